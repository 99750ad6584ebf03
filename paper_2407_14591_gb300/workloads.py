"""Seeded synthetic inputs: lattices, term lists and start vectors.

This module holds no arithmetic of the method. It only draws random numbers and lists the
bonds of the lattices, in a neutral form ``(kind, i, j, coef)`` that both the CUDA path (via
the binding) and the CPU oracle (in tests and in the bench's CPU baseline) consume. It imports
nothing from the rest of the package.

Random numbers come from numpy's PCG64 with seed ``20240719 + workload number``; vectors are
drawn as U[-1, 1] in FP64, normalised per right-hand side in FP64 and only then cast.
Disorder (couplings, fields, Hubbard U) is drawn from the same generator after the vector.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20240719

__all__ = [
    "SEED_BASE",
    "Workload",
    "rng_for",
    "random_vector",
    "chain_bonds",
    "square_bonds",
    "heisenberg_terms",
    "workload",
    "batched_chains",
]


def rng_for(number: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + number))


def random_vector(rng: np.random.Generator, D: int, nrhs: int = 1, dtype=np.float64) -> np.ndarray:
    """U[-1,1] entries drawn in FP64, each right-hand side normalised to 1 in FP64, then cast.

    Shape (D,) for nrhs == 1, else (D, nrhs) (row i holds the nrhs values of basis state i).
    """
    x = rng.uniform(-1.0, 1.0, size=(D, nrhs))
    x /= np.linalg.norm(x, axis=0, keepdims=True)
    x = x.astype(dtype)
    return x[:, 0].copy() if nrhs == 1 else x


def chain_bonds(L: int, periodic: bool = True) -> list[tuple[int, int]]:
    """Nearest-neighbour bonds (i, i+1) of a chain; the periodic one adds (L-1, 0)."""
    n = L if periodic else L - 1
    return [(i, (i + 1) % L) for i in range(n)]


def square_bonds(Lx: int, Ly: int) -> tuple[list[tuple[int, int]], list[tuple[int, int]]]:
    """Periodic Lx x Ly square lattice, site = x + Lx*y: (nearest, next-nearest) bond lists.

    Nearest: (x,y)-(x+1,y) and (x,y)-(x,y+1). Next-nearest: (x,y)-(x+1,y+1) and
    (x,y)-(x+1,y-1). Each list has 2 Lx Ly bonds.
    """
    def s(x, y):
        return (x % Lx) + Lx * (y % Ly)

    nn, nnn = [], []
    for y in range(Ly):
        for x in range(Lx):
            nn.append((s(x, y), s(x + 1, y)))
            nn.append((s(x, y), s(x, y + 1)))
            nnn.append((s(x, y), s(x + 1, y + 1)))
            nnn.append((s(x, y), s(x + 1, y - 1)))
    return nn, nnn


def heisenberg_terms(bonds, J, delta: float = 1.0) -> list[tuple[str, int, int, float]]:
    """J_b (Sx Sx + Sy Sy + delta Sz Sz) per bond, as XY and ZZ terms. J may be a scalar or a
    per-bond sequence."""
    Js = np.broadcast_to(np.asarray(J, dtype=np.float64), (len(bonds),))
    out = []
    for (i, j), Jb in zip(bonds, Js):
        out.append(("XY", i, j, float(Jb)))
        out.append(("ZZ", i, j, float(Jb) * delta))
    return out


def field_terms(h) -> list[tuple[str, int, int, float]]:
    return [("Z", i, -1, float(hi)) for i, hi in enumerate(h)]


@dataclass
class Workload:
    name: str
    L: int
    Q: int
    N: int
    n_sub: int
    terms: list = field(default_factory=list)
    number: int = 0
    nrhs: int = 1
    notes: str = ""


def workload(number: int, n_sub: int | None = None, draw_vector: bool = True, D: int | None = None):
    """The five seeded workloads; returns (Workload, x or None).

    ``D`` must be the sector dimension when ``draw_vector`` is set (the caller knows it from
    its own sector object); the disorder draws follow the vector draw in the same generator.

    1  periodic Heisenberg chain L=20, N=10, J=1, delta=1; n_sub=2.
    2  J1-J2 Heisenberg on the periodic 6x5 square lattice (site = x + 6y), N=15, J1=1, J2=0.5;
       n_sub in {2, 3, 5}.
    3  periodic Bose-Hubbard chain Q=4, L=14, N=14, t=1, U_i ~ U[2, 6]; n_sub=2.
    5  periodic disordered XXZ chain L=24, N=12, delta=1, J_b ~ U[0.5, 1.5], h_i ~ U[-3, 3].
    Workload 4 (many chains at once) is ``batched_chains``.
    """
    rng = rng_for(number)
    x = None
    if number == 1:
        w = Workload("heisenberg_chain_L20_N10", 20, 2, 10, 2 if n_sub is None else n_sub, number=1)
        w.terms = heisenberg_terms(chain_bonds(20), 1.0, 1.0)
        if draw_vector:
            x = random_vector(rng, D)
    elif number == 2:
        w = Workload("j1j2_square_6x5_N15", 30, 2, 15, 2 if n_sub is None else n_sub, number=2)
        nn, nnn = square_bonds(6, 5)
        w.terms = heisenberg_terms(nn, 1.0, 1.0) + heisenberg_terms(nnn, 0.5, 1.0)
        if draw_vector:
            x = random_vector(rng, D)
    elif number == 3:
        w = Workload("bose_hubbard_Q4_L14_N14", 14, 4, 14, 2 if n_sub is None else n_sub, number=3)
        if draw_vector:
            x = random_vector(rng, D)
        U = rng.uniform(2.0, 6.0, size=14)
        w.terms = [("HOP", i, j, 1.0) for i, j in chain_bonds(14)] + [("U", i, -1, float(U[i])) for i in range(14)]
    elif number == 5:
        w = Workload("disordered_xxz_L24_N12", 24, 2, 12, 2 if n_sub is None else n_sub, number=5)
        if draw_vector:
            x = random_vector(rng, D)
        Jb = rng.uniform(0.5, 1.5, size=24)
        h = rng.uniform(-3.0, 3.0, size=24)
        w.terms = heisenberg_terms(chain_bonds(24), Jb, 1.0) + field_terms(h)
    else:
        raise ValueError("workload number must be 1, 2, 3 or 5 (4 is batched_chains)")
    return w, x


def batched_chains(count: int = 64, nrhs: int = 8, L_range=(16, 26), draw=True):
    """Workload 4: ``count`` periodic XXZ chains (J=1, delta=1, h_i ~ U[-5, 5]).

    L ~ U{16..26}; N ~ U{floor(L/2)-3 .. floor(L/2)}. All (L, N) pairs are drawn first, then
    each chain's fields in order. Vectors are drawn by ``batched_vectors`` once the caller knows
    each sector's dimension. Returns a list of Workload.
    """
    rng = rng_for(4)
    Ls = rng.integers(L_range[0], L_range[1] + 1, size=count)
    Ns = np.array([rng.integers(L // 2 - 3, L // 2 + 1) for L in Ls])
    out = []
    for c, (L, N) in enumerate(zip(Ls, Ns)):
        h = rng.uniform(-5.0, 5.0, size=int(L))
        w = Workload(f"xxz_chain_{c}_L{L}_N{N}", int(L), 2, int(N), 0, number=4, nrhs=nrhs)
        w.terms = heisenberg_terms(chain_bonds(int(L)), 1.0, 1.0) + field_terms(h)
        out.append(w)
    return out


def batched_vectors(dims, nrhs: int = 8, dtype=np.float64):
    """Start vectors of workload 4, one (D, nrhs) array per chain, from the jumped PCG64 stream
    of the same seed (so they do not depend on how much disorder was drawn)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4).jumped())  # a stream apart from the disorder
    return [random_vector(rng, int(D), nrhs, dtype) for D in dims]
