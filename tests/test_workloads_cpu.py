"""The seeded input generators (CPU): reproducible draws, the stated recipe (x ~ U[-1, 1] drawn in
FP64 and normalised per right-hand side, disorder drawn after x), the lattices' bond counts and the
workload-4 ranges. They hold none of the method's arithmetic; the same generators feed the
oracle and the library.
"""

import numpy as np

from oracle import sector_dim
from paper_2407_14591_gb300 import workloads as wl


def test_vectors_are_seeded_normalised_and_in_range():
    a = wl.random_vector(wl.rng_for(1), 1000)
    b = wl.random_vector(wl.rng_for(1), 1000)
    assert np.array_equal(a, b)
    assert abs(np.linalg.norm(a) - 1.0) < 1e-14
    m = wl.random_vector(wl.rng_for(2), 500, nrhs=3)
    assert m.shape == (500, 3)
    assert np.allclose(np.linalg.norm(m, axis=0), 1.0, atol=1e-14)
    # the same generator's U[-1, 1] draw, each column divided by its FP64 norm
    raw = wl.rng_for(2).uniform(-1.0, 1.0, size=(500, 3))
    assert np.array_equal(m, raw / np.linalg.norm(raw, axis=0, keepdims=True))
    f = wl.random_vector(wl.rng_for(1), 1000, dtype=np.float32)
    assert f.dtype == np.float32 and np.array_equal(f, a.astype(np.float32))


def test_disorder_is_drawn_after_the_vector():
    """Workload 5's couplings and fields follow the vector draw in the same generator, so they
    depend on the sector dimension the caller passes, and repeat exactly for the same one."""
    D = sector_dim(24, 2, 12)
    w1, x1 = wl.workload(5, D=D)
    w2, x2 = wl.workload(5, D=D)
    assert w1.terms == w2.terms and np.array_equal(x1, x2)
    rng = wl.rng_for(5)
    x = wl.random_vector(rng, D)
    Jb = rng.uniform(0.5, 1.5, size=24)
    h = rng.uniform(-3.0, 3.0, size=24)
    assert np.array_equal(x, x1)
    zz = [c for k, i, j, c in w1.terms if k == "ZZ"]
    z = [c for k, i, j, c in w1.terms if k == "Z"]
    assert np.allclose(zz, Jb) and np.allclose(z, h)
    assert all(0.5 <= c <= 1.5 for c in zz) and all(-3.0 <= c <= 3.0 for c in z)


def test_lattices_and_workload_shapes():
    nn, nnn = wl.square_bonds(6, 5)
    assert len(nn) == len(nnn) == 60
    assert len({tuple(sorted(b)) for b in nn}) == 60 and len({tuple(sorted(b)) for b in nnn}) == 60
    assert all(0 <= i < 30 and 0 <= j < 30 and i != j for i, j in nn + nnn)
    assert len(wl.chain_bonds(20)) == 20 and len(wl.chain_bonds(20, periodic=False)) == 19
    w2, _ = wl.workload(2, draw_vector=False)
    assert (w2.L, w2.Q, w2.N) == (30, 2, 15) and sector_dim(30, 2, 15) == 155117520
    w3, _ = wl.workload(3, draw_vector=False)
    assert (w3.L, w3.Q, w3.N) == (14, 4, 14) and sector_dim(14, 4, 14) == 6472168
    assert sum(1 for k, *_ in w3.terms if k == "HOP") == 14 and sum(1 for k, *_ in w3.terms if k == "U") == 14


def test_workload4_chain_ranges_and_vectors():
    chains = wl.batched_chains()
    assert len(chains) == 64
    for w in chains:
        assert 16 <= w.L <= 26 and w.L // 2 - 3 <= w.N <= w.L // 2 and w.nrhs == 8
        h = [c for k, i, j, c in w.terms if k == "Z"]
        assert len(h) == w.L and all(-5.0 <= c <= 5.0 for c in h)
    again = wl.batched_chains()
    assert [(w.L, w.N, w.terms) for w in chains] == [(w.L, w.N, w.terms) for w in again]
    dims = [sector_dim(w.L, 2, w.N) for w in chains[:3]]
    v = wl.batched_vectors(dims, nrhs=8)
    assert [a.shape for a in v] == [(d, 8) for d in dims]
    assert all(np.allclose(np.linalg.norm(a, axis=0), 1.0, atol=1e-13) for a in v)
