"""Pins for the oracle's operator terms, product y = H x and Lanczos (CPU only).

The main pin is an independent textbook construction: the full Q^L-dimensional Hamiltonian built
from Kronecker products of single-site matrices, restricted to the sector's rows and columns and
permuted into canonical order. Further pins: Hermiticity, term-by-term linearity, E0 = -2 for the
4-site Heisenberg ring, free fermions (Jordan-Wigner) for XX chains with fields, and the t = 0
Bose-Hubbard chain by brute force over occupations.
"""

import itertools
from functools import reduce

import numpy as np
import pytest
import scipy.sparse as sp

import oracle.hamiltonian as oh
from conftest import read_golden
from oracle import OracleSector, lanczos, matvec, matvec_rows
from paper_2407_14591_gb300 import workloads as wl


def site_ops(Q):
    b = np.zeros((Q, Q))
    for n in range(1, Q):
        b[n - 1, n] = np.sqrt(n)  # b|n> = sqrt(n)|n-1>
    num = np.diag(np.arange(Q, dtype=float))
    return b, num


def embed(op, i, L, Q):
    mats = [sp.identity(Q, format="csr")] * L
    mats = mats[:i] + [sp.csr_matrix(op)] + mats[i + 1:]
    return reduce(lambda a, b: sp.kron(a, b, format="csr"), mats)


def dense_full(L, Q, terms):
    """Full-space H from Kronecker products; site 0 is the leftmost factor."""
    b, num = site_ops(Q)
    bd = b.T
    dimf = Q ** L
    H = sp.csr_matrix((dimf, dimf))
    if Q == 2:
        splus, sminus, sz = bd, b, num - 0.5 * np.eye(2)  # particle = up spin
    for kind, i, j, c in terms:
        if kind == "XY":
            H += c * 0.5 * (embed(splus, i, L, Q) @ embed(sminus, j, L, Q) + embed(sminus, i, L, Q) @ embed(splus, j, L, Q))
        elif kind == "ZZ":
            H += c * embed(sz, i, L, Q) @ embed(sz, j, L, Q)
        elif kind == "Z":
            H += c * embed(sz, i, L, Q)
        elif kind == "HOP":
            H += -c * (embed(bd, i, L, Q) @ embed(b, j, L, Q) + embed(bd, j, L, Q) @ embed(b, i, L, Q))
        elif kind == "NN":
            H += c * embed(num, i, L, Q) @ embed(num, j, L, Q)
        elif kind == "N":
            H += c * embed(num, i, L, Q)
        elif kind == "U":
            H += 0.5 * c * embed(num @ (num - np.eye(Q)), i, L, Q)
    return H.tocsr()


def full_index(sec, words):
    """Kronecker-order index sum_i d_i Q^(L-1-i) of each word."""
    d = sec.digits(words)
    return (d * (sec.Q ** np.arange(sec.L - 1, -1, -1))).sum(axis=1)


def restricted(sec, terms):
    H = dense_full(sec.L, sec.Q, terms)
    f = full_index(sec, sec.basis)
    return H[f][:, f].toarray()


def oracle_dense(sec, terms):
    return matvec(sec, terms, np.eye(sec.dim))


def random_terms(rng, L, Q, nbonds):
    kinds_pair = ["XY", "ZZ"] if Q == 2 else ["HOP", "NN"]
    kinds_site = ["Z"] if Q == 2 else ["N", "U"]
    terms = []
    for _ in range(nbonds):
        i, j = rng.choice(L, size=2, replace=False)
        for k in kinds_pair:
            terms.append((k, int(i), int(j), float(rng.uniform(-1.5, 1.5))))
    for i in range(L):
        for k in kinds_site:
            terms.append((k, i, -1, float(rng.uniform(-2, 2))))
    if Q == 2:  # a boson hop on Q=2 is a hard-core hop; include it too
        terms.append(("HOP", 0, L - 1, 0.7))
        terms.append(("NN", 1, 2, -0.3))
        terms.append(("U", 0, -1, 5.0))  # n(n-1) = 0 for Q = 2
    return terms


@pytest.mark.parametrize("L,Q,N,n_sub,nb", [(8, 2, 4, 2, 10), (9, 2, 3, 3, 12), (10, 2, 5, 4, 9),
                                             (6, 3, 6, 2, 7), (5, 4, 7, 2, 6), (6, 3, 4, 6, 6),
                                             (5, 4, 5, 1, 6)])
def test_matvec_equals_restricted_kronecker(L, Q, N, n_sub, nb):
    rng = np.random.default_rng(1000 + L * 10 + Q)
    terms = random_terms(rng, L, Q, nb)
    sec = OracleSector(L, Q, N, n_sub=n_sub)
    np.testing.assert_allclose(oracle_dense(sec, terms), restricted(sec, terms), rtol=0, atol=1e-13)


def test_j1j2_small_lattice_kronecker():
    nn, nnn = wl.square_bonds(4, 3)
    terms = wl.heisenberg_terms(nn, 1.0) + wl.heisenberg_terms(nnn, 0.5)
    sec = OracleSector(12, 2, 6, n_sub=3)
    x = np.random.default_rng(5).uniform(-1, 1, sec.dim)
    H = restricted(sec, terms)
    np.testing.assert_allclose(matvec(sec, terms, x), H @ x, rtol=0, atol=1e-12)


def test_hermitian_linear_and_rows():
    rng = np.random.default_rng(7)
    sec = OracleSector(14, 2, 6, n_sub=3)
    nn, nnn = wl.square_bonds(7, 2)
    t1 = wl.heisenberg_terms(nn, rng.uniform(0.5, 1.5, len(nn)), 0.7)
    t2 = wl.field_terms(rng.uniform(-1, 1, 14))
    u, v = rng.uniform(-1, 1, (2, sec.dim))
    Hu, Hv = matvec(sec, t1 + t2, u), matvec(sec, t1 + t2, v)
    assert abs(u @ Hv - Hu @ v) <= 1e-12 * np.abs(Hu).max() * np.abs(v).sum()
    np.testing.assert_allclose(Hv, matvec(sec, t1, v) + matvec(sec, t2, v), rtol=0, atol=1e-13)
    rows = rng.choice(sec.dim, 300, replace=False)
    np.testing.assert_allclose(matvec_rows(sec, t1 + t2, v, rows), Hv[rows], rtol=0, atol=1e-13)
    V = rng.uniform(-1, 1, (sec.dim, 3))
    np.testing.assert_allclose(matvec(sec, t1 + t2, V)[:, 1], matvec(sec, t1 + t2, V[:, 1]), rtol=0, atol=1e-13)


def test_heisenberg_ring_L4():
    sec = OracleSector(4, 2, 2, n_sub=2)
    terms = wl.heisenberg_terms(wl.chain_bonds(4), 1.0)
    assert np.linalg.eigvalsh(oracle_dense(sec, terms))[0] == pytest.approx(-2.0, abs=1e-14)
    rng = np.random.default_rng(0)
    res = lanczos(lambda v: matvec(sec, terms, v), rng.uniform(-1, 1, sec.dim), 10)
    assert res["E0"] == pytest.approx(-2.0, abs=1e-13)


def free_fermion_e0(L, N, J, h, periodic):
    """XX chain with fields via Jordan-Wigner: sum of the N lowest single-particle levels
    minus sum(h)/2; a periodic boundary hop carries the sign (-1)^(N-1)."""
    hsp = np.diag(np.asarray(h, dtype=float))
    for b, (i, j) in enumerate(wl.chain_bonds(L, periodic)):
        s = (-1.0) ** (N - 1) if (periodic and b == L - 1) else 1.0
        hsp[i, j] += s * J[b] / 2
        hsp[j, i] += s * J[b] / 2
    return np.sort(np.linalg.eigvalsh(hsp))[:N].sum() - 0.5 * np.sum(h)


@pytest.mark.parametrize("L,N,periodic,n_sub", [(10, 4, False, 2), (10, 5, True, 3), (12, 5, True, 2),
                                                 (16, 8, True, 2), (16, 7, False, 4)])
def test_free_fermion_e0(L, N, periodic, n_sub):
    rng = np.random.default_rng(L * 100 + N)
    bonds = wl.chain_bonds(L, periodic)
    J = rng.uniform(0.5, 1.5, len(bonds))
    h = rng.uniform(-1, 1, L)
    terms = wl.heisenberg_terms(bonds, J, 0.0) + wl.field_terms(h)
    sec = OracleSector(L, 2, N, n_sub=n_sub)
    x0 = rng.uniform(-1, 1, sec.dim)
    res = lanczos(lambda v: matvec(sec, terms, v), x0, 120)
    assert res["E0"] == pytest.approx(free_fermion_e0(L, N, J, h, periodic), abs=1e-10)


def test_bose_hubbard_t0_brute_force():
    L, Q, N = 6, 4, 7
    U = np.random.default_rng(3).uniform(2, 6, L)
    terms = [("HOP", i, j, 0.0) for i, j in wl.chain_bonds(L)] + [("U", i, -1, float(U[i])) for i in range(L)]
    sec = OracleSector(L, Q, N, n_sub=2)
    best = min(sum(U[i] / 2 * n[i] * (n[i] - 1) for i in range(L))
               for n in itertools.product(range(Q), repeat=L) if sum(n) == N)
    assert np.linalg.eigvalsh(oracle_dense(sec, terms))[0] == pytest.approx(best, abs=1e-12)


def test_lanczos_matches_dense_and_breakdown():
    w, _ = wl.workload(3, draw_vector=False)
    sec = OracleSector(6, 4, 6, n_sub=2)
    terms = [("HOP", i, j, 1.0) for i, j in wl.chain_bonds(6)] + [("U", i, -1, 3.0 + 0.1 * i) for i in range(6)]
    ev = np.linalg.eigvalsh(oracle_dense(sec, terms))
    res = lanczos(lambda v: matvec(sec, terms, v), np.random.default_rng(2).uniform(-1, 1, sec.dim), 200,
                  want_vector=True)
    assert res["E0"] == pytest.approx(ev[0], abs=1e-10)
    assert res["steps_done"] <= sec.dim  # stops at an invariant subspace, not an error
    psi = res["vector"]
    r = matvec(sec, terms, psi) - res["E0"] * psi
    assert np.linalg.norm(r) < 1e-8


def test_planted_mistakes_are_caught(monkeypatch):
    """A dropped factor or a wrong amplitude in the oracle makes the Kronecker pin fail."""
    rng = np.random.default_rng(11)
    sec2 = OracleSector(8, 2, 4, n_sub=2)
    t2 = random_terms(rng, 8, 2, 8)
    sec4 = OracleSector(5, 4, 6, n_sub=2)
    t4 = random_terms(rng, 5, 4, 6)
    ref2, ref4 = restricted(sec2, t2), restricted(sec4, t4)
    orig = oh._offdiag_images

    def xy_without_half(sector, kind, i, j, c, words):
        for pos, new, amp in orig(sector, kind, i, j, c, words):
            yield pos, new, amp * (2.0 if kind == "XY" else 1.0)

    monkeypatch.setattr(oh, "_offdiag_images", xy_without_half)
    assert not np.allclose(oracle_dense(sec2, t2), ref2, atol=1e-10)

    def hop_without_sqrt(sector, kind, i, j, c, words):
        for pos, new, amp in orig(sector, kind, i, j, c, words):
            yield pos, new, (np.sign(amp) * abs(c) if kind == "HOP" else amp)

    monkeypatch.setattr(oh, "_offdiag_images", hop_without_sqrt)
    assert not np.allclose(oracle_dense(sec4, t4), ref4, atol=1e-10)
    monkeypatch.setattr(oh, "_offdiag_images", orig)
    orig_diag = oh._diag_term
    monkeypatch.setattr(oh, "_diag_term", lambda s, k, i, j, c, w: orig_diag(s, k, i, j, -c if k == "ZZ" else c, w))
    assert not np.allclose(oracle_dense(sec2, t2), ref2, atol=1e-10)


def test_lanczos_golden_workload1_matches_sparse_eigensolver():
    """The stored oracle Lanczos E0 of workload 1 (L = 20 ring, N = 10) equals the smallest
    eigenvalue (ARPACK) of the Heisenberg Hamiltonian written out independently of the oracle:
    basis = all 20-bit words with ten set bits (any order), S+S- + S-S+ / 2 as pair flips located
    through a dense word -> position table, SzSz = +-1/4 on the diagonal."""
    import scipy.sparse as sps
    from scipy.sparse.linalg import eigsh

    rows = dict((r[0], r[1:]) for r in read_golden("lanczos_workload1.txt"))
    E0 = float(rows["E0"][0])
    L = 20
    words = np.arange(1 << L, dtype=np.int64)
    pop = np.zeros(1 << L, dtype=np.int64)
    for b in range(L):
        pop += (words >> b) & 1
    states = words[pop == 10]
    pos = np.full(1 << L, -1, dtype=np.int64)
    pos[states] = np.arange(states.size)
    diag = np.zeros(states.size)
    r_idx, c_idx = [], []
    for i in range(L):
        j = (i + 1) % L
        bi, bj = (states >> i) & 1, (states >> j) & 1
        diag += np.where(bi == bj, 0.25, -0.25)
        m = np.flatnonzero(bi != bj)
        r_idx.append(m)
        c_idx.append(pos[states[m] ^ ((1 << i) | (1 << j))])
    r_idx, c_idx = np.concatenate(r_idx), np.concatenate(c_idx)
    assert (c_idx >= 0).all()
    H = sps.csr_matrix((np.full(r_idx.size, 0.5), (r_idx, c_idx)), shape=(states.size,) * 2) + sps.diags(diag)
    ev = eigsh(H, k=1, which="SA", tol=1e-13)[0][0]
    assert abs(E0 - ev) <= 1e-9 * abs(ev)


@pytest.mark.parametrize("L,Q,N,n_sub,nb", [(8, 2, 4, 2, 10), (9, 2, 3, 3, 12), (6, 3, 6, 2, 7), (5, 4, 7, 2, 6),
                                             (6, 3, 4, 6, 6)])
def test_diagonal_equals_kronecker_diagonal(L, Q, N, n_sub, nb):
    """oracle.diagonal(sector, terms) is <sigma|H|sigma> of the restricted Kronecker-built H, for
    the whole basis and for a subset of words given explicitly."""
    rng = np.random.default_rng(2000 + L * 10 + Q)
    terms = random_terms(rng, L, Q, nb)
    sec = OracleSector(L, Q, N, n_sub=n_sub)
    ref = np.diag(restricted(sec, terms))
    np.testing.assert_allclose(oh.diagonal(sec, terms), ref, rtol=0, atol=1e-13)
    pick = rng.choice(sec.dim, min(sec.dim, 17), replace=False)
    np.testing.assert_allclose(oh.diagonal(sec, terms, sec.basis[pick]), ref[pick], rtol=0, atol=1e-13)


def test_diagonal_planted_mistake_is_caught(monkeypatch):
    """A flipped sign of the Sz Sz term or a dropped 1/2 of the Hubbard term fails the pin."""
    rng = np.random.default_rng(21)
    sec2, sec4 = OracleSector(8, 2, 4, n_sub=2), OracleSector(5, 4, 6, n_sub=2)
    t2, t4 = random_terms(rng, 8, 2, 8), random_terms(rng, 5, 4, 6)
    ref2, ref4 = np.diag(restricted(sec2, t2)), np.diag(restricted(sec4, t4))
    orig = oh._diag_term
    monkeypatch.setattr(oh, "_diag_term", lambda s, k, i, j, c, w: orig(s, k, i, j, -c if k == "ZZ" else c, w))
    assert not np.allclose(oh.diagonal(sec2, t2), ref2, atol=1e-10)
    monkeypatch.setattr(oh, "_diag_term", lambda s, k, i, j, c, w: orig(s, k, i, j, 2 * c if k == "U" else c, w))
    assert not np.allclose(oh.diagonal(sec4, t4), ref4, atol=1e-10)


@pytest.mark.parametrize("Lw,L,Q,N", [(66, 12, 2, 3), (70, 10, 2, 2), (33, 7, 4, 3)])
def test_wide_words_embedding_equals_narrow_oracle(Lw, L, Q, N):
    """Terms on the first L sites of an Lw-site lattice (words wider than 64 bits): the states
    with every particle on those sites form an invariant block, and on it the wide product equals
    the one-word product of the L-site lattice (itself pinned to the Kronecker construction),
    word w mapping to w << Nbits (Lw - L); x supported on the block gives y zero elsewhere."""
    rng = np.random.default_rng(Lw + L + Q)
    terms = random_terms(rng, L, Q, L + 2)
    narrow = OracleSector(L, Q, N, n_sub=2)
    wide = OracleSector(Lw, Q, N, n_sub=0)
    assert wide.wide and not narrow.wide
    nb = (Q - 1).bit_length()
    shift = nb * (Lw - L)
    rows = wide.index_of_many(wide.words_array([int(w) << shift for w in narrow.basis]))
    x = rng.uniform(-1, 1, narrow.dim)
    xw = np.zeros(wide.dim)
    xw[rows] = x
    yw = matvec(wide, terms, xw)
    np.testing.assert_allclose(yw[rows], matvec(narrow, terms, x), rtol=0, atol=1e-13)
    rest = np.ones(wide.dim, dtype=bool)
    rest[rows] = False
    assert np.all(yw[rest] == 0.0)
    np.testing.assert_allclose(matvec_rows(wide, terms, xw, rows[:50]), yw[rows[:50]], rtol=0, atol=1e-13)


def test_wide_words_free_fermion_e0():
    """A disordered periodic XX chain of 66 sites with 2 particles (66-bit words): the oracle
    Lanczos E0 equals the Jordan-Wigner free-fermion value."""
    L, N = 66, 2
    rng = np.random.default_rng(66)
    bonds = wl.chain_bonds(L, True)
    J = rng.uniform(0.5, 1.5, len(bonds))
    h = rng.uniform(-1, 1, L)
    terms = wl.heisenberg_terms(bonds, J, 0.0) + wl.field_terms(h)
    sec = OracleSector(L, 2, N, n_sub=5)
    assert sec.wide
    res = lanczos(lambda v: matvec(sec, terms, v), rng.uniform(-1, 1, sec.dim), 100)
    assert res["E0"] == pytest.approx(free_fermion_e0(L, N, J, h, True), abs=1e-10)
