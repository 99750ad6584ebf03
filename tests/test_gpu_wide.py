"""States of two words (64 < L * Nbits <= 128) on the GPU, through the two-word C-ABI forms.

Bit-exact whole-sector unrank / rank against the oracle's sorted list (exact Python integers),
the two-word batches on one-word sectors, the error word, the product y = H x against the
oracle (FP64 bar 1e-12 max-relative, FP32 bar 1e-5 relative L2), and Lanczos on a 66-site
free-fermion chain against the Jordan-Wigner energy.
"""

import numpy as np
import pytest
import torch

from oracle import OracleSector, matvec as o_matvec
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"
MASK64 = (1 << 64) - 1


def words_tensor(words):
    """(n, 2) int64 tensor of two-word states (low word first) from Python integers."""
    lo = np.array([int(w) & MASK64 for w in words], dtype=np.uint64).view(np.int64)
    hi = np.array([int(w) >> 64 for w in words], dtype=np.uint64).view(np.int64)
    return torch.from_numpy(np.stack([lo, hi], axis=1)).to(DEV)


def words_of(t):
    a = t.cpu().numpy().view(np.uint64)
    return [int(lo) | (int(hi) << 64) for lo, hi in a]


@pytest.mark.parametrize("L,Q,N,n_sub", [(70, 2, 3, 5), (33, 4, 3, 3), (128, 2, 2, 8), (100, 2, 3, 7), (42, 8, 2, 0),
                                          (65, 2, 64, 5), (64, 4, 2, 6)])
def test_wide_unrank_rank_whole_sector_bit_exact(L, Q, N, n_sub):
    s = b.make_sector(L, Q, N, n_sub)
    assert s.wide
    o = OracleSector(L, Q, N, partition=s.partition)
    assert s.dim == o.dim
    idx = torch.arange(s.dim, device=DEV, dtype=torch.int64)
    st = s.state_at_batch2(idx)
    back = s.index_of_batch2(st)
    torch.cuda.synchronize()
    s.check_device()
    assert words_of(st) == [int(w) for w in o.basis]
    assert torch.equal(back, idx)
    for i in (0, s.dim // 3, s.dim - 1):  # the host forms agree
        assert s.state_at(i) == int(o.basis[i]) and s.index_of(int(o.basis[i])) == i


def test_two_word_batches_on_a_one_word_sector():
    s = b.make_sector(20, 2, 10, 2)
    idx = torch.arange(s.dim, device=DEV, dtype=torch.int64)
    st1 = s.state_at_batch(idx)
    st2 = s.state_at_batch2(idx)
    torch.cuda.synchronize()
    assert torch.equal(st2[:, 0], st1) and torch.all(st2[:, 1] == 0)
    assert torch.equal(s.index_of_batch2(st2), idx)
    s.check_device()


def test_wide_batch_error_word():
    s = b.make_sector(70, 2, 2, 5)
    out = s.state_at_batch2(torch.tensor([0, s.dim, 5], device=DEV, dtype=torch.int64))
    torch.cuda.synchronize()
    assert out[1].tolist() == [-1, -1] and words_of(out[:1]) == [s.state_at(0)]
    with pytest.raises(b.DQError) as e:
        s.check_device()
    assert e.value.code == b.DQ_EDEVICE
    bad = words_tensor([s.state_at(7), (1 << 70) | 1, 0b111, (1 << 69) | (1 << 3)])
    got = s.index_of_batch2(bad)
    torch.cuda.synchronize()
    assert got.tolist() == [7, -1, -1, s.index_of((1 << 69) | (1 << 3))]
    with pytest.raises(b.DQError):
        s.check_device()
    s.check_device()


def random_terms(rng, L, Q, nbonds):
    kinds_pair, kinds_site = (["XY", "ZZ", "HOP", "NN"], ["Z", "N"]) if Q == 2 else (["HOP", "NN"], ["N", "U"])
    terms = []
    for _ in range(nbonds):
        i, j = rng.choice(L, size=2, replace=False)
        for k in kinds_pair:
            if rng.random() < 0.7:
                terms.append((k, int(i), int(j), float(rng.uniform(-1.5, 1.5))))
    for i in rng.choice(L, size=min(L, 12), replace=False):
        for k in kinds_site:
            terms.append((k, int(i), -1, float(rng.uniform(-2, 2))))
    return terms


@pytest.mark.parametrize("L,Q,N,n_sub,nb", [(70, 2, 2, 5, 40), (66, 2, 3, 5, 10), (33, 4, 3, 3, 30), (128, 2, 2, 8, 60),
                                             (42, 8, 2, 0, 30)])
def test_wide_matvec_vs_oracle(L, Q, N, n_sub, nb):
    rng = np.random.default_rng(L * 7 + Q * 3 + N)
    terms = random_terms(rng, L, Q, nb)
    s = b.make_sector(L, Q, N, n_sub)
    t = b.make_terms(s, terms)
    assert t.path == "general"
    o = OracleSector(L, Q, N, partition=s.partition)
    for nrhs in (1, 3):
        x = rng.uniform(-1, 1, (o.dim, nrhs))
        x = x[:, 0].copy() if nrhs == 1 else x
        ref = o_matvec(o, terms, x)
        y = b.matvec(s, t, torch.from_numpy(x).to(DEV)).cpu().numpy()
        s.check_device()
        assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref)), nrhs
        x32 = x.astype(np.float32)
        ref32 = o_matvec(o, terms, x32.astype(np.float64))
        y32 = b.matvec(s, t, torch.from_numpy(x32).to(DEV)).double().cpu().numpy()
        assert np.linalg.norm(y32 - ref32) <= 1e-5 * np.linalg.norm(ref32), nrhs


def test_wide_lanczos_free_fermions():
    """A disordered periodic XX chain of 66 sites with 3 particles (D = 45,760, 66-bit words):
    the GPU Lanczos E0 against the Jordan-Wigner free-fermion energy."""
    L, N = 66, 3
    rng = np.random.default_rng(166)
    bonds = wl.chain_bonds(L, True)
    J = rng.uniform(0.5, 1.5, L)
    h = rng.uniform(-1, 1, L)
    terms = wl.heisenberg_terms(bonds, J, 0.0) + wl.field_terms(h)
    hsp = np.diag(h)
    for bnd, (i, j) in enumerate(bonds):
        sg = (-1.0) ** (N - 1) if bnd == L - 1 else 1.0
        hsp[i, j] += sg * J[bnd] / 2
        hsp[j, i] += sg * J[bnd] / 2
    exact = np.sort(np.linalg.eigvalsh(hsp))[:N].sum() - 0.5 * h.sum()
    s = b.make_sector(L, 2, N, 0)
    assert s.wide
    t = b.make_terms(s, terms)
    res = b.lanczos(s, t, torch.from_numpy(rng.uniform(-1, 1, s.dim)).to(DEV), 300)
    assert abs(res["E0"] - exact) <= 1e-10 * abs(exact)
