"""CUDA path against the oracle, through the C-ABI (GPU only).

Bar: indices and states bit-exact; FP64 y within max_i |y_i - y_ref_i| / max_i |y_ref_i| <= 1e-12;
FP32-vector y within ||y - y_ref||_2 / ||y_ref||_2 <= 1e-5 of the FP64 oracle applied to the same
(FP32) input; Lanczos E0 within 1e-10 (FP64) or 1e-6 (FP32) relative of the oracle's E0.
"""

import numpy as np
import pytest
import torch

from oracle import OracleSector, lanczos as o_lanczos, matvec as o_matvec, matvec_rows as o_matvec_rows
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5
DEV = "cuda"


def maxrel(y, ref):
    return float(np.max(np.abs(y - ref)) / np.max(np.abs(ref)))


def rel2(y, ref):
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


_SECTORS = {}


def oracle_sector(L, Q, N, partition):
    key = (L, Q, N, tuple(partition))
    if key not in _SECTORS:
        _SECTORS[key] = OracleSector(L, Q, N, partition=partition)
    return _SECTORS[key]


def gpu_matvec(sec, terms, x_np, dtype=torch.float64):
    t = b.make_terms(sec, terms)
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV, dtype)
    y = b.matvec(sec, t, x)
    torch.cuda.synchronize()
    sec.check_device()
    return y.double().cpu().numpy()


# ---------------------------------------------------------------- rank / unrank -------------

@pytest.mark.parametrize("L,Q,N,n_sub", [(20, 2, 10, 2), (14, 4, 14, 2), (24, 2, 12, 2), (12, 3, 9, 3),
                                          (16, 2, 8, 16), (10, 5, 17, 4), (5, 16, 30, 2), (18, 2, 7, 1),
                                          (64, 2, 2, 4), (64, 2, 3, 3), (32, 4, 3, 3)])
def test_unrank_rank_whole_sector_bit_exact(L, Q, N, n_sub):
    s = b.make_sector(L, Q, N, n_sub)
    o = oracle_sector(L, Q, N, s.partition)
    idx = torch.arange(s.dim, device=DEV, dtype=torch.int64)
    st = s.state_at_batch(idx)
    back = s.index_of_batch(st)
    torch.cuda.synchronize()
    s.check_device()
    assert np.array_equal(st.cpu().numpy().view(np.uint64), o.basis)
    assert torch.equal(back, idx)


def test_rank_unrank_sampled_large_sector():
    for n_sub in (2, 3, 5):
        s = b.make_sector(30, 2, 15, n_sub)
        g = torch.Generator(device="cpu").manual_seed(20240721 + n_sub)
        idx = torch.randint(0, s.dim, (1 << 24,), generator=g).to(DEV)
        idx[:4096] = torch.arange(4096, device=DEV)
        idx[-4096:] = torch.arange(s.dim - 4096, s.dim, device=DEV)
        back = s.index_of_batch(s.state_at_batch(idx))
        torch.cuda.synchronize()
        s.check_device()
        assert torch.equal(back, idx)
        # spot check against the host functions
        for i in idx[:64].tolist() + idx[-64:].tolist():
            assert s.index_of(s.state_at(i)) == i


def test_batch_error_word_and_empty():
    s = b.make_sector(10, 2, 5, 2)
    bad = torch.tensor([0, s.dim, 5], device=DEV, dtype=torch.int64)
    out = s.state_at_batch(bad)
    torch.cuda.synchronize()
    assert out[1].item() == -1 and out[0].item() == s.state_at(0)
    with pytest.raises(b.DQError) as e:
        s.check_device()
    assert e.value.code == b.DQ_EDEVICE
    s.check_device()  # cleared
    words = torch.tensor([s.state_at(3), 0, (1 << 10) | 0b11111], device=DEV, dtype=torch.int64)
    out = s.index_of_batch(words)
    torch.cuda.synchronize()
    assert out.tolist()[0] == 3 and out.tolist()[1] == -1 and out.tolist()[2] == -1
    with pytest.raises(b.DQError):
        s.check_device()
    empty = torch.empty(0, device=DEV, dtype=torch.int64)
    assert s.state_at_batch(empty).numel() == 0


# ---------------------------------------------------------------- matvec ---------------------

def random_terms(rng, L, Q, nbonds, disorder=True):
    if Q == 2:
        kinds_pair, kinds_site = ["XY", "ZZ", "HOP", "NN"], ["Z", "N"]
    else:
        kinds_pair, kinds_site = ["HOP", "NN"], ["N", "U"]
    terms = []
    for _ in range(nbonds):
        i, j = rng.choice(L, size=2, replace=False)
        for k in kinds_pair:
            if rng.random() < 0.7:
                terms.append((k, int(i), int(j), float(rng.uniform(-1.5, 1.5)) if disorder else 1.0))
    for i in range(L):
        for k in kinds_site:
            if rng.random() < 0.5:
                terms.append((k, i, -1, float(rng.uniform(-2, 2))))
    return terms


SMALL = [(12, 2, 6, 2), (12, 2, 5, 3), (13, 2, 6, 13), (12, 2, 6, 1), (10, 3, 9, 2), (8, 4, 11, 3), (9, 3, 7, 9),
         (7, 5, 12, 2), (6, 16, 30, 2), (16, 2, 8, 4), (11, 2, 0, 2), (11, 2, 11, 3), (5, 4, 15, 2), (14, 2, 1, 5),
         (64, 2, 2, 4), (64, 2, 3, 3), (32, 4, 3, 3)]  # the last three: words of all 64 bits


@pytest.mark.parametrize("L,Q,N,n_sub", SMALL)
def test_matvec_small_random_operators_fp64(L, Q, N, n_sub):
    rng = np.random.default_rng(31 * L + 7 * Q + N + n_sub)
    terms = random_terms(rng, L, Q, 2 * L)
    s = b.make_sector(L, Q, N, n_sub)
    o = oracle_sector(L, Q, N, s.partition)
    x = rng.uniform(-1, 1, o.dim)
    ref = o_matvec(o, terms, x)
    y = gpu_matvec(s, terms, x)
    if np.max(np.abs(ref)) == 0:
        assert np.max(np.abs(y)) == 0
    else:
        assert maxrel(y, ref) <= TOL64


@pytest.mark.parametrize("nrhs", [2, 3, 8, 11])
def test_matvec_multi_rhs(nrhs):
    rng = np.random.default_rng(nrhs)
    terms = random_terms(rng, 14, 2, 20)
    s = b.make_sector(14, 2, 7, 2)
    o = oracle_sector(14, 2, 7, s.partition)
    X = rng.uniform(-1, 1, (o.dim, nrhs))
    ref = o_matvec(o, terms, X)
    Y = gpu_matvec(s, terms, X)
    assert maxrel(Y, ref) <= TOL64
    Y32 = gpu_matvec(s, terms, X.astype(np.float32), torch.float32)
    ref32 = o_matvec(o, terms, X.astype(np.float32).astype(np.float64))
    assert rel2(Y32, ref32) <= TOL32


def _workload(number, n_sub=None):
    w, _ = wl.workload(number, n_sub=n_sub, draw_vector=False)
    s = b.make_sector(w.L, w.Q, w.N, w.n_sub)
    w, x = wl.workload(number, n_sub=n_sub, D=s.dim)
    return w, s, x


@pytest.mark.parametrize("number", [1, 3, 5])
def test_matvec_workloads_full_fp64_and_fp32(number):
    w, s, x = _workload(number)
    o = oracle_sector(w.L, w.Q, w.N, s.partition)
    ref = o_matvec(o, w.terms, x)
    y = gpu_matvec(s, w.terms, x)
    assert maxrel(y, ref) <= TOL64
    x32 = x.astype(np.float32)
    ref32 = o_matvec(o, w.terms, x32.astype(np.float64))
    y32 = gpu_matvec(s, w.terms, x32, torch.float32)
    assert rel2(y32, ref32) <= TOL32


@pytest.mark.slow
@pytest.mark.parametrize("n_sub", [2, 3, 5])
def test_matvec_j1j2_full_size_sampled_rows(n_sub):
    """155,117,520-dimensional sector, in the launch configuration the bench times: the GPU y
    against oracle rows (gather reading) on the first and last 4096 rows and 2^16 random rows,
    with FP64 and FP32 vectors (the FP32 product against the oracle applied to the rounded x),
    plus Hermiticity <u, H v> = <H u, v> over the whole vector."""
    w, s, x = _workload(2, n_sub=n_sub)
    o = OracleSector(w.L, w.Q, w.N, partition=s.partition)  # not cached: 2.5 GB per partition
    rng = np.random.default_rng(2)
    rows = np.concatenate([np.arange(4096), rng.choice(s.dim, 1 << 16, replace=False), np.arange(s.dim - 4096, s.dim)])
    ref = o_matvec_rows(o, w.terms, x, rows)
    x32 = x.astype(np.float32)
    ref32 = o_matvec_rows(o, w.terms, x32, rows)
    del o
    xt = torch.from_numpy(x).to(DEV)
    t = b.make_terms(s, w.terms)
    y = b.matvec(s, t, xt)
    torch.cuda.synchronize()
    s.check_device()
    rows_d = torch.from_numpy(rows).to(DEV)
    got = y[rows_d].cpu().numpy()
    assert maxrel(got, ref) <= TOL64
    y32 = b.matvec(s, t, torch.from_numpy(x32).to(DEV))
    s.check_device()
    assert rel2(y32[rows_d].double().cpu().numpy(), ref32) <= TOL32
    del y32
    g = torch.Generator(device="cpu").manual_seed(7)
    u = (torch.rand(s.dim, generator=g, dtype=torch.float64) * 2 - 1).to(DEV)
    Hu = b.matvec(s, t, u)
    lhs, rhs = torch.dot(u, y).item(), torch.dot(Hu, xt).item()
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1.0)


def test_degenerate_sectors():
    for L, Q, N, n_sub in [(8, 2, 0, 2), (8, 2, 8, 2), (5, 4, 15, 2), (1, 2, 1, 1), (2, 3, 2, 2)]:
        s = b.make_sector(L, Q, N, n_sub)
        o = oracle_sector(L, Q, N, s.partition)
        terms = [("HOP", 0, L - 1, 0.7), ("N", 0, -1, 1.5)] if L > 1 else [("N", 0, -1, 1.5)]
        if Q == 2 and L > 1:
            terms += [("XY", 0, 1, 1.0), ("ZZ", 0, 1, 0.5), ("Z", 1, -1, 0.25)]
        x = np.linspace(-1, 1, o.dim) + 0.5
        ref = o_matvec(o, terms, x)
        y = gpu_matvec(s, terms, x)
        assert np.allclose(y, ref, rtol=0, atol=1e-13 * max(1.0, np.max(np.abs(ref))))


# ---------------------------------------------------------------- Lanczos --------------------

def test_lanczos_heisenberg_ring_L4():
    s = b.make_sector(4, 2, 2, 2)
    t = b.make_terms(s, wl.heisenberg_terms(wl.chain_bonds(4), 1.0))
    v0 = torch.tensor([0.3, -0.2, 0.5, 0.1, 0.7, -0.4], device=DEV, dtype=torch.float64)
    res = b.lanczos(s, t, v0, 10)
    assert res["E0"] == pytest.approx(-2.0, abs=1e-12)
    assert res["steps_done"] <= 6


def test_lanczos_workload1_vs_oracle():
    w, s, x = _workload(1)
    o = oracle_sector(w.L, w.Q, w.N, s.partition)
    ref = o_lanczos(lambda v: o_matvec(o, w.terms, v), x, 100)
    t = b.make_terms(s, w.terms)
    res = b.lanczos(s, t, torch.from_numpy(x).to(DEV), 100)
    assert abs(res["E0"] - ref["E0"]) <= 1e-10 * abs(ref["E0"])
    np.testing.assert_allclose(res["alpha"][:20], ref["alpha"][:20], rtol=1e-9, atol=1e-9)
    res32 = b.lanczos(s, t, torch.from_numpy(x).to(DEV, torch.float32), 100)
    assert abs(res32["E0"] - ref["E0"]) <= 1e-6 * abs(ref["E0"])


def test_lanczos_free_fermions_disordered():
    L, N = 20, 9
    rng = np.random.default_rng(99)
    J = rng.uniform(0.5, 1.5, L)
    h = rng.uniform(-1, 1, L)
    terms = wl.heisenberg_terms(wl.chain_bonds(L), J, 0.0) + wl.field_terms(h)
    hsp = np.diag(h)
    for bnd, (i, j) in enumerate(wl.chain_bonds(L)):
        sg = (-1.0) ** (N - 1) if bnd == L - 1 else 1.0
        hsp[i, j] += sg * J[bnd] / 2
        hsp[j, i] += sg * J[bnd] / 2
    exact = np.sort(np.linalg.eigvalsh(hsp))[:N].sum() - 0.5 * h.sum()
    s = b.make_sector(L, 2, N, 3)
    t = b.make_terms(s, terms)
    v0 = torch.from_numpy(rng.uniform(-1, 1, s.dim)).to(DEV)
    res = b.lanczos(s, t, v0, 200)
    assert abs(res["E0"] - exact) <= 1e-10 * abs(exact)
