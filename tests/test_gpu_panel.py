"""The panel kernel (Q = 2, two subsystems; exact fixed-point sums) against the oracle (GPU only).

Covers the geometry of the 6x5 J1-J2 workload at particle numbers small enough for a full oracle
sweep, square and chain clusters with odd lengths, mixed term kinds with uniform fields, extreme
vector scales, all-zero and non-finite input, and FP32 vectors.
"""

import numpy as np
import pytest
import torch

from oracle import OracleSector, matvec as o_matvec
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


def j1j2_terms(Lx, Ly, J2=0.5, delta=1.0):
    nn, nnn = wl.square_bonds(Lx, Ly)
    return wl.heisenberg_terms(nn, 1.0, delta) + wl.heisenberg_terms(nnn, J2, delta)


def run_both(L, N, terms, n_sub=2, scale=1.0, seed=0, want_panel=True):
    s = b.make_sector(L, 2, N, n_sub)
    t = b.make_terms(s, terms)
    if want_panel:  # the class-sum panel kernel, or its warp-per-panel form for P_1 of 8-10 sites
        assert t.path == ("panel_w" if 8 <= s.partition[-1] <= 10 else "panel"), s.partition
    o = OracleSector(L, 2, N, partition=s.partition)
    x = np.random.default_rng(seed).uniform(-1, 1, o.dim) * scale
    ref = o_matvec(o, terms, x)
    y = b.matvec(s, t, torch.from_numpy(x).to(DEV)).cpu().numpy()
    torch.cuda.synchronize()
    s.check_device()
    x32 = x.astype(np.float32)
    ref32 = o_matvec(o, terms, x32.astype(np.float64))
    y32 = b.matvec(s, t, torch.from_numpy(x32).to(DEV)).double().cpu().numpy()
    return y, ref, y32, ref32


def check(y, ref, y32, ref32):
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.linalg.norm(y32 - ref32) <= 1e-5 * np.linalg.norm(ref32)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 27, 29])
def test_j1j2_6x5_geometry_small_N(N):
    check(*run_both(30, N, j1j2_terms(6, 5), seed=N))


@pytest.mark.parametrize("Lx,Ly,N", [(4, 4, 8), (4, 4, 1), (4, 4, 15), (5, 4, 10), (5, 4, 7), (6, 4, 12), (3, 3, 4)])
def test_square_clusters(Lx, Ly, N):
    check(*run_both(Lx * Ly, N, j1j2_terms(Lx, Ly, J2=0.25, delta=0.5), seed=Lx * 10 + N))


@pytest.mark.parametrize("L,N", [(17, 8), (21, 10), (19, 3), (4, 2), (2, 1), (24, 12)])
def test_chains_odd_and_tiny(L, N):
    terms = wl.heisenberg_terms(wl.chain_bonds(L), 1.0, 1.0)
    check(*run_both(L, N, terms, seed=L))


def test_mixed_kinds_uniform_field():
    L = 18
    nn = wl.chain_bonds(L)
    terms = ([("HOP", i, j, 0.5) for i, j in nn] + [("NN", i, j, 0.75) for i, j in nn] +
             [("ZZ", i, (i + 2) % L, -0.5) for i in range(L)] + [("Z", i, -1, 0.375) for i in range(L)] +
             [("N", i, -1, 0.25) for i in range(L)] + [("XY", i, (i + 3) % L, 0.5) for i in range(L)])
    check(*run_both(L, 7, terms, seed=3))


@pytest.mark.parametrize("lat", [(4, 4), (11, 2)])  # P_1 of 8 sites (warp-panel), 11 sites (panel)
@pytest.mark.parametrize("scale", [1e-200, 1e-30, 1e30, 1e200])
def test_extreme_scales(scale, lat):
    terms = j1j2_terms(*lat)
    L = lat[0] * lat[1]
    y, ref, _, _ = run_both(L, L // 2, terms, scale=scale, seed=9)
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("lat,path", [((4, 4), "panel_w"), ((11, 2), "panel")])
def test_zero_and_nonfinite_input(lat, path):
    L = lat[0] * lat[1]
    s = b.make_sector(L, 2, L // 2, 2)
    t = b.make_terms(s, j1j2_terms(*lat))
    assert t.path == path
    x = torch.zeros(s.dim, dtype=torch.float64, device=DEV)
    y = b.matvec(s, t, x)
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0
    s.check_device()
    x[5] = float("nan")
    b.matvec(s, t, x)
    with pytest.raises(b.DQError) as e:
        s.check_device()
    assert e.value.code == b.DQ_EDEVICE
    s.check_device()


def test_disorder_takes_the_per_bond_panel_kernel():
    """Per-bond couplings leave the class-sum panel kernel for the per-bond one (P_1 of at most 13
    sites); with three subsystems they take the general kernel, and uniform couplings with three
    subsystems of 6, 5 and 5 sites the panel kernel with a tail of two."""
    L = 16
    J = np.random.default_rng(1).uniform(0.5, 1.5, L)
    terms = wl.heisenberg_terms(wl.chain_bonds(L), J)
    s = b.make_sector(L, 2, 8, 2)
    assert b.make_terms(s, terms).path == "panel_pb"
    s3 = b.make_sector(L, 2, 8, 3)
    assert b.make_terms(s3, wl.heisenberg_terms(wl.chain_bonds(L), 1.0)).path == "panel"
    assert b.make_terms(s3, terms).path == "general"
    check(*run_both(L, 8, terms, seed=5, want_panel=False))
    s30 = b.make_sector(30, 2, 15, 2)  # P_1 of 15 sites: the general kernel
    assert b.make_terms(s30, wl.heisenberg_terms(wl.chain_bonds(30), np.linspace(0.5, 1.5, 30))).path == "general"


def test_repeated_calls_and_two_terms_objects():
    s = b.make_sector(20, 2, 10, 2)
    t1 = b.make_terms(s, j1j2_terms(5, 4))
    t2 = b.make_terms(s, wl.heisenberg_terms(wl.chain_bonds(20), 1.0))
    o = OracleSector(20, 2, 10, partition=s.partition)
    rng = np.random.default_rng(4)
    for _ in range(2):
        x = rng.uniform(-1, 1, o.dim)
        xt = torch.from_numpy(x).to(DEV)
        y1 = b.matvec(s, t1, xt).cpu().numpy()
        y2 = b.matvec(s, t2, xt).cpu().numpy()
        r1 = o_matvec(o, j1j2_terms(5, 4), x)
        r2 = o_matvec(o, wl.heisenberg_terms(wl.chain_bonds(20), 1.0), x)
        assert np.max(np.abs(y1 - r1)) <= 1e-12 * np.max(np.abs(r1))
        assert np.max(np.abs(y2 - r2)) <= 1e-12 * np.max(np.abs(r2))


def test_timing_hooks_count_and_time_the_main_kernel():
    """dq_timing_*: three kernels per product on the panel paths (two prepass kernels and the
    warp-panel or the per-bond panel kernel), positive times."""
    s = b.make_sector(20, 2, 10, 2)
    terms = wl.heisenberg_terms(wl.chain_bonds(20), 1.0, 1.0)
    tp = b.make_terms(s, terms)
    assert tp.path == "panel_w"
    tg = b.make_terms(s, terms + [("Z", 3, -1, 0.3)])  # a non-uniform field: the per-bond panel path
    assert tg.path == "panel_pb"
    x = torch.rand(s.dim, dtype=torch.float64, device=DEV)
    b.matvec(s, tp, x)
    torch.cuda.synchronize()
    b.timing_enable(True)
    for _ in range(3):
        b.matvec(s, tp, x)
    b.matvec(s, tg, x)
    ms, calls, kernels = b.timing_read()
    b.timing_enable(False)
    assert calls == 4 and kernels == 3 * 3 + 3
    assert ms > 0.0
    b.matvec(s, tp, x)  # timing off: nothing more is recorded
    assert b.timing_read()[1] == 4


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_products_replay_from_a_cuda_graph(dtype):
    """dq_matvec captured in a CUDA graph (after one eager call has set up its scratch) gives,
    on replay with new x, exactly what an eager call gives: the warp-panel, panel and general
    paths."""
    rng = np.random.default_rng(12)
    cases = [(b.make_sector(20, 2, 10, 2), wl.heisenberg_terms(wl.chain_bonds(20), 1.0, 1.0), "panel_w"),
             (b.make_sector(22, 2, 11, 2), wl.heisenberg_terms(wl.chain_bonds(22), 1.0, 1.0), "panel"),
             (b.make_sector(14, 2, 7, 3), wl.heisenberg_terms(wl.chain_bonds(14), rng.uniform(0.5, 1.5, 14), 1.0)
              + wl.field_terms(rng.uniform(-3, 3, 14)), "general")]
    for s, terms, path in cases:
        t = b.make_terms(s, terms)
        assert t.path == path
        x = torch.rand(s.dim, dtype=dtype, device=DEV)
        y = torch.empty_like(x)
        b.matvec(s, t, x, y)  # first call: scratch
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            b.matvec(s, t, x, y)
        for _ in range(2):
            x.copy_(torch.rand(s.dim, dtype=dtype, device=DEV) - 0.5)
            g.replay()
            torch.cuda.synchronize()
            ref = b.matvec(s, t, x)
            assert torch.equal(y, ref)
        s.check_device()
