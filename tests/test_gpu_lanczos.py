"""Lanczos through the C-ABI (GPU only): E0 against the oracle and dense diagonalisation on small
sectors, FP32 vectors against FP64 vectors on the full-size workloads, and the residual
||H psi - E0 psi|| / |E0| of the Ritz vector the call returns; each for the FP64 passes over the
basis and for their double-single form (``double_single``).

Bars: E0 within 1e-10 relative (FP64 vectors) or 1e-6 (FP32 vectors, FP64 recurrence) of the
reference; on full-size sectors, where no dense reference exists, FP32 E0 within 1e-6 of FP64 E0.
"""

import numpy as np
import pytest
import torch

from oracle import OracleSector, lanczos as o_lanczos, matvec as o_matvec
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


def bose_hubbard_terms(L, U, t=1.0):
    return [("HOP", i, j, t) for i, j in wl.chain_bonds(L)] + [("U", i, -1, float(U[i])) for i in range(L)]


def residual(s, t, res):
    """||H psi - E0 psi|| / |E0| in FP64 for the Ritz vector returned with E0."""
    psi = res["psi"]
    hpsi = b.matvec(s, t, psi).double()
    r = torch.linalg.norm(hpsi - res["E0"] * psi.double()).item()
    return r / abs(res["E0"]), torch.linalg.norm(psi.double()).item()


def _workload(number):
    w, _ = wl.workload(number, draw_vector=False)
    s = b.make_sector(w.L, w.Q, w.N, w.n_sub)
    w, x = wl.workload(number, D=s.dim)
    return w, s, x


@pytest.mark.parametrize("ds", [False, True])
def test_bose_hubbard_small_sector_vs_oracle_and_dense(ds):
    """Q = 4 Bose-Hubbard ring, L = 8, N = 8 (D = 3823), U_i ~ U[2, 6]: the GPU Lanczos with full
    re-orthogonalisation against the smallest eigenvalue of the oracle-built dense H (and the
    oracle's own Lanczos), for FP64 and FP32 vectors; the Ritz vector's residual."""
    L, Q, N = 8, 4, 8
    rng = np.random.default_rng(20240719 + 3)
    x0 = rng.uniform(-1, 1, 3823)
    U = rng.uniform(2.0, 6.0, L)
    terms = bose_hubbard_terms(L, U)
    s = b.make_sector(L, Q, N, 2)
    o = OracleSector(L, Q, N, partition=s.partition)
    assert o.dim == s.dim == 3823
    H = o_matvec(o, terms, np.eye(o.dim))
    ev = float(np.linalg.eigvalsh(H)[0])
    ref = o_lanczos(lambda v: o_matvec(o, terms, v), x0, 150)
    assert abs(ref["E0"] - ev) <= 1e-10 * abs(ev)
    t = b.make_terms(s, terms)
    for dtype, tol, rtol in ((torch.float64, 1e-10, 1e-8), (torch.float32, 1e-6, 1e-5)):
        res = b.lanczos(s, t, torch.from_numpy(x0).to(DEV, dtype), 150, reorth=True, want_vector=True,
                        double_single=ds)
        assert res["steps_done"] == 150
        assert abs(res["E0"] - ref["E0"]) <= tol * abs(ref["E0"]), dtype
        r, nrm = residual(s, t, res)
        assert abs(nrm - 1.0) <= 1e-6 and r <= rtol, (dtype, r)
    # the first coefficients follow the oracle's recurrence
    res = b.lanczos(s, t, torch.from_numpy(x0).to(DEV), 30, reorth=True, double_single=ds)
    np.testing.assert_allclose(res["alpha"], ref["alpha"][:30], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(res["beta"][:29], ref["beta"][:29], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("ds", [False, True])
def test_plain_recurrence_and_reorth_agree_on_workload1(ds):
    """Workload 1 (L = 20 ring, N = 10): the plain three-term recurrence and full
    re-orthogonalisation give the oracle's E0 (stored golden value) and a small residual."""
    from conftest import read_golden

    rows = dict((r[0], r[1:]) for r in read_golden("lanczos_workload1.txt"))
    e_ref = float(rows["E0"][0])
    w, s, x = _workload(1)
    t = b.make_terms(s, w.terms)
    for reorth in (2, 1, 0):
        res = b.lanczos(s, t, torch.from_numpy(x).to(DEV), 100, reorth=reorth, want_vector=True, double_single=ds)
        assert abs(res["E0"] - e_ref) <= 1e-10 * abs(e_ref), reorth
        r, _ = residual(s, t, res)
        assert r <= 1e-7, (reorth, r)


@pytest.mark.parametrize("ds", [False, True])
def test_breakdown_stops_early_with_exact_e0(ds):
    """A sector smaller than the step count: the recurrence meets an invariant subspace and stops
    without error, and E0 is the exact smallest eigenvalue (dense oracle H)."""
    L, Q, N = 6, 3, 5
    rng = np.random.default_rng(5)
    terms = [("HOP", i, j, float(rng.uniform(0.5, 1.5))) for i, j in wl.chain_bonds(L)] + \
            [("U", i, -1, float(rng.uniform(1, 3))) for i in range(L)]
    s = b.make_sector(L, Q, N, 2)
    o = OracleSector(L, Q, N, partition=s.partition)
    ev = float(np.linalg.eigvalsh(o_matvec(o, terms, np.eye(o.dim)))[0])
    t = b.make_terms(s, terms)
    res = b.lanczos(s, t, torch.from_numpy(rng.uniform(-1, 1, s.dim)).to(DEV), 4 * s.dim, reorth=True,
                    want_vector=True, double_single=ds)
    assert res["steps_done"] <= s.dim
    assert abs(res["E0"] - ev) <= 1e-10 * abs(ev)
    assert residual(s, t, res)[0] <= 1e-9


@pytest.mark.slow
def test_workload3_full_size_fp32_vectors_match_fp64():
    """Workload 3 (Bose-Hubbard Q = 4, L = 14, N = 14, D = 6,472,168) with full
    re-orthogonalisation, 100 steps from the seeded start vector: FP32 vectors with the FP64
    recurrence give E0 within 1e-6 of FP64 vectors, the double-single passes within 1e-10 (FP64
    vectors) and 1e-6 (FP32 vectors); the FP64 Ritz vector's residual is small."""
    w, s, x = _workload(3)
    t = b.make_terms(s, w.terms)
    r64 = b.lanczos(s, t, torch.from_numpy(x).to(DEV), 100, reorth=True, want_vector=True)
    res64, _ = residual(s, t, r64)
    del r64["psi"]
    assert r64["steps_done"] == 100 and res64 <= 1e-5
    for dtype, ds, tol in ((torch.float32, False, 1e-6), (torch.float64, True, 1e-10), (torch.float32, True, 1e-6)):
        r = b.lanczos(s, t, torch.from_numpy(x).to(DEV, dtype), 100, reorth=True, want_vector=True, double_single=ds)
        res, _ = residual(s, t, r)
        rel = abs(r["E0"] - r64["E0"]) / abs(r64["E0"])
        print(f"workload 3 {dtype} double_single={ds}: E0 {r['E0']:.15f} (FP64 {r64['E0']:.15f}) rel {rel:.2e} "
              f"residual {res:.2e} (FP64 {res64:.2e})")
        assert r["steps_done"] == 100
        assert rel <= tol, (dtype, ds)


@pytest.mark.slow
def test_workload2_full_size_reorth_fp32_vectors_match_fp64():
    """Workload 2 at full size (D = 155,117,520) with full re-orthogonalisation, 60 steps: FP32
    vectors with the FP64 recurrence against FP64 vectors (E0 within 1e-6), the double-single
    passes within 1e-10 (FP64 vectors) and 1e-6 (FP32 vectors), E0 below the Rayleigh quotient
    of v0, and the FP64 Ritz vector's residual below that of v0."""
    w, s, x = _workload(2)
    t = b.make_terms(s, w.terms)
    v64 = torch.from_numpy(x).to(DEV)
    hv = b.matvec(s, t, v64)
    rq = (torch.dot(v64, hv) / torch.dot(v64, v64)).item()
    r0 = (torch.linalg.norm(hv - rq * v64) / abs(rq)).item()
    del hv
    r64 = b.lanczos(s, t, v64, 60, reorth=True, want_vector=True)
    res64, _ = residual(s, t, r64)
    del r64["psi"]
    assert r64["steps_done"] == 60 and r64["E0"] < rq and res64 < r0
    for dtype, ds, tol in ((torch.float32, False, 1e-6), (torch.float64, True, 1e-10), (torch.float32, True, 1e-6)):
        r = b.lanczos(s, t, v64.to(dtype), 60, reorth=True, double_single=ds)
        rel = abs(r["E0"] - r64["E0"]) / abs(r64["E0"])
        print(f"workload 2 {dtype} double_single={ds}: E0 {r['E0']:.12f} (FP64 {r64['E0']:.12f}) rel {rel:.2e}; "
              f"FP64 residual {res64:.2e} (v0: {r0:.2e})")
        assert r["steps_done"] == 60
        assert rel <= tol, (dtype, ds)
