"""The warp-panel product (Q = 2, three or more subsystems, the last of 8 to 10 sites; uniform
couplings of at most two hop amplitudes and four Sz Sz coefficients) against the oracle: FP64
(max-relative 1e-12) and FP32 vectors (relative L2 1e-5 against the oracle applied to the
rounded x), on chains and the 6x5 lattice with three and four subsystems, extreme particle
numbers, a non-finite input, and workload 2 with three subsystems at full size on sampled rows.
"""

import numpy as np
import pytest
import torch

from oracle import OracleSector, matvec as o_matvec, matvec_rows as o_matvec_rows
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


def check(s, t, terms, o, x):
    ref = o_matvec(o, terms, x)
    y = b.matvec(s, t, torch.from_numpy(x).to(DEV)).cpu().numpy()
    s.check_device()
    if np.max(np.abs(ref)) == 0:
        assert np.max(np.abs(y)) == 0
    else:
        assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    x32 = x.astype(np.float32)
    ref32 = o_matvec(o, terms, x32.astype(np.float64))
    y32 = b.matvec(s, t, torch.from_numpy(x32).to(DEV)).double().cpu().numpy()
    if np.linalg.norm(ref32) > 0:
        assert np.linalg.norm(y32 - ref32) <= 1e-5 * np.linalg.norm(ref32)


def j1j2_chain_terms(L, J1=1.0, J2=0.5, delta=1.0):
    nn = wl.chain_bonds(L)
    nnn = [(i, (i + 2) % L) for i in range(L)]
    return wl.heisenberg_terms(nn, J1, delta) + wl.heisenberg_terms(nnn, J2, delta)


@pytest.mark.parametrize("L,N,n_sub", [(24, 12, 3), (24, 9, 3), (24, 1, 3), (24, 23, 3), (24, 0, 3), (24, 24, 3),
                                       (27, 6, 3), (30, 4, 3), (32, 3, 4), (32, 29, 4)])
def test_chains(L, N, n_sub):
    rng = np.random.default_rng(L * 37 + N * 3 + n_sub)
    terms = j1j2_chain_terms(L) + [("Z", i, -1, 0.3) for i in range(L)]  # a uniform field
    s = b.make_sector(L, 2, N, n_sub)
    t = b.make_terms(s, terms)
    assert t.path == "panel_w", s.partition
    o = OracleSector(L, 2, N, partition=s.partition)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))


@pytest.mark.parametrize("N,delta", [(7, 1.0), (6, 0.75)])
def test_j1j2_lattice_three_subsystems(N, delta):
    """The 6x5 J1-J2 lattice of workload 2 at smaller particle numbers (D = 2,035,800 and
    593,775), three subsystems of ten sites; delta != 1 gives different XY and ZZ classes (the
    panel kernels take dyadic coefficients only)."""
    nn, nnn = wl.square_bonds(6, 5)
    terms = wl.heisenberg_terms(nn, 1.0, delta) + wl.heisenberg_terms(nnn, 0.5, delta)
    s = b.make_sector(30, 2, N, 3)
    t = b.make_terms(s, terms)
    assert t.path == "panel_w"
    o = OracleSector(30, 2, N, partition=s.partition)
    rng = np.random.default_rng(N)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))


def test_nonfinite_input_gives_nan_and_error_word():
    terms = j1j2_chain_terms(24)
    s = b.make_sector(24, 2, 12, 3)
    t = b.make_terms(s, terms)
    assert t.path == "panel_w"
    x = torch.rand(s.dim, dtype=torch.float64, device=DEV)
    x[123] = float("inf")
    y = b.matvec(s, t, x)
    torch.cuda.synchronize()
    assert torch.isnan(y).all()
    with pytest.raises(b.DQError) as e:
        s.check_device()
    assert e.value.code == b.DQ_EDEVICE
    s.check_device()


def test_disorder_and_wide_last_subsystem_take_other_kernels():
    """Per-bond couplings (more classes than the panel kernels hold) and a last subsystem outside
    8..10 sites leave the warp-panel kernel; the disordered product still matches the oracle."""
    rng = np.random.default_rng(4)
    L, N = 24, 10
    terms = wl.heisenberg_terms(wl.chain_bonds(L), rng.uniform(0.5, 1.5, L))
    s = b.make_sector(L, 2, N, 3)
    t = b.make_terms(s, terms)
    assert t.path == "general"
    o = OracleSector(L, 2, N, partition=s.partition)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))
    s5 = b.make_sector(30, 2, 5, 5)  # subsystems of six sites: the panel kernel with a tail of two
    t5 = b.make_terms(s5, j1j2_chain_terms(30))
    assert t5.path == "panel"


@pytest.mark.slow
def test_workload2_three_subsystems_full_size_sampled_rows():
    """Workload 2 (D = 155,117,520) with three subsystems on the warp-panel kernel: oracle rows on
    the first and last 4096 rows and 2^16 random rows, FP64 and FP32."""
    w, _ = wl.workload(2, n_sub=3, draw_vector=False)
    s = b.make_sector(w.L, w.Q, w.N, w.n_sub)
    w, x = wl.workload(2, n_sub=3, D=s.dim)
    t = b.make_terms(s, w.terms)
    assert t.path == "panel_w"
    o = OracleSector(w.L, w.Q, w.N, partition=s.partition)
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([np.arange(4096), rng.choice(s.dim, 1 << 16, replace=False),
                                     np.arange(s.dim - 4096, s.dim)]))
    ref = o_matvec_rows(o, w.terms, x, rows)
    x32 = x.astype(np.float32)
    ref32 = o_matvec_rows(o, w.terms, x32, rows)
    del o
    rows_d = torch.from_numpy(rows).to(DEV)
    y = b.matvec(s, t, torch.from_numpy(x).to(DEV))
    s.check_device()
    got = y[rows_d].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    del y
    y32 = b.matvec(s, t, torch.from_numpy(x32).to(DEV))
    s.check_device()
    g32 = y32[rows_d].double().cpu().numpy()
    assert np.linalg.norm(g32 - ref32) <= 1e-5 * np.linalg.norm(ref32)
