"""The panel product with P_1 = the last two subsystems (Q = 2, three or more subsystems whose last
one is shorter than 8 or longer than 10 sites, the two together at most 15 sites; uniform
couplings) against the oracle: FP64 (max-relative 1e-12) and FP32 vectors (relative L2 1e-5
against the oracle applied to the rounded x), on chains with three to six subsystems, extreme
particle numbers, the 6x5 lattice with four and five subsystems, and a non-finite input (workload
2 with five subsystems at full size is in the full-size parity test).
"""

import numpy as np
import pytest
import torch

from oracle import OracleSector, matvec as o_matvec
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
    s.check_device()
    if np.linalg.norm(ref32) > 0:
        assert np.linalg.norm(y32 - ref32) <= 1e-5 * np.linalg.norm(ref32)


def j1j2_chain_terms(L, J1=1.0, J2=0.5, delta=1.0):
    nn = wl.chain_bonds(L)
    nnn = [(i, (i + 2) % L) for i in range(L)]
    return wl.heisenberg_terms(nn, J1, delta) + wl.heisenberg_terms(nnn, J2, delta)


# (L, N, n_sub): partitions (6,6,6), (7,7,7), (6,6,6,6), (6,6,5,5), (4,4,4,4,4), (4,4,4,4,4,4),
# (5,5,4): tails of 12, 14, 12, 10, 8, 8 and 9 sites
CASES = [(18, 9, 3), (21, 10, 3), (24, 12, 4), (24, 1, 4), (24, 23, 4), (24, 0, 4), (24, 24, 4), (22, 11, 4),
         (20, 10, 5), (24, 7, 6), (14, 7, 3)]


@pytest.mark.parametrize("L,N,n_sub", CASES)
def test_chains(L, N, n_sub):
    rng = np.random.default_rng(L * 41 + N * 5 + n_sub)
    terms = j1j2_chain_terms(L) + [("Z", i, -1, 0.25) for i in range(L)]  # a uniform field
    s = b.make_sector(L, 2, N, n_sub)
    t = b.make_terms(s, terms)
    assert t.path == "panel", s.partition
    o = OracleSector(L, 2, N, partition=s.partition)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))


@pytest.mark.parametrize("N,n_sub,delta", [(7, 5, 1.0), (6, 5, 0.75), (7, 4, 1.0)])
def test_j1j2_lattice_tail(N, n_sub, delta):
    """The 6x5 J1-J2 lattice of workload 2 at smaller particle numbers (D = 2,035,800 and
    593,775): five subsystems of six sites (a tail of 12 sites, panels of at most 924 rows) and
    four subsystems (8,8,7,7: a tail of 14 sites); delta != 1 gives different XY and ZZ
    classes."""
    nn, nnn = wl.square_bonds(6, 5)
    terms = wl.heisenberg_terms(nn, 1.0, delta) + wl.heisenberg_terms(nnn, 0.5, delta)
    s = b.make_sector(30, 2, N, n_sub)
    t = b.make_terms(s, terms)
    assert t.path == "panel"
    o = OracleSector(30, 2, N, partition=s.partition)
    rng = np.random.default_rng(N * 10 + n_sub)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))


def test_nonfinite_input_gives_nan_and_error_word():
    terms = j1j2_chain_terms(24)
    s = b.make_sector(24, 2, 12, 4)
    t = b.make_terms(s, terms)
    assert t.path == "panel"
    x = torch.rand(s.dim, dtype=torch.float64, device=DEV)
    x[77] = float("nan")
    y = b.matvec(s, t, x)
    torch.cuda.synchronize()
    assert torch.isnan(y).all()
    with pytest.raises(b.DQError) as e:
        s.check_device()
    assert e.value.code == b.DQ_EDEVICE
    s.check_device()


def test_wide_tail_and_disorder_take_the_general_kernel():
    """A tail of more than 15 sites (three subsystems of 11: the last two hold 22) and per-bond
    couplings with three or more subsystems stay on the general kernel."""
    s = b.make_sector(33, 2, 3, 3)
    assert s.partition == [11, 11, 11]
    t = b.make_terms(s, j1j2_chain_terms(33))
    assert t.path == "general"
    o = OracleSector(33, 2, 3, partition=s.partition)
    check(s, t, j1j2_chain_terms(33), o, np.random.default_rng(2).uniform(-1, 1, o.dim))
    rng = np.random.default_rng(8)
    terms = wl.heisenberg_terms(wl.chain_bonds(18), rng.uniform(0.5, 1.5, 18))
    s2 = b.make_sector(18, 2, 9, 3)
    t2 = b.make_terms(s2, terms)
    assert t2.path == "general"
    o = OracleSector(18, 2, 9, partition=s2.partition)
    check(s2, t2, terms, o, rng.uniform(-1, 1, o.dim))
