"""The boson panel product (Q > 2, two subsystems; site functions and hops with any coefficient per
site and per bond) against the oracle: FP64 (max-relative 1e-12) and FP32 vectors (relative L2
1e-5 against the oracle applied to the rounded x), on Bose-Hubbard chains and a ladder with Q = 3,
4, 5 and 8, disordered hops and fields, extreme particle numbers (empty, one particle, full), a
non-finite input, bit-for-bit agreement with the general kernel on FP64 vectors, and the
operators it leaves to the general kernel (n_i n_j pairs, more than two subsystems). Workload 3 at
full size is in the full-size parity test.
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
    return y


def bose_terms(rng, bonds, L, t=None, U=(2.0, 6.0), mu=None):
    tb = np.ones(len(bonds)) if t is None else t
    terms = [("HOP", int(i), int(j), float(c)) for (i, j), c in zip(bonds, tb)]
    terms += [("U", i, -1, float(u)) for i, u in enumerate(rng.uniform(U[0], U[1], L))]
    if mu is not None:
        terms += [("N", i, -1, float(m)) for i, m in enumerate(rng.uniform(-mu, mu, L))]
    return terms


@pytest.mark.parametrize("L,Q,N", [(14, 4, 14), (12, 4, 12), (10, 4, 7), (9, 4, 20), (12, 3, 12), (10, 3, 5),
                                   (8, 8, 10), (8, 8, 3), (10, 4, 0), (10, 4, 1), (10, 4, 30), (7, 5, 9)])
def test_bose_hubbard_chains(L, Q, N):
    rng = np.random.default_rng(L * 100 + Q * 10 + N)
    terms = bose_terms(rng, wl.chain_bonds(L), L, mu=1.0)
    s = b.make_sector(L, Q, N, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_q", (s.partition, s.dim)
    o = OracleSector(L, Q, N, partition=s.partition)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))


def test_disordered_hops_on_a_ladder():
    """A 2 x 6 ladder (legs and rungs, open ends) with a hop amplitude per bond, Q = 4, N = 9."""
    rng = np.random.default_rng(21)
    L = 12
    bonds = [(i, i + 1) for i in range(5)] + [(6 + i, 7 + i) for i in range(5)] + [(i, 6 + i) for i in range(6)]
    terms = bose_terms(rng, bonds, L, t=rng.uniform(0.3, 1.7, len(bonds)), mu=2.0)
    s = b.make_sector(L, 4, 9, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_q"
    o = OracleSector(L, 4, 9, partition=s.partition)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))


def test_bitwise_equal_to_the_general_kernel():
    """The panel kernel uses the general kernel's integer coefficients and sums exactly, so on
    FP64 vectors it returns the general kernel's y bit for bit (the general kernel runs for two
    right-hand sides, here two copies of x)."""
    rng = np.random.default_rng(5)
    L = 14
    terms = bose_terms(rng, wl.chain_bonds(L), L, t=rng.uniform(0.5, 1.5, L), mu=1.0)
    s = b.make_sector(L, 4, L, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_q"
    x = torch.from_numpy(rng.uniform(-1, 1, s.dim)).to(DEV)
    y1 = b.matvec(s, t, x)
    y2 = b.matvec(s, t, torch.stack([x, x], dim=1).contiguous())
    s.check_device()
    assert torch.equal(y1, y2[:, 0]) and torch.equal(y1, y2[:, 1])


def test_nonfinite_input_gives_nan_and_error_word():
    rng = np.random.default_rng(9)
    terms = bose_terms(rng, wl.chain_bonds(12), 12)
    s = b.make_sector(12, 4, 12, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_q"
    x = torch.rand(s.dim, dtype=torch.float64, device=DEV)
    x[1234] = float("inf")
    y = b.matvec(s, t, x)
    torch.cuda.synchronize()
    assert torch.isnan(y).all()
    with pytest.raises(b.DQError) as e:
        s.check_device()
    assert e.value.code == b.DQ_EDEVICE
    s.check_device()


def test_pairs_and_three_subsystems_take_the_general_kernel():
    rng = np.random.default_rng(3)
    L = 10
    terms = bose_terms(rng, wl.chain_bonds(L), L) + [("NN", i, (i + 1) % L, 0.7) for i in range(L)]
    s = b.make_sector(L, 4, 10, 2)
    t = b.make_terms(s, terms)
    assert t.path == "general"
    o = OracleSector(L, 4, 10, partition=s.partition)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))
    s3 = b.make_sector(12, 4, 12, 3)
    assert b.make_terms(s3, bose_terms(rng, wl.chain_bonds(12), 12)).path == "general"
