"""The per-bond panel product (Q = 2, two subsystems, P_1 of at most 13 sites, a coefficient per
bond and per site) against the oracle, FP64 (max-relative 1e-12) and FP32 vectors (relative L2
1e-5 against the oracle applied to the rounded x): disordered chains and lattices, every term
kind, extreme particle numbers, a non-finite input and workload 5 at full size.
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
    if np.linalg.norm(ref32) > 0:
        assert np.linalg.norm(y32 - ref32) <= 1e-5 * np.linalg.norm(ref32)


def disordered_terms(rng, bonds, L, kinds=("XY", "ZZ"), fields=True):
    terms = []
    for i, j in bonds:
        for k in kinds:
            terms.append((k, int(i), int(j), float(rng.uniform(-1.5, 1.5))))
    if fields:
        terms += [("Z", i, -1, float(rng.uniform(-3, 3))) for i in range(L)]
    return terms


@pytest.mark.parametrize("L,N", [(14, 7), (15, 6), (17, 8), (20, 10), (22, 9), (26, 13), (9, 1), (12, 11)])
def test_disordered_chains(L, N):
    rng = np.random.default_rng(L * 31 + N)
    terms = disordered_terms(rng, wl.chain_bonds(L), L)
    s = b.make_sector(L, 2, N, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_pb"
    o = OracleSector(L, 2, N, partition=s.partition)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))


@pytest.mark.parametrize("Lx,Ly,N", [(4, 4, 8), (5, 4, 9), (4, 3, 5)])
def test_disordered_lattices_all_kinds(Lx, Ly, N):
    """Square lattices with NN and NNN bonds, every pair kind with its own coefficient (XY, ZZ,
    hard-core HOP, NN) and per-site Z and N fields."""
    rng = np.random.default_rng(Lx * 10 + Ly)
    nn, nnn = wl.square_bonds(Lx, Ly)
    L = Lx * Ly
    terms = disordered_terms(rng, nn + nnn, L, kinds=("XY", "ZZ", "HOP", "NN"))
    terms += [("N", i, -1, float(rng.uniform(-1, 1))) for i in range(L)]
    s = b.make_sector(L, 2, N, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_pb"
    o = OracleSector(L, 2, N, partition=s.partition)
    check(s, t, terms, o, rng.uniform(-1, 1, o.dim))


def test_hop_only_zz_only_and_empty_sectors():
    rng = np.random.default_rng(3)
    L = 16
    for kinds, fields in ((("XY",), False), (("ZZ",), True), (("HOP",), False)):
        terms = disordered_terms(rng, wl.chain_bonds(L), L, kinds=kinds, fields=fields)
        for N in (0, 1, 8, 16):
            s = b.make_sector(L, 2, N, 2)
            t = b.make_terms(s, terms)
            assert t.path == "panel_pb"
            o = OracleSector(L, 2, N, partition=s.partition)
            check(s, t, terms, o, rng.uniform(-1, 1, o.dim) + 0.25)


def test_nonfinite_input_gives_nan_and_error_word():
    rng = np.random.default_rng(9)
    terms = disordered_terms(rng, wl.chain_bonds(14), 14)
    s = b.make_sector(14, 2, 7, 2)
    t = b.make_terms(s, terms)
    assert t.path == "panel_pb"
    x = torch.rand(s.dim, dtype=torch.float64, device=DEV)
    x[11] = float("nan")
    y = b.matvec(s, t, x)
    torch.cuda.synchronize()
    assert torch.isnan(y).all()
    with pytest.raises(b.DQError) as e:
        s.check_device()
    assert e.value.code == b.DQ_EDEVICE
    s.check_device()


def test_workload5_full_size():
    """Workload 5 (disordered XXZ chain L = 24, N = 12, D = 2,704,156) on the per-bond panel
    kernel against the oracle's column form on the whole sector."""
    w, _ = wl.workload(5, draw_vector=False)
    s = b.make_sector(w.L, w.Q, w.N, w.n_sub)
    w, x = wl.workload(5, D=s.dim)
    t = b.make_terms(s, w.terms)
    assert t.path == "panel_pb"
    o = OracleSector(w.L, w.Q, w.N, partition=s.partition)
    check(s, t, w.terms, o, x)
