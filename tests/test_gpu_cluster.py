"""The cluster-merged operator of App. C (dq_make_cluster_terms) on the GPU.

Each cluster's terms are merged into one sparse matrix over its digit patterns; the product
applies one column per cluster and row. Checked against the oracle (which applies the terms one
by one) on chains, square lattices, bosons and two-word states, for FP64 (max-relative 1e-12)
and FP32 vectors (relative L2 1e-5, against the oracle on the rounded x), several right-hand
sides, and through Lanczos against the stored oracle E0 of workload 1.
"""

import numpy as np
import pytest
import torch

from conftest import read_golden
from oracle import OracleSector, matvec as o_matvec
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


def random_terms(rng, L, Q, bonds):
    kinds_pair, kinds_site = (["XY", "ZZ", "HOP", "NN"], ["Z", "N"]) if Q == 2 else (["HOP", "NN"], ["N", "U"])
    terms = []
    for i, j in bonds:
        for k in kinds_pair:
            if rng.random() < 0.8:
                terms.append((k, int(i), int(j), float(rng.uniform(-1.5, 1.5))))
    for i in range(L):
        for k in kinds_site:
            if rng.random() < 0.6:
                terms.append((k, i, -1, float(rng.uniform(-2, 2))))
    return terms


CASES = [  # (L, Q, N, n_sub, bonds, cluster sites)
    (16, 2, 8, 2, wl.chain_bonds(16), 11),
    (14, 2, 6, 3, sum(wl.square_bonds(7, 2), []), 8),
    (12, 2, 6, 4, sum(wl.square_bonds(4, 3), []), 12),
    (10, 3, 9, 2, wl.chain_bonds(10), 6),
    (8, 4, 9, 3, wl.chain_bonds(8), 5),
    (70, 2, 3, 5, wl.chain_bonds(70), 10),
    (33, 4, 3, 3, wl.chain_bonds(33), 6),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_cluster_product_vs_oracle(case):
    L, Q, N, n_sub, bonds, m = CASES[case]
    rng = np.random.default_rng(500 + case)
    terms = random_terms(rng, L, Q, bonds)
    s = b.make_sector(L, Q, N, n_sub)
    t = b.make_cluster_terms(s, terms, m)
    assert t.path == "cluster"
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


def test_cluster_form_equals_per_term_form_and_lanczos():
    """Workload 1 (L = 20 ring, N = 10) with 11-site clusters: the same product as the per-term
    operator within 1e-12, and the stored oracle Lanczos E0."""
    rows = dict((r[0], r[1:]) for r in read_golden("lanczos_workload1.txt"))
    e_ref = float(rows["E0"][0])
    w, _ = wl.workload(1, draw_vector=False)
    s = b.make_sector(w.L, w.Q, w.N, w.n_sub)
    w, x = wl.workload(1, D=s.dim)
    t = b.make_terms(s, w.terms)
    tc = b.make_cluster_terms(s, w.terms, 11)
    assert len(tc.clusters()[0]) == 2
    xt = torch.from_numpy(x).to(DEV)
    y, yc = b.matvec(s, t, xt), b.matvec(s, tc, xt)
    assert torch.max(torch.abs(y - yc)).item() <= 1e-12 * torch.max(torch.abs(y)).item()
    res = b.lanczos(s, tc, xt, 100)
    assert abs(res["E0"] - e_ref) <= 1e-10 * abs(e_ref)
