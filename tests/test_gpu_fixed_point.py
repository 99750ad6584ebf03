"""The exact fixed-point FP64 path of the general product (GPU only).

FP64 vectors with a Q = 2 operator are scaled per column to 57-bit integers and summed in 128-bit
integers; these tests check what that design must get right beyond the parity tests: columns of
very different magnitude keep their full relative accuracy, coefficients spanning many orders of
magnitude stay within the norm-wise bound, and an Inf or NaN gives NaN output and the error word.
"""

import numpy as np
import pytest
import torch

from oracle import OracleSector, matvec as o_matvec
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


def xxz_terms(L, rng, field=3.0):
    J = rng.uniform(0.5, 1.5, L)
    h = rng.uniform(-field, field, L)
    return wl.heisenberg_terms(wl.chain_bonds(L), J, 1.0) + wl.field_terms(h)


@pytest.mark.parametrize("n_sub", [1, 3])
def test_columns_of_very_different_scale(n_sub):
    """Each column has its own scale: a column 1e-200 times another is as accurate as it."""
    rng = np.random.default_rng(7)
    L, N = 14, 7
    terms = xxz_terms(L, rng)
    s = b.make_sector(L, 2, N, n_sub)
    t = b.make_terms(s, terms)
    assert t.path == "general"
    o = OracleSector(L, 2, N, partition=s.partition)
    scales = np.array([1e-200, 1.0, 1e150, 3e-5, -2.0])
    x = rng.uniform(-1, 1, (o.dim, len(scales))) * scales
    ref = o_matvec(o, terms, x)
    y = b.matvec(s, t, torch.from_numpy(x).to(DEV)).cpu().numpy()
    s.check_device()
    for c in range(len(scales)):
        assert np.max(np.abs(y[:, c] - ref[:, c])) <= 1e-13 * np.max(np.abs(ref[:, c])), c


@pytest.mark.parametrize("n_sub,path", [(2, "panel_pb"), (3, "general")])
def test_coefficients_over_sixteen_decades(n_sub, path):
    """Coefficients from 1e-8 to 1e8 share one power-of-two grid; the error stays norm-wise tiny
    (the per-bond panel kernel and the general kernel)."""
    rng = np.random.default_rng(11)
    L, N = 13, 6
    J = 10.0 ** rng.uniform(-8, 8, L)
    h = 10.0 ** rng.uniform(-8, 8, L) * rng.choice([-1, 1], L)
    terms = wl.heisenberg_terms(wl.chain_bonds(L), J, 0.7) + wl.field_terms(h)
    s = b.make_sector(L, 2, N, n_sub)
    t = b.make_terms(s, terms)
    assert t.path == path
    o = OracleSector(L, 2, N, partition=s.partition)
    x = rng.uniform(-1, 1, o.dim)
    ref = o_matvec(o, terms, x)
    y = b.matvec(s, t, torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_general_nonfinite_input_gives_nan_and_error_word():
    rng = np.random.default_rng(3)
    s = b.make_sector(12, 2, 6, 3)
    t = b.make_terms(s, xxz_terms(12, rng))
    assert t.path == "general"
    x = torch.rand(s.dim, 2, dtype=torch.float64, device=DEV)
    b.matvec(s, t, x)
    s.check_device()
    x[17, 1] = float("inf")
    y = b.matvec(s, t, x)
    torch.cuda.synchronize()
    assert torch.isnan(y).all()
    with pytest.raises(b.DQError) as e:
        s.check_device()
    assert e.value.code == b.DQ_EDEVICE
    s.check_device()


@pytest.mark.parametrize("path", ["panel", "panel_w", "panel_pb", "general"])
def test_graded_column_elementwise_bound(path):
    """One column whose entries span twenty decades (|x_i| = 10^-20u, u ~ U[0, 1], random signs):
    every y_i meets the element-wise bound of the block fixed-point FP64 form,
        |y_i - y_ref,i| <= 2^-52 |y_ref,i| + 2^-50 max_j|x_j| (sum_j |h_ij| + n_i max|h|),
    n_i the nonzeros of row i, i.e. the error is absolute in units of the column maximum, not
    relative to |y_i|. The element-wise relative errors are printed for the record."""
    rng = np.random.default_rng(17)
    L, N = (16, 4) if path == "panel_w" else (14, 7)  # D = 1820 or 3432: a dense H for the bound
    if path in ("panel", "panel_w"):
        terms = wl.heisenberg_terms(wl.chain_bonds(L), 1.0, 1.0) + wl.field_terms(np.full(L, 0.375))
        n_sub = 2
    else:
        terms = xxz_terms(L, rng)
        n_sub = 2 if path == "panel_pb" else 3
    s = b.make_sector(L, 2, N, n_sub)
    t = b.make_terms(s, terms)
    assert t.path == path
    o = OracleSector(L, 2, N, partition=s.partition)
    H = o_matvec(o, terms, np.eye(o.dim))
    x = 10.0 ** (-20.0 * rng.uniform(0, 1, o.dim)) * rng.choice([-1.0, 1.0], o.dim)
    x[rng.integers(o.dim)] = 1.0
    ref = o_matvec(o, terms, x)
    y = b.matvec(s, t, torch.from_numpy(x).to(DEV)).cpu().numpy()
    s.check_device()
    absH = np.abs(H)
    bound = 2.0 ** -52 * np.abs(ref) + 2.0 ** -50 * np.max(np.abs(x)) * (
        absH.sum(axis=1) + (absH > 0).sum(axis=1) * absH.max())
    err = np.abs(y - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    rel = err / np.maximum(np.abs(ref), 1e-300)
    big = np.abs(ref) >= 1e-3 * np.max(np.abs(ref))
    print(f"{path}: element-wise relative error: median {np.median(rel):.1e}, max {rel.max():.1e}; "
          f"over |y_i| >= 1e-3 max|y|: max {rel[big].max():.1e}; smallest |y_i| {np.abs(ref).min():.1e}")
    assert rel[big].max() <= 1e-11
