"""Differentiable product and Krylov time evolution (GPU), against references independent of the
CUDA path: per-term oracle products, dense matrices built by the oracle, scipy/torch matrix
exponentials, and central finite differences with step 1e-6."""

import numpy as np
import pytest
import scipy.linalg as sla
import torch

from oracle import OracleSector, matvec as o_matvec
from paper_2407_14591_gb300 import autograd as ag
from paper_2407_14591_gb300 import binding as b
from paper_2407_14591_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda"


def xxz_operator(sector, L, delta=1.0):
    """theta = (J_0..J_{L-1}, h_0..h_{L-1}) on a periodic chain."""
    params = []
    for bnd, (i, j) in enumerate(wl.chain_bonds(L)):
        params.append(("XY", i, j, bnd, 1.0))
        params.append(("ZZ", i, j, bnd, delta))
    for i in range(L):
        params.append(("Z", i, -1, L + i, 1.0))
    return ag.ParamOperator(sector, params, n_params=2 * L)


def theta_draw(L, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(0.5, 1.5, L), rng.uniform(-3, 3, L)])


def oracle_terms(op, theta):
    return [(k, i, j, s * theta[p]) for (k, i, j, p, s) in op.params]


def test_matvec_forward_backward_vs_oracle_and_fd():
    L, N = 12, 6
    s = b.make_sector(L, 2, N, 2)
    o = OracleSector(L, 2, N, partition=s.partition)
    op = xxz_operator(s, L)
    th = theta_draw(L, 1)
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, o.dim)
    r = rng.uniform(-1, 1, o.dim)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    xt = torch.tensor(x, device=DEV, requires_grad=True)
    y = ag.matvec(op, xt, theta)
    ref = o_matvec(o, oracle_terms(op, th), x)
    assert np.max(np.abs(y.detach().cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    loss = torch.dot(torch.tensor(r, device=DEV), y)
    loss.backward()
    # reference: dtheta_k = sum_q scale_q <r, T_q x>, each T_q applied by the oracle
    g_ref = np.zeros(2 * L)
    for (k, i, j, p, sc) in op.params:
        g_ref[p] += sc * r @ o_matvec(o, [(k, i, j, 1.0)], x)
    np.testing.assert_allclose(theta.grad.numpy(), g_ref, rtol=1e-12, atol=1e-12 * np.abs(g_ref).max())
    dx_ref = o_matvec(o, oracle_terms(op, th), r)  # H^T r = H r
    np.testing.assert_allclose(xt.grad.cpu().numpy(), dx_ref, rtol=0, atol=1e-12 * np.abs(dx_ref).max())
    # central finite differences (the loss is linear in theta, so only rounding remains)
    h = 1e-6
    for k in (0, 3, L + 2, 2 * L - 1):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        with torch.no_grad():
            lp = torch.dot(torch.tensor(r, device=DEV), ag.matvec(op, xt, torch.tensor(tp))).item()
            lm = torch.dot(torch.tensor(r, device=DEV), ag.matvec(op, xt, torch.tensor(tm))).item()
        assert (lp - lm) / (2 * h) == pytest.approx(theta.grad[k].item(), rel=1e-7, abs=1e-9)


def test_nrhs2_complex_gradient_is_real_part():
    L, N = 10, 4
    s = b.make_sector(L, 2, N, 2)
    op = xxz_operator(s, L)
    th = torch.tensor(theta_draw(L, 3))
    rng = np.random.default_rng(4)
    psi = torch.tensor(rng.uniform(-1, 1, s.dim) + 1j * rng.uniform(-1, 1, s.dim), device=DEV)
    dpsi = torch.tensor(rng.uniform(-1, 1, s.dim) + 1j * rng.uniform(-1, 1, s.dim), device=DEV)
    g2 = b.term_grads(s, [p[:3] for p in op.params], torch.view_as_real(psi), torch.view_as_real(dpsi))
    gr = b.term_grads(s, [p[:3] for p in op.params], psi.real.contiguous(), dpsi.real.contiguous())
    gi = b.term_grads(s, [p[:3] for p in op.params], psi.imag.contiguous(), dpsi.imag.contiguous())
    torch.testing.assert_close(g2, gr + gi, rtol=1e-13, atol=1e-13)


def dense_reference(o, op, th, psi0, obs_site, t):
    """psi(t) = expm(-i H t) psi0 and d<S^z_site>/dtheta with dense torch matrices built from
    the oracle's products of each term (no CUDA kernel involved)."""
    D = o.dim
    mats = []
    for (k, i, j, p, sc) in op.params:
        mats.append(o_matvec(o, [(k, i, j, 1.0)], np.eye(D)))
    Hk = torch.tensor(np.stack(mats), dtype=torch.float64)
    idx = torch.tensor([p for (_, _, _, p, _) in op.params])
    scl = torch.tensor([sc for (_, _, _, _, sc) in op.params], dtype=torch.float64)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    coefs = scl * theta[idx]
    H = torch.einsum("q,qab->ab", coefs, Hk)
    U = torch.linalg.matrix_exp(-1j * t * H.to(torch.complex128))
    psi = U @ torch.tensor(psi0, dtype=torch.complex128)
    Od = torch.tensor(np.diag(o_matvec(o, [("Z", obs_site, -1, 1.0)], np.eye(D))), dtype=torch.float64)
    val = torch.sum(Od * (psi.conj() * psi).real)
    val.backward()
    return psi.detach().numpy(), val.item(), theta.grad.numpy()


@pytest.mark.parametrize("use_checkpoint", [True, False])
def test_krylov_evolution_and_gradient_vs_dense(use_checkpoint):
    L, N, dt, steps = 10, 5, 0.1, 20
    s = b.make_sector(L, 2, N, 2)
    o = OracleSector(L, 2, N, partition=s.partition)
    op = xxz_operator(s, L)
    obs = ag.ParamOperator(s, [], fixed=[("Z", 0, -1, 1.0)])
    th = theta_draw(L, 5)
    rng = np.random.default_rng(6)
    psi0 = rng.uniform(-1, 1, o.dim) + 1j * rng.uniform(-1, 1, o.dim)
    psi0 /= np.linalg.norm(psi0)
    psi_ref, val_ref, g_ref = dense_reference(o, op, th, psi0, 0, dt * steps)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    psi = ag.evolve(op, theta, torch.tensor(psi0, device=DEV), dt, steps, m=16, use_checkpoint=use_checkpoint)
    assert np.linalg.norm(psi.detach().cpu().numpy() - psi_ref) <= 1e-10
    val = ag.expectation(obs, psi)
    assert val.item() == pytest.approx(val_ref, abs=1e-11)
    val.backward()
    np.testing.assert_allclose(theta.grad.numpy(), g_ref, rtol=1e-6, atol=1e-8)


def test_krylov_gradient_finite_differences():
    L, N, dt, steps = 10, 4, 0.1, 20
    s = b.make_sector(L, 2, N, 2)
    op = xxz_operator(s, L)
    obs = ag.ParamOperator(s, [], fixed=[("Z", 0, -1, 1.0)])
    th = theta_draw(L, 7)
    rng = np.random.default_rng(8)
    psi0 = torch.tensor(rng.uniform(-1, 1, s.dim) + 1j * rng.uniform(-1, 1, s.dim), device=DEV)
    psi0 = psi0 / torch.linalg.vector_norm(psi0)

    def f(t):
        return ag.expectation(obs, ag.evolve(op, t, psi0, dt, steps))

    theta = torch.tensor(th, requires_grad=True)
    f(theta).backward()
    h = 1e-6
    for k in (1, 4, L, L + 7):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        with torch.no_grad():
            fd = (f(torch.tensor(tp)).item() - f(torch.tensor(tm)).item()) / (2 * h)
        assert fd == pytest.approx(theta.grad[k].item(), rel=1e-5, abs=1e-7)


@pytest.mark.slow
def test_workload5_size_gradient():
    """Disordered XXZ chain L = 24, N = 12 (D = 2,704,156): forward y = H(theta) x in FP64 and
    FP32, backward, and the gradient of <psi(t)|S^z_0|psi(t)> through 20 checkpointed Krylov
    steps, checked by central finite differences on two parameters."""
    w, _ = wl.workload(5, draw_vector=False)
    s = b.make_sector(24, 2, 12, 2)
    w, x = wl.workload(5, D=s.dim)
    op = xxz_operator(s, 24)
    th = np.array([t[3] for t in w.terms if t[0] == "XY"] + [t[3] for t in w.terms if t[0] == "Z"])
    theta = torch.tensor(th, requires_grad=True)
    # the workload's own terms and the parametrised operator agree
    y_ref = b.matvec(s, b.make_terms(s, w.terms), torch.from_numpy(x).to(DEV))
    y = ag.matvec(op, torch.from_numpy(x).to(DEV), theta)
    assert torch.max(torch.abs(y - y_ref)).item() <= 1e-12 * torch.max(torch.abs(y_ref)).item()
    y32 = ag.matvec(op, torch.from_numpy(x).to(DEV, torch.float32), theta)
    assert (torch.linalg.norm(y32.double() - y_ref) / torch.linalg.norm(y_ref)).item() <= 1e-5
    obs = ag.ParamOperator(s, [], fixed=[("Z", 0, -1, 1.0)])
    rng = np.random.default_rng(9)
    psi0 = torch.tensor(x + 1j * rng.uniform(-1, 1, s.dim) / np.sqrt(s.dim), device=DEV)
    psi0 = psi0 / torch.linalg.vector_norm(psi0)

    def f(t):
        return ag.expectation(obs, ag.evolve(op, t, psi0, 0.1, 20))

    f(theta).backward()
    h = 1e-6
    for k in (0, 24 + 5):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        with torch.no_grad():
            fd = (f(torch.tensor(tp)).item() - f(torch.tensor(tm)).item()) / (2 * h)
        assert fd == pytest.approx(theta.grad[k].item(), rel=1e-4, abs=1e-8)
