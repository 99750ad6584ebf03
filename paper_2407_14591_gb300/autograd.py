"""Differentiable product y = H(theta) x and differentiable Krylov time evolution.

``ParamOperator`` describes H(theta) = sum_q scale_q theta[k_q] T_q + sum_f c_f T_f: a list of
parametrised terms (kind, i, j, k, scale) and fixed terms (kind, i, j, coef). ``matvec`` is a
``torch.autograd.Function`` whose adjoint is written by hand:

* dx = H(theta)^T dy = H(theta) dy (all terms are real and Hermitian), one more product;
* dtheta_k = sum_{q: k_q = k} scale_q <dy, T_q x>, from the library's per-term reductions
  (``dq_term_grads``).

``evolve`` applies exp(-i H dt) ``steps`` times with a Lanczos (Krylov) approximation of
dimension m, on complex vectors stored as two real columns (two right-hand sides of the
product). Each time step can be checkpointed (``torch.utils.checkpoint``): only the state at
step boundaries is kept and the Krylov basis is recomputed in the backward pass.

Every product runs in the CUDA library; torch only holds vectors and does the small m x m
algebra (tridiagonal eigendecomposition and exponential).
"""

from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

from . import binding as b

__all__ = ["ParamOperator", "matvec", "evolve", "expectation"]


class ParamOperator:
    """H(theta) on one sector. ``params``: (kind, i, j, k, scale) with coefficient scale*theta[k];
    ``fixed``: (kind, i, j, coef)."""

    def __init__(self, sector: b.Sector, params, fixed=(), n_params: int | None = None):
        self.sector = sector
        self.params = [(p[0], int(p[1]), int(p[2]), int(p[3]), float(p[4])) for p in params]
        self.fixed = [(f[0], int(f[1]), int(f[2]), float(f[3])) for f in fixed]
        self.n_params = n_params if n_params is not None else (max((p[3] for p in self.params), default=-1) + 1)
        self.index = torch.tensor([p[3] for p in self.params], dtype=torch.long)
        self.scale = torch.tensor([p[4] for p in self.params], dtype=torch.float64)
        self._cache_key = None
        self._cache_terms = None

    def term_list(self, theta) -> list:
        th = theta.detach().to("cpu", torch.float64)
        out = [(k, i, j, s * float(th[p])) for (k, i, j, p, s) in self.params]
        return out + list(self.fixed)

    def compile(self, theta) -> b.Terms:
        key = theta.detach().to("cpu", torch.float64).numpy().tobytes() if theta is not None else b""
        if key != self._cache_key:
            self._cache_terms = b.make_terms(self.sector, self.term_list(theta) if theta is not None else self.fixed)
            self._cache_key = key
        return self._cache_terms


class _Matvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, theta, op):
        t = op.compile(theta)
        xc = x.contiguous()
        y = b.matvec(op.sector, t, xc)
        ctx.op = op
        ctx.terms = t
        ctx.save_for_backward(xc, theta)
        return y

    @staticmethod
    def backward(ctx, dy):
        x, theta = ctx.saved_tensors
        op = ctx.op
        dyc = dy.contiguous()
        dx = dtheta = None
        if ctx.needs_input_grad[0]:
            dx = b.matvec(op.sector, ctx.terms, dyc)
        if ctx.needs_input_grad[1] and op.params:
            g = b.term_grads(op.sector, [p[:3] for p in op.params], x, dyc)
            d = torch.zeros(op.n_params, dtype=torch.float64, device=g.device)
            d.index_add_(0, op.index.to(g.device), g * op.scale.to(g.device))
            dtheta = d.to(theta.dtype).to(theta.device)
        return dx, dtheta, None


def matvec(op: ParamOperator, x, theta):
    """y = H(theta) x; differentiable in x and theta. x: (D,) or (D, nrhs) CUDA tensor."""
    if theta is None:
        theta = torch.zeros(max(op.n_params, 1), dtype=torch.float64)
    return _Matvec.apply(x, theta, op)


def _apply_c(op, vc, theta):
    """H applied to a complex vector (its real and imaginary parts as two right-hand sides)."""
    yr = matvec(op, torch.view_as_real(vc), theta)
    return torch.view_as_complex(yr)


def _krylov_step(psi_r, theta, op, dt: float, m: int, breakdown: float = 1e-12):
    """One step psi <- exp(-i H dt) psi, Lanczos on the complex vector psi (given as (D, 2))."""
    psi = torch.view_as_complex(psi_r)
    nrm = torch.linalg.vector_norm(psi)
    v = psi / nrm
    V = [v]
    alphas, betas = [], []
    m = min(m, op.sector.dim)
    for k in range(m):
        w = _apply_c(op, V[k], theta)
        a = torch.real(torch.vdot(V[k], w))
        alphas.append(a)
        w = w - a * V[k]
        if k > 0:
            w = w - betas[-1] * V[k - 1]
        B = torch.stack(V, dim=1)
        for _ in range(2):  # full re-orthogonalisation (classical Gram-Schmidt, twice)
            w = w - B @ (B.conj().T @ w)
        if k == m - 1:
            break
        bt = torch.linalg.vector_norm(w)
        if float(bt.detach()) < breakdown * max(1.0, float(torch.stack(alphas).detach().abs().max())):
            break
        betas.append(bt)
        V.append(w / bt)
    n = len(alphas)
    T = torch.diag(torch.stack(alphas))
    if n > 1:
        off = torch.stack(betas[: n - 1])
        T = T + torch.diag(off, 1) + torch.diag(off, -1)
    lam, U = torch.linalg.eigh(T)
    Uc = U.to(torch.complex128)
    coef = Uc @ (torch.exp(-1j * dt * lam.to(torch.complex128)) * Uc[0, :])
    out = nrm * (torch.stack(V[:n], dim=1) @ coef.to(psi.dtype))
    return torch.view_as_real(out)


def evolve(op: ParamOperator, theta, psi0, dt: float, steps: int, m: int = 16, use_checkpoint: bool = True):
    """psi(steps*dt) = exp(-i H(theta) dt)^steps psi0 (complex128 CUDA vector), differentiable."""
    psi_r = torch.view_as_real(psi0.contiguous())
    for _ in range(steps):
        if use_checkpoint:
            psi_r = checkpoint(_krylov_step, psi_r, theta, op, dt, m, use_reentrant=False)
        else:
            psi_r = _krylov_step(psi_r, theta, op, dt, m)
    return torch.view_as_complex(psi_r)


def expectation(obs: ParamOperator, psi, theta=None):
    """<psi| O |psi> (real part) for an operator O, differentiable in psi (and theta)."""
    return torch.real(torch.vdot(psi, _apply_c(obs, psi, theta)))
