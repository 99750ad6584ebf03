"""Oracle Lanczos: ground-state energy from a Krylov recurrence, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper computes ground states with a matrix-free Lanczos whose only use of H is the product
H v (Sec. 2.1, Sec. 4.4; App. D calls ``lanczos``), with Eigen solving the small tridiagonal
problem. This oracle runs the textbook recurrence

    w = H v_k;  alpha_k = <v_k, w>;  w -= alpha_k v_k + beta_{k-1} v_{k-1};
    full re-orthogonalisation of w against v_0..v_k (classical Gram-Schmidt, applied twice);
    beta_k = ||w||;  v_{k+1} = w / beta_k,

and takes the smallest eigenvalue of the tridiagonal matrix T (diagonal alpha, off-diagonal
beta) from LAPACK through ``scipy.linalg.eigvalsh_tridiagonal`` (a library step).
"""

from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal, eigvalsh_tridiagonal

__all__ = ["lanczos"]


def lanczos(apply_h, v0: np.ndarray, steps: int, reorth: bool = True, breakdown_tol: float = 1e-14,
            want_vector: bool = False) -> dict:
    """Run up to ``steps`` Lanczos steps from ``v0``; returns E0, alpha, beta, steps_done.

    Stops early when beta_k < breakdown_tol * ||T|| (an invariant subspace was found); that is
    not an error. With ``want_vector`` the Ritz vector of E0 is returned as well.
    """
    v = np.asarray(v0, dtype=np.float64).copy()
    v /= np.linalg.norm(v)
    V = [v]
    alpha, beta = [], []
    v_prev = np.zeros_like(v)
    b_prev = 0.0
    for k in range(steps):
        w = apply_h(V[k])
        a = float(np.dot(V[k], w))
        w = w - a * V[k] - b_prev * v_prev
        if reorth:
            B = np.stack(V, axis=1)
            for _ in range(2):
                w = w - B @ (B.T @ w)
        b = float(np.linalg.norm(w))
        alpha.append(a)
        tnorm = max(max(abs(t) for t in alpha), max(beta) if beta else 0.0, b)
        if k == steps - 1 or b < breakdown_tol * tnorm:
            beta.append(b)
            break
        beta.append(b)
        v_prev, b_prev = V[k], b
        V.append(w / b)
    m = len(alpha)
    off = np.array(beta[: m - 1], dtype=np.float64)
    a_arr = np.array(alpha, dtype=np.float64)
    out = {"alpha": a_arr, "beta": np.array(beta, dtype=np.float64), "steps_done": m}
    if m == 1:
        out["E0"] = float(a_arr[0])
        if want_vector:
            out["vector"] = V[0].copy()
        return out
    if want_vector:
        evals, evecs = eigh_tridiagonal(a_arr, off, select="i", select_range=(0, 0))
        out["E0"] = float(evals[0])
        out["vector"] = np.stack(V[:m], axis=1) @ evecs[:, 0]
    else:
        out["E0"] = float(eigvalsh_tridiagonal(a_arr, off, select="i", select_range=(0, 0))[0])
    return out
