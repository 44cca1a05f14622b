"""Condition number of the Wilson-clover operator D, estimated by Lanczos on
the Hermitian positive definite D^H D (the solution-error criterion: two
solutions whose residuals are r1 and r2 relative to |b| differ by at most
cond(D) (r1 + r2) relative to the solution).

TEST INFRASTRUCTURE ONLY: used by the tests, never by the library.  The
operator comes from the C oracle; D^H is applied as gamma_5 D gamma_5
(gamma_5-hermiticity, pinned in tests/test_oracle.py).

Lanczos with full re-orthogonalisation (twice per step) from one random
start vector builds the tridiagonal T_k = Q_k^H (D^H D) Q_k; its largest and
smallest eigenvalues approach sigma_max^2 and sigma_min^2 of D from inside
(the smallest Ritz value is never below sigma_min^2, so the ratio is a lower
bound on cond(D) that tightens with k).  An invariant subspace (beta = 0)
ends the iteration early with exact values for the start vector's
components.
"""
from __future__ import annotations

import numpy as np

from oracle import pyoracle as ora

_G5 = np.array([1.0, 1.0, -1.0, -1.0])[None, :, None]  # gamma_5 = diag(1, 1, -1, -1) on the spin index


def apply_DhD(L, U, A, kappa: float, x: np.ndarray) -> np.ndarray:
    """D^H D x for one spinor field (V, 4, 3), with D^H = g5 D g5."""
    y = ora.apply_D(L, U, A, kappa, x)
    return _G5 * ora.apply_D(L, U, A, kappa, _G5 * y)


def lanczos_extremes(L, U, A, kappa: float, steps: int = 80, seed: int = 0):
    """(sigma_max, sigma_min, steps taken) of D from `steps` Lanczos steps on D^H D."""
    V = int(np.prod(L))
    g = np.random.Generator(np.random.Philox(int(seed)))
    q = g.standard_normal((V, 4, 3)) + 1j * g.standard_normal((V, 4, 3))
    q /= np.linalg.norm(q)
    Q = [q]
    alpha, beta = [], []
    scale = None
    for j in range(steps):
        w = apply_DhD(L, U, A, kappa, Q[j])
        a = np.vdot(Q[j], w).real
        alpha.append(a)
        w = w - a * Q[j]
        if j > 0:
            w = w - beta[-1] * Q[j - 1]
        for _ in range(2):  # full re-orthogonalisation against every earlier vector
            for qi in Q:
                w = w - np.vdot(qi, w) * qi
        b = np.linalg.norm(w)
        scale = max(scale or 0.0, abs(a), b)
        if b <= 1e-12 * scale or j == steps - 1:
            break
        beta.append(b)
        Q.append(w / b)
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    theta = np.linalg.eigvalsh(T)
    return float(np.sqrt(theta[-1])), float(np.sqrt(max(theta[0], 0.0))), k


def cond_estimate(L, U, A, kappa: float, steps: int = 80, seed: int = 0) -> dict:
    smax, smin, k = lanczos_extremes(L, U, A, kappa, steps, seed)
    return {"sigma_max": smax, "sigma_min": smin, "cond": smax / smin if smin > 0 else float("inf"),
            "lanczos_steps": k}
