"""FGMRES with deflated restarts (FGMRES-DR), the outer solver of
arXiv:1502.04025, Sec. 3.1, written from the definitions of deflated
restarting (harmonic Ritz vectors kept across restarts) for flexible GMRES.

TEST INFRASTRUCTURE ONLY: used by the tests, never by the library.  The
operator and the Schwarz preconditioner come from the C oracle; the small
dense linear algebra (least squares, the harmonic Ritz eigenproblem, QR)
from numpy.

One cycle (flexible Arnoldi, modified Gram-Schmidt):
    z_j = M v_j,  w = D z_j,  h_ij = <v_i, w>,  w -= h_ij v_i,
    h_{j+1,j} = |w|,  v_{j+1} = w / h_{j+1,j}
so that D Z_j = V_{j+1} Hbar_j.  The iterate minimises |c - Hbar y| with
c = V^H r_0.  At a deflated restart after m steps:
    rho   = c - Hbar_m y                         (the residual, in basis V_{m+1})
    F     = H_m + H_m^{-H} l^H l                 (l = last row of Hbar_m)
    g_1..g_k = eigenvectors of F with the k eigenvalues of smallest modulus
              (harmonic Ritz vectors)
    P_{k+1} = orthonormal basis of [[g_1..g_k ; 0], rho]   ((m+1) x (k+1))
    V_{k+1} <- V_{m+1} P_{k+1},  Z_k <- Z_m P_k,  Hbar_k <- P_{k+1}^H Hbar_m P_k,
    c <- P_{k+1}^H rho
and the Arnoldi process continues from step k.  With k = 0 this is plain
restarted FGMRES(m).
"""
from __future__ import annotations

import numpy as np

from oracle import pyoracle as ora


class Problem:
    def __init__(self, L, dom, U, A, Ainv, kappa, use_sap=True, nmr=4, ncy=4):
        self.L, self.dom, self.U, self.A, self.Ainv, self.kappa = L, dom, U, A, Ainv, kappa
        self.use_sap, self.nmr, self.ncy = use_sap, nmr, ncy

    def D(self, x):
        return ora.apply_D(self.L, self.U, self.A, self.kappa, x.reshape(-1, 4, 3)).reshape(-1)

    def M(self, v):
        if not self.use_sap:
            return v.copy()
        psi, _ = ora.sap(self.L, self.dom, self.U, self.A, self.Ainv, self.kappa, v.reshape(-1, 4, 3), self.nmr,
                         2 * self.ncy)
        return psi.reshape(-1)


def _lstsq(H, c):
    y, *_ = np.linalg.lstsq(H, c, rcond=None)
    return y, c - H @ y


def harmonic_ritz(Hbar_m):
    """Eigenpairs of H_m + H_m^{-H} l^H l (l the last row of Hbar_m), sorted by |theta|."""
    m = Hbar_m.shape[1]
    Hm = Hbar_m[:m, :m]
    l = Hbar_m[m:m + 1, :m]
    F = Hm + np.linalg.solve(Hm.conj().T, l.conj().T @ l)
    theta, G = np.linalg.eig(F)
    order = np.argsort(np.abs(theta), kind="stable")
    return theta[order], G[:, order]


def fgmres_dr(P: Problem, b, tol, m, k, max_cycles=100, state_hook=None):
    """Returns (x, info); state_hook(V, Z, Hbar, c) is called after every deflated restart."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    n = b.size
    bnorm = np.linalg.norm(b)
    x = np.zeros(n, dtype=np.complex128)
    r = b - P.D(x)
    beta = np.linalg.norm(r)
    V = np.zeros((m + 1, n), dtype=np.complex128)
    Z = np.zeros((m, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    c = np.zeros(m + 1, dtype=np.complex128)
    V[0] = r / beta
    c[0] = beta
    j0 = 0
    iters = 0
    hist = []
    converged = False
    thetas = []
    for cycle in range(max_cycles):
        jm = j0
        for j in range(j0, m):
            Z[j] = P.M(V[j])
            w = P.D(Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V[j + 1] = w / H[j + 1, j]
            iters += 1
            jm = j + 1
            _, res = _lstsq(H[:j + 2, :j + 1], c[:j + 2])
            est = np.linalg.norm(res) / bnorm
            hist.append(est)
            if est <= tol:
                break
        y, rho = _lstsq(H[:jm + 1, :jm], c[:jm + 1])
        x = x + Z[:jm].T @ y
        rtrue = b - P.D(x)
        rel = np.linalg.norm(rtrue) / bnorm
        hist.append(rel)
        if rel <= tol:
            converged = True
            break
        if k == 0 or jm < m:
            beta = np.linalg.norm(rtrue)
            V[:] = 0
            Z[:] = 0
            H[:] = 0
            c[:] = 0
            V[0] = rtrue / beta
            c[0] = beta
            j0 = 0
            continue
        theta, G = harmonic_ritz(H)
        thetas.append(theta[:k].copy())
        Q, _ = np.linalg.qr(np.vstack([G[:, :k], np.zeros((1, k))]))
        q = rho - Q @ (Q.conj().T @ rho)
        q = q - Q @ (Q.conj().T @ q)  # twice, for a tiny residual vector
        q = q / np.linalg.norm(q)
        Pk1 = np.hstack([Q, q[:, None]])
        Pk = Q[:m, :]
        Vn = Pk1.T @ V
        Zn = Pk.T @ Z
        Hn = Pk1.conj().T @ H @ Pk
        cn = Pk1.conj().T @ rho
        V[:] = 0
        Z[:] = 0
        H[:] = 0
        c[:] = 0
        V[:k + 1] = Vn
        Z[:k] = Zn
        H[:k + 1, :k] = Hn
        c[:k + 1] = cn
        j0 = k
        if state_hook is not None:
            state_hook(V[:k + 1].copy(), Z[:k].copy(), H[:k + 1, :k].copy(), c[:k + 1].copy())
    return x, {"converged": converged, "iters": iters, "history": np.array(hist), "thetas": thetas}
