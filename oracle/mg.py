"""Two-level aggregation multigrid preconditioner with the Schwarz method as
its smoother (arXiv:1502.04025, Sec. 2.4: a Krylov solver preconditioned by
a V-cycle whose smoother is the domain-decomposition preconditioner of
Sec. 3), written out plainly in FP64.

TEST INFRASTRUCTURE ONLY: used by the tests, never by the library.  The
operator and the Schwarz smoother come from the C oracle; the rest is numpy.

The paper names the method and prints none of it.  The reading (shared with
the library, listed in the design notes):
  aggregates   the Schwarz domains, each split by chirality (spins {0,1} and
               {2,3}, the eigenspaces of gamma5), so that the prolongator
               commutes with gamma5
  setup        nv given random vectors w_k; `setup_iters` times each is
               replaced by M_SAP w_k (`setup_ncy` Schwarz cycles of `nmr` MR
               steps) and normalised; then, on every aggregate and chirality
               block, w_0..w_{nv-1} restricted to the block are orthonormalised
               by modified Gram-Schmidt, twice.  The block vectors are the
               columns of the prolongator P.
  coarse       D_c = P^H D P (coarse index (aggregate, chirality, k))
  V-cycle      e_c ~ D_c^{-1} P^H v by one GMRES cycle of `coarse_iters` steps
               from zero (or, for the pins, an exact solve), z = P e_c,
               r = v - D z, z += M_SAP(r) (`post_ncy` Schwarz cycles)
  bootstrap    the adaptive setup, `bootstrap` times: w_k = the V-cycle of the
               method built so far applied to the k-th prolongator column
               (column k of every block, as one fine field), normalised; P and
               D_c rebuilt from the new w_k
"""
from __future__ import annotations

import numpy as np

from oracle import pyoracle as ora


def aggregates(L, dom):
    """Aggregate (lexicographic domain-block index) of every site, and their count."""
    L = tuple(L)
    V = int(np.prod(L))
    n = np.arange(V)
    x = n % L[0]
    y = (n // L[0]) % L[1]
    z = (n // (L[0] * L[1])) % L[2]
    t = n // (L[0] * L[1] * L[2])
    nb = [L[i] // dom[i] for i in range(4)]
    a = (x // dom[0]) + nb[0] * ((y // dom[1]) + nb[1] * ((z // dom[2]) + nb[2] * (t // dom[3])))
    return a, int(np.prod(nb))


class TwoLevel:
    def __init__(self, L, dom, U, A, Ainv, kappa, w0, setup_iters=2, setup_ncy=2, nmr=4, post_ncy=2,
                 coarse_iters=24, bootstrap=0):
        self.L, self.dom, self.U, self.A, self.Ainv, self.kappa = tuple(L), tuple(dom), U, A, Ainv, kappa
        self.nmr, self.post_ncy, self.coarse_iters = nmr, post_ncy, coarse_iters
        self.V = int(np.prod(L))
        self.agg, self.nagg = aggregates(L, dom)
        w = np.array(w0, dtype=np.complex128).reshape(-1, self.V, 4, 3)
        self.nv = w.shape[0]
        # setup: smooth the random vectors with the Schwarz method
        for _ in range(setup_iters):
            for k in range(self.nv):
                w[k] = self.sap(w[k], setup_ncy)
                w[k] /= np.linalg.norm(w[k])
        self.w_smoothed = w.copy()
        self.sites = [np.nonzero(self.agg == a)[0] for a in range(self.nagg)]
        self.nc = self.nagg * 2 * self.nv
        self.build(w)
        for _ in range(bootstrap):
            cols = self.basis()
            w = np.array([self.vcycle(cols[k]) for k in range(self.nv)])
            for k in range(self.nv):
                w[k] /= np.linalg.norm(w[k])
            self.build(w)

    def build(self, w):
        """Prolongator from the test vectors w (nv, V, 4, 3): per aggregate and
        chirality, MGS twice over the nv vectors, so block (a, chi) is a
        (6 * sites, nv) matrix with orthonormal columns; then D_c."""
        self.Pb = {}
        for a in range(self.nagg):
            s = self.sites[a]
            for chi in range(2):
                blk = w[:, s, 2 * chi:2 * chi + 2, :].reshape(self.nv, -1).copy()
                for _ in range(2):
                    for k in range(self.nv):
                        for l in range(k):
                            blk[k] -= np.vdot(blk[l], blk[k]) * blk[l]
                        blk[k] /= np.linalg.norm(blk[k])
                self.Pb[a, chi] = blk.T.copy()
        self.Dc = self.coarse_matrix()

    def basis(self):
        """The prolongator's columns as fine fields: (nv, V, 4, 3), column k of every block."""
        out = np.zeros((self.nv, self.V, 4, 3), dtype=np.complex128)
        for (a, chi), blk in self.Pb.items():
            out[:, self.sites[a], 2 * chi:2 * chi + 2, :] = blk.T.reshape(self.nv, -1, 2, 3)
        return out

    # -- fine-grid pieces
    def D(self, x):
        return ora.apply_D(self.L, self.U, self.A, self.kappa, np.asarray(x).reshape(self.V, 4, 3))

    def sap(self, eta, ncy):
        psi, _ = ora.sap(self.L, self.dom, self.U, self.A, self.Ainv, self.kappa,
                         np.asarray(eta).reshape(self.V, 4, 3), self.nmr, 2 * ncy)
        return psi

    # -- transfer operators; coarse vectors are (nagg, 2, nv)
    def restrict(self, v):
        v = np.asarray(v).reshape(self.V, 4, 3)
        out = np.zeros((self.nagg, 2, self.nv), dtype=np.complex128)
        for (a, chi), blk in self.Pb.items():
            out[a, chi] = blk.conj().T @ v[self.sites[a], 2 * chi:2 * chi + 2, :].reshape(-1)
        return out

    def prolong(self, ec):
        ec = np.asarray(ec).reshape(self.nagg, 2, self.nv)
        out = np.zeros((self.V, 4, 3), dtype=np.complex128)
        for (a, chi), blk in self.Pb.items():
            out[self.sites[a], 2 * chi:2 * chi + 2, :] = (blk @ ec[a, chi]).reshape(-1, 2, 3)
        return out

    def coarse_matrix(self):
        """D_c = P^H D P, column by column (D applied to each prolonged unit vector)."""
        Dc = np.zeros((self.nc, self.nc), dtype=np.complex128)
        for j in range(self.nc):
            e = np.zeros(self.nc, dtype=np.complex128)
            e[j] = 1.0
            Dc[:, j] = self.restrict(self.D(self.prolong(e))).reshape(-1)
        return Dc

    def coarse_solve(self, rc):
        """One GMRES cycle of coarse_iters steps on D_c e = rc from e = 0
        (modified Gram-Schmidt, least squares); fewer on an exact breakdown."""
        b = np.asarray(rc).reshape(-1)
        beta = np.linalg.norm(b)
        x = np.zeros_like(b)
        if beta == 0:
            return x.reshape(self.nagg, 2, self.nv)
        m = self.coarse_iters
        Vb = np.zeros((m + 1, b.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        Vb[0] = b / beta
        jm = 0
        for j in range(m):
            w = self.Dc @ Vb[j]
            for i in range(j + 1):
                H[i, j] = np.vdot(Vb[i], w)
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            jm = j + 1
            if H[j + 1, j] == 0:
                break
            Vb[j + 1] = w / H[j + 1, j]
        c = np.zeros(jm + 1, dtype=np.complex128)
        c[0] = beta
        y, *_ = np.linalg.lstsq(H[:jm + 1, :jm], c, rcond=None)
        return (Vb[:jm].T @ y).reshape(self.nagg, 2, self.nv)

    def vcycle(self, v, exact_coarse=False):
        v = np.asarray(v).reshape(self.V, 4, 3)
        rc = self.restrict(v)
        if exact_coarse:
            ec = np.linalg.solve(self.Dc, rc.reshape(-1)).reshape(rc.shape)
        else:
            ec = self.coarse_solve(rc)
        z = self.prolong(ec)
        if self.post_ncy > 0:
            z = z + self.sap(v - self.D(z), self.post_ncy)
        return z
