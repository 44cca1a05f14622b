"""Pins of the FGMRES-DR reference (oracle/fgmres_dr.py): it reduces to
restarted FGMRES without deflation, keeps the flexible Arnoldi relation
across a deflated restart, reaches the dense LU solution, its harmonic Ritz
values approach the smallest eigenvalues of the operator, and deflation cuts
the iteration count on a slowly converging system."""
import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

L44 = (4, 4, 4, 4)
DOM2 = (2, 2, 2, 2)


@pytest.fixture(scope="module")
def prob(ora):
    from oracle import fgmres_dr as dr

    U = inputs.gauge_field(L44, 0.5, 1001)
    kappa = 0.13
    A = ora.clover(L44, U, 1.0, kappa)
    Ainv = ora.invert_clover(L44, A)
    return dict(dr=dr, U=U, A=A, Ainv=Ainv, kappa=kappa)


def _dense(ora, p):
    V = inputs.volume(L44)
    N = 12 * V
    M = np.zeros((N, N), dtype=np.complex128)
    e = np.zeros((V, 4, 3), dtype=np.complex128)
    f = e.reshape(-1)
    for k in range(N):
        f[k] = 1
        M[:, k] = ora.apply_D(L44, p["U"], p["A"], p["kappa"], e).reshape(-1)
        f[k] = 0
    return M


def test_no_deflation_is_restarted_fgmres(ora, prob):
    dr = prob["dr"]
    P = dr.Problem(L44, DOM2, prob["U"], prob["A"], prob["Ainv"], prob["kappa"], use_sap=False)
    b = inputs.gaussian_source(L44, 2201).reshape(-1)
    x, info = dr.fgmres_dr(P, b, 1e-10, m=8, k=0, max_cycles=60)
    xc, ic = ora.fgmres(L44, DOM2, prob["U"], prob["A"], prob["Ainv"], prob["kappa"], b.reshape(-1, 4, 3), 1e-10,
                        m=8, max_restarts=59, use_sap=False)
    assert info["converged"] and ic["converged"]
    assert info["iters"] == ic["iters"]
    assert np.allclose(info["history"], ic["history"], rtol=1e-6, atol=1e-14)
    assert np.linalg.norm(x - xc.reshape(-1)) <= 1e-8 * np.linalg.norm(x)


def test_deflated_restart_keeps_the_arnoldi_relation(ora, prob):
    dr = prob["dr"]
    P = dr.Problem(L44, DOM2, prob["U"], prob["A"], prob["Ainv"], prob["kappa"], use_sap=True, nmr=2, ncy=1)
    b = inputs.gaussian_source(L44, 2202).reshape(-1)
    seen = []

    def hook(V, Z, H, c):
        k = Z.shape[0]
        DZ = np.stack([P.D(Z[i]) for i in range(k)])
        seen.append((np.linalg.norm(DZ - (H.T @ V)) / np.linalg.norm(DZ),
                     np.abs(V.conj() @ V.T - np.eye(k + 1)).max(), np.linalg.norm(c)))

    x, info = dr.fgmres_dr(P, b, 1e-12, m=6, k=3, max_cycles=40, state_hook=hook)
    assert info["converged"] and len(seen) >= 8
    # The relation holds at every deflated restart.  So does orthonormality,
    # to the accuracy the restart can give it: the least-squares residual
    # rho, recycled as the last basis vector, carries an absolute error of
    # order eps |b|, so after normalisation the basis is orthonormal to about
    # eps |b| / |rho| (|rho| = |c|), which grows as the solve converges.  A
    # recombination that mixes the wrong columns breaks it by O(1).
    eps, bn = np.finfo(float).eps, np.linalg.norm(b)
    for rel_rel, orth, cn in seen:
        assert rel_rel <= 1e-11
        assert orth <= 16 * eps * bn / cn, (orth, cn)


def test_deflation_reaches_lu_and_cuts_iterations(ora, prob):
    dr = prob["dr"]
    M = _dense(ora, prob)
    b = inputs.gaussian_source(L44, 2203).reshape(-1)
    x_lu = np.linalg.solve(M, b)
    P = dr.Problem(L44, DOM2, prob["U"], prob["A"], prob["Ainv"], prob["kappa"], use_sap=False)
    x0, i0 = dr.fgmres_dr(P, b, 1e-11, m=10, k=0, max_cycles=200)
    x1, i1 = dr.fgmres_dr(P, b, 1e-11, m=10, k=5, max_cycles=200)
    assert i0["converged"] and i1["converged"]
    assert np.linalg.norm(x1 - x_lu) <= 1e-8 * np.linalg.norm(x_lu)
    assert i1["iters"] < i0["iters"]
    # the harmonic Ritz values of the last deflated restart approach the
    # eigenvalues of D of smallest modulus
    ev = np.linalg.eigvals(M)
    smallest = ev[np.argsort(np.abs(ev))]
    th = i1["thetas"][-1][0]
    assert abs(th - smallest[np.argmin(np.abs(smallest[:24] - th))]) <= 0.05 * abs(th)
