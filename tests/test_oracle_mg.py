"""Pins of the two-level multigrid reference (oracle/mg.py): its prolongator
respects chirality and is orthonormal per block, its coarse operator keeps
the gamma5-hermiticity of D, a complete basis makes the coarse correction
the exact inverse (dense LU), the coarse correction removes every error in
the range of P, the multigrid-preconditioned FGMRES reaches the LU
solution in fewer steps than the Schwarz-preconditioned one near the
critical kappa, and a bootstrap pass without post-smoothing keeps the
coarse space (the exact coarse correction does not change)."""
import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

L44, DOM2 = (4, 4, 4, 4), (2, 2, 2, 2)


@pytest.fixture(scope="module")
def field(ora):
    U = inputs.gauge_field(L44, 0.5, 1001)
    kappa = 0.13
    A = ora.clover(L44, U, 1.0, kappa)
    Ainv = ora.invert_clover(L44, A)
    return U, A, Ainv, kappa


def _mg(field, nv, seed=4001, **kw):
    from oracle import mg
    U, A, Ainv, kappa = field
    w0 = inputs.gaussian_source(L44, seed, nrhs=nv)
    return mg.TwoLevel(L44, DOM2, U, A, Ainv, kappa, w0, **kw)


def test_prolongator_blocks(field):
    M = _mg(field, 4)
    B = M.basis()
    for (a, chi), blk in M.Pb.items():
        assert np.allclose(blk.conj().T @ blk, np.eye(M.nv), atol=1e-13)
    # columns vanish off their aggregate and their chirality: restricting a
    # field supported on chirality 0 gives zero chirality-1 coarse entries
    v = inputs.gaussian_source(L44, 4002)
    v[:, 2:, :] = 0
    assert np.abs(M.restrict(v)[:, 1, :]).max() == 0
    assert B.shape == (M.nv, 256, 4, 3)


def test_coarse_operator_is_gamma5_hermitian(field):
    M = _mg(field, 4)
    g = np.tile(np.repeat([1.0, -1.0], M.nv), M.nagg)
    Dc = M.Dc
    assert np.linalg.norm(Dc.conj().T - g[:, None] * Dc * g[None, :]) <= 1e-12 * np.linalg.norm(Dc)
    # and it is not Hermitian itself (the check above is not vacuous)
    assert np.linalg.norm(Dc.conj().T - Dc) > 1e-3 * np.linalg.norm(Dc)


def test_coarse_gmres_is_the_krylov_minimiser(field):
    """One cycle of j steps minimises |rc - D_c e| over the Krylov space
    K_j(D_c, rc) (checked with an explicit power basis and numpy's least
    squares), and reaches the exact solution when j = dim D_c."""
    M = _mg(field, 2)
    rng = np.random.default_rng(11)
    rc = rng.standard_normal(M.nc) + 1j * rng.standard_normal(M.nc)
    for j in (1, 3, 8):
        M.coarse_iters = j
        e = M.coarse_solve(rc).reshape(-1)
        K = np.stack([np.linalg.matrix_power(M.Dc, p) @ rc for p in range(j)], axis=1)
        y, *_ = np.linalg.lstsq(M.Dc @ K, rc, rcond=None)
        assert np.linalg.norm(e - K @ y) <= 1e-8 * np.linalg.norm(K @ y)
    M.coarse_iters = M.nc
    e = M.coarse_solve(rc).reshape(-1)
    assert np.linalg.norm(M.Dc @ e - rc) <= 1e-9 * np.linalg.norm(rc)


def test_coarse_correction_removes_range_of_P(field):
    M = _mg(field, 4)
    rng = np.random.default_rng(7)
    ec = rng.standard_normal((M.nagg, 2, M.nv)) + 1j * rng.standard_normal((M.nagg, 2, M.nv))
    e = M.prolong(ec)
    corr = M.prolong(np.linalg.solve(M.Dc, M.restrict(M.D(e)).reshape(-1)))
    assert np.linalg.norm(e - corr) <= 1e-11 * np.linalg.norm(e)


def test_complete_basis_gives_the_exact_inverse(ora, field):
    # 16 sites x 6 components per aggregate-chirality block: nv = 96 spans it
    M = _mg(field, 96, setup_iters=1, setup_ncy=1, post_ncy=0)
    U, A, Ainv, kappa = field
    b = inputs.gaussian_source(L44, 4003)
    z = M.vcycle(b, exact_coarse=True)
    Dm = np.stack([ora.apply_D(L44, U, A, kappa, e.reshape(256, 4, 3)).reshape(-1)
                   for e in np.eye(256 * 12, dtype=np.complex128)], axis=1)
    x = np.linalg.solve(Dm, b.reshape(-1))
    assert np.linalg.norm(z.reshape(-1) - x) <= 1e-10 * np.linalg.norm(x)


def test_multigrid_fgmres_reaches_lu_in_fewer_steps(ora, field):
    from oracle import fgmres_dr as dr
    U, A, Ainv, _ = field
    kappa = 0.138  # close to critical on this field: small eigenvalues
    A = ora.clover(L44, U, 1.0, kappa)
    Ainv = ora.invert_clover(L44, A)
    from oracle import mg
    w0 = inputs.gaussian_source(L44, 4001, nrhs=8)
    M = mg.TwoLevel(L44, DOM2, U, A, Ainv, kappa, w0, setup_iters=3, setup_ncy=2, nmr=4, post_ncy=2,
                    coarse_iters=24)
    b = inputs.gaussian_source(L44, 4004)

    class MGProblem(dr.Problem):
        def M(self, v):
            return M.vcycle(v).reshape(-1)

    P_mg = MGProblem(L44, DOM2, U, A, Ainv, kappa)
    P_sap = dr.Problem(L44, DOM2, U, A, Ainv, kappa, use_sap=True, nmr=4, ncy=2)
    x_mg, info_mg = dr.fgmres_dr(P_mg, b.reshape(-1), 1e-10, m=16, k=0, max_cycles=50)
    x_sap, info_sap = dr.fgmres_dr(P_sap, b.reshape(-1), 1e-10, m=16, k=0, max_cycles=50)
    assert info_mg["converged"] and info_sap["converged"]
    r = b.reshape(-1) - ora.apply_D(L44, U, A, kappa, x_mg.reshape(256, 4, 3)).reshape(-1)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    assert info_mg["iters"] < info_sap["iters"]


def test_bootstrap_without_smoothing_keeps_the_coarse_space(field):
    """Without post-smoothing every V-cycle output lies in range(P), so a
    bootstrap pass rebuilds P with the same span per block: the exact coarse
    correction P D_c^{-1} P^H is unchanged, while the columns themselves
    change.  A pass that rebuilt the wrong blocks, or left D_c stale, fails."""
    M0 = _mg(field, 3, post_ncy=0)
    M1 = _mg(field, 3, post_ncy=0, bootstrap=1)
    assert np.abs(M1.basis() - M0.basis()).max() > 1e-3
    v = inputs.gaussian_source(L44, 4010)
    z0, z1 = M0.vcycle(v, exact_coarse=True), M1.vcycle(v, exact_coarse=True)
    assert np.linalg.norm(z1 - z0) <= 1e-10 * np.linalg.norm(z0)
    # with smoothing the span moves
    M2 = _mg(field, 3, post_ncy=2, bootstrap=1)
    M2.post_ncy = 0
    assert np.linalg.norm(M2.vcycle(v, exact_coarse=True) - z0) > 1e-3 * np.linalg.norm(z0)
