"""GPU two-level multigrid preconditioner against the reference
(oracle/mg.py): the prolongator built from the same random vectors, the
coarse correction (one GMRES cycle on D_c = P^H D P, prolonged), the V-cycle
with Schwarz post-smoothing, and FGMRES with the V-cycle as preconditioner."""
import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

pytestmark = pytest.mark.gpu

L44, DOM2 = (4, 4, 4, 4), (2, 2, 2, 2)


@pytest.fixture(scope="module")
def q():
    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import qdd

    return qdd


@pytest.fixture(scope="module")
def ctx(q):
    c = q.qdd_create(0, 0)
    yield c
    q.qdd_destroy(c)


def _problem(q, ctx, ora, L, dom, kappa, eps=0.5, seed=1001):
    U = inputs.gauge_field(L, eps, seed)
    A = ora.clover(L, U, 1.0, kappa)
    Ainv = ora.invert_clover(L, A)
    g = q.qdd_create_gauge_field(ctx, L, dom, U)
    q.qdd_set_clover(g, 1.0, kappa)
    return U, A, Ainv, g


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("L,dom", [(L44, DOM2), ((8, 8, 8, 8), (4, 4, 4, 4))])
def test_basis_and_coarse_correction_match_reference(q, ctx, ora, L, dom):
    from oracle import mg
    U, A, Ainv, g = _problem(q, ctx, ora, L, dom, 0.13)
    nv = 4
    w0 = inputs.gaussian_source(L, 4001, nrhs=nv)
    kw = dict(setup_iters=2, setup_ncy=2, nmr=4, post_ncy=0, coarse_iters=16)
    ref = mg.TwoLevel(L, dom, U, A, Ainv, 0.13, w0, **kw)
    q.qdd_mg_setup(g, np.ascontiguousarray(w0), nv=nv, sap_prec="f64", **kw)
    V = int(np.prod(L))
    B = q.qdd_mg_get_basis(g, nv, V)
    # FP64 smoothing on both sides; the library stores P in FP32
    assert _rel(B, ref.basis()) <= 1e-6
    # coarse correction z = P e, e from 16 GMRES steps on D_c (FP32 on the GPU)
    v = inputs.gaussian_source(L, 4005)
    z = q.qdd_mg_vcycle(g, np.ascontiguousarray(v))
    assert _rel(z, ref.vcycle(v)) <= 1e-4
    q.qdd_destroy_gauge(g)


def test_bootstrap_matches_reference(q, ctx, ora):
    """The adaptive setup pass: each test vector replaced by the V-cycle of
    the first build applied to its prolongator column, P and D_c rebuilt."""
    from oracle import mg
    U, A, Ainv, g = _problem(q, ctx, ora, L44, DOM2, 0.13)
    nv = 4
    w0 = inputs.gaussian_source(L44, 4001, nrhs=nv)
    kw = dict(setup_iters=2, setup_ncy=2, nmr=4, post_ncy=2, coarse_iters=16, bootstrap=1)
    ref = mg.TwoLevel(L44, DOM2, U, A, Ainv, 0.13, w0, **kw)
    q.qdd_mg_setup(g, np.ascontiguousarray(w0), nv=nv, sap_prec="f64", **kw)
    V = int(np.prod(L44))
    # FP32 coarse cycle inside the bootstrap V-cycles, FP32 storage of P
    assert _rel(q.qdd_mg_get_basis(g, nv, V), ref.basis()) <= 1e-3
    v = inputs.gaussian_source(L44, 4006)
    assert _rel(q.qdd_mg_vcycle(g, np.ascontiguousarray(v)), ref.vcycle(v)) <= 1e-3
    with pytest.raises(q.QddError):
        q.qdd_mg_setup(g, np.ascontiguousarray(w0), nv=nv, bootstrap=-1)
    q.qdd_destroy_gauge(g)


def test_vcycle_with_post_smoothing_matches_reference(q, ctx, ora):
    from oracle import mg
    U, A, Ainv, g = _problem(q, ctx, ora, L44, DOM2, 0.13)
    nv = 4
    w0 = inputs.gaussian_source(L44, 4001, nrhs=nv)
    kw = dict(setup_iters=2, setup_ncy=2, nmr=4, post_ncy=2, coarse_iters=16)
    ref = mg.TwoLevel(L44, DOM2, U, A, Ainv, 0.13, w0, **kw)
    q.qdd_mg_setup(g, np.ascontiguousarray(w0), nv=nv, sap_prec="f64", **kw)
    v = inputs.gaussian_source(L44, 4006)
    z = q.qdd_mg_vcycle(g, np.ascontiguousarray(v))
    assert _rel(z, ref.vcycle(v)) <= 1e-4
    q.qdd_destroy_gauge(g)


@pytest.mark.parametrize("sap_prec", ["f64", "f32"])
def test_multigrid_fgmres_converges_in_fewer_steps(q, ctx, ora, sap_prec):
    from oracle import mg, fgmres_dr as dr
    kappa = 0.138  # close to critical on this field
    U, A, Ainv, g = _problem(q, ctx, ora, L44, DOM2, kappa)
    nv = 8
    w0 = inputs.gaussian_source(L44, 4001, nrhs=nv)
    kw = dict(setup_iters=3, setup_ncy=2, nmr=4, post_ncy=2, coarse_iters=24)
    q.qdd_mg_setup(g, np.ascontiguousarray(w0), nv=nv, sap_prec=sap_prec, **kw)
    b = inputs.gaussian_source(L44, 4004)
    common = dict(tol=1e-10, restart_m=16, max_restarts=50, arnoldi_prec="f64")
    x_mg, r_mg = q.qdd_solve(g, b, use_sap=2, **common)
    x_sap, r_sap = q.qdd_solve(g, b, use_sap=1, nmr=4, ncy=2, sap_prec=sap_prec, **common)
    assert r_mg["converged"] and r_sap["converged"]
    r = b - ora.apply_D(L44, U, A, kappa, x_mg)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    assert r_mg["iters"] < r_sap["iters"]
    # the reference takes about as many steps
    ref = mg.TwoLevel(L44, DOM2, U, A, Ainv, kappa, w0, **kw)

    class MGProblem(dr.Problem):
        def M(self, v):
            return ref.vcycle(v).reshape(-1)

    _, info = dr.fgmres_dr(MGProblem(L44, DOM2, U, A, Ainv, kappa), b.reshape(-1), 1e-10, m=16, k=0,
                           max_cycles=50)
    assert abs(r_mg["iters"] - info["iters"]) <= max(3, info["iters"] // 5)
    q.qdd_destroy_gauge(g)


def test_multigrid_parameter_checks(q, ctx, ora):
    U, A, Ainv, g = _problem(q, ctx, ora, L44, DOM2, 0.13)
    b = inputs.gaussian_source(L44, 4007)
    with pytest.raises(q.QddError):  # no setup yet
        q.qdd_solve(g, b, use_sap=2)
    w0 = np.ascontiguousarray(inputs.gaussian_source(L44, 4001, nrhs=2))
    with pytest.raises(q.QddError):
        q.qdd_mg_setup(g, w0, nv=0)
    q.qdd_mg_setup(g, w0, nv=2, setup_iters=1)
    with pytest.raises(q.QddError):  # one right-hand side only
        q.qdd_solve(g, np.ascontiguousarray(inputs.gaussian_source(L44, 4008, nrhs=2)), use_sap=2, nrhs=2)
    q.qdd_destroy_gauge(g)
