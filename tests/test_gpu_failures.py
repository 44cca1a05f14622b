"""Failure detection on the host side of the solver: a solve that runs out of
restarts returns QDD_ENOCONV with its last iterate and a filled report, and
a non-finite right-hand side is reported as QDD_ENAN without disturbing the
gauge object (the next solve on it converges).  Nothing here faults, traps
or stalls the GPU."""
import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

pytestmark = pytest.mark.gpu

L, DOM = (8, 8, 8, 8), (4, 4, 4, 4)


@pytest.fixture(scope="module")
def q():
    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import qdd

    return qdd


@pytest.fixture(scope="module")
def setup(q, ora):
    ctx = q.qdd_create(0, 0)
    U = inputs.gauge_field(L, 0.5, 1001)
    g = q.qdd_create_gauge_field(ctx, L, DOM, U)
    q.qdd_set_clover(g, 1.0, 0.12)
    A = ora.clover(L, U, 1.0, 0.12)
    yield q, g, U, A
    q.qdd_destroy_gauge(g)
    q.qdd_destroy(ctx)


def test_nonconvergence_returns_the_last_iterate_and_its_true_residual(setup, ora):
    q, g, U, A = setup
    b = inputs.gaussian_source(L, 2020)
    kw = dict(tol=1e-10, restart_m=2, max_restarts=0, sap_prec="f32")
    with pytest.raises(q.QddError) as e:
        q.qdd_solve(g, b, **kw)
    assert e.value.status == q.QDD_ENOCONV
    x, rep = q.qdd_solve(g, b, allow_noconv=True, **kw)
    assert not rep["converged"] and rep["iters"] == 2 and rep["restarts"] == 0
    r = b - ora.apply_D(L, U, A, 0.12, x)
    true = np.linalg.norm(r) / np.linalg.norm(b)
    assert 1e-10 < true < 1e-1  # progress, but not the tolerance
    assert abs(rep["true_rel_res"] - true) <= 1e-6 * true


def test_non_finite_source_is_reported_and_the_gauge_stays_usable(setup, ora):
    q, g, U, A = setup
    b = inputs.gaussian_source(L, 2021)
    bad = b.copy()
    bad[17, 2, 1] = np.nan
    with pytest.raises(q.QddError) as e:
        q.qdd_solve(g, bad, tol=1e-10, sap_prec="f32")
    assert e.value.status == q.QDD_ENAN
    bad[17, 2, 1] = np.inf
    with pytest.raises(q.QddError) as e:
        q.qdd_solve(g, bad, tol=1e-10, sap_prec="f32")
    assert e.value.status == q.QDD_ENAN
    x, rep = q.qdd_solve(g, b, tol=1e-10, sap_prec="f32")
    assert rep["converged"]
    r = b - ora.apply_D(L, U, A, 0.12, x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
