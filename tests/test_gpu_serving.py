"""Serving loop: requests on different lattices, kappa values and numbers of
right-hand sides, submitted together, overlap on the device and are batched
where they share a gauge field; every result equals the one the same request
gets alone.  Admission by the HBM budget rejects what can never fit."""
import time

import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import qdd

    return qdd


def _gauge(q, ctx, L, dom, eps, seed, csw, kappa):
    U = inputs.gauge_field(L, eps, seed)
    g = q.qdd_create_gauge_field(ctx, L, dom, U)
    q.qdd_set_clover(g, csw, kappa)
    return g, U


def test_results_same_alone_and_in_the_mix(q, ora):
    ctx = q.qdd_create(0, 0)
    q.qdd_serve_config(ctx, 3)
    L1, d1 = (8, 8, 8, 8), (4, 4, 4, 4)
    L2, d2 = (16, 8, 8, 8), (8, 4, 4, 4)
    gA, UA = _gauge(q, ctx, L1, d1, 0.5, 1001, 1.0, 0.120)
    gB, _ = _gauge(q, ctx, L1, d1, 0.5, 1001, 1.0, 0.130)   # same links, other kappa
    gC, UC = _gauge(q, ctx, L2, d2, 0.5, 1004, 1.0, 0.125)
    p = q.qdd_default_params(tol=1e-10, sap_prec="f32")
    reqs = []
    for k, (g, L, nrhs, seed) in enumerate([(gA, L1, 1, 2101), (gB, L1, 2, 2102), (gC, L2, 1, 2103),
                                             (gA, L1, 3, 2104), (gC, L2, 2, 2105), (gA, L1, 1, 2106),
                                             (gB, L1, 1, 2107)]):
        b = inputs.gaussian_source(L, seed, nrhs=nrhs)
        b = np.ascontiguousarray(b)
        reqs.append((g, L, nrhs, b))
    alone = []
    for g, L, nrhs, b in reqs:
        pr = q.qdd_default_params(tol=1e-10, sap_prec="f32", nrhs=nrhs)
        x, rep = q.qdd_solve(g, b, pr)
        assert rep["converged"]
        alone.append(x)
    # submit everything at once; same-gauge requests get batched
    xs, tickets = [], []
    t0 = time.perf_counter()
    for g, L, nrhs, b in reqs:
        pr = q.qdd_default_params(tol=1e-10, sap_prec="f32", nrhs=nrhs)
        x = np.zeros_like(b)
        xs.append(x)
        tickets.append(q.qdd_submit(ctx, g, b, x, pr))
    lat = []
    for t in tickets:
        st, rep = q.qdd_poll(ctx, t, 60.0)
        assert st == q.QDD_OK, q.qdd_last_error()
        assert rep["converged"] and rep["true_rel_res"] <= 1e-10
        lat.append(rep["seconds"])
    assert time.perf_counter() - t0 < 60
    for x, xa in zip(xs, alone):
        assert np.array_equal(x, xa)
    # and the answers are right: residual through the oracle for two of them
    A = ora.clover(L1, UA, 1.0, 0.12)
    b0 = reqs[0][3]
    r = b0 - ora.apply_D(L1, UA, A, 0.12, xs[0])
    assert np.linalg.norm(r) / np.linalg.norm(b0) <= 1e-10
    AC = ora.clover(L2, UC, 1.0, 0.125)
    b2 = reqs[2][3]
    r = b2 - ora.apply_D(L2, UC, AC, 0.125, xs[2])
    assert np.linalg.norm(r) / np.linalg.norm(b2) <= 1e-10
    for g in (gA, gB, gC):
        q.qdd_destroy_gauge(g)
    q.qdd_destroy(ctx)


def test_admission_rejects_what_cannot_fit(q):
    L, dom = (8, 8, 8, 8), (4, 4, 4, 4)
    U = inputs.gauge_field(L, 0.5, 1001)
    # a budget that holds the gauge field and clover but no Krylov workspace
    ctx = q.qdd_create(0, 60 << 20)
    g = q.qdd_create_gauge_field(ctx, L, dom, U)
    q.qdd_set_clover(g, 1.0, 0.12)
    used, budget = q.qdd_memory(ctx)
    assert used <= budget
    b = np.ascontiguousarray(inputs.gaussian_source(L, 2001, nrhs=12))
    x = np.zeros_like(b)
    t = q.qdd_submit(ctx, g, b, x, q.qdd_default_params(nrhs=12, restart_m=64))
    st, _ = q.qdd_poll(ctx, t, 30.0)
    assert st == q.QDD_EBUDGET
    # the synchronous path reports the same budget error
    with pytest.raises(q.QddError) as e:
        q.qdd_solve(g, b, q.qdd_default_params(nrhs=12, restart_m=64))
    assert e.value.status == q.QDD_EBUDGET
    q.qdd_destroy_gauge(g)
    q.qdd_destroy(ctx)


def test_autotune_picks_a_converged_shape(q, ora):
    """The autotuner times every candidate and returns the fastest converged
    one; shapes the geometry rules reject are logged and skipped."""
    ctx = q.qdd_create(0, 0)
    L = (16, 8, 8, 8)
    U = inputs.gauge_field(L, 0.5, 1001)
    b = inputs.gaussian_source(L, 2001)
    p = q.qdd_default_params(tol=1e-10, sap_prec="f32")
    cands = [(4, 4, 4, 4), (8, 4, 4, 4), (4, 2, 2, 2), (16, 4, 4, 4)]  # the last leaves one block in x
    res, log = q.qdd_autotune(ctx, L, U, 1.0, 0.125, b, p, cands, nmr_candidates=(2, 4))
    timed = [c for c in log if "ms" in c]
    assert res["n_tried"] == len(timed) and len(timed) >= 4
    assert any("error" in c for c in log)
    best = min((c for c in timed if c["converged"]), key=lambda c: c["ms"])
    assert tuple(best["dom"]) == res["dom"] and best["nmr"] == res["nmr"]
    for c in timed:
        assert 0 < c["wave_load"] <= 1
    # the chosen setting solves the problem
    g = q.qdd_create_gauge_field(ctx, L, res["dom"], U)
    q.qdd_set_clover(g, 1.0, 0.125)
    x, rep = q.qdd_solve(g, b, q.qdd_default_params(tol=1e-10, sap_prec="f32", nmr=res["nmr"]))
    A = ora.clover(L, U, 1.0, 0.125)
    r = b - ora.apply_D(L, U, A, 0.125, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    q.qdd_destroy_gauge(g)
    q.qdd_destroy(ctx)


def test_poll_unknown_ticket_and_timeout(q):
    ctx = q.qdd_create(0, 0)
    st, _ = q.qdd_poll(ctx, 12345, 0.0)
    assert st == q.QDD_EINVAL
    q.qdd_destroy(ctx)
