"""GPU parity of the paired-thread Schwarz kernel (form 3 of
qdd_set_schwarz_variant: two threads per even/odd site pair, each with two
of the four directions and one clover block) against the FP64 oracle.

It runs where the half domain fills whole warps: 4^4 domains (128 threads
per half), 8x4^3 domains (256) and 4x4x2x2 domains (32); with FP32 links it
is also the default form (0).  On other shapes the one-thread form runs.

The checks are those of the one-thread form: per site against the oracle
(test_gpu_parity's tolerances), the residual the sweeps maintain equal to
eta - D psi, several right-hand sides each equal to its single-source
result bit for bit, nmr = 0, and a mixed-precision solve to a true FP64
residual of 1e-10.  Against the one-thread form (form 2, same storage) the
outputs agree to the rounding of FP32 arithmetic: the two partial hop sums
and the MR dot products are added in another order.
"""
import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

from test_gpu_parity import check, problem, rel, site_err

pytestmark = pytest.mark.gpu

PAIR_GEOMS = [
    ((8, 8, 8, 8), (4, 4, 4, 4)),    # 128-site half domains (the 16-bit workloads' shape)
    ((16, 8, 8, 8), (8, 4, 4, 4)),   # 256-site half domains (the FP32 workload's shape)
    ((8, 8, 4, 4), (4, 4, 2, 2)),    # 32-site half domains: one warp per half
]
LOWP_TOL = {"f32": 2e-5, "h16": 5e-3, "f16": 1e-2, "bf16": 6e-2}


@pytest.fixture(scope="module")
def q():
    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import qdd

    return qdd


@pytest.fixture(scope="module")
def ctx(q):
    return q.qdd_create(0, 0)


class form:
    """Run a block with the given Schwarz kernel form on a gauge field."""

    def __init__(self, q, g, variant):
        self.q, self.g, self.v = q, g, variant

    def __enter__(self):
        self.q.qdd_set_schwarz_variant(self.g, self.v)

    def __exit__(self, *exc):
        self.q.qdd_set_schwarz_variant(self.g, 0)


@pytest.mark.parametrize("prec", ["f32", "h16", "f16", "bf16"])
@pytest.mark.parametrize("L,dom", PAIR_GEOMS)
def test_pair_form_matches_oracle(q, ctx, ora, L, dom, prec):
    P = problem(q, ctx, ora, L, dom)
    eta = inputs.gaussian_source(L, 3002)
    psi_o, _ = ora.sap(L, dom, P.U, P.A, P.Ainv, P.kappa, eta, 4, 8)
    with form(q, P.g, 3):
        psi = q.qdd_sap_apply(P.g, eta, 4, 8, prec)
    with form(q, P.g, 2):
        psi1 = q.qdd_sap_apply(P.g, eta, 4, 8, prec)
    tol = LOWP_TOL[prec]
    check(psi, psi_o, tol, 4 * tol, f"sap pair {prec} {L}")
    # against the one-thread form: rounding of the FP32 arithmetic only
    d = rel(psi, psi1)
    print(f"PAIR {prec} {L}: |psi_pair - psi_one_thread| / |psi_one_thread| = {d:.2e}")
    assert d <= (2e-6 if prec == "f32" else tol / 4)


@pytest.mark.parametrize("L,dom", PAIR_GEOMS)
def test_pair_form_residual_and_multi_rhs(q, ctx, ora, L, dom):
    P = problem(q, ctx, ora, L, dom)
    eta = np.ascontiguousarray(inputs.gaussian_source(L, 3004, nrhs=2))
    with form(q, P.g, 3):
        psi, rho = q.qdd_sap_apply(P.g, eta, 4, 8, "f32", nrhs=2, want_rho=True)
        singles = [q.qdd_sap_apply(P.g, np.ascontiguousarray(eta[r]), 4, 8, "f32", want_rho=True) for r in range(2)]
    for r in range(2):
        res = eta[r] - ora.apply_D(L, P.U, P.A, P.kappa, psi[r])
        assert np.linalg.norm(rho[r] - res) <= 2e-5 * np.linalg.norm(eta[r])
        assert site_err(rho[r] - res + eta[r], eta[r]) <= 8e-5
        assert np.array_equal(singles[r][0], psi[r]) and np.array_equal(singles[r][1], rho[r])


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_pair_form_nmr_zero_and_one(q, ctx, ora, prec):
    P = problem(q, ctx, ora, (8, 8, 8, 8), (4, 4, 4, 4))
    eta = inputs.gaussian_source(P.L, 3003)
    for nmr in (0, 1):
        psi_o, _ = ora.sap(P.L, P.dom, P.U, P.A, P.Ainv, P.kappa, eta, nmr, 4)
        with form(q, P.g, 3):
            psi = q.qdd_sap_apply(P.g, eta, nmr, 4, prec)
        tol = LOWP_TOL[prec]
        check(psi, psi_o, tol, 4 * tol, f"sap pair {prec} nmr {nmr}")


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
def test_pair_form_solve(q, ctx, ora, prec):
    P = problem(q, ctx, ora, (8, 8, 8, 8), (4, 4, 4, 4))
    b = inputs.gaussian_source(P.L, 2001)
    with form(q, P.g, 3):
        x, rep = q.qdd_solve(P.g, b, tol=1e-10, sap_prec=prec, arnoldi_prec="df64", relax_eta=1e-6)
    with form(q, P.g, 2):
        _, rep1 = q.qdd_solve(P.g, b, tol=1e-10, sap_prec=prec, arnoldi_prec="df64", relax_eta=1e-6)
    r = b - ora.apply_D(P.L, P.U, P.A, P.kappa, x)
    res = np.linalg.norm(r) / np.linalg.norm(b)
    print(f"PAIR solve {prec}: {rep['iters']} iterations (one-thread form: {rep1['iters']}), true residual {res:.2e}")
    assert rep["converged"] and res <= 1e-10
    assert abs(rep["iters"] - rep1["iters"]) <= 1
