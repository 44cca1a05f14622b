"""Parity at the full sizes of the two largest workloads, on sampled sites.

32^3x64 (eps 0.7, c_sw 1.5, kappa 0.1355; FP16-stored Schwarz, 12 point
sources) and 48^3x96 (the same couplings; BF16-stored Schwarz, one Z2
source), 4^4 domains, in the launch configuration the benchmark times.  The
FP64 oracle cannot apply the operator to a whole 48^3x96 field, let alone
solve it, in test time; it evaluates D at sampled sites instead
(apply_D_sites, the clover built per site from the links), which is enough
for:
  * the operator in every storage the solves use (FP64, double-float, FP32,
    the workload's 16-bit storage): per site and in the 2-norm over the
    sample, with the tolerances of tests/test_gpu_parity.py;
  * the Schwarz method: the residual it maintains equals eta - D psi at the
    sampled sites (FP32 storage), and the 16-bit run's output agrees with
    the FP32 one site by site;
  * the solve: every right-hand side's residual b - D x, evaluated by the
    oracle at the sampled sites (and at the point sources' site), is below
    1e-10 |b| both in the 2-norm over the sample and at every sampled site.
"""
import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = {
    "32^3x64 f16 12 point sources": dict(L=(32, 32, 32, 64), dom=(4, 4, 4, 4), eps=0.7, csw=1.5, kappa=0.1355,
                                         gauge_seed=1003, source_seed=2003, sap_prec="f16", source="point12"),
    "48^3x96 bf16 z2": dict(L=(48, 48, 48, 96), dom=(4, 4, 4, 4), eps=0.7, csw=1.5, kappa=0.1355,
                            gauge_seed=1004, source_seed=2004, sap_prec="bf16", source="z2"),
}
NSITES = 512
TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-5, "f16": 4e-3, "bf16": 3e-2}
SITE_TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-5, "f16": 24 * 2.0 ** -11, "bf16": 24 * 2.0 ** -8}


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def site_err(got, want):
    g = np.asarray(got).reshape(-1, 12)
    w = np.asarray(want).reshape(-1, 12)
    num = np.abs(g - w).max(1)
    den = np.abs(w).max(1)
    return float((num / np.maximum(den, 1e-3 * den.max())).max())


@pytest.fixture(scope="module")
def q():
    from paper_1502_04025_gb300 import build

    build.build()
    from paper_1502_04025_gb300 import qdd

    return qdd


class Big:
    def __init__(self, q, name, c):
        self.q, self.name, self.c = q, name, c
        self.L = c["L"]
        self.V = inputs.volume(self.L)
        self.ctx = q.qdd_create(0, 0)
        self.U = inputs.gauge_field(self.L, c["eps"], c["gauge_seed"])
        self.g = q.qdd_create_gauge_field(self.ctx, self.L, c["dom"], self.U)
        q.qdd_set_clover(self.g, c["csw"], c["kappa"])
        rng = np.random.Generator(np.random.Philox(4242))
        self.sites = np.sort(np.unique(np.concatenate(
            [[0], rng.choice(self.V, size=NSITES, replace=False)])))

    def D_at_sites(self, ora, x):
        return ora.apply_D_sites(self.L, self.U, self.c["csw"], self.c["kappa"], x, self.sites)

    def close(self):
        self.q.qdd_destroy_gauge(self.g)
        self.q.qdd_destroy(self.ctx)


@pytest.fixture(scope="module", params=list(CASES))
def big(request, q):
    b = Big(q, request.param, CASES[request.param])
    yield b
    b.close()


def test_operator_at_sampled_sites(big, ora):
    q = big.q
    x = inputs.gaussian_source(big.L, big.c["source_seed"])
    want = big.D_at_sites(ora, x)
    for prec in ("f64", "df64", "f32", big.c["sap_prec"]):
        got = q.qdd_apply_D(big.g, x, prec)[big.sites]
        e_g, e_s = rel(got, want), site_err(got, want)
        print(f"PARITY fullsize {big.name} dslash {prec} global {e_g:.3e} site {e_s:.3e}")
        assert e_g <= TOL[prec] and e_s <= SITE_TOL[prec], (prec, e_g, e_s)


def test_schwarz_residual_and_storage_at_sampled_sites(big, ora):
    q = big.q
    eta = inputs.gaussian_source(big.L, big.c["source_seed"] + 100)
    psi32, rho32 = q.qdd_sap_apply(big.g, eta, 4, 8, "f32", want_rho=True)
    # the maintained residual is eta - D psi (FP32 arithmetic and storage)
    res = eta[big.sites] - big.D_at_sites(ora, psi32)
    e = site_err(rho32[big.sites] - res + eta[big.sites], eta[big.sites])
    r_norm = np.linalg.norm(rho32[big.sites]) / np.linalg.norm(eta[big.sites])
    print(f"PARITY fullsize {big.name} schwarz f32 residual identity site {e:.3e} (|rho|/|eta| {r_norm:.3e})")
    assert e <= 1e-5 and r_norm < 0.5
    # the workload's 16-bit storage against FP32, site by site
    p = big.c["sap_prec"]
    psi16 = q.qdd_sap_apply(big.g, eta, 4, 8, p)
    e_g, e_s = rel(psi16[big.sites], psi32[big.sites]), site_err(psi16[big.sites], psi32[big.sites])
    tol = {"f16": 1e-2, "bf16": 6e-2}[p]
    print(f"PARITY fullsize {big.name} schwarz {p} vs f32 global {e_g:.3e} site {e_s:.3e}")
    assert e_g <= tol and e_s <= 4 * tol


def test_solve_residual_at_sampled_sites(big, ora):
    q = big.q
    c = big.c
    if c["source"] == "point12":
        b = np.ascontiguousarray(inputs.point_sources(big.L))
    else:
        b = inputs.z2_source(big.L, c["source_seed"])
    nrhs = 12 if c["source"] == "point12" else 1
    x, rep = q.qdd_solve(big.g, b, tol=1e-10, restart_m=16, nmr=4, ncy=4, sap_prec=c["sap_prec"],
                         arnoldi_prec="df64", relax_eta=1e-6, reorth=0, nrhs=nrhs, max_restarts=200)
    assert rep["converged"] and rep["true_rel_res"] <= 1e-10
    bs, xs = b.reshape(nrhs, big.V, 4, 3), x.reshape(nrhs, big.V, 4, 3)
    worst_norm = worst_site = 0.0
    for r in range(nrhs):
        res = bs[r][big.sites] - big.D_at_sites(ora, xs[r])
        bn = np.linalg.norm(bs[r])
        worst_norm = max(worst_norm, np.linalg.norm(res) / bn)
        worst_site = max(worst_site, np.sqrt((np.abs(res.reshape(-1, 12)) ** 2).sum(1)).max() / bn)
    print(f"PARITY fullsize {big.name} solve iters {rep['iters']} reported {rep['true_rel_res']:.3e} "
          f"sampled |r_S|/|b| {worst_norm:.3e} worst site {worst_site:.3e}")
    assert worst_norm <= 1e-10 and worst_site <= 1e-10


def test_solve_16c32_iterations_match_the_oracle():
    """The 16^3x32 workload (FP32 Schwarz on 8x4^3 domains, FP64 outer) takes
    the FP64 oracle's SAP-FGMRES iteration count within one (stored in
    oracle/iterations_16c32.json by oracle/measure_iterations.py, which runs
    only the oracle), and its true residual meets the tolerance."""
    import json
    import os

    from paper_1502_04025_gb300 import build, inputs

    build.build()
    from paper_1502_04025_gb300 import qdd

    with open(os.path.join(os.path.dirname(__file__), "..", "oracle", "iterations_16c32.json")) as f:
        ref = json.load(f)
    w = ref["workload"]
    L, dom = tuple(w["L"]), tuple(w["dom"])
    ctx = qdd.qdd_create(0, 0)
    g = qdd.qdd_create_gauge_field(ctx, L, dom, inputs.gauge_field(L, w["eps"], w["gauge_seed"]))
    try:
        qdd.qdd_set_clover(g, w["csw"], w["kappa"])
        b = inputs.gaussian_source(L, w["source_seed"])
        x, rep = qdd.qdd_solve(g, b, tol=w["tol"], restart_m=w["m"], nmr=w["nmr"], ncy=w["ncy"], sap_prec="f32",
                               arnoldi_prec="df64", relax_eta=1e-6)
        print(f"16^3x32: {rep['iters']} iterations (oracle {ref['iterations']}), true residual "
              f"{rep['true_rel_res']:.2e} (oracle {ref['true_rel_res']:.2e})")
        assert rep["converged"] and rep["true_rel_res"] <= w["tol"]
        assert abs(rep["iters"] - ref["iterations"]) <= 1
        # the estimated residual history follows the oracle's, step by step, to the
        # FP32 preconditioner's rounding
        hist = rep["history"][: len(ref["history"]) - 1]
        for k, (h, r) in enumerate(zip(hist, ref["history"])):
            assert abs(h - r) <= 1e-3 * r + 1e-12, (k, h, r)
    finally:
        qdd.qdd_destroy_gauge(g)
        qdd.qdd_destroy(ctx)
