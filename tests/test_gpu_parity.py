"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
the same seeded inputs.

Every comparison is made per site: the largest component error at a site,
relative to the largest component of the expected value at that site
(site_err), so that one wrong site cannot hide in a global norm.  The
relative 2-norm over the whole output (rel) is checked as well.

Tolerances.  Per site (SITE_TOL), from the rounding of the stored operands:
a site's output is the clover term (6x6 blocks, 6 products per component)
plus 8 hops of kappa (1 -+ gamma) U x (3 products per colour, two spin
components), so its error is at most about (12 + 8 * 12 * kappa) u ~ 24 u
times the site's scale, u the unit roundoff of the stored links, clover
and spinors (2^-24 FP32, 2^-11 FP16, 2^-8 BF16; FP16 links/clover with
FP32 spinors: about 12 u).  Over the whole output (TOL):
  FP64 arithmetic            1e-12  (rounding order only)
  double-float (FP32 pairs)  1e-12  (links, clover, input split to 2x24 bits; ~2^-46 per operation)
  FP32 arithmetic            1e-5   (the operator-apply bound of the target)
  FP16 links/clover, FP32 spinors  2e-3  (2^-11 per link/clover component)
  FP16 storage + FP32 arith  4e-3   (2^-11 per stored component, ~10 terms)
  BF16 storage + FP32 arith  3e-2   (2^-8 per stored component)
"""
import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-5, "h16": 2e-3, "f16": 4e-3, "bf16": 3e-2}
SITE_TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-5, "h16": 12 * 2.0 ** -11, "f16": 24 * 2.0 ** -11,
            "bf16": 24 * 2.0 ** -8}


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def site_err(got, want, ncomp=12):
    """Max over sites of (max component |got - want|) / (max component |want|)
    at that site (ncomp components per site: 12 for a spinor, 144 for the
    clover matrix); sites whose expected value is below 1e-3 of the field's
    largest are measured against that floor instead."""
    g = np.asarray(got).reshape(-1, ncomp)
    w = np.asarray(want).reshape(-1, ncomp)
    num = np.abs(g - w).max(1)
    den = np.abs(w).max(1)
    return float((num / np.maximum(den, 1e-3 * den.max())).max())


def check(got, want, tol_global, tol_site, what=""):
    e_g, e_s = rel(got, want), site_err(got, want)
    print(f"PARITY {what} global {e_g:.3e} (tol {tol_global:.1e}) site {e_s:.3e} (tol {tol_site:.1e})")
    assert e_g <= tol_global and e_s <= tol_site, (what, e_g, e_s)


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


class Problem:
    def __init__(self, q, ctx, ora, L, dom, eps, csw, kappa, seed):
        self.L, self.dom, self.csw, self.kappa = L, dom, csw, kappa
        self.V = inputs.volume(L)
        self.U = inputs.gauge_field(L, eps, seed)
        self.g = q.qdd_create_gauge_field(ctx, L, dom, self.U)
        q.qdd_set_clover(self.g, csw, kappa)
        self.A = ora.clover(L, self.U, csw, kappa)
        self.Ainv = ora.invert_clover(L, self.A)


_problems = {}


def problem(q, ctx, ora, L, dom, eps=0.5, csw=1.0, kappa=0.12, seed=1001):
    key = (tuple(L), tuple(dom), eps, csw, kappa, seed)
    if key not in _problems:
        _problems[key] = Problem(q, ctx, ora, L, dom, eps, csw, kappa, seed)
    return _problems[key]


GEOMS = [
    ((8, 8, 8, 8), (4, 4, 4, 4)),      # config-1 geometry: 16 domains of 256 sites
    ((4, 4, 4, 4), (2, 2, 2, 2)),      # 8-site half domains: partial-warp reductions
    ((8, 4, 4, 12), (4, 2, 2, 2)),     # ragged: 6 blocks in t, 32-site domains
    ((16, 8, 8, 8), (8, 4, 4, 4)),     # 8x4^3 domains of 512 sites (config-2 shape)
    ((12, 8, 4, 4), (6, 4, 2, 2)),     # 48-site half domains: one and a half warps per domain
]


@pytest.mark.parametrize("L,dom", GEOMS)
def test_clover_matches_oracle(q, ctx, ora, L, dom):
    P = problem(q, ctx, ora, L, dom, eps=0.7, csw=1.5, kappa=0.1355)
    blocks = q.qdd_get_clover(P.g, P.V, 0)
    full = np.zeros((P.V, 12, 12), dtype=np.complex128)
    full[:, :6, :6] = blocks[:, 0]
    full[:, 6:, 6:] = blocks[:, 1]
    assert rel(full, P.A) <= 1e-13 and site_err(full, P.A, 144) <= 1e-13
    # Schwarz form: A on even sites, A^{-1} on odd sites
    sform = q.qdd_get_clover(P.g, P.V, 1)
    sfull = np.zeros_like(full)
    sfull[:, :6, :6] = sform[:, 0]
    sfull[:, 6:, 6:] = sform[:, 1]
    c = np.stack(np.unravel_index(np.arange(P.V), L[::-1]), 1)[:, ::-1]
    odd = (c.sum(1) % 2) == 1
    assert rel(sfull[~odd], P.A[~odd]) <= 1e-13 and site_err(sfull[~odd], P.A[~odd], 144) <= 1e-13
    assert rel(sfull[odd], P.Ainv[odd]) <= 1e-12 and site_err(sfull[odd], P.Ainv[odd], 144) <= 1e-12


@pytest.mark.parametrize("L,dom", GEOMS)
@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "h16", "f16", "bf16"])
def test_dslash_matches_oracle(q, ctx, ora, L, dom, prec):
    P = problem(q, ctx, ora, L, dom)
    x = inputs.gaussian_source(L, 2001)
    want = ora.apply_D(L, P.U, P.A, P.kappa, x)
    got = q.qdd_apply_D(P.g, x, prec)
    check(got, want, TOL[prec], SITE_TOL[prec], f"dslash {L} {prec}")
    if prec in ("f64", "df64"):
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("prec", ["f32", "h16", "f16", "bf16"])
def test_two_row_links_match_whole_links(q, ctx, ora, prec):
    """SU(3) links: the FP32/16-bit operator rebuilds each link's third row
    from the first two; it matches the oracle and the whole-link kernel."""
    P = problem(q, ctx, ora, (16, 8, 8, 8), (8, 4, 4, 4), seed=1003)
    assert q.qdd_link_compression(P.g) == (True, True)
    x = inputs.gaussian_source(P.L, 2003)
    want = ora.apply_D(P.L, P.U, P.A, P.kappa, x)
    two = q.qdd_apply_D(P.g, x, prec)
    q.qdd_set_link_compression(P.g, False)
    try:
        assert q.qdd_link_compression(P.g) == (False, True)
        three = q.qdd_apply_D(P.g, x, prec)
    finally:
        q.qdd_set_link_compression(P.g, True)
    check(two, want, TOL[prec], SITE_TOL[prec], f"two rows {prec}")
    check(three, want, TOL[prec], SITE_TOL[prec], f"three rows {prec}")
    # the rebuilt row differs from the stored one by the storage rounding of the first two
    assert rel(two, three) <= {"f32": 1e-6, "h16": 2e-3, "f16": 4e-3, "bf16": 3e-2}[prec]
    assert site_err(two, three) <= SITE_TOL[prec]


def test_links_that_are_not_su3_keep_three_rows(q, ctx, ora):
    L, dom = (8, 8, 8, 8), (4, 4, 4, 4)
    U = inputs.gauge_field(L, 0.5, 1004)
    rng = np.random.default_rng(7)
    U = U * (1.0 + 1e-3 * rng.standard_normal(U.shape[:-2] + (1, 1)))  # unitary no more
    g = q.qdd_create_gauge_field(ctx, L, dom, np.ascontiguousarray(U))
    try:
        q.qdd_set_clover(g, 1.0, 0.12)
        assert q.qdd_link_compression(g) == (False, False)
        with pytest.raises(q.QddError):
            q.qdd_set_link_compression(g, True)
        A = ora.clover(L, U, 1.0, 0.12)
        x = inputs.gaussian_source(L, 2004)
        check(q.qdd_apply_D(g, x, "f32"), ora.apply_D(L, U, A, 0.12, x), TOL["f32"], SITE_TOL["f32"], "not su3")
    finally:
        q.qdd_destroy_gauge(g)


@pytest.mark.parametrize("prec,half_ulp", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_16bit_storage_round_trip_bound(q, ctx, prec, half_ulp):
    """With kappa = 0 the operator is the identity (A = 1, hops scaled by 0), so a
    16-bit apply returns its input rounded twice (stored with a per-site scale
    = max |component|, round to nearest; then the output likewise): every
    component lies within 2 half-ulps of the site's scale of the input."""
    L, dom = (8, 8, 8, 8), (4, 4, 4, 4)
    g = q.qdd_create_gauge_field(ctx, L, dom, inputs.gauge_field(L, 0.5, 1001))
    try:
        q.qdd_set_clover(g, 1.0, 0.0)
        x = inputs.gaussian_source(L, 2031) * np.exp(inputs.gaussian_source(L, 2032).real)[..., :1, :1]
        y = q.qdd_apply_D(g, x, prec)
        scale = np.maximum(np.abs(x.real), np.abs(x.imag)).max(axis=(1, 2))
        err = np.maximum(np.abs((y - x).real), np.abs((y - x).imag)).max(axis=(1, 2))
        assert (err <= (2 * half_ulp + 1e-6) * scale).all()
        assert (err > 0).any()  # the storage really is 16-bit
        y64 = q.qdd_apply_D(g, x, "f64")
        assert np.abs(y64 - x).max() <= 1e-15 * np.abs(x).max()
    finally:
        q.qdd_destroy_gauge(g)


def test_dslash_multi_rhs(q, ctx, ora):
    P = problem(q, ctx, ora, (8, 8, 8, 8), (4, 4, 4, 4))
    xs = inputs.gaussian_source(P.L, 2002, nrhs=3)
    got = q.qdd_apply_D(P.g, np.ascontiguousarray(xs), "f64", nrhs=3)
    for r in range(3):
        check(got[r], ora.apply_D(P.L, P.U, P.A, P.kappa, xs[r]), TOL["f64"], SITE_TOL["f64"], "multi rhs")


@pytest.mark.parametrize("L,dom", GEOMS)  # the 8x4^3 shape runs with the FP64 links unstaged (295 KB)
@pytest.mark.parametrize("n_half", [1, 2, 5, 8])
def test_sap_f64_matches_oracle(q, ctx, ora, L, dom, n_half):
    P = problem(q, ctx, ora, L, dom)
    eta = inputs.gaussian_source(L, 3001)
    psi_o, rho_o = ora.sap(L, dom, P.U, P.A, P.Ainv, P.kappa, eta, 4, n_half)
    psi, rho = q.qdd_sap_apply(P.g, eta, 4, n_half, "f64", want_rho=True)
    check(psi, psi_o, 1e-12, 1e-11, f"sap f64 psi {L} {n_half}")
    # the residual at a site is compared with the site's scale of eta (it is small where the block solve converged)
    assert site_err(rho - rho_o + eta, eta) <= 1e-11 and rel(rho, rho_o) <= 1e-11


@pytest.mark.parametrize("prec", ["f32", "h16", "f16", "bf16"])
@pytest.mark.parametrize("L,dom", [GEOMS[0], GEOMS[3], GEOMS[4]])
def test_sap_lowp_matches_oracle(q, ctx, ora, L, dom, prec):
    P = problem(q, ctx, ora, L, dom)
    eta = inputs.gaussian_source(L, 3002)
    psi_o, _ = ora.sap(L, dom, P.U, P.A, P.Ainv, P.kappa, eta, 4, 8)
    psi = q.qdd_sap_apply(P.g, eta, 4, 8, prec)
    # 8 half-sweeps of 4 MR steps: storage rounding enters every step; per site up to 4x the global bound
    tol = {"f32": 2e-5, "h16": 5e-3, "f16": 1e-2, "bf16": 6e-2}[prec]
    check(psi, psi_o, tol, 4 * tol, f"sap {prec} {L}")


@pytest.mark.parametrize("L,dom", [GEOMS[0], GEOMS[1], GEOMS[2], GEOMS[3]])
def test_sap_residual_and_multi_rhs(q, ctx, ora, L, dom):
    """The residual the Schwarz sweeps maintain (with the pending face inflow
    applied to the next colour) equals eta - D psi, and each of several
    right-hand sides gets exactly its single-source result."""
    P = problem(q, ctx, ora, L, dom)
    eta = np.ascontiguousarray(inputs.gaussian_source(L, 3004, nrhs=2))
    psi_o, _ = ora.sap(L, dom, P.U, P.A, P.Ainv, P.kappa, eta[1], 4, 8)
    psi, rho = q.qdd_sap_apply(P.g, eta, 4, 8, "f32", nrhs=2, want_rho=True)
    check(psi[1], psi_o, 2e-5, 8e-5, f"sap f32 rhs 1 {L}")
    for r in range(2):
        res = eta[r] - ora.apply_D(L, P.U, P.A, P.kappa, psi[r])
        assert np.linalg.norm(rho[r] - res) <= 2e-5 * np.linalg.norm(eta[r])
        assert site_err(rho[r] - res + eta[r], eta[r]) <= 8e-5
        psi1, rho1 = q.qdd_sap_apply(P.g, np.ascontiguousarray(eta[r]), 4, 8, "f32", want_rho=True)
        assert np.array_equal(psi1, psi[r]) and np.array_equal(rho1, rho[r])


def test_sap_nmr_zero_and_multi_rhs(q, ctx, ora):
    P = problem(q, ctx, ora, (8, 8, 8, 8), (4, 4, 4, 4))
    etas = inputs.gaussian_source(P.L, 3003, nrhs=2)
    for nmr in (0, 1):
        psi = q.qdd_sap_apply(P.g, np.ascontiguousarray(etas), nmr, 4, "f64", nrhs=2)
        for r in range(2):
            psi_o, _ = ora.sap(P.L, P.dom, P.U, P.A, P.Ainv, P.kappa, etas[r], nmr, 4)
            check(psi[r], psi_o, 1e-12, 1e-11, f"sap nmr {nmr}")


def _true_rel(ora, P, x, b):
    r = b - ora.apply_D(P.L, P.U, P.A, P.kappa, x)
    return np.linalg.norm(r) / np.linalg.norm(b)


def test_solve_config1_fp64(q, ctx, ora):
    """8^4, eps 0.5, c_sw 1.0, kappa 0.12, 4^4 domains, nmr 4, ncy 4,
    FGMRES(16), tol 1e-10, all FP64."""
    P = problem(q, ctx, ora, (8, 8, 8, 8), (4, 4, 4, 4))
    b = inputs.gaussian_source(P.L, 2001)
    x, rep = q.qdd_solve(P.g, b, tol=1e-10, restart_m=16, nmr=4, ncy=4, sap_prec="f64")
    assert rep["converged"] and rep["true_rel_res"] <= 1e-10
    assert _true_rel(ora, P, x, b) <= 1e-10
    x_o, info = ora.fgmres(P.L, P.dom, P.U, P.A, P.Ainv, P.kappa, b, 1e-12, m=16, max_restarts=50, use_sap=True,
                           nmr=4, ncy=4)
    assert info["converged"]
    x2, rep2 = q.qdd_solve(P.g, b, tol=1e-12, restart_m=16, nmr=4, ncy=4, sap_prec="f64")
    check(x2, x_o, 1e-9, 1e-8, "solve 8^4 f64")
    # same method, same iteration count up to the Gram-Schmidt variant
    assert abs(rep2["iters"] - info["iters"]) <= 2


@pytest.mark.parametrize("prec,arn", [("f32", "f64"), ("f16", "f64"), ("bf16", "f64"), ("f32", "f32"),
                                      ("f32", "df64"), ("f64", "df64"), ("h16", "df64")])
def test_solve_mixed_precision(q, ctx, ora, prec, arn):
    P = problem(q, ctx, ora, (16, 8, 8, 8), (8, 4, 4, 4), kappa=0.125)
    b = inputs.gaussian_source(P.L, 2002)
    x, rep = q.qdd_solve(P.g, b, tol=1e-10, sap_prec=prec, arnoldi_prec=arn)
    assert rep["converged"]
    assert _true_rel(ora, P, x, b) <= 1e-10


def test_half_precision_storage_keeps_the_iteration_count(q, ctx, ora):
    """Sec. 3.3: half-precision links and clover (spinors in single precision)
    in the Schwarz method had no noticeable effect on the outer iteration
    count; here that holds within 10% (at least one step) of the FP32
    preconditioner, and for the all-16-bit storages too."""
    P = problem(q, ctx, ora, (16, 8, 8, 8), (8, 4, 4, 4), kappa=0.125)
    b = inputs.gaussian_source(P.L, 2014)
    _, r32 = q.qdd_solve(P.g, b, tol=1e-10, sap_prec="f32")
    for prec in ("h16", "f16", "bf16"):
        _, r = q.qdd_solve(P.g, b, tol=1e-10, sap_prec=prec)
        assert r["converged"]
        assert r["iters"] <= r32["iters"] + max(1, r32["iters"] // 10), (prec, r["iters"], r32["iters"])


def test_solve_df64_arnoldi_same_iterations(q, ctx, ora):
    """The double-float Arnoldi operator keeps the FP64 iteration count."""
    P = problem(q, ctx, ora, (16, 8, 8, 8), (8, 4, 4, 4), kappa=0.125)
    b = inputs.gaussian_source(P.L, 2012)
    x1, r1 = q.qdd_solve(P.g, b, tol=1e-10, sap_prec="f32", arnoldi_prec="f64")
    x2, r2 = q.qdd_solve(P.g, b, tol=1e-10, sap_prec="f32", arnoldi_prec="df64")
    assert r1["iters"] == r2["iters"] and r1["restarts"] == r2["restarts"]
    assert rel(x2, x1) <= 1e-9


def test_solve_relaxed_arnoldi(q, ctx, ora):
    """Relaxed (inexact-Krylov) Arnoldi operator: FP32 once the residual is
    small; still reaches the FP64 true residual with at most one more step."""
    P = problem(q, ctx, ora, (16, 8, 8, 8), (8, 4, 4, 4), kappa=0.125)
    b = inputs.gaussian_source(P.L, 2013)
    x1, r1 = q.qdd_solve(P.g, b, tol=1e-10, sap_prec="f32", arnoldi_prec="f64")
    x2, r2 = q.qdd_solve(P.g, b, tol=1e-10, sap_prec="f32", arnoldi_prec="f64", relax_eta=1e-6)
    assert r2["converged"] and _true_rel(ora, P, x2, b) <= 1e-10
    assert r2["iters"] <= r1["iters"] + 1
    with pytest.raises(q.QddError):
        q.qdd_solve(P.g, b, tol=1e-10, sap_prec="f64", relax_eta=1e-6)


def test_solve_plain_gmres_and_multi_rhs(q, ctx, ora):
    P = problem(q, ctx, ora, (8, 8, 8, 8), (4, 4, 4, 4))
    bs = np.ascontiguousarray(inputs.point_sources(P.L)[:4])
    xb, rep = q.qdd_solve(P.g, bs, tol=1e-10, nrhs=4, sap_prec="f32")
    assert rep["converged"]
    for r in range(4):
        xr, _ = q.qdd_solve(P.g, np.ascontiguousarray(bs[r]), tol=1e-10, nrhs=1, sap_prec="f32")
        assert np.array_equal(xr, xb[r])  # batching does not change any arithmetic
        assert _true_rel(ora, P, xb[r], bs[r]) <= 1e-10
    x0, rep0 = q.qdd_solve(P.g, np.ascontiguousarray(bs[0]), tol=1e-10, use_sap=0, max_restarts=200)
    assert rep0["converged"] and _true_rel(ora, P, x0, bs[0]) <= 1e-10
    assert rep0["iters"] > rep["iters"]


def test_solve_from_page_locked_host_buffers(q, ctx, ora):
    """Host buffers, pageable or page-locked (the bench's end-to-end case),
    give the same bits, also in place (the solution written over the
    source); the source is read only."""
    import torch

    P = problem(q, ctx, ora, (8, 8, 8, 8), (4, 4, 4, 4))
    b = np.ascontiguousarray(inputs.gaussian_source(P.L, 2001, nrhs=2))
    x_staged, rep = q.qdd_solve(P.g, b, tol=1e-10, nrhs=2, sap_prec="f32")
    bp = torch.from_numpy(b).pin_memory()
    xp = torch.zeros_like(bp).pin_memory()
    x_mapped, rep2 = q.qdd_solve(P.g, bp.numpy(), x=xp.numpy(), tol=1e-10, nrhs=2, sap_prec="f32")
    assert rep["converged"] and rep2["iters"] == rep["iters"]
    assert np.array_equal(x_mapped, x_staged) and np.array_equal(xp.numpy(), x_staged)
    assert np.array_equal(bp.numpy(), b)  # the source is read only
    q.qdd_solve(P.g, bp.numpy(), x=bp.numpy(), tol=1e-10, nrhs=2, sap_prec="f32")
    assert np.array_equal(bp.numpy(), x_staged)
    for r in range(2):
        assert _true_rel(ora, P, x_mapped[r], b[r]) <= 1e-10


def test_cdot_multi_matches_numpy(q, ctx):
    import torch

    g = torch.Generator().manual_seed(5)
    n = 100_003  # ragged against the block size
    v = torch.randn(17, n, dtype=torch.complex128, generator=g).cuda()
    w = torch.randn(n, dtype=torch.complex128, generator=g).cuda()
    out = q.qdd_cdot_multi(ctx, v, w).cpu().numpy()
    want = np.conj(v.cpu().numpy()) @ w.cpu().numpy()
    assert np.abs(out - want).max() <= 1e-12 * np.abs(want).max()
