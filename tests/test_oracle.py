"""Pins of the FP64 CPU oracle against what the mathematics fixes.

Every check here compares the oracle with something other than itself:
the Clifford algebra, the closed-form free-field spectrum, the closed-form
clover term of a constant abelian field, gamma_5-hermiticity, gauge
covariance, dense linear algebra (numpy LU / least squares) on small
lattices, and the defining properties of MR, SAP and GMRES.
"""
import numpy as np
import pytest

from paper_1502_04025_gb300 import inputs

L44 = (4, 4, 4, 4)
DOM2 = (2, 2, 2, 2)


def cdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def match_multiset(got, want, tol):
    """Greedy nearest matching of two complex multisets."""
    got = list(got)
    assert len(got) == len(want)
    for w in want:
        i = int(np.argmin(np.abs(np.array(got) - w)))
        assert abs(got[i] - w) < tol, (got[i], w)
        got.pop(i)


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def site_coords(L):
    V = inputs.volume(L)
    n = np.arange(V)
    x = n % L[0]
    y = (n // L[0]) % L[1]
    z = (n // (L[0] * L[1])) % L[2]
    t = n // (L[0] * L[1] * L[2])
    return np.stack([x, y, z, t], axis=1)


def dense_D(ora, L, U, A, kappa):
    V = inputs.volume(L)
    N = 12 * V
    M = np.zeros((N, N), dtype=np.complex128)
    e = np.zeros((V, 4, 3), dtype=np.complex128)
    flat = e.reshape(-1)
    for k in range(N):
        flat[k] = 1.0
        M[:, k] = ora.apply_D(L, U, A, kappa, e).reshape(-1)
        flat[k] = 0.0
    return M


@pytest.fixture(scope="module")
def problem44(ora):
    L = L44
    U = inputs.gauge_field(L, 0.5, 1001)
    csw, kappa = 1.0, 0.12
    A = ora.clover(L, U, csw, kappa)
    Ainv = ora.invert_clover(L, A)
    return dict(L=L, U=U, csw=csw, kappa=kappa, A=A, Ainv=Ainv)


@pytest.fixture(scope="module")
def dense44(ora, problem44):
    p = problem44
    return dense_D(ora, p["L"], p["U"], p["A"], p["kappa"])


# ---------------------------------------------------------------- gammas

def test_gamma_clifford_algebra(ora):
    g = [ora.gamma(m) for m in range(5)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T, atol=0)
        for b in range(4):
            ac = g[a] @ g[b] + g[b] @ g[a]
            assert np.allclose(ac, 2 * np.eye(4) * (a == b), atol=1e-15)
    assert np.allclose(g[4], g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)
    # chiral basis: gamma_5 diagonal, so sigma_{mu nu} is block diagonal
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]), atol=1e-15)
    for a in range(4):
        for b in range(4):
            s = 0.5j * (g[a] @ g[b] - g[b] @ g[a])
            assert np.allclose(s[:2, 2:], 0) and np.allclose(s[2:, :2], 0)


# ------------------------------------------------------------ free field

def _free_eigs(p, kappa):
    c = np.sum(np.cos(p))
    s = np.sqrt(np.sum(np.sin(p) ** 2))
    return 1 - 2 * kappa * c + 2j * kappa * s, 1 - 2 * kappa * c - 2j * kappa * s


@pytest.mark.parametrize("k", [(0, 0, 0, 0), (1, 0, 0, 0), (0, 2, 1, 3), (1, 1, 1, 1), (2, 3, 0, 5)])
def test_free_field_plane_waves(ora, k):
    """U = 1: D maps e^{ip.n} chi to e^{ip.n} D(p) chi, and the 12x12 D(p) has
    eigenvalues 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p), six-fold each."""
    L = (4, 4, 6, 8)
    kappa, csw = 0.11, 1.7  # the clover term vanishes for unit links
    U = inputs.unit_gauge_field(L)
    A = ora.clover(L, U, csw, kappa)
    p = 2 * np.pi * np.array(k) / np.array(L)
    phase = np.exp(1j * site_coords(L) @ p)
    Dp = np.zeros((12, 12), dtype=np.complex128)
    for j in range(12):
        chi = np.zeros(12, dtype=np.complex128)
        chi[j] = 1
        psi = (phase[:, None] * chi[None, :]).reshape(-1, 4, 3)
        out = ora.apply_D(L, U, A, kappa, psi).reshape(-1, 12)
        col = out[0] / phase[0]
        assert np.allclose(out, phase[:, None] * col[None, :], atol=1e-14)
        Dp[:, j] = col
    lp, lm = _free_eigs(p, kappa)
    match_multiset(np.linalg.eigvals(Dp), [lp] * 6 + [lm] * 6, 1e-7)
    # the degenerate eigenvalues perturb like sqrt(eps); the trace and the
    # characteristic moments pin them to full precision
    for k in (1, 2, 3):
        mom = np.trace(np.linalg.matrix_power(Dp, k))
        assert abs(mom - 6 * (lp ** k + lm ** k)) <= 1e-12 * max(1.0, abs(mom))


def test_free_field_dense_spectrum(ora):
    """Dense spectrum of the free operator on a small lattice is the
    closed-form multiset over all lattice momenta."""
    L = (2, 2, 4, 4)
    kappa = 0.13
    U = inputs.unit_gauge_field(L)
    A = ora.clover(L, U, 1.0, kappa)
    M = dense_D(ora, L, U, A, kappa)
    ev = np.linalg.eigvals(M)
    want = []
    for kx in range(L[0]):
        for ky in range(L[1]):
            for kz in range(L[2]):
                for kt in range(L[3]):
                    p = 2 * np.pi * np.array([kx, ky, kz, kt]) / np.array(L)
                    lp, lm = _free_eigs(p, kappa)
                    want += [lp] * 6 + [lm] * 6
    match_multiset(ev, want, 1e-6)


# ---------------------------------------------------------------- clover

def test_clover_unit_links_is_identity(ora):
    L = (4, 4, 4, 4)
    A = ora.clover(L, inputs.unit_gauge_field(L), 1.9, 0.13)
    assert np.allclose(A, np.eye(12)[None], atol=0)


def _abelian_field(L, kflux):
    """Links diag(e^{i th}, e^{-i th}, 1) with a constant plaquette angle
    phi = 2 pi kflux / (Lx Ly) in the (x, y) plane and none elsewhere."""
    V = inputs.volume(L)
    phi = 2 * np.pi * kflux / (L[0] * L[1])
    c = site_coords(L)
    th = np.zeros((V, 4))
    th[:, 1] = phi * c[:, 0]
    last = c[:, 0] == L[0] - 1
    th[last, 0] = -phi * L[0] * c[last, 1]
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = np.exp(1j * th)
    U[:, :, 1, 1] = np.exp(-1j * th)
    U[:, :, 2, 2] = 1
    return U, phi


def test_clover_constant_abelian_field(ora):
    """For a constant abelian field F_xy = i sin(phi) diag(1,-1,0) and all
    other F vanish, so A = 1 - kappa c_sw sin(phi) sigma_xy (x) diag(1,-1,0)."""
    L = (4, 6, 4, 4)
    csw, kappa = 1.3, 0.12
    U, phi = _abelian_field(L, 1)
    A = ora.clover(L, U, csw, kappa)
    g = [ora.gamma(m) for m in range(4)]
    sxy = 0.5j * (g[0] @ g[1] - g[1] @ g[0])
    want = np.eye(12) - kappa * csw * np.sin(phi) * np.kron(sxy, np.diag([1.0, -1.0, 0.0]))
    for n in [0, 5, 17, inputs.volume(L) - 1]:
        assert np.allclose(A[n], want, atol=1e-14)
    F = ora.field_strength(L, U, 7, 0, 1)
    assert np.allclose(F, 1j * np.sin(phi) * np.diag([1, -1, 0]), atol=1e-14)
    for mu, nu in [(0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]:
        assert np.allclose(ora.field_strength(L, U, 7, mu, nu), 0, atol=1e-14)


def test_clover_trace_removed(ora):
    """F_{mu nu} is taken traceless: for the abelian field diag(e^{i th},
    e^{i th}, e^{-2i th}) the plaquette phases give F = i diag(s1, s1, -s2)
    (s1 = sin phi, s2 = sin 2 phi), whose trace is removed before use."""
    L = (4, 6, 4, 4)
    csw, kappa = 1.1, 0.13
    U1, phi = _abelian_field(L, 1)
    th = np.angle(U1[:, :, 0, 0])
    U = np.zeros_like(U1)
    U[:, :, 0, 0] = U[:, :, 1, 1] = np.exp(1j * th)
    U[:, :, 2, 2] = np.exp(-2j * th)
    F0 = 1j * np.diag([np.sin(phi), np.sin(phi), -np.sin(2 * phi)])
    Fhat = F0 - np.trace(F0) / 3 * np.eye(3)
    assert np.allclose(ora.field_strength(L, U, 9, 0, 1), Fhat, atol=1e-14)
    g = [ora.gamma(m) for m in range(4)]
    sxy = 0.5j * (g[0] @ g[1] - g[1] @ g[0])
    want = np.eye(12) + 1j * kappa * csw * np.kron(sxy, Fhat)
    A = ora.clover(L, U, csw, kappa)
    assert np.allclose(A[9], want, atol=1e-14)
    # and for a random SU(3) field every F is traceless
    Ur = inputs.gauge_field(L, 0.8, 5)
    for n in (0, 33, 101):
        for mu, nu in [(0, 1), (1, 3), (2, 3)]:
            assert abs(np.trace(ora.field_strength(L, Ur, n, mu, nu))) < 1e-15


def test_clover_hermitian_and_inverse(ora, problem44):
    A, Ainv = problem44["A"], problem44["Ainv"]
    assert np.allclose(A, np.conj(np.transpose(A, (0, 2, 1))), atol=1e-15)
    prod = np.einsum("nij,njk->nik", A, Ainv)
    assert np.allclose(prod, np.eye(12)[None], atol=1e-13)
    # chirality blocks: no coupling between spins {0,1} and {2,3}
    assert np.allclose(A[:, :6, 6:], 0, atol=0) and np.allclose(A[:, 6:, :6], 0, atol=0)


# ----------------------------------------------------- operator symmetry

def test_gamma5_hermiticity(ora):
    L = (4, 4, 4, 6)
    U = inputs.gauge_field(L, 0.7, 7)
    kappa, csw = 0.13, 1.5
    A = ora.clover(L, U, csw, kappa)
    x = inputs.gaussian_source(L, 11)
    y = inputs.gaussian_source(L, 12)
    g5 = np.array([1, 1, -1, -1])[None, :, None]
    lhs = cdot(y, g5 * ora.apply_D(L, U, A, kappa, x))
    rhs = np.conj(cdot(x, g5 * ora.apply_D(L, U, A, kappa, y)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gauge_covariance(ora):
    L = (4, 4, 6, 4)
    U = inputs.gauge_field(L, 0.6, 21)
    kappa, csw = 0.125, 1.2
    V = inputs.volume(L)
    g = inputs.random_su3((V,), 22)
    c = site_coords(L)
    Ug = np.empty_like(U)
    for mu in range(4):
        cc = c.copy()
        cc[:, mu] = (cc[:, mu] + 1) % L[mu]
        nf = cc[:, 0] + L[0] * (cc[:, 1] + L[1] * (cc[:, 2] + L[2] * cc[:, 3]))
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.transpose(g[nf], (0, 2, 1)))
    x = inputs.gaussian_source(L, 23)
    gx = np.einsum("nab,nsb->nsa", g, x)
    A = ora.clover(L, U, csw, kappa)
    Ag = ora.clover(L, Ug, csw, kappa)
    lhs = ora.apply_D(L, Ug, Ag, kappa, gx)
    rhs = np.einsum("nab,nsb->nsa", g, ora.apply_D(L, U, A, kappa, x))
    assert rel(lhs, rhs) <= 1e-13


def test_apply_D_sites_matches_full(ora, problem44):
    p = problem44
    x = inputs.gaussian_source(p["L"], 31)
    full = ora.apply_D(p["L"], p["U"], p["A"], p["kappa"], x)
    sites = np.array([0, 1, 63, 128, 255])
    part = ora.apply_D_sites(p["L"], p["U"], p["csw"], p["kappa"], x, sites)
    assert np.allclose(part, full[sites], atol=1e-14)


# ------------------------------------------------------------ dense solve

def test_fgmres_plain_matches_dense_lu(ora, problem44, dense44):
    p = problem44
    b = inputs.gaussian_source(p["L"], 2001)
    x_lu = np.linalg.solve(dense44, b.reshape(-1)).reshape(b.shape)
    x, info = ora.fgmres(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], b, 1e-12, m=16,
                         max_restarts=100, use_sap=False)
    assert info["converged"]
    assert info["true_rel_res"] <= 1e-12
    sv = np.linalg.svd(dense44, compute_uv=False)
    cond = sv[0] / sv[-1]
    assert rel(x, x_lu) <= 2 * cond * 1e-12


def test_fgmres_sap_matches_dense_lu(ora, problem44, dense44):
    p = problem44
    b = inputs.gaussian_source(p["L"], 2002)
    x_lu = np.linalg.solve(dense44, b.reshape(-1)).reshape(b.shape)
    x, info = ora.fgmres(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], b, 1e-12, m=16,
                         max_restarts=50, use_sap=True, nmr=4, ncy=4)
    assert info["converged"]
    r = b - ora.apply_D(p["L"], p["U"], p["A"], p["kappa"], x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-12
    assert rel(x, x_lu) <= 1e-10
    # SAP must cut the iteration count against the unpreconditioned solve
    _, info0 = ora.fgmres(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], b, 1e-12, m=16,
                          max_restarts=100, use_sap=False)
    assert info["iters"] < info0["iters"]


def test_gmres_residuals_equal_dense_minimum(ora, problem44, dense44):
    """With M = 1 the j-th GMRES residual is min over the Krylov space
    K_j(D, b) of |b - D x|, computed here by numpy least squares."""
    p = problem44
    b = inputs.gaussian_source(p["L"], 2003).reshape(-1)
    _, info = ora.fgmres(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], b.reshape(-1, 4, 3), 1e-30,
                         m=8, max_restarts=0, use_sap=False)
    hist = info["history"][:8]
    K = np.zeros((b.size, 8), dtype=np.complex128)
    v = b / np.linalg.norm(b)
    for j in range(8):
        K[:, j] = v
        v = dense44 @ v
        v /= np.linalg.norm(v)
    for j in range(1, 9):
        Q, _ = np.linalg.qr(K[:, :j])
        y, *_ = np.linalg.lstsq(dense44 @ Q, b, rcond=None)
        rmin = np.linalg.norm(b - dense44 @ (Q @ y)) / np.linalg.norm(b)
        assert abs(hist[j - 1] - rmin) <= 1e-9 * max(rmin, 1e-3)


def test_one_cycle_solution_is_the_krylov_minimiser(ora, problem44, dense44):
    """After one cycle of m steps (no restart) with M = 1, x is the
    minimiser of |b - D x| over K_m(D, b) (numpy least squares), and the
    true residual equals the last Givens estimate."""
    p = problem44
    b = inputs.gaussian_source(p["L"], 2004).reshape(-1)
    m = 6
    x, info = ora.fgmres(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], b.reshape(-1, 4, 3), 1e-30,
                         m=m, max_restarts=0, use_sap=False)
    K = np.zeros((b.size, m), dtype=np.complex128)
    v = b / np.linalg.norm(b)
    for j in range(m):
        K[:, j] = v
        v = dense44 @ v
        v /= np.linalg.norm(v)
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(dense44 @ Q, b, rcond=None)
    assert rel(x.reshape(-1), Q @ y) <= 1e-10
    assert abs(info["true_rel_res"] - info["history"][m - 1]) <= 1e-10 * info["true_rel_res"]


# -------------------------------------------------------------- MR / SAP

def _domain_sites(L, dom, d):
    nb = [L[i] // dom[i] for i in range(4)]
    b = [d % nb[0], (d // nb[0]) % nb[1], (d // (nb[0] * nb[1])) % nb[2], d // (nb[0] * nb[1] * nb[2])]
    c = site_coords(L)
    mask = np.ones(len(c), dtype=bool)
    for i in range(4):
        mask &= (c[:, i] // dom[i]) == b[i]
    return np.nonzero(mask)[0], sum(b) % 2


def _domain_index(sites):
    return (sites[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)


def test_mr_residual_monotone_and_odd_zero(ora, problem44):
    p = problem44
    eta = inputs.gaussian_source(p["L"], 41)
    norms = []
    for nmr in range(0, 7):
        _, rho = ora.sap(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], eta, nmr, 1)
        s, col = _domain_sites(p["L"], DOM2, 0)
        assert col == 0
        c = site_coords(p["L"])[s]
        odd = (c.sum(1) % 2) == 1
        # after the block solve the odd half of the domain residual is zero
        assert np.abs(rho[s[odd]]).max() <= 1e-13 * np.abs(eta).max()
        norms.append(np.linalg.norm(rho[s]))
    assert all(norms[i + 1] <= norms[i] * (1 + 1e-14) for i in range(len(norms) - 1))


def test_mr_first_step_is_the_dense_minimiser(ora, problem44, dense44):
    """One MR step from zero: r1 = bhat - alpha* p with p = Dhat bhat and
    alpha* = <p, bhat>/<p, p>, the minimiser of |bhat - alpha p|, built
    here from the dense Dirichlet block and its even-odd Schur complement."""
    p = problem44
    eta = inputs.gaussian_source(p["L"], 45)
    _, rho = ora.sap(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], eta, 1, 1)
    s, _ = _domain_sites(p["L"], DOM2, 0)
    par = site_coords(p["L"])[s].sum(1) % 2
    e_idx, o_idx = _domain_index(s[par == 0]), _domain_index(s[par == 1])
    D = dense44
    Dee, Deo = D[np.ix_(e_idx, e_idx)], D[np.ix_(e_idx, o_idx)]
    Doe, Doo = D[np.ix_(o_idx, e_idx)], D[np.ix_(o_idx, o_idx)]
    Dhat = Dee - Deo @ np.linalg.solve(Doo, Doe)
    eflat = eta.reshape(-1)
    bhat = eflat[e_idx] - Deo @ np.linalg.solve(Doo, eflat[o_idx])
    pv = Dhat @ bhat
    alpha = np.vdot(pv, bhat) / np.vdot(pv, pv)
    r1 = bhat - alpha * pv
    assert rel(rho.reshape(-1)[e_idx], r1) <= 1e-13
    # any other step length leaves a larger residual
    for da in (1e-3, 1e-3j):
        assert np.linalg.norm(bhat - (alpha + da) * pv) > np.linalg.norm(r1)


def test_mr_converges_to_dense_domain_inverse(ora, problem44, dense44):
    p = problem44
    eta = inputs.gaussian_source(p["L"], 42)
    psi, _ = ora.sap(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], eta, 200, 1)
    for d in range(16):
        s, col = _domain_sites(p["L"], DOM2, d)
        if col != 0:
            assert np.abs(psi[s]).max() == 0.0
            continue
        idx = _domain_index(s)
        DL = dense44[np.ix_(idx, idx)]
        want = np.linalg.solve(DL, eta.reshape(-1)[idx])
        assert rel(psi.reshape(-1)[idx], want) <= 1e-12


def test_sap_residual_bookkeeping(ora, problem44):
    """After every half-sweep the maintained residual equals eta - D psi."""
    p = problem44
    eta = inputs.gaussian_source(p["L"], 43)
    for n_half in (1, 2, 3, 8):
        psi, rho = ora.sap(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], eta, 4, n_half)
        r = eta - ora.apply_D(p["L"], p["U"], p["A"], p["kappa"], psi)
        assert rel(rho, r) <= 1e-13


def test_sap_exact_blocks_equal_block_gauss_seidel(ora, problem44, dense44):
    """With (numerically) exact block solves, SAP is block Gauss-Seidel over
    the two colours; reproduced here with dense numpy block solves."""
    p = problem44
    eta = inputs.gaussian_source(p["L"], 44).reshape(-1)
    psi_ora, _ = ora.sap(p["L"], DOM2, p["U"], p["A"], p["Ainv"], p["kappa"], eta.reshape(-1, 4, 3), 300, 4)
    doms = [_domain_sites(p["L"], DOM2, d) for d in range(16)]
    psi = np.zeros_like(eta)
    for hs in range(4):
        colour = hs % 2
        r = eta - dense44 @ psi
        for s, col in doms:
            if col != colour:
                continue
            idx = _domain_index(s)
            psi[idx] += np.linalg.solve(dense44[np.ix_(idx, idx)], r[idx])
    assert rel(psi_ora.reshape(-1), psi) <= 1e-11


def test_domain_colouring(ora):
    L, dom = (8, 8, 8, 8), (4, 4, 4, 4)
    cols = [ora.domain_colour(L, dom, d) for d in range(16)]
    assert cols[0] == 0 and sum(cols) == 8
    assert ora.domain_colour((8, 8, 8, 8), (8, 4, 4, 4), 0) == -1  # one block in x: rejected
