"""The seeded gauge fields are SU(3) to rounding: U U^+ = 1 and det U = 1 for
every link, eps = 0 gives unit links, and the third row of every link is the
complex conjugate of the cross product of its first two (the identity the
two-row operator copies rely on; it fails for a field that is not SU(3))."""
import numpy as np

from paper_1502_04025_gb300 import inputs


def _third_row(U):
    r0, r1 = U[..., 0, :], U[..., 1, :]
    return np.conj(np.cross(r0, r1))


def test_gauge_field_is_su3():
    U = inputs.gauge_field((4, 4, 4, 6), 0.7, 1001).reshape(-1, 3, 3)
    eye = np.eye(3)
    dev = np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - eye).max()
    assert dev <= 1e-13
    assert np.abs(np.linalg.det(U) - 1.0).max() <= 1e-13
    # a nontrivial field: far from the unit links
    assert np.abs(U - eye).max() > 0.1


def test_zero_eps_gives_unit_links():
    U = inputs.gauge_field((4, 4, 4, 4), 0.0, 1002).reshape(-1, 3, 3)
    assert np.abs(U - np.eye(3)).max() <= 1e-14


def test_third_row_is_the_conjugated_cross_product():
    U = inputs.gauge_field((4, 4, 4, 4), 0.5, 1003)
    assert np.abs(_third_row(U) - U[..., 2, :]).max() <= 1e-13
    # a U(3) link with det != 1 breaks it
    V = U * np.exp(0.3j)
    assert np.abs(_third_row(V) - V[..., 2, :]).max() > 1e-2


def test_sources():
    L = (4, 4, 4, 4)
    z = inputs.z2_source(L, 2005)
    assert np.allclose(np.abs(z), 1.0, atol=1e-15)
    assert set(np.round(z.ravel() * np.sqrt(2)).tolist()) == {1 + 1j, 1 - 1j, -1 + 1j, -1 - 1j}
    P = inputs.point_sources(L, site=5).reshape(12, -1)
    assert np.array_equal(np.abs(P).sum(1), np.ones(12))
    assert np.array_equal(np.nonzero(P)[1], 5 * 12 + np.arange(12))  # site 5, spin*3 + colour in order
    g = inputs.gaussian_source(L, 2001)
    assert abs(g.real.std() - 1) < 0.05 and abs(g.imag.std() - 1) < 0.05


def test_exponential_matches_the_eigendecomposition():
    """The C helper's Taylor series with scaling and squaring gives the same
    SU(3) matrices as exp(i eps H) through numpy's eigen-decomposition of H,
    for small and large eps (several squarings)."""
    h = inputs.rng(77).standard_normal((4000, 4, 8))
    for eps in (0.1, 0.7, 3.0):
        a = inputs._su3_from_normals(h, eps)
        b = inputs.su3_from_normals_eigh(h, eps)
        assert np.abs(a - b).max() <= 1e-14
