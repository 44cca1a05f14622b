"""Pins of the oracle's condition-number estimate (oracle/spectrum.py):
the free-field operator's singular values in closed form, and the dense SVD
of the operator on a small random gauge field."""
import numpy as np
import pytest

from oracle import spectrum
from paper_1502_04025_gb300 import inputs


def _free_singular_values(L, kappa):
    """For unit links the clover term is 1 and D(p) = a + i b.gamma with
    a = 1 - 2 kappa sum cos p, b_mu = 2 kappa sin p_mu; gamma-matrices
    anticommute, so D(p)^H D(p) = a^2 + |b|^2: every singular value is
    sqrt(a^2 + |b|^2) over the momenta p_mu = 2 pi k / L_mu."""
    ps = np.meshgrid(*[2 * np.pi * np.arange(n) / n for n in L], indexing="ij")
    a = 1 - 2 * kappa * sum(np.cos(p) for p in ps)
    b2 = 4 * kappa ** 2 * sum(np.sin(p) ** 2 for p in ps)
    return np.sqrt(a ** 2 + b2)


@pytest.mark.parametrize("L,kappa", [((4, 4, 4, 4), 0.12), ((4, 4, 2, 6), 0.1)])
def test_free_field_closed_form(ora, L, kappa):
    U = inputs.unit_gauge_field(L)
    A = ora.clover(L, U, 1.0, kappa)
    sv = _free_singular_values(L, kappa)
    # few distinct singular values (one Krylov direction each): the extremes come out exact
    est = spectrum.cond_estimate(L, U, A, kappa, steps=40)
    assert est["sigma_max"] == pytest.approx(sv.max(), rel=1e-10)
    assert est["sigma_min"] == pytest.approx(sv.min(), rel=1e-10)
    assert est["cond"] == pytest.approx(sv.max() / sv.min(), rel=1e-9)


def test_random_field_matches_dense_svd(ora):
    L, kappa = (4, 2, 2, 2), 0.13
    U = inputs.gauge_field(L, 0.7, 1009)
    A = ora.clover(L, U, 1.5, kappa)
    V = int(np.prod(L))
    n = 12 * V
    D = np.empty((n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1.0
        D[:, k] = ora.apply_D(L, U, A, kappa, e.reshape(V, 4, 3)).ravel()
    s = np.linalg.svd(D, compute_uv=False)
    full = spectrum.cond_estimate(L, U, A, kappa, steps=n)
    assert full["sigma_max"] == pytest.approx(s[0], rel=1e-10)
    assert full["sigma_min"] == pytest.approx(s[-1], rel=1e-8)
    # a short run approaches both ends from inside: a lower bound on cond(D)
    short = spectrum.cond_estimate(L, U, A, kappa, steps=12)
    assert s[-1] * (1 - 1e-12) <= short["sigma_min"] and short["sigma_max"] <= s[0] * (1 + 1e-12)
    assert short["cond"] <= s[0] / s[-1] * (1 + 1e-12)
