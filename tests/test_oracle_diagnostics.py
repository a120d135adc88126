"""Oracle pins of the high-order diagnostics and entropy proxies (cavity
study and cylinder audit of the paper): Maxwellian values, exact values for
constructed moment vectors, invariances; and of the coefficient
under-relaxation."""

import numpy as np

import oracle as O
from paper_2606_15622_gb300 import populations as P


def _moments_with(theta_diag=None, Theta=None, n=10.0):
    """A moment vector with a given second-moment tensor (other slots 0)."""
    m = np.zeros(O.NMOM)
    m[O.M_N] = n
    T = np.diag(theta_diag) if Theta is None else np.asarray(Theta, dtype=float)
    for a, (i, j) in enumerate(O.SYM2):
        m[O.M_U2 + a] = T[i, j]
    m[O.M_THETA] = np.trace(T) / 3.0
    return m


def test_maxwellian_cells_reach_the_equilibrium_values():
    n, theta = 300_000, 0.8
    pop = P.maxwellian_cells([n], theta=theta, mean=(1.0, 2.0, -3.0), seed=11)
    m = O.moments(pop.v64, pop.offsets)
    m6 = O.speed_moment6(pop.v64, pop.offsets)
    d = O.diagnostics(m, m6)[0]
    # within a few standard errors of the Gaussian values
    np.testing.assert_allclose(d[0:6], 5.0 * np.array([1, 0, 0, 1, 0, 1]), atol=0.1)
    assert abs(d[6]) < 0.3 and abs(d[7] - 105.0) < 3.0
    assert 0.0 <= d[8] < 1e-3 and d[9] < 1e-3


def test_covariance_entropy_deficit_exact_values():
    # Theta = diag(1, 2, 3): theta = 2, det(Theta / theta) = 6 / 8
    d = O.diagnostics(_moments_with([1.0, 2.0, 3.0]), [0.0])[0]
    assert abs(d[8] - (-0.5 * np.log(6.0 / 8.0))) < 1e-15
    # isotropic covariance: D_G = 0 exactly
    assert O.diagnostics(_moments_with([2.5, 2.5, 2.5]), [0.0])[0][8] == 0.0
    # rotation invariance of D_G
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    T = Q @ np.diag([0.5, 1.0, 4.0]) @ Q.T
    d_rot = O.diagnostics(_moments_with(Theta=T), [0.0])[0][8]
    d_diag = O.diagnostics(_moments_with([0.5, 1.0, 4.0]), [0.0])[0][8]
    assert abs(d_rot - d_diag) < 1e-12
    assert d_diag > 0


def test_entropy_terms_and_invalid_cells():
    m = _moments_with([1.5, 1.5, 1.5], n=40.0)
    d = O.diagnostics(m, [0.0], rho=np.array([2.0]), theta_inf=0.5, rho_inf=4.0, dg_inf=0.25)[0]
    ds = 1.5 * np.log(1.5 / 0.5) - np.log(2.0 / 4.0)
    assert abs(d[10] - ds) < 1e-15 and abs(d[11] - (ds + 0.25)) < 1e-15
    # heat-flux term: b = (q, 0, 0) -> D_q = (q / (2 theta^1.5))^2 / 5
    m2 = m.copy()
    m2[O.M_U3 + O.SYM3.index((0, 0, 0))] = 0.9
    d2 = O.diagnostics(m2, [0.0])[0]
    assert abs(d2[9] - (0.9 / (2 * 1.5 ** 1.5)) ** 2 / 5) < 1e-15
    bad = np.stack([_moments_with([1.0, 1.0, 1.0], n=1.0), _moments_with([0.0, 0.0, 0.0])])
    assert np.isnan(O.diagnostics(bad, [0.0, 0.0])).all()


def test_relaxation_blends_linearly():
    a, b = np.arange(9.0), -np.arange(9.0)
    np.testing.assert_array_equal(O.coeffs_relax(a, b, 1.0), a)
    np.testing.assert_array_equal(O.coeffs_relax(a, b, 0.0), b)
    np.testing.assert_allclose(O.coeffs_relax(a, b, 0.2), 0.2 * a + 0.8 * b, rtol=0, atol=1e-15)
