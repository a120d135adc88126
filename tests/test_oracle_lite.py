"""Oracle pins of the LITE moment pass and the 16 network inputs (Sec. 4,
Phase 1-2 item 1 and Phase 3 item 2): closed forms for constructed particle
sets, agreement with the independently written full-moment oracle (C) and
with library routines (numpy covariance and determinant), Maxwellian limits,
Galilean invariance."""

import numpy as np

import oracle as O
from oracle import lite as L
from paper_2606_15622_gb300 import populations as P


def test_axis_set_closed_forms():
    # six particles +-a e_x, +-b e_y, +-c e_z: U = 0, u = diag(a^2, b^2, c^2) / 3,
    # theta = (a^2 + b^2 + c^2) / 9, odd symmetry gives b_i = 0
    a, b, c = 1.0, 2.0, 3.0
    v = np.array([[a, -a, 0, 0, 0, 0], [0, 0, b, -b, 0, 0], [0, 0, 0, 0, c, -c]])
    m = L.lite_moments(v, [0, 6])[0]
    assert m[L.L_N] == 6
    np.testing.assert_allclose(m[L.L_U:L.L_U + 3], 0.0, atol=1e-15)
    assert abs(m[L.L_THETA] - 14.0 / 9.0) < 1e-15
    np.testing.assert_allclose(m[L.L_U2:L.L_U2 + 6], [1 / 3, 0, 0, 4 / 3, 0, 3.0], atol=1e-15)
    np.testing.assert_allclose(m[L.L_B:L.L_B + 3], 0.0, atol=1e-15)
    f = L.lite_features(m, [0.25])[0]
    assert abs(f[14] - (1 / 3) * (4 / 3) * 3.0) < 1e-14  # DM2 = a^2 b^2 c^2 / 27
    assert f[15] == 4.0                                   # nu = 1 / tau
    np.testing.assert_allclose(f[5:11], [1 / 3 - 14 / 9, 0, 0, 4 / 3 - 14 / 9, 0, 3 - 14 / 9], atol=1e-15)


def test_skewed_set_heat_flux():
    # x velocities {-1, -1, 2}: mean 0, <c_x^2> = 2, <c_x^3> = 2, so b_x = 2 and q_x = 1
    v = np.array([[-1.0, -1.0, 2.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]) + np.array([[5.0], [-1.0], [0.5]])
    m = L.lite_moments(v, [0, 3])[0]
    np.testing.assert_allclose(m[L.L_U:L.L_U + 3], [5.0, -1.0, 0.5], atol=1e-15)
    assert abs(m[L.L_THETA] - 2.0 / 3.0) < 1e-15
    np.testing.assert_allclose(m[L.L_B:L.L_B + 3], [2.0, 0.0, 0.0], atol=1e-14)
    f = L.lite_features(m, [1.0])[0]
    np.testing.assert_allclose(f[11:14], [1.0, 0.0, 0.0], atol=1e-14)
    assert f[14] == 0.0  # rank-one second-moment tensor
    np.testing.assert_allclose(f[5:11], [2 - 2 / 3, 0, 0, -2 / 3, 0, -2 / 3], atol=1e-15)


def test_against_full_moment_oracle_and_numpy():
    pop = P.cavity(nx=8, ny=6, mean_ppc=60.0, seed=4)
    m = L.lite_moments(pop.v64, pop.offsets)
    full = O.moments(pop.v64, pop.offsets)
    ok = pop.counts > 0
    np.testing.assert_array_equal(m[:, L.L_N], full[:, O.M_N])
    np.testing.assert_allclose(m[ok, L.L_U:L.L_U + 3], full[ok, O.M_U:O.M_U + 3], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(m[ok, L.L_THETA], full[ok, O.M_THETA], rtol=1e-12)
    np.testing.assert_allclose(m[ok, L.L_U2:L.L_U2 + 6], full[ok, O.M_U2:O.M_U2 + 6], rtol=1e-11, atol=1e-13)
    u3 = full[:, O.M_U3:O.M_U3 + 10]
    idx = {t: s for s, t in enumerate(O.SYM3)}
    b = np.stack([sum(u3[:, idx[tuple(sorted((i, j, j)))]] for j in range(3)) for i in range(3)], axis=1)
    np.testing.assert_allclose(m[ok, L.L_B:L.L_B + 3], b[ok], rtol=1e-10, atol=1e-12)
    # second moments = the biased covariance; DM2 = its determinant
    f = L.lite_features(m[ok], pop.tau[ok])
    for k, cell in enumerate(np.flatnonzero(ok)[:40]):
        a, e = pop.offsets[cell], pop.offsets[cell + 1]
        cov = np.cov(pop.v64[:, a:e], bias=True)
        np.testing.assert_allclose([cov[i, j] for (i, j) in L.SYM2], m[cell, L.L_U2:L.L_U2 + 6], rtol=1e-10,
                                   atol=1e-13)
        assert abs(f[k, 14] - np.linalg.det(cov)) <= 1e-10 * abs(np.linalg.det(cov)) + 1e-15
        assert abs(f[k, 5] + f[k, 8] + f[k, 10]) <= 1e-12 * f[k, 1]  # Pi is traceless


def test_maxwellian_limits_and_galilean_invariance():
    theta = 0.7
    pop = P.maxwellian_cells([400_000], theta=theta, mean=(0.0, 0.0, 0.0), seed=3)
    m = L.lite_moments(pop.v64, pop.offsets)[0]
    f = L.lite_features(m, [2.0])[0]
    assert abs(f[1] - theta) < 0.01
    assert np.all(np.abs(f[5:11]) < 0.01)
    assert np.all(np.abs(f[11:14]) < 0.01)
    assert abs(f[14] - theta ** 3) < 0.01
    shifted = pop.v64 + np.array([[3.0], [-2.0], [0.25]])
    m2 = L.lite_moments(shifted, pop.offsets)[0]
    np.testing.assert_allclose(m2[L.L_THETA:], m[L.L_THETA:], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(m2[L.L_U:L.L_U + 3], m[L.L_U:L.L_U + 3] + [3.0, -2.0, 0.25], atol=1e-12)


def test_empty_cells_are_zero():
    v = np.array([[1.0, 2.0], [0.0, 1.0], [3.0, 3.0]])
    m = L.lite_moments(v, [0, 0, 2, 2])
    assert np.all(m[0] == 0) and np.all(m[2] == 0) and m[1, L.L_N] == 2
