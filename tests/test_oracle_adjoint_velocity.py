"""Pins of the oracle's reference gradient (complex step) and of its velocity
update (Eqs. update_vel, update_N, update_alpha; Sec. 3.9-3.10)."""

import os

import numpy as np
import pytest

import oracle as O
from paper_2606_15622_gb300 import populations as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_jacobian_matches_central_differences(cavity_pop):
    pop = cavity_pop.subset([11, 222, 3333, 9999])
    m = O.moments(pop.v64, pop.offsets)
    for c in range(pop.n_cells):
        J = O.closure_jacobian(m[c], pop.tau[c])
        assert np.all(J[:, :4] == 0)  # N, U do not enter the closure
        for k in [4, 5, 8, 12, 17, 22, 26, 27, 29]:
            h = 1e-6 * max(abs(m[c, k]), 1e-3)
            mp, mm = m[c].copy(), m[c].copy()
            mp[k] += h
            mm[k] -= h
            fd = (O.closure(mp[None], pop.tau[c:c + 1])[0][0] - O.closure(mm[None], pop.tau[c:c + 1])[0][0]) / (2 * h)
            scale = np.abs(fd).max() + 1e-3 * np.abs(J).max()
            assert np.abs(J[:, k] - fd).max() < 1e-5 * scale, (c, k)


def test_velocity_gradient_matches_central_differences():
    cav = P.cavity(seed=21, nx=8, ny=8, mean_ppc=10, ppc_range=(8, 14))
    pop = cav.subset([0, 5, 17])
    m = O.moments(pop.v64, pop.offsets)
    rng = np.random.default_rng(1)
    g = rng.standard_normal((pop.n_cells, 9))
    gm, gv = O.closure_backward(pop.v64, pop.offsets, pop.tau, m, g)

    def loss(v):
        Y, _ = O.closure(O.moments(v, pop.offsets), pop.tau)
        return (g * Y).sum()

    for d in range(3):
        for p in rng.choice(pop.n_particles, 6, replace=False):
            h = 1e-6
            vp, vm = pop.v64.copy(), pop.v64.copy()
            vp[d, p] += h
            vm[d, p] -= h
            fd = (loss(vp) - loss(vm)) / (2 * h)
            assert abs(gv[d, p] - fd) < 1e-6 * (abs(fd) + np.abs(gv).max() * 1e-2), (d, p)
    # translation invariance of the closure: the gradient sums to 0 per cell
    for c in range(pop.n_cells):
        s = gv[:, pop.offsets[c]:pop.offsets[c + 1]].sum(axis=1)
        assert np.abs(s).max() < 1e-9 * np.abs(gv).max()


def test_philox_known_answers():
    for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        w = [int(x, 16) for x in ln.split()]
        out = O.philox4x32_10(w[0:4], w[4:6])
        assert list(out) == w[6:10]


def test_normals_are_the_inverse_distribution_of_the_philox_words():
    """xi_k of particle p = Phi^-1(u), u = (floor(w / 2^9) + 1/2) 2^-23 of
    word j = 3p + k of the step's Philox stream (word j % 4 of the block on
    counter j // 4; the published known answers pin the blocks); Phi^-1
    checked against scipy's ndtri and against tabulated quantiles.  Particles
    1000..1007 span blocks 750..755, two of them split between blocks."""
    from scipy.special import ndtri
    seed, step = 0x0123456789ABCDEF, 0x1122334455667788
    xi = O.normals(8, seed, step, first_index=1000)
    blocks = {}
    for k in range(8):
        p = 1000 + k
        for i in range(3):
            j = 3 * p + i
            b = j // 4
            if b not in blocks:
                blocks[b] = O.philox4x32_10([b & 0xFFFFFFFF, b >> 32, step & 0xFFFFFFFF, step >> 32],
                                            [seed & 0xFFFFFFFF, seed >> 32])
            u = ((int(blocks[b][j % 4]) >> 9) + 0.5) * 2.0 ** -23
            np.testing.assert_allclose(xi[i, k], ndtri(u), rtol=1e-12, atol=1e-13)
    assert sorted(blocks) == list(range(750, 756))
    # the map through the oracle at tabulated points: Phi^-1(0.975) = 1.959963984540054,
    # Phi^-1(0.5) = 0, Phi(1) = 0.8413447460685429; the extreme uniforms
    for u, x in [(0.975, 1.959963984540054), (0.025, -1.959963984540054), (0.5, 0.0),
                 (0.8413447460685429, 1.0), (2.0 ** -24, ndtri(2.0 ** -24)), (1 - 2.0 ** -24, ndtri(1 - 2.0 ** -24))]:
        assert abs(ndtri(u) - x) < 1e-12


def test_normals_are_standard_normal():
    n = 400_000
    xi = O.normals(n, seed=1234, step=7)
    for d in range(3):
        x = xi[d]
        assert abs(x.mean()) < 6 / np.sqrt(n)
        assert abs(x.var() - 1) < 6 * np.sqrt(2 / n)
        assert abs((x ** 4).mean() - 3) < 6 * np.sqrt(96 / n)
    # the three components are uncorrelated
    assert abs((xi[0] * xi[1]).mean()) < 6 / np.sqrt(n)
    assert abs((xi[0] * xi[2]).mean()) < 6 / np.sqrt(n)
    # counters differ by step and by particle
    assert not np.array_equal(O.normals(8, 1234, 7), O.normals(8, 1234, 8))
    np.testing.assert_array_equal(O.normals(4, 1234, 7, first_index=3), O.normals(7, 1234, 7)[:, 3:])


def _cell_energy(v, offs, U):
    out = []
    for c in range(offs.size - 1):
        vc = v[:, offs[c]:offs[c + 1]] - U[c][:, None]
        out.append((vc * vc).sum(0).mean())
    return np.array(out)


def test_alpha_conserves_expected_energy(cavity_pop):
    """Eq. update_alpha is defined so that the expected energy E|M^{n+1}-U|^2
    over the noise equals 3 theta.  Averaging the cell energy over many
    independent noise draws must reproduce 3 theta within CLT bounds."""
    pop = cavity_pop.subset([4, 1000, 7777])
    m = O.moments(pop.v64, pop.offsets)
    Y, fl = O.closure(m, pop.tau, eps2_hat=1e-2)
    dt = 0.3
    U = m[:, 1:4]
    draws = []
    for s in range(3000):
        vn, alpha, _ = O.velocity_update(pop.v64, pop.offsets, m, Y, pop.tau, fl, dt, eps2_hat=1e-2,
                                         seed=99, step=s)
        draws.append(_cell_energy(vn, pop.offsets, U))
    draws = np.array(draws)
    mean, se = draws.mean(0), draws.std(0) / np.sqrt(draws.shape[0])
    assert np.all(alpha != 1.0)
    assert np.all(np.abs(mean - 3 * m[:, 4]) < 6 * se)


def test_linear_fallback_is_the_exact_ou_step():
    pop = P.maxwellian_cells([50, 60], theta=[1.5, 0.7], tau=[0.8, 2.0], seed=3)
    m = O.moments(pop.v64, pop.offsets)
    Y, _ = O.closure(m, pop.tau)
    fl = np.array([O.FLAG_SINGULAR, O.FLAG_FEW], dtype=np.int32)
    xi = np.random.default_rng(0).standard_normal((3, pop.n_particles))
    dt = 0.25
    vn, alpha, _ = O.velocity_update(pop.v64, pop.offsets, m, Y, pop.tau, fl, dt, xi=xi)
    np.testing.assert_array_equal(alpha, [1.0, 1.0])
    for c in range(2):
        s = slice(pop.offsets[c], pop.offsets[c + 1])
        a = np.exp(-dt / pop.tau[c])
        U = m[c, 1:4][:, None]
        ou = (pop.v64[:, s] - U) * a + np.sqrt(m[c, 4] * (1 - a * a)) * xi[:, s] + U
        np.testing.assert_allclose(vn[:, s], ou, rtol=1e-14, atol=1e-14)


def test_update_keeps_the_cell_mean_without_noise(cavity_pop):
    """<N> = <A> + <M'>/tau = 0 for the cubic drift, so with xi = 0 the cell
    mean velocity is U after the step (momentum)."""
    pop = cavity_pop.subset(np.arange(0, 16384, 1500))
    m = O.moments(pop.v64, pop.offsets)
    Y, fl = O.closure(m, pop.tau)
    vn, _, _ = O.velocity_update(pop.v64, pop.offsets, m, Y, pop.tau, fl, 0.4,
                                 xi=np.zeros_like(pop.v64))
    for c in range(pop.n_cells):
        s = slice(pop.offsets[c], pop.offsets[c + 1])
        np.testing.assert_allclose(vn[:, s].mean(1), m[c, 1:4], rtol=0, atol=1e-12 * np.sqrt(m[c, 4]) * 10)


def test_small_step_is_nearly_identity(cavity_pop):
    pop = cavity_pop.subset([17, 18])
    m = O.moments(pop.v64, pop.offsets)
    Y, fl = O.closure(m, pop.tau)
    dt = 1e-9
    vn, alpha, _ = O.velocity_update(pop.v64, pop.offsets, m, Y, pop.tau, fl, dt, seed=1, step=1)
    assert np.abs(alpha - 1).max() < 1e-7
    assert np.abs(vn - pop.v64).max() < 1e-3  # noise ~ sqrt(2 theta dt / tau)


def test_drift_averages_from_moments_equal_particle_sums(cavity_pop):
    """The cell averages of Eq. update_alpha in closed form from the moments
    and <|c|^6> (what a one-pass update uses) against direct sums over the
    particles of N.N and M'.N, N from Eq. update_N."""
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 331))
    eps2_hat = 0.05
    m = O.moments(pop.v64, pop.offsets)
    y, fl = O.closure(m, pop.tau, eps2_hat=eps2_hat)
    m6 = O.speed_moment6(pop.v64, pop.offsets)
    checked = 0
    for k in np.flatnonzero(fl == 0):
        a, b = pop.offsets[k], pop.offsets[k + 1]
        tau, th = pop.tau[k], m[k, O.M_THETA]
        e2 = eps2_hat / (tau * th)
        C = np.array([[y[k, O.SYM2.index(tuple(sorted((i, j))))] for j in range(3)] for i in range(3)])
        A = C + np.eye(3) / tau
        G = y[k, 6:9]
        c = pop.v64[:, a:b] - m[k, O.M_U:O.M_U + 3, None]
        r2 = (c * c).sum(0)
        u3 = m[k, O.M_U3:O.M_U3 + 10]
        bvec = np.array([sum(u3[O.SYM3.index(tuple(sorted((i, j, j))))] for j in range(3)) for i in range(3)])
        N = A @ c + G[:, None] * (r2 - 3 * th) - e2 * (c * r2 - bvec[:, None])
        nn_p, mn_p = (N * N).sum(0).mean(), (c * N).sum(0).mean()
        sym = lambda base: np.array([[m[k, base + O.SYM2.index(tuple(sorted((i, j))))] for j in range(3)]
                                     for i in range(3)])
        u, w = sym(O.M_U2), sym(O.M_W)
        z = m[k, O.M_Z:O.M_Z + 3]
        s4 = np.trace(w)
        mn_m = np.sum(A * u) + G @ bvec - e2 * s4
        nn_m = (np.sum((A @ A) * u) + G @ G * (s4 - 9 * th ** 2) + e2 ** 2 * (m6[k] - bvec @ bvec)
                + 2 * G @ A @ bvec - 2 * e2 * np.sum(A * w) - 2 * e2 * G @ (z - 3 * th * bvec))
        scale = np.mean((np.abs(A @ c) + np.abs(G[:, None] * r2) + e2 * np.abs(c * r2)).sum(0) ** 2)
        assert abs(nn_m - nn_p) <= 1e-10 * scale
        assert abs(mn_m - mn_p) <= 1e-10 * np.sqrt(scale * (r2.mean()))
        checked += 1
    assert checked > 20
