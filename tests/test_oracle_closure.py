"""Pins of the oracle's 9x9 closure (Eq. system9x9, Table 1, Sec. 3.4-3.7).

The pins do not reuse the oracle's matrix formula: they check moment
matching directly at the particle level (Eq. moment_match with the drift of
Eq. cubic_drift), Table 1 entry by entry, the equilibrium reduction to the
linear model (Eq. linear_drift), the Prandtl numbers the paper states, the
invariances of the physics, and the elimination against exact rationals.
"""

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2606_15622_gb300 import populations as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS_SWEEP = [0.0, 1e-3, 1e-1]


def _unpack(Y):
    C = np.array([[Y[0], Y[1], Y[2]], [Y[1], Y[3], Y[4]], [Y[2], Y[4], Y[5]]])
    return C, np.array(Y[6:9])


def _productions(vcell, C, G, tau, eps2_hat):
    """FP productions of psi = c_i c_j and psi = c_i |c|^2 computed particle by
    particle from the cubic drift (Eq. cubic_drift) and the isotropic
    diffusion D = 2 theta / tau:
        S_ij = <A_i c_j + A_j c_i> + (2 theta / tau) delta_ij
        H_i  = <A_k (delta_ik |c|^2 + 2 c_i c_k)> + (theta / tau) <10 c_i>
    together with the moments they must relax (u_ij, theta, b_i)."""
    U = vcell.mean(axis=1, keepdims=True)
    c = vcell - U
    c2 = (c * c).sum(0)
    u = c @ c.T / c.shape[1]
    theta = np.trace(u) / 3.0
    b = (c * c2).mean(axis=1)
    eps2 = eps2_hat / (tau * theta)
    A = C @ c + G[:, None] * (c2 - 3 * theta)[None, :] - eps2 * (c * c2 - b[:, None])
    S = (A @ c.T + c @ A.T) / c.shape[1] + (2 * theta / tau) * np.eye(3)
    H = np.array([(A[i] * c2 + 2 * c[i] * (A * c).sum(0)).mean() for i in range(3)]) \
        + (theta / tau) * 10 * c.mean(axis=1)
    return S, H, u, theta, b, A


@pytest.mark.parametrize("eps2_hat", EPS_SWEEP)
def test_particle_level_moment_matching(cavity_pop, eps2_hat):
    """The solved Y makes the FP production of stress equal the Maxwell-
    molecule rate -(2/tau)(u_ij - theta delta_ij) and of heat flux
    -(4/(3 tau)) b_i (Pr = 2/3), checked by direct summation over particles."""
    cells = np.arange(3, cavity_pop.n_cells, 331)
    pop = cavity_pop.subset(cells)
    m = O.moments(pop.v64, pop.offsets)
    Y, fl = O.closure(m, pop.tau, eps2_hat=eps2_hat)
    assert not fl.any()
    for c in range(pop.n_cells):
        vc = pop.v64[:, pop.offsets[c]:pop.offsets[c + 1]]
        tau = pop.tau[c]
        C, G = _unpack(Y[c])
        S, H, u, theta, b, A = _productions(vc, C, G, tau, eps2_hat)
        scale = np.abs(C).max() * theta + np.abs(G).max() * theta ** 1.5 * 10 + theta / tau
        assert np.abs(S - (-(2 / tau) * (u - theta * np.eye(3)))).max() < 1e-11 * scale
        assert np.abs(H - (-(4 / (3 * tau)) * b)).max() < 1e-11 * scale * np.sqrt(theta)
        # momentum: <A> = 0 for the cubic drift; energy: <A.c> = -3 theta / tau
        assert np.abs(A.mean(axis=1)).max() < 1e-12 * scale
        assert abs((A * (vc - vc.mean(1, keepdims=True))).sum(0).mean() + 3 * theta / tau) < 1e-11 * scale


def test_linear_model_prandtl_three_halves(cavity_pop):
    """Sec. 3.3: with A = -c/tau and D = 2 theta/tau the stress relaxes at
    2/tau towards theta delta_ij and the heat flux at 3/tau, i.e. Pr = 3/2 for
    the linear model, as the paper states.  (With D = theta/tau the stress
    would relax towards theta/2 -- that reading is ruled out.)"""
    pop = cavity_pop.subset(np.arange(10, cavity_pop.n_cells, 997))
    for c in range(pop.n_cells):
        vc = pop.v64[:, pop.offsets[c]:pop.offsets[c + 1]]
        tau = pop.tau[c]
        S, H, u, theta, b, _ = _productions(vc, -np.eye(3) / tau, np.zeros(3), tau, 0.0)
        np.testing.assert_allclose(S, -(2 / tau) * (u - theta * np.eye(3)), atol=1e-12 * theta / tau)
        np.testing.assert_allclose(H, -(3 / tau) * b, atol=1e-12 * theta ** 1.5 / tau)
    stress_rate, heat_rate = 2.0, 3.0
    assert heat_rate / stress_rate == 1.5


def _parse_expr(expr, u, b):
    env = {f"u{i + 1}{j + 1}": u[i, j] for i in range(3) for j in range(3)}
    env.update({f"b{i + 1}": b[i] for i in range(3)})
    total = 0.0
    for term in expr.split("+"):
        if "*" in term:
            k, sym = term.split("*")
            total += float(k) * env[sym]
        elif term in env:
            total += env[term]
        else:
            total += float(term)
    return total


def test_stress_rows_reproduce_table1(cavity_pop):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_VW.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 36 + 18
    pop = cavity_pop.subset([7, 123, 4567])
    m = O.moments(pop.v64, pop.offsets)
    for c in range(pop.n_cells):
        u = np.zeros((3, 3))
        for a, (i, j) in enumerate(O.SYM2):
            u[i, j] = u[j, i] = m[c, O.M_U2 + a]
        u3 = {idx: m[c, O.M_U3 + a] for a, idx in enumerate(O.SYM3)}
        b = np.array([u3[tuple(sorted((i, 0, 0)))] + u3[tuple(sorted((i, 1, 1)))] + u3[tuple(sorted((i, 2, 2)))]
                      for i in range(3)])
        A, _ = O.assemble(m[c], pop.tau[c], 1e-3)
        for blk, r, col, expr in rows:
            r, col = int(r) - 1, int(col) - 1
            if blk == "W":
                col += 6
            assert A[r, col] == pytest.approx(_parse_expr(expr, u, b), rel=1e-14, abs=1e-15), (blk, r, col)


def _maxwellian_moments(theta, n=1000, U=(0.3, -0.2, 1.0)):
    m = np.zeros(O.NMOM)
    m[O.M_N] = n
    m[1:4] = U
    m[O.M_THETA] = theta
    for a, (i, j) in enumerate(O.SYM2):
        if i == j:
            m[O.M_U2 + a] = theta
            m[O.M_W + a] = 5 * theta ** 2
    return m


@pytest.mark.parametrize("eps2_hat", EPS_SWEEP)
@pytest.mark.parametrize("theta,tau", [(1.0, 1.0), (2.5, 0.4), (40.0, 0.2)])
def test_equilibrium_reduces_to_linear_model(eps2_hat, theta, tau):
    """Exact Maxwellian moments give C = (-1 + 5 eps2_hat)/tau I and G = 0;
    at eps2_hat = 0 this is the linear drift -c/tau (Eq. linear_drift)."""
    Y, fl = O.closure(_maxwellian_moments(theta)[None], np.array([tau]), eps2_hat=eps2_hat)
    assert fl[0] == 0
    C, G = _unpack(Y[0])
    np.testing.assert_allclose(C, (-1 + 5 * eps2_hat) / tau * np.eye(3), rtol=1e-14, atol=1e-14 / tau)
    assert np.abs(G).max() < 1e-14 / (tau * np.sqrt(theta))


def test_large_maxwellian_cell_converges_to_linear_model():
    n = 1_000_000
    pop = P.maxwellian_cells([n], theta=1.3, tau=0.7, seed=11)
    m = O.moments(pop.v64, pop.offsets)
    Y, fl = O.closure(m, pop.tau, eps2_hat=0.0)
    C, G = _unpack(Y[0])
    # O(N^-1/2) deviation of sampled moments; 10 / sqrt(N) leaves a wide margin
    assert np.abs(C * 0.7 + np.eye(3)).max() < 10 / np.sqrt(n) * 10
    assert np.abs(G * 0.7 * np.sqrt(1.3)).max() < 10 / np.sqrt(n) * 10


def _rot_perm_cases():
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    perm = np.eye(3)[[2, 0, 1]]
    refl = np.diag([1.0, -1.0, 1.0])
    return {"rotation": q, "permutation": perm, "reflection": refl}


@pytest.mark.parametrize("case", ["rotation", "permutation", "reflection"])
def test_closure_is_rotation_covariant(cavity_pop, case):
    q = _rot_perm_cases()[case]
    pop = cavity_pop.subset(np.arange(1, cavity_pop.n_cells, 503))
    m0 = O.moments(pop.v64, pop.offsets)
    m1 = O.moments(q @ pop.v64, pop.offsets)
    Y0, f0, cond, _ = O.closure(m0, pop.tau, want_cond=True)
    Y1, f1 = O.closure(m1, pop.tau)
    assert not f0.any() and not f1.any()
    for c in range(pop.n_cells):
        C0, G0 = _unpack(Y0[c])
        C1, G1 = _unpack(Y1[c])
        tol = 1e-13 * cond[c] * np.abs(Y0[c]).max()
        assert np.abs(C1 - q @ C0 @ q.T).max() < tol
        assert np.abs(G1 - q @ G0).max() < tol


def test_closure_is_galilean_invariant_and_scales(cavity_pop):
    pop = cavity_pop.subset(np.arange(2, cavity_pop.n_cells, 401))
    m0 = O.moments(pop.v64, pop.offsets)
    Y0, _, cond, _ = O.closure(m0, pop.tau, want_cond=True)
    # Galilean: v -> v + a (Mach-10 sized shift)
    Y1, _ = O.closure(O.moments(pop.v64 + np.array([[12.9], [1.0], [-2.0]]), pop.offsets), pop.tau)
    err = np.abs(Y1 - Y0).max(axis=1) / np.abs(Y0).max(axis=1)
    assert np.all(err < 1e-12 * cond)
    # velocity scale s: C (1/time) unchanged, G (1/(time velocity)) -> G / s
    s = 3.0
    Y2, _ = O.closure(O.moments(s * pop.v64, pop.offsets), pop.tau)
    np.testing.assert_allclose(Y2[:, :6], Y0[:, :6], rtol=0, atol=1e-12 * np.abs(Y0).max())
    np.testing.assert_allclose(Y2[:, 6:] * s, Y0[:, 6:], rtol=0, atol=1e-12 * np.abs(Y0).max())


def _exact_solve(A, r):
    n = 9
    M = [[Fraction(float(A[i, j])) for j in range(n)] + [Fraction(float(r[i]))] for i in range(n)]
    for k in range(n):
        p = next(i for i in range(k, n) if M[i][k] != 0)
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            f = M[i][k] / M[k][k]
            for j in range(k, n + 1):
                M[i][j] -= f * M[k][j]
    y = [Fraction(0)] * n
    for k in range(n - 1, -1, -1):
        s = M[k][n] - sum(M[k][j] * y[j] for j in range(k + 1, n))
        y[k] = s / M[k][k]
    return np.array([float(x) for x in y])


@pytest.mark.parametrize("seed", [0, 1])
def test_elimination_against_exact_rationals(seed):
    pop = P.integer_cells([12, 16, 20, 30], lo=-3, hi=3, seed=seed)
    m = O.moments(pop.v64, pop.offsets)
    for c in range(pop.n_cells):
        A, r = O.assemble(m[c], 1.0, 1e-3)
        y, f = O.solve(A, r)
        assert f == 0
        ye = _exact_solve(A, r)
        kappa = np.linalg.cond(A, np.inf)
        assert np.abs(y - ye).max() <= 50 * kappa * 2.2e-16 * np.abs(ye).max()


def test_backward_error_of_the_solve(cavity_pop):
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 61))
    m = O.moments(pop.v64, pop.offsets)
    Y, fl = O.closure(m, pop.tau)
    for c in range(pop.n_cells):
        A, r = O.assemble(m[c], pop.tau[c], O.DEFAULT_EPS2_HAT)
        res = np.abs(A @ Y[c] - r).max()
        assert res <= 1e-14 * (np.abs(A).sum(1).max() * np.abs(Y[c]).max() + np.abs(r).max())


def test_degenerate_cells_fall_back_to_linear_drift():
    tau = np.array([0.5, 0.5, 0.5, 0.5, 0.5])
    rng = np.random.default_rng(0)
    v = rng.standard_normal((3, 3 + 10 + 10))
    v[:, 3:13] = 1.25  # ten identical particles: theta = 0
    v[1, 20] = np.nan
    offs = np.array([0, 3, 13, 23, 23, 23], dtype=np.int64)
    m = O.moments(v, offs)
    Y, fl = O.closure(m, tau[:5])
    assert fl[0] & O.FLAG_FEW
    assert fl[1] & O.FLAG_SINGULAR
    assert fl[2] & O.FLAG_NONFINITE
    assert fl[3] & O.FLAG_FEW and fl[4] & O.FLAG_FEW
    lin = np.array([-2.0, 0, 0, -2.0, 0, -2.0, 0, 0, 0])
    for c in range(5):
        np.testing.assert_array_equal(Y[c], lin)


def test_four_particle_cells_are_singular():
    """Brute force over random cells: with four particles the 9x9 system is
    singular whatever the velocities (the smallest pivot ratio is at the
    rounding level), with five it is generically regular.  The FP32-moment
    GPU mode relies on this to flag four-particle cells without a solve."""
    rng = np.random.default_rng(11)
    for n, want_singular in ((4, True), (5, False)):
        ratios = []
        for _ in range(200):
            v = rng.standard_normal((3, n)) * rng.uniform(0.3, 3) + rng.uniform(-5, 5, (3, 1))
            m = O.moments(v, np.array([0, n]))
            for e2 in (0.0, 1e-3, 1e-1):
                _, fl, _, mp = O.closure(m, np.array([rng.uniform(0.5, 2.0)]), eps2_hat=e2, want_cond=True)
                ratios.append(mp[0])
        ratios = np.array(ratios)
        if want_singular:
            assert ratios.max() < 1e-12
        else:
            assert np.median(ratios) > 1e-3 and (ratios < 1e-12).mean() < 0.01
