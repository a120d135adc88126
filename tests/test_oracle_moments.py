"""Pins of the oracle's per-cell central moments (Sec. 3.6 definition of
u^(p)_{i1..in} = <|c|^p c_i1 .. c_in>, <.> the mean over the cell)."""

from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2606_15622_gb300 import populations as P


def _exact_moments(vcell):
    """Brute force with exact rationals: mean, then central products."""
    n = vcell.shape[1]
    pts = [[Fraction(int(vcell[d, p])) for d in range(3)] for p in range(n)]
    U = [sum(p[d] for p in pts) / n for d in range(3)]
    cs = [[p[d] - U[d] for d in range(3)] for p in pts]
    out = [Fraction(n)] + U + [None] + [Fraction(0)] * 25
    for a, (i, j) in enumerate(O.SYM2):
        out[O.M_U2 + a] = sum(c[i] * c[j] for c in cs) / n
        out[O.M_W + a] = sum((c[0] ** 2 + c[1] ** 2 + c[2] ** 2) * c[i] * c[j] for c in cs) / n
    for a, (i, j, k) in enumerate(O.SYM3):
        out[O.M_U3 + a] = sum(c[i] * c[j] * c[k] for c in cs) / n
    for i in range(3):
        out[O.M_Z + i] = sum((c[0] ** 2 + c[1] ** 2 + c[2] ** 2) ** 2 * c[i] for c in cs) / n
    out[O.M_THETA] = (out[O.M_U2] + out[O.M_U2 + 3] + out[O.M_U2 + 5]) / 3
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_moments_match_exact_rationals_on_integer_cells(seed):
    pop = P.integer_cells([1, 2, 3, 5, 8, 13], lo=-4, hi=4, seed=seed)
    m = O.moments(pop.v64, pop.offsets)
    for c in range(pop.n_cells):
        ex = _exact_moments(pop.v64[:, pop.offsets[c]:pop.offsets[c + 1]])
        scale = max(1.0, max(abs(float(x)) for x in ex))
        for k in range(O.NMOM):
            assert abs(m[c, k] - float(ex[k])) <= 1e-14 * scale, (c, k, m[c, k], ex[k])


def test_gaussian_closed_forms_within_clt_bounds():
    """Large Maxwellian cells: <c_i c_j> = theta delta_ij, odd moments 0,
    <|c|^2 c_i c_j> = 5 theta^2 delta_ij (so <c_1^4> + <c_1^2 c_2^2> +
    <c_1^2 c_3^2> = 3 + 1 + 1 theta^2), <|c|^4> = 15 theta^2, <|c|^4 c_i> = 0."""
    n = 400_000
    theta = 1.7
    pop = P.maxwellian_cells([n], theta=theta, mean=(3.0, -1.0, 0.5), seed=7)
    m = O.moments(pop.v64, pop.offsets)[0]
    c = pop.v64 - pop.v64.mean(axis=1, keepdims=True)
    c2 = (c * c).sum(0)

    def bound(samples):  # 6 standard errors of a sample mean
        return 6.0 * samples.std() / np.sqrt(n)

    for a, (i, j) in enumerate(O.SYM2):
        ex = theta if i == j else 0.0
        assert abs(m[O.M_U2 + a] - ex) < bound(c[i] * c[j])
        ex4 = 5 * theta ** 2 if i == j else 0.0
        assert abs(m[O.M_W + a] - ex4) < bound(c2 * c[i] * c[j])
    for a, (i, j, k) in enumerate(O.SYM3):
        assert abs(m[O.M_U3 + a]) < bound(c[i] * c[j] * c[k])
    for i in range(3):
        assert abs(m[O.M_Z + i]) < bound(c2 * c2 * c[i])
    s4 = m[O.M_W] + m[O.M_W + 3] + m[O.M_W + 5]
    assert abs(s4 - 15 * theta ** 2) < bound(c2 * c2)
    assert abs(m[O.M_THETA] - theta) < bound(c2 / 3)
    # <c_1^4> = 3 theta^2 per component, from the same particles
    assert abs((c[0] ** 4).mean() - 3 * theta ** 2) < bound(c[0] ** 4)
    # <|c|^6> = 3 * 5 * 7 theta^3 (chi-square with 3 degrees of freedom)
    m6 = O.speed_moment6(pop.v64, pop.offsets)[0]
    assert abs(m6 - 105 * theta ** 3) < bound(c2 ** 3)


def test_galilean_invariance(cavity_pop):
    pop = cavity_pop.subset(np.arange(0, 16384, 97))
    m0 = O.moments(pop.v64, pop.offsets)
    shift = np.array([[12.9], [-3.0], [0.25]])
    m1 = O.moments(pop.v64 + shift, pop.offsets)
    np.testing.assert_allclose(m1[:, 1:4], m0[:, 1:4] + shift.T, rtol=1e-13, atol=1e-12)
    scale = np.abs(m0[:, 4:]).max(axis=1, keepdims=True)
    assert np.all(np.abs(m1[:, 4:] - m0[:, 4:]) <= 1e-11 * scale)


def _tensors(m):
    u = np.zeros((3, 3)); w = np.zeros((3, 3)); u3 = np.zeros((3, 3, 3))
    for a, (i, j) in enumerate(O.SYM2):
        u[i, j] = u[j, i] = m[O.M_U2 + a]
        w[i, j] = w[j, i] = m[O.M_W + a]
    import itertools
    for a, idx in enumerate(O.SYM3):
        for perm in itertools.permutations(idx):
            u3[perm] = m[O.M_U3 + a]
    return u, u3, w, m[O.M_Z:O.M_Z + 3]


def test_rotation_covariance(cavity_pop):
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    pop = cavity_pop.subset(np.arange(5, 16384, 211))
    m0 = O.moments(pop.v64, pop.offsets)
    m1 = O.moments(q @ pop.v64, pop.offsets)
    for c in range(pop.n_cells):
        u, u3, w, z = _tensors(m0[c])
        U, U3, Wt, Z = _tensors(m1[c])
        sc = max(1.0, np.abs(m0[c, 4:]).max())
        assert np.abs(U - q @ u @ q.T).max() < 1e-12 * sc
        assert np.abs(Wt - q @ w @ q.T).max() < 1e-12 * sc
        assert np.abs(U3 - np.einsum("ia,jb,kc,abc->ijk", q, q, q, u3)).max() < 1e-12 * sc
        assert np.abs(Z - q @ z).max() < 1e-12 * sc


def test_empty_and_single_particle_cells():
    v = np.array([[1.5], [-2.0], [0.25]])
    offs = np.array([0, 0, 1, 1], dtype=np.int64)
    m = O.moments(v, offs)
    assert np.all(m[0] == 0) and np.all(m[2] == 0)
    assert m[1, O.M_N] == 1
    np.testing.assert_array_equal(m[1, 1:4], v[:, 0])
    assert np.all(m[1, 4:] == 0)


def test_speed_moment6_matches_exact_rationals():
    """<|c|^6> of small integer-velocity cells against exact rational
    arithmetic (mean, centring and the sixth power done in fractions)."""
    from fractions import Fraction
    pop = P.integer_cells([1, 2, 5, 8, 13], lo=-4, hi=4, seed=3)
    got = O.speed_moment6(pop.v64, pop.offsets)
    for k in range(pop.n_cells):
        a, b = pop.offsets[k], pop.offsets[k + 1]
        vs = [[Fraction(int(x)) for x in pop.v64[d, a:b]] for d in range(3)]
        n = b - a
        mean = [sum(col) / n for col in vs]
        ex = sum(sum((vs[d][p] - mean[d]) ** 2 for d in range(3)) ** 3 for p in range(n)) / n
        assert abs(got[k] - float(ex)) <= 1e-12 * max(1.0, abs(float(ex)))
