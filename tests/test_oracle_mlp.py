"""Pins of the learned-closure reference (oracle/mlp.py)."""

import numpy as np
import torch

import oracle as O
from oracle import mlp as M
from paper_2606_15622_gb300 import populations as P


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 10
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(M.bf16_round(x), ref)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(1)
    prm = M.init_params(3)
    x = rng.standard_normal((7, M.IN))
    x[:, M.NFEAT:] = 0
    g = rng.standard_normal((7, M.OUT))
    out, cache = M.forward(prm, x, keep=True)
    dW, db, dx = M.backward(prm, cache, g)
    h = 1e-6
    for l, (i, j) in [(0, (5, 3)), (2, (17, 100)), (4, (2, 64)), (3, (127, 0))]:
        p1 = {"W": [w.copy() for w in prm["W"]], "b": prm["b"]}
        p2 = {"W": [w.copy() for w in prm["W"]], "b": prm["b"]}
        p1["W"][l][i, j] += h
        p2["W"][l][i, j] -= h
        fd = ((M.forward(p1, x) - M.forward(p2, x)) * g).sum() / (2 * h)
        assert abs(fd - dW[l][i, j]) < 1e-6 * max(1.0, abs(fd))
    for l, i in [(1, 7), (4, 3)]:
        p1 = {"W": prm["W"], "b": [b.copy() for b in prm["b"]]}
        p2 = {"W": prm["W"], "b": [b.copy() for b in prm["b"]]}
        p1["b"][l][i] += h
        p2["b"][l][i] -= h
        fd = ((M.forward(p1, x) - M.forward(p2, x)) * g).sum() / (2 * h)
        assert abs(fd - db[l][i]) < 1e-6 * max(1.0, abs(fd))


def test_silu_gradient_closed_form():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.silu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_targets_are_scale_invariant(cavity_pop):
    """The dimensionless map: scaling velocities by s leaves features and
    targets unchanged (C -> C, G -> G/s, theta -> s^2 theta)."""
    pop = cavity_pop.subset(np.arange(0, 16384, 401))
    m0 = O.moments(pop.v64, pop.offsets)
    y0, _ = O.closure(m0, pop.tau)
    m1 = O.moments(2.5 * pop.v64, pop.offsets)
    y1, _ = O.closure(m1, pop.tau)
    np.testing.assert_allclose(M.raw_features(m1), M.raw_features(m0), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(M.targets(y1, m1, pop.tau), M.targets(y0, m0, pop.tau), rtol=1e-8, atol=1e-10)


def test_energy_residual_vanishes_for_exact_closure(cavity_pop):
    pop = cavity_pop.subset(np.arange(0, 16384, 211))
    m = O.moments(pop.v64, pop.offsets)
    y, fl = O.closure(m, pop.tau, eps2_hat=0.01)
    e = M.energy_residual(M.targets(y, m, pop.tau), m, 0.01)
    assert np.abs(e[fl == 0]).max() < 1e-10
    # and the linear drift C = -I/tau, G = 0 has e = 1 - 1 - eps2_hat s4_hat / 3
    lin = np.zeros_like(y)
    lin[:, [0, 3, 5]] = -1.0 / pop.tau[:, None]
    e_lin = M.energy_residual(M.targets(lin, m, pop.tau), m, 0.0)
    assert np.abs(e_lin).max() < 1e-12


def test_drift_matrix_matches_particle_sums(cavity_pop):
    """d^T Q d equals tau^2/theta <|dA|^2> summed particle by particle."""
    pop = cavity_pop.subset([3, 999, 5000])
    m = O.moments(pop.v64, pop.offsets)
    Q = M.drift_matrix(m)
    rng = np.random.default_rng(2)
    for c in range(pop.n_cells):
        d = rng.standard_normal(9)
        vc = pop.v64[:, pop.offsets[c]:pop.offsets[c + 1]]
        cc = vc - vc.mean(1, keepdims=True)
        th = m[c, 4]
        tau = pop.tau[c]
        dC = np.zeros((3, 3))
        for a, (i, j) in enumerate(M.SYM2):
            dC[i, j] = dC[j, i] = d[a] / tau
        dG = d[6:] / (tau * np.sqrt(th))
        c2 = (cc * cc).sum(0)
        dA = dC @ cc + dG[:, None] * (c2 - 3 * th)[None, :]
        direct = (dA * dA).sum(0).mean() * tau ** 2 / th
        assert abs(d @ Q[c] @ d - direct) < 1e-10 * max(1.0, direct)


def test_adam_first_step_is_sign_times_lr():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -0.25, 0.0])
    p2, m, v = M.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.1)
    np.testing.assert_allclose(p2[:2], p[:2] - 0.1 * np.sign(g[:2]), rtol=1e-6)
    assert p2[2] == p[2]


def test_vectorised_philox_known_answers():
    """The numpy Philox of the dropout probe against the published known
    answers (the same file that pins the C generator of the noise)."""
    import os
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = [[int(x, 16) for x in ln.split()] for ln in open(golden) if ln.strip() and not ln.startswith("#")]
    for w in rows:
        out = M.philox4x32_10(np.array(w[0:4], dtype=np.uint64), (w[4], w[5]))
        assert list(out) == w[6:10]


def test_dropout_masks_rate_and_independence():
    n, rate = 2000, 0.2
    s = M.dropout_scales(np.arange(n), 3, seed=99, rate=rate)
    dropped = s == 0.0
    # Bernoulli(rate) within 5 standard errors, per layer; kept units scaled by 1/(1-rate)
    for l in range(4):
        assert abs(dropped[l].mean() - rate) < 5 * np.sqrt(rate * (1 - rate) / dropped[l].size)
    assert np.allclose(s[~dropped], np.float32(1.25))
    # other passes, seeds and cells draw other masks
    assert (M.dropout_scales(np.arange(n), 4, 99, rate) != s).mean() > 0.2
    assert (M.dropout_scales(np.arange(n), 3, 98, rate) != s).mean() > 0.2
    assert (s[:, :-1] != s[:, 1:]).mean() > 0.2
    # a cell's masks depend on its index, not on its place in the batch
    assert np.array_equal(M.dropout_scales(np.arange(n) + 1, 3, 99, rate)[:, :-1], s[:, 1:])
    # rate 0 keeps everything unscaled
    assert np.all(M.dropout_scales(np.arange(10), 0, 1, 0.0) == 1.0)


def test_sensitivity_special_cases():
    prm = M.init_params(3)
    rng = np.random.default_rng(0)
    x = M.bf16_round(rng.standard_normal((50, M.IN)).astype(np.float32)).astype(np.float64)
    x[:, M.NFEAT:] = 0
    y_mu, y_sigma = np.zeros(16), np.ones(16)
    tau, theta = np.full(50, 2.0), np.full(50, 4.0)
    # rate 0: every pass is the plain forward; no spread, mean = forward / scale
    sig, mean = M.sensitivity(prm, x, y_mu, y_sigma, tau, theta, np.arange(50), 3, 0.0, seed=1)
    assert np.all(sig == 0.0)
    ref = M.forward(prm, x, bf16=True)[:, :9]
    np.testing.assert_allclose(mean[:, :6], ref[:, :6] / 2.0, rtol=1e-15)
    np.testing.assert_allclose(mean[:, 6:], ref[:, 6:] / 4.0, rtol=1e-15)
    # with dropout: the aggregates are the norms of the per-coefficient sigmas,
    # sigma equals the 1/N spread of the passes computed by hand
    sig, _ = M.sensitivity(prm, x, y_mu, y_sigma, tau, theta, np.arange(50), 5, 0.2, seed=7)
    ys = np.stack([M.forward_dropout(prm, x, M.dropout_scales(np.arange(50), k, 7, 0.2))[:, :9] for k in range(5)])
    by_hand = np.sqrt(((ys - ys.mean(0)) ** 2).mean(0))
    np.testing.assert_allclose(sig[:, :6], by_hand[:, :6] / 2.0, rtol=1e-12)
    np.testing.assert_allclose(sig[:, 6:9], by_hand[:, 6:] / 4.0, rtol=1e-12)
    np.testing.assert_allclose(sig[:, 9], np.linalg.norm(sig[:, :6], axis=1), rtol=1e-14)
    np.testing.assert_allclose(sig[:, 10], np.linalg.norm(sig[:, 6:9], axis=1), rtol=1e-14)
    assert np.all(sig[:, 9] > 0)
