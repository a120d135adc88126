"""GPU learned closure (features, fused BF16 MLP, loss, backward, Adam,
surrogate with exact fallback) against the numpy reference oracle/mlp.py.

Tolerances: the GPU and the reference round the same BF16 inputs, weights
and activations; they differ by FP32 accumulation order, which moves a few
activations by one BF16 ulp (2^-8 relative) and propagates -- outputs agree
to 2e-2 of their largest magnitude and 3e-3 on average; gradients (BF16
dZ operands) to 3e-2 relative per layer.
"""

import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp as M
from paper_2606_15622_gb300 import api, surrogate as S
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu


def _surrogate_with_random_params(seed=5):
    s = S.Surrogate(eps2_hat=1e-3, seed=seed)
    prm = M.init_params(seed)
    s.set_params(prm["W"], prm["b"])
    return s, prm


def _inputs(n, seed):
    x = np.random.default_rng(seed).standard_normal((n, M.IN)).astype(np.float32)
    x[:, M.NFEAT:] = 0
    return M.bf16_round(x)


@pytest.mark.parametrize("n", [1, 127, 1000, 4099])
def test_forward_matches_reference(n):
    s, prm = _surrogate_with_random_params()
    x = _inputs(n, n)
    xd = torch.from_numpy(x).cuda().to(torch.bfloat16)
    out = s.forward(xd, standardized=True).cpu().numpy()
    ref = M.forward(prm, x.astype(np.float64), bf16=True)
    err = np.abs(out - ref)
    assert err.max() <= 2e-2 * np.abs(ref).max()
    assert err.mean() <= 3e-3 * np.abs(ref).mean()
    # element by element: a relative bound (a few BF16 ulps of the output)
    # plus an absolute one at the scale of the output column, which carries
    # the one-ulp flips of hidden activations through the last layer
    col = np.sqrt((ref ** 2).mean(0, keepdims=True)) if n > 1 else np.abs(ref)
    bound = 2.0 ** -6 * np.abs(ref) + 2.0 ** -6 * col
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("n", [1, 128, 129, 255, 256, 40000])
def test_tensor_core_inference_matches_training_forward(n):
    """The inference pass (persistent tcgen05 kernel, two tile groups a CTA)
    and the training pass (a 128-row tile a CTA, saving the activations)
    round at the same points; they differ only by FP32 accumulation order.
    Sizes cover one row, exact and ragged 128-row tiles, both groups of a CTA
    and many tiles per CTA."""
    s, prm = _surrogate_with_random_params(seed=8)
    x = torch.from_numpy(_inputs(n, 100 + n)).cuda().to(torch.bfloat16)
    o_tc = s.forward(x, standardized=True)
    o_tr = s.forward(x, standardized=True, save=True)[0]
    torch.cuda.synchronize()
    a, b = o_tc.cpu().numpy(), o_tr.cpu().numpy()
    assert np.isfinite(a).all()
    err = np.abs(a - b)
    assert err.max() <= 2e-2 * np.abs(b).max()
    assert err.mean() <= 3e-3 * np.abs(b).mean()


def test_forward_saves_activations_and_unstandardizes():
    s, prm = _surrogate_with_random_params()
    s.y_mu[:9] = torch.linspace(-1, 1, 9, device="cuda")
    s.y_sigma[:9] = torch.linspace(0.5, 2, 9, device="cuda")
    s._net = None
    x = torch.from_numpy(_inputs(300, 1)).cuda().to(torch.bfloat16)
    o_std, h, z = s.forward(x, standardized=True, save=True)
    o_raw_t = s.forward(x, standardized=False, save=True)[0]
    o_inf = s.forward(x, standardized=True)
    o_raw = s.forward(x, standardized=False)
    torch.cuda.synchronize()
    # each kernel undoes the standardisation of its own output exactly
    np.testing.assert_allclose((o_std * s.y_sigma + s.y_mu).cpu().numpy()[:, :9], o_raw_t.cpu().numpy()[:, :9],
                               rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose((o_inf * s.y_sigma + s.y_mu).cpu().numpy()[:, :9], o_raw.cpu().numpy()[:, :9],
                               rtol=1e-6, atol=1e-6)
    # saved activations are SiLU of the saved pre-activations, rounded to BF16
    h, z = S.saved_rows(h), S.saved_rows(z)
    assert h.shape == z.shape == (4, 300, 128)
    # in the documented layout: every layer's pre-activations against the
    # oracle's (BF16 operands, FP32 results)
    _, (hs_ref, zs_ref) = M.forward(prm, x.float().cpu().numpy().astype(np.float64), bf16=True, keep=True)
    for l in range(4):
        zr = zs_ref[l]
        err = np.abs(z[l].cpu().numpy() - zr)
        assert np.all(err <= 2.0 ** -6 * np.abs(zr) + 2.0 ** -6 * np.sqrt((zr ** 2).mean(0, keepdims=True))), l
    np.testing.assert_allclose(h.float().cpu().numpy(), M.bf16_round(M.silu(z.cpu().numpy())), rtol=1e-2, atol=1e-3)


def _loss_args(n, seed):
    rng = np.random.default_rng(seed)
    pop = P.cavity(seed=seed, nx=32, ny=32)
    m = O.moments(pop.v64, pop.offsets)[:n]
    y, fl = O.closure(m, pop.tau[:n])
    t_true = M.targets(y, m, pop.tau[:n])
    out = rng.standard_normal((n, M.OUT)) * 0.5
    y_mu = np.zeros(16)
    y_sigma = np.ones(16)
    y_mu[:9] = t_true.mean(0)
    y_sigma[:9] = t_true.std(0) + 1e-3
    f = M.raw_features(m)
    aux = np.zeros((n, 16))
    aux[:, :6] = f[:, :6]
    aux[:, 6] = f[:, 6] + f[:, 9] + f[:, 11]
    aux[:, 7] = f[:, 7] + f[:, 12] + f[:, 14]
    aux[:, 8] = f[:, 8] + f[:, 13] + f[:, 15]
    aux[:, 9] = f[:, 16] + f[:, 19] + f[:, 21]
    return out, t_true, aux, y_mu, y_sigma, m


def test_loss_gradient_matches_reference_finite_differences():
    n = 64
    out, t_true, aux, y_mu, y_sigma, m = _loss_args(n, 3)
    w = np.array([1.0] * 6 + [2.0] * 3, dtype=np.float32)
    lam_d, lam_e, eps2 = 0.1, 1.0, 1e-3
    dev = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    dout = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    doutb = torch.empty((n, 16), dtype=torch.bfloat16, device="cuda")
    ls = torch.zeros(1, dtype=torch.float32, device="cuda")
    import ctypes
    L = api.lib()
    keep = [dev(out), dev(t_true), dev(aux), dev(y_mu), dev(y_sigma)]  # alive until the kernel has run
    rc = L.fp_surrogate_loss(*[api._ptr(t) for t in keep], n, (ctypes.c_float * 9)(*w.tolist()), lam_d, lam_e,
                             eps2, 1.0, api._ptr(dout), api._ptr(doutb), api._ptr(ls), api._stream(None))
    assert rc == 0
    torch.cuda.synchronize()
    ref_loss = M.loss(out, t_true, m, y_mu[:9], y_sigma[:9], eps2, w, lam_d, lam_e)
    assert abs(float(ls.item()) / n - ref_loss) <= 1e-4 * abs(ref_loss)
    g = dout.cpu().numpy()
    h = 1e-5
    rng = np.random.default_rng(0)
    for _ in range(20):
        r, a = rng.integers(n), rng.integers(9)
        op, om = out.copy(), out.copy()
        op[r, a] += h
        om[r, a] -= h
        fd = (M.loss(op, t_true, m, y_mu[:9], y_sigma[:9], eps2, w, lam_d, lam_e)
              - M.loss(om, t_true, m, y_mu[:9], y_sigma[:9], eps2, w, lam_d, lam_e)) / (2 * h) * n
        assert abs(g[r, a] - fd) <= 2e-3 * max(1.0, abs(fd)), (r, a, g[r, a], fd)
    assert np.all(g[:, 9:] == 0)


def test_backward_matches_reference():
    n = 2048
    s, prm = _surrogate_with_random_params(7)
    x = _inputs(n, 11)
    xd = torch.from_numpy(x).cuda().to(torch.bfloat16)
    out, h, z = s.forward(xd, standardized=True, save=True)
    dout = np.random.default_rng(2).standard_normal((n, 16)).astype(np.float32) / n
    dout[:, 9:] = 0
    dd = torch.from_numpy(dout).cuda()
    grads = torch.zeros(S.param_count(), dtype=torch.float32, device="cuda")
    ws = torch.empty(int(api.lib().fp_mlp_backward_workspace_bytes(n)), dtype=torch.uint8, device="cuda")
    import ctypes
    dd_bf = dd.to(torch.bfloat16)
    rc = api.lib().fp_mlp_backward(ctypes.byref(s.net()), api._ptr(xd), api._ptr(h), api._ptr(z),
                                   api._ptr(dd_bf), api._ptr(dd), n, api._ptr(grads), api._ptr(ws),
                                   ws.numel(), api._stream(None))
    assert rc == 0
    torch.cuda.synchronize()
    # reference: FP64 reverse mode on the BF16-rounded forward
    pb = {"W": [M.bf16_round(w).astype(np.float64) for w in prm["W"]], "b": prm["b"]}
    _, cache = M.forward(pb, x.astype(np.float64), bf16=True, keep=True)
    dW, db, _ = M.backward(pb, cache, M.bf16_round(dout).astype(np.float64))
    g = grads.cpu().numpy()
    for l in range(5):
        gw = g[S.param_offset(0, l):S.param_offset(0, l) + dW[l].size].reshape(dW[l].shape)
        gb = g[S.param_offset(1, l):S.param_offset(1, l) + db[l].size]
        assert np.linalg.norm(gw - dW[l]) <= 3e-2 * np.linalg.norm(dW[l]), l
        assert np.linalg.norm(gb - db[l]) <= 3e-2 * np.linalg.norm(db[l]) + 1e-12, l


def test_adam_matches_reference():
    n = 5000
    rng = np.random.default_rng(1)
    p, g = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
    m, v = np.zeros(n, np.float32), np.zeros(n, np.float32)
    P_, G_, M_, V_ = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    sh = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    pr, mr, vr = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in (1, 2, 3):
        rc = api.lib().fp_adam_step(api._ptr(P_), api._ptr(G_), api._ptr(M_), api._ptr(V_), n, 1e-2, 0.9, 0.999,
                                    1e-8, t, api._ptr(sh), api._stream(None))
        assert rc == 0
        pr, mr, vr = M.adam_step(pr, g.astype(np.float64), mr, vr, t, lr=1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(P_.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    assert torch.equal(sh, P_.to(torch.bfloat16))


def test_fused_training_step_matches_the_four_calls_and_the_oracle():
    """fp_surrogate_train_step (the loss fused into the forward's last layer,
    Adam into the gradient tile sum) against the four calls it fuses, its
    loss against the oracle's, and its parameter update against the oracle's
    Adam applied to its own gradient.  1000 rows: seven full 128-row tiles and
    a ragged one."""
    n = 1000
    _, t_true, aux, y_mu, y_sigma, m = _loss_args(n, 5)
    x = _inputs(n, 21)
    dev = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    xd, td, ad = dev(x, torch.bfloat16), dev(t_true), dev(aux)
    trainers = []
    for fused in (True, False):
        s, prm = _surrogate_with_random_params(9)
        s.y_mu.copy_(dev(y_mu))
        s.y_sigma.copy_(dev(y_sigma))
        s._net = None
        trainers.append(S.Trainer(s, batch=n, fused=fused))
    tf, tu = trainers
    out = tf.s.forward(xd, standardized=True).cpu().numpy().astype(np.float64)
    p0, m0, v0 = (a.cpu().numpy().astype(np.float64) for a in (tf.s.params, tf.m, tf.v))
    for tr in trainers:
        tr.step(xd, td, ad, 1.0 / n)
    torch.cuda.synchronize()
    # the same loss and gradient as the four calls (FP32 order of the fused kernels)
    lf, lu = float(tf.loss_acc.item()), float(tu.loss_acc.item())
    assert abs(lf - lu) <= 1e-5 * abs(lu)
    gf, gu = tf.grads.cpu().numpy().astype(np.float64), tu.grads.cpu().numpy().astype(np.float64)
    for l in range(5):
        for which in (0, 1):
            a, b = S.param_offset(which, l), (S.param_offset(1, l) if which == 0 else
                                              (S.param_offset(0, l + 1) if l < 4 else S.param_count()))
            assert np.linalg.norm(gf[a:b] - gu[a:b]) <= 1e-3 * np.linalg.norm(gu[a:b]) + 1e-12, (l, which)
    # the loss against the oracle's, on the network's standardised outputs
    ref = M.loss(out, t_true, m, y_mu[:9], y_sigma[:9], 1e-3, tf.w.astype(np.float64), tf.lam_drift,
                 tf.lam_energy)
    assert abs(lf / n - ref) <= 1e-4 * abs(ref)
    # Adam on the step's own gradient
    pr, mr, vr = M.adam_step(p0, gf, m0, v0, 1, lr=tf.lr)
    np.testing.assert_allclose(tf.s.params.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(tf.m.cpu().numpy(), mr, rtol=1e-5, atol=1e-9)
    # 1 - beta2 evaluated in FP32 is 1e-3 (1 - 1.3e-5)
    np.testing.assert_allclose(tf.v.cpu().numpy(), vr, rtol=3e-5, atol=1e-12)
    assert torch.equal(tf.s.shadow, tf.s.params.to(torch.bfloat16))


def test_surrogate_fallback_is_exact_for_flagged_cells(cavity_pop):
    """An untrained network fails the energy check on essentially every cell;
    those cells must come back with the exact FP64 closure."""
    s, _ = _surrogate_with_random_params(3)
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 9))
    mom = torch.from_numpy(O.moments(pop.v64, pop.offsets)).cuda()
    tau = torch.from_numpy(pop.tau).cuda()
    y, fl = s.closure(mom, tau)
    torch.cuda.synchronize()
    y, fl = y.cpu().numpy(), fl.cpu().numpy()
    yr, flr = O.closure(mom.cpu().numpy(), pop.tau)
    fb = (fl & api.FLAG_FALLBACK) != 0
    assert fb.mean() > 0.95
    err = np.linalg.norm(y[fb] - yr[fb], axis=1) / np.linalg.norm(yr[fb], axis=1)
    assert err.max() <= 1e-10
    assert np.all((fl[fb] & api.FALLBACK_FLAGS) == flr[fb])


def test_training_reduces_error_below_linear_closure():
    """Train on 60k cells for a few epochs with the library's kernels: the
    loss falls and the trained network's coefficients (on held-out cells,
    before any fallback) beat the linear-drift closure by a wide margin."""
    train = P.training_cells(60000, seed=101)
    ts = S.TrainingSet(train, eps2_hat=1e-3)
    s = S.Surrogate(eps2_hat=1e-3, seed=9)
    s.init_params()
    S.fit_scalers(s, ts)
    tr = S.Trainer(s, batch=4096, lr=2e-3)
    hist = tr.fit(ts, epochs=6, seed=1)
    assert hist[-1] < 0.5 * hist[0]
    test = P.training_cells(4000, seed=202)
    tt = S.TrainingSet(test, eps2_hat=1e-3)
    x = tt.inputs(s)
    pred = s.forward(x, standardized=False)[:, :9]
    torch.cuda.synchronize()
    err_net = ((pred - tt.t).norm(dim=1) / tt.t.norm(dim=1)).median().item()
    lin = torch.zeros_like(tt.t)
    lin[:, [0, 3, 5]] = -1.0
    err_lin = ((lin - tt.t).norm(dim=1) / tt.t.norm(dim=1)).median().item()
    assert err_net < 0.5 * err_lin, (err_net, err_lin)
