"""GPU LITE path (moment pass up to the heat flux, the 16 network inputs, the
learned closure on them) against the oracle (oracle/lite.py, oracle/mlp.py).

Tolerances: the LITE pass sums in FP32 with compensation, so each moment
agrees with the FP64 oracle to 1e-5 of its natural scale (theta^(k/2) for
order k); N is exact.  Standardised inputs are rounded to BF16 on both
sides, which may land one BF16 ulp apart (2^-7 relative).  The network
outputs agree as in the full-input network's tests (2e-2 of the largest
magnitude, 3e-3 on average).
"""

import numpy as np
import pytest
import torch

from oracle import lite as L
from oracle import mlp as M
from paper_2606_15622_gb300 import api, surrogate as S
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu

COUNTS = [0, 1, 2, 3, 4, 7, 8, 9, 15, 16, 17, 127, 128, 129, 130, 1000, 5000, 70000, 0, 5]


def _scale(m):
    th = np.maximum(m[:, L.L_THETA], 1e-300)
    return np.sqrt(th)


def _check_lite(got, ref):
    np.testing.assert_array_equal(got[:, L.L_N], ref[:, L.L_N])
    s = _scale(ref)[:, None]
    assert np.all(np.abs(got[:, L.L_U:L.L_U + 3] - ref[:, L.L_U:L.L_U + 3]) <= 1e-5 * s + 1e-6 *
                  np.abs(ref[:, L.L_U:L.L_U + 3]))
    assert np.all(np.abs(got[:, L.L_THETA] - ref[:, L.L_THETA]) <= 1e-5 * s[:, 0] ** 2)
    assert np.all(np.abs(got[:, L.L_U2:L.L_U2 + 6] - ref[:, L.L_U2:L.L_U2 + 6]) <= 1e-5 * s ** 2)
    assert np.all(np.abs(got[:, L.L_B:L.L_B + 3] - ref[:, L.L_B:L.L_B + 3]) <= 1e-5 * s ** 3)


@pytest.mark.parametrize("vdtype", ["f32", "f64"])
def test_lite_moments_match_oracle(vdtype):
    pop = P.maxwellian_cells(COUNTS, theta=0.6, mean=(2.0, -1.0, 0.5), seed=21)
    v = pop.v32.astype(np.float64) if vdtype == "f32" else pop.v64
    vd = torch.from_numpy(pop.v32 if vdtype == "f32" else pop.v64).cuda()
    got = api.fp_moments_lite(vd, torch.from_numpy(pop.offsets).cuda()).cpu().numpy()
    ref = L.lite_moments(v, pop.offsets)
    _check_lite(got, ref)


@pytest.mark.parametrize("vdtype", ["f32", "f64"])
def test_lite_moments_match_oracle_on_cavity(cavity_pop, vdtype):
    """FP32 velocities take the shared-memory streamed gather, FP64 ones the
    direct one."""
    pop = cavity_pop
    v = pop.v32 if vdtype == "f32" else pop.v64
    got = api.fp_moments_lite(torch.from_numpy(v).cuda(), torch.from_numpy(pop.offsets).cuda())
    torch.cuda.synchronize()
    _check_lite(got.cpu().numpy(), L.lite_moments(v.astype(np.float64), pop.offsets))


def test_lite_moments_unaligned_velocities():
    """Velocities not 16-byte aligned (a view one float into a buffer) take
    the direct gather; results agree all the same."""
    pop = P.maxwellian_cells([5, 300, 0, 3000, 17], theta=1.3, seed=8)
    n = pop.n_particles
    buf = torch.zeros(3 * n + 1, dtype=torch.float32, device="cuda")
    buf[1:].copy_(torch.from_numpy(pop.v32.reshape(-1)))
    v = buf[1:].view(3, n)
    got = api.fp_moments_lite(v, torch.from_numpy(pop.offsets).cuda()).cpu().numpy()
    _check_lite(got, L.lite_moments(pop.v32.astype(np.float64), pop.offsets))


def test_lite_moments_full_size_sampled():
    """The cylinder population at full size: sampled cells against the
    oracle (computed one by one)."""
    pop = P.cylinder()
    got = api.fp_moments_lite(torch.from_numpy(pop.v32).cuda(), torch.from_numpy(pop.offsets).cuda()).cpu().numpy()
    rng = np.random.default_rng(0)
    cells = np.unique(np.concatenate([rng.choice(pop.n_cells, 300, replace=False), [0, pop.n_cells - 1],
                                      np.argsort(pop.counts)[-3:]]))
    for c in cells:
        a, e = pop.offsets[c], pop.offsets[c + 1]
        ref = L.lite_moments(pop.v32[:, a:e].astype(np.float64), [0, e - a])
        _check_lite(got[c:c + 1], ref)


def _lite_surrogate(seed=5):
    s = S.Surrogate(eps2_hat=1e-3, seed=seed, features="lite")
    prm = M.init_params(seed)
    s.set_params(prm["W"], prm["b"])
    return s, prm


def _set_scalers(s, f):
    nf = S.NFEAT_LITE
    s.x_mu[:nf] = torch.from_numpy(f.mean(0)).float()
    s.x_sigma[:nf] = torch.from_numpy(f.std(0).clip(1e-6)).float()
    s.y_mu[:9] = torch.linspace(-1.0, 0.5, 9)
    s.y_sigma[:9] = torch.linspace(0.2, 1.0, 9)
    s._net = None


def _ref_inputs(s, f):
    mu = s.x_mu.cpu().numpy().astype(np.float64)
    sg = s.x_sigma.cpu().numpy().astype(np.float64)
    x = np.zeros((f.shape[0], M.IN))
    x[:, :S.NFEAT_LITE] = (f - mu[:S.NFEAT_LITE]) / sg[:S.NFEAT_LITE]
    return M.bf16_round(x.astype(np.float32)).astype(np.float64)


def test_lite_features_match_oracle(cavity_pop):
    pop = cavity_pop
    lite = L.lite_moments(pop.v64, pop.offsets)
    f = L.lite_features(lite, pop.tau)
    s, _ = _lite_surrogate()
    ok = pop.counts >= 4
    _set_scalers(s, f[ok])
    x, fl = s.lite_features(torch.from_numpy(lite).cuda(), torch.from_numpy(pop.tau).cuda())
    torch.cuda.synchronize()
    x, fl = x.float().cpu().numpy(), fl.cpu().numpy()
    xr = _ref_inputs(s, f)
    assert np.all(x[:, S.NFEAT_LITE:] == 0)
    d = np.abs(x - xr)[ok]
    assert np.all(d <= 2.0 ** -7 * np.abs(xr[ok]) + 1e-4)  # inputs formed in FP32, rounded to BF16
    few = (pop.counts < api.default_params().min_particles)
    np.testing.assert_array_equal((fl & api.FLAG_FEW) != 0, few)
    np.testing.assert_array_equal((fl & api.FLAG_SINGULAR) != 0, lite[:, L.L_THETA] <= 0)
    assert np.all((fl & api.FLAG_NONFINITE) == 0)


def test_lite_feature_flags_on_constructed_rows():
    s, _ = _lite_surrogate()
    rows = np.zeros((5, L.NLITE))
    rows[:, L.L_N] = [10, 2, 10, 10, 10]
    rows[:, L.L_THETA] = [1.0, 1.0, 0.0, 1.0, 1.0]
    rows[:, L.L_U2 + 0] = rows[:, L.L_U2 + 3] = rows[:, L.L_U2 + 5] = rows[:, L.L_THETA]
    rows[3, L.L_B + 1] = np.nan
    tau = np.array([1.0, 1.0, 1.0, 1.0, -1.0])
    s.x_min[:S.NFEAT_LITE] = -1e6
    s.x_max[:S.NFEAT_LITE] = 1e6
    s.x_max[0] = 5.0  # rho box: N = 10 is outside, N = 2 inside
    s.x_sigma[0] = 1.0
    s._net = None
    x, fl = s.lite_features(torch.from_numpy(rows).cuda(), torch.from_numpy(tau).cuda())
    fl = fl.cpu().numpy()
    assert fl[0] == api.FLAG_RANGE
    assert fl[1] == api.FLAG_FEW
    assert fl[2] == api.FLAG_RANGE | api.FLAG_SINGULAR
    assert fl[3] & api.FLAG_NONFINITE and fl[4] & api.FLAG_NONFINITE


def test_lite_closure_matches_oracle(cavity_pop):
    pop = cavity_pop
    vd, offd = torch.from_numpy(pop.v64).cuda(), torch.from_numpy(pop.offsets).cuda()
    taud = torch.from_numpy(pop.tau).cuda()
    lite_ref = L.lite_moments(pop.v64, pop.offsets)
    f = L.lite_features(lite_ref, pop.tau)
    s, prm = _lite_surrogate(seed=7)
    ok = pop.counts >= 4
    _set_scalers(s, f[ok])
    lite = api.fp_moments_lite(vd, offd)
    y, fl = s.closure_lite(lite, taud)
    torch.cuda.synchronize()
    y, fl = y.cpu().numpy(), fl.cpu().numpy()
    # oracle: inputs -> network -> un-standardised targets -> coefficients
    out = M.forward(prm, _ref_inputs(s, f), bf16=True)[:, :9]
    t = out * s.y_sigma[:9].cpu().numpy() + s.y_mu[:9].cpu().numpy()
    th = lite_ref[:, L.L_THETA]
    yr = np.zeros((pop.n_cells, 9))
    yr[ok, :6] = t[ok, :6] / pop.tau[ok, None]
    yr[ok, 6:] = t[ok, 6:] / (pop.tau[ok] * np.sqrt(th[ok]))[:, None]
    lin = np.zeros(9)
    lin[[0, 3, 5]] = 1.0
    yr[~ok] = -lin[None, :] / pop.tau[~ok, None]
    assert np.all(((fl & api.FALLBACK_FLAGS) != 0) == ~ok)
    np.testing.assert_array_equal(y[~ok], yr[~ok])
    td = np.empty_like(y)
    td[:, :6] = y[:, :6] * pop.tau[:, None]
    td[:, 6:] = y[:, 6:] * (pop.tau * np.sqrt(np.where(ok, th, 1.0)))[:, None]
    err = np.abs(td - t)[ok]
    assert err.max() <= 2e-2 * np.abs(t[ok]).max()
    assert err.mean() <= 3e-3 * np.abs(t[ok]).mean()


def test_lite_weight_file_round_trip(tmp_path):
    s, _ = _lite_surrogate(seed=3)
    p = str(tmp_path / "lite.fpw")
    s.save(p)
    r = S.Surrogate.load(p)
    assert r.features_set == "lite" and r.nfeat == S.NFEAT_LITE
    assert torch.equal(r.params, s.params)
    with pytest.raises(api.FPError):
        r.closure(torch.zeros((1, api.NMOM), dtype=torch.float64, device="cuda"),
                  torch.ones(1, dtype=torch.float64, device="cuda"))


def test_lite_training_beats_linear_closure():
    """A short LITE training run with the library's kernels: the loss falls
    and held-out coefficients beat the linear-drift closure."""
    ts = S.TrainingSet(P.training_cells(60000, seed=101), eps2_hat=1e-3, features="lite")
    assert ts.f.shape[1] == S.NFEAT_LITE
    s = S.Surrogate(eps2_hat=1e-3, seed=9, features="lite")
    s.init_params()
    S.fit_scalers(s, ts)
    tr = S.Trainer(s, batch=4096, lr=2e-3)
    hist = tr.fit(ts, epochs=6, seed=1)
    assert hist[-1] < 0.5 * hist[0]
    tt = S.TrainingSet(P.training_cells(4000, seed=202), eps2_hat=1e-3, features="lite")
    pred = s.forward(tt.inputs(s), standardized=False)[:, :9]
    torch.cuda.synchronize()
    err_net = ((pred - tt.t).norm(dim=1) / tt.t.norm(dim=1)).median().item()
    lin = torch.zeros_like(tt.t)
    lin[:, [0, 3, 5]] = -1.0
    err_lin = ((lin - tt.t).norm(dim=1) / tt.t.norm(dim=1)).median().item()
    assert err_net < err_lin, (err_net, err_lin)


def test_lite_argument_errors():
    s, _ = _lite_surrogate()
    lite = torch.zeros((4, L.NLITE), dtype=torch.float64, device="cuda")
    tau = torch.ones(4, dtype=torch.float64, device="cuda")
    # the fused closure needs no workspace: an empty one is accepted
    assert api.lib().fp_surrogate_lite_workspace_bytes(4) == 0
    s.closure_lite(lite, tau, workspace=torch.empty(0, dtype=torch.uint8, device="cuda"))
    # a full-input network refuses LITE vectors
    with pytest.raises(api.FPError):
        S.Surrogate(eps2_hat=1e-3, seed=1).closure_lite(lite, tau)
    with pytest.raises(api.FPError):
        api.fp_moments_lite(torch.zeros((3, 4), dtype=torch.float16, device="cuda"),
                            torch.tensor([0, 4], dtype=torch.int64, device="cuda"))
