"""The learned closure's inputs and training rows, element by element against
oracle/mlp.py and oracle/lite.py.

fp_surrogate_features forms each raw input in FP32 from the FP64 moments,
standardises it in FP32 and rounds to BF16; the oracle does the same in FP64
and rounds once.  The two then differ by at most one BF16 ulp of the value,
plus the FP32 cancellation of the standardisation (x - mu) / sigma when the
raw input lies near its mean (2^-22 of (|x| + |mu|) / sigma).
fp_surrogate_training_rows: the raw inputs to FP32 rounding of the FP64
definitions, the dimensionless targets to half an FP32 ulp, the auxiliary
moments to the FP32 rounding of their three-term sums.
"""

import numpy as np
import pytest
import torch

import oracle as O
from oracle import lite as L
from oracle import mlp as M
from paper_2606_15622_gb300 import api, surrogate as S

pytestmark = pytest.mark.gpu


def _bf16_ulp(x):
    a = np.abs(np.asarray(x, dtype=np.float64))
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 0.0)


def _surrogate(features, f, margin_box=True):
    s = S.Surrogate(eps2_hat=1e-3, seed=3, features=features)
    prm = M.init_params(3)
    s.set_params(prm["W"], prm["b"])
    nf = f.shape[1]
    s.x_mu[:nf] = torch.from_numpy(f.mean(0)).float()
    s.x_sigma[:nf] = torch.from_numpy(f.std(0).clip(1e-6)).float()
    s.x_min[:nf] = torch.from_numpy(f.min(0)).float()
    s.x_max[:nf] = torch.from_numpy(f.max(0)).float()
    s._net = None
    return s


def _check_inputs(x, f, s):
    nf = f.shape[1]
    mu = s.x_mu[:nf].cpu().numpy().astype(np.float64)
    sg = s.x_sigma[:nf].cpu().numpy().astype(np.float64)
    xr = M.bf16_round(((f - mu) / sg).astype(np.float64)).astype(np.float64)
    exact = (f - mu) / sg
    tol = _bf16_ulp(exact) + 2.0 ** -22 * (np.abs(f) + np.abs(mu)) / sg
    d = np.abs(x[:, :nf] - xr)
    assert np.all(d <= tol), (d / np.maximum(tol, 1e-300)).max()
    assert np.all(x[:, nf:] == 0)


def test_full_features_match_oracle_elementwise(cavity_pop):
    pop = cavity_pop
    m = O.moments(pop.v64, pop.offsets)
    ok = (pop.counts >= 4) & (m[:, O.M_THETA] > 0)
    f = M.raw_features(m)
    s = _surrogate("full", f[ok])
    x, fl = s.features(torch.from_numpy(m).cuda(), torch.from_numpy(pop.tau).cuda())
    torch.cuda.synchronize()
    x, fl = x.float().cpu().numpy().astype(np.float64), fl.cpu().numpy()
    _check_inputs(x[ok], f[ok], s)
    few = pop.counts < api.default_params().min_particles
    np.testing.assert_array_equal((fl & api.FLAG_FEW) != 0, few)
    np.testing.assert_array_equal((fl & api.FLAG_SINGULAR) != 0, ~(m[:, O.M_THETA] > 0))
    # every fitted cell lies inside the box it was fitted on
    assert np.all((fl[ok] & api.FLAG_RANGE) == 0)


def test_full_feature_flags_on_constructed_rows():
    """Maxwellian moment rows (theta = 1: u = I, w = 5 I, the rest 0) inside a
    unit box, with one input pushed out per row, too few particles, theta = 0,
    a NaN moment and a non-positive tau."""
    base = np.zeros(O.NMOM)
    base[O.M_N] = 50
    base[O.M_THETA] = 1.0
    for k in (0, 3, 5):
        base[O.M_U2 + k] = 1.0
        base[O.M_W + k] = 5.0
    rows = np.tile(base, (7, 1))
    rows[1, O.M_U3 + 4] = 3.0          # u_123 / theta^1.5 = 3: outside [-1 - m, 1 + m]
    rows[2, O.M_Z + 1] = -4.0          # z_2 / theta^2.5 = -4: outside
    rows[3, O.M_N] = 2                 # too few
    rows[4, O.M_THETA] = 0.0           # theta = 0
    rows[5, O.M_W + 2] = np.nan        # non-finite
    tau = np.ones(7)
    tau[6] = 0.0                       # tau must be positive
    f = M.raw_features(base[None])
    s = _surrogate("full", np.vstack([f, f]))
    nf = M.NFEAT
    s.x_mu[:nf] = 0
    s.x_sigma[:nf] = 1
    s.x_min[:nf] = torch.from_numpy(np.minimum(f[0], 0) - 1).float()
    s.x_max[:nf] = torch.from_numpy(np.maximum(f[0], 0) + 1).float()
    s._net = None
    _, fl = s.features(torch.from_numpy(rows).cuda(), torch.from_numpy(tau).cuda())
    fl = fl.cpu().numpy()
    assert fl[0] == 0
    assert fl[1] == api.FLAG_RANGE and fl[2] == api.FLAG_RANGE
    assert fl[3] == api.FLAG_FEW
    assert fl[4] & api.FLAG_SINGULAR
    assert fl[5] & api.FLAG_NONFINITE and fl[6] & api.FLAG_NONFINITE


def test_lite_inputs_match_oracle_elementwise(cavity_pop):
    pop = cavity_pop
    lite = L.lite_moments(pop.v64, pop.offsets)
    ok = (pop.counts >= 4) & (lite[:, L.L_THETA] > 0)
    f = L.lite_features(lite, pop.tau)
    s = _surrogate("lite", f[ok])
    x, _ = s.lite_features(torch.from_numpy(lite).cuda(), torch.from_numpy(pop.tau).cuda())
    torch.cuda.synchronize()
    x = x.float().cpu().numpy().astype(np.float64)
    # DM2 = det u is formed in FP32 from rounded entries: its own rounding
    # (a few FP32 ulps of the products u^3) enters before the standardisation
    nf = f.shape[1]
    mu = s.x_mu[:nf].cpu().numpy().astype(np.float64)
    sg = s.x_sigma[:nf].cpu().numpy().astype(np.float64)
    exact = (f - mu) / sg
    u = lite[:, L.L_U2:L.L_U2 + 6]
    det_scale = np.abs(u).max(1) ** 3
    xr = M.bf16_round(exact.astype(np.float64)).astype(np.float64)
    tol = _bf16_ulp(exact) + 2.0 ** -22 * (np.abs(f) + np.abs(mu)) / sg
    tol[:, 14] += 2.0 ** -20 * det_scale / sg[14]
    # Pi_ii = u_ii - theta is a difference of two rounded FP32 numbers
    th = lite[:, L.L_THETA]
    for j, k in ((5, 0), (8, 3), (10, 5)):
        tol[:, j] += 2.0 ** -22 * (np.abs(u[:, k]) + th) / sg[j]
    d = np.abs(x[:, :nf] - xr)[ok]
    assert np.all(d <= tol[ok]), (d / tol[ok]).max()


def test_training_rows_match_oracle(cavity_pop):
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 5))
    m = O.moments(pop.v64, pop.offsets)
    y, fl = O.closure(m, pop.tau)
    lite = L.lite_moments(pop.v64, pop.offsets)
    dm, dt, dy, dl = (torch.from_numpy(a).cuda() for a in (m, pop.tau, y, lite))
    raw, targ, aux = api.fp_surrogate_training_rows(dm, dt, coeffs=dy)
    raw_l, _, _ = api.fp_surrogate_training_rows(dm, dt, lite=dl, lite_inputs=True, targets=False, aux=False)
    torch.cuda.synchronize()
    raw, targ, aux, raw_l = (t.cpu().numpy().astype(np.float64) for t in (raw, targ, aux, raw_l))
    ok = (pop.counts >= 4) & (m[:, O.M_THETA] > 0)
    f = M.raw_features(m)
    np.testing.assert_allclose(raw[ok, :M.NFEAT], f[ok], rtol=2.0 ** -21, atol=0)
    assert np.all(raw[:, M.NFEAT:] == 0)
    t = M.targets(y, m, pop.tau)
    np.testing.assert_allclose(targ[:, :M.NOUT], t, rtol=2.0 ** -24, atol=0)
    assert np.all(targ[:, M.NOUT:] == 0)
    b = np.stack([f[:, 6] + f[:, 9] + f[:, 11], f[:, 7] + f[:, 12] + f[:, 14], f[:, 8] + f[:, 13] + f[:, 15]], 1)
    s4 = f[:, 16] + f[:, 19] + f[:, 21]
    ref = np.concatenate([f[:, :6], b, s4[:, None]], 1)
    scale = np.abs(f[:, [6, 9, 11, 7, 12, 14, 8, 13, 15]]).max(1)[:, None]
    err = np.abs(aux[:, :10] - ref)[ok]
    assert np.all(err[:, :6] <= 2.0 ** -22 * np.abs(ref[ok, :6]))
    assert np.all(err[:, 6:9] <= 2.0 ** -20 * scale[ok])
    assert np.all(err[:, 9] <= 2.0 ** -20 * np.abs(ref[ok, 9]))
    fl_l = L.lite_features(lite, pop.tau)
    det_scale = np.abs(lite[:, L.L_U2:L.L_U2 + 6]).max(1) ** 3
    tol = 2.0 ** -21 * np.abs(fl_l) + 2.0 ** -21 * np.abs(lite[:, [L.L_THETA]])
    tol[:, 14] += 2.0 ** -20 * det_scale
    assert np.all(np.abs(raw_l[ok, :16] - fl_l[ok]) <= tol[ok])


def test_training_rows_argument_errors():
    t = torch.ones(4, dtype=torch.float64, device="cuda")
    m = torch.zeros((4, O.NMOM), dtype=torch.float64, device="cuda")
    with pytest.raises(api.FPError):
        api.fp_surrogate_training_rows(None, t, coeffs=None)  # targets need coefficients
    with pytest.raises(api.FPError):
        api.fp_surrogate_training_rows(m, t, lite=None, lite_inputs=True, targets=False, aux=False)
