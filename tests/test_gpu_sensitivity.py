"""GPU coefficient-sensitivity probe (dropout at inference) against the
oracle (oracle/mlp.py: the same Philox masks, the BF16-emulating forward).

The masks are integer decisions on the same generator words, so they agree
exactly; the passes then differ as the plain forward passes do (FP32
accumulation order, one BF16 ulp here and there), which moves each sigma by
a few per cent of its size at most: |d sigma| <= 0.05 sigma + 2e-3 of the
cell's coefficient scale.
"""

import numpy as np
import pytest
import torch

import oracle as O
from oracle import lite as L
from oracle import mlp as M
from paper_2606_15622_gb300 import api, surrogate as S

pytestmark = pytest.mark.gpu


def _net(features, seed):
    s = S.Surrogate(eps2_hat=1e-3, seed=seed, features=features)
    prm = M.init_params(seed)
    s.set_params(prm["W"], prm["b"])
    return s, prm


def _scalers(s, f):
    nf = f.shape[1]
    s.x_mu[:nf] = torch.from_numpy(f.mean(0)).float()
    s.x_sigma[:nf] = torch.from_numpy(f.std(0).clip(1e-6)).float()
    s.y_mu[:9] = torch.tensor([-1.0, 0.01, -0.02, -1.0, 0.0, -1.0, 0.05, -0.03, 0.02])
    s.y_sigma[:9] = torch.linspace(0.05, 0.2, 9)
    s._net = None


def _x_ref(s, f):
    nf = f.shape[1]
    x = np.zeros((f.shape[0], M.IN))
    x[:, :nf] = (f - s.x_mu[:nf].cpu().numpy()) / s.x_sigma[:nf].cpu().numpy()
    return M.bf16_round(x.astype(np.float32)).astype(np.float64)


def _case(features, pop):
    if features == "full":
        mom = O.moments(pop.v64, pop.offsets)
        f = M.raw_features(mom)
        theta = mom[:, O.M_THETA]
    else:
        mom = L.lite_moments(pop.v64, pop.offsets)
        f = L.lite_features(mom, pop.tau)
        theta = mom[:, L.L_THETA]
    return mom, f, theta


@pytest.mark.parametrize("features", ["full", "lite"])
def test_sensitivity_matches_oracle(cavity_pop, features):
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 8))
    mom, f, theta = _case(features, pop)
    ok = pop.counts >= 4
    s, prm = _net(features, 11)
    _scalers(s, f[ok])
    sens, mean, fl = s.sensitivity(torch.from_numpy(mom).cuda(), torch.from_numpy(pop.tau).cuda(), n_passes=6,
                                   rate=0.2, seed=2024)
    torch.cuda.synchronize()
    sens, mean, fl = sens.cpu().numpy(), mean.cpu().numpy(), fl.cpu().numpy()
    bad = (fl & api.FALLBACK_FLAGS) != 0
    np.testing.assert_array_equal(bad, ~ok)
    assert np.all(np.isnan(sens[bad])) and np.all(np.isnan(mean[bad]))
    cells = np.flatnonzero(ok)
    ref, mref = M.sensitivity(prm, _x_ref(s, f)[cells], s.y_mu.cpu().numpy(), s.y_sigma.cpu().numpy(),
                              pop.tau[cells], theta[cells], cells, 6, 0.2, 2024)
    scale = np.abs(mref).max(axis=1, keepdims=True)
    g = sens[cells]
    assert np.all(np.abs(g[:, :9] - ref[:, :9]) <= 0.05 * ref[:, :9] + 2e-3 * scale)
    assert np.all(np.abs(g[:, 9:] - ref[:, 9:]) <= 0.05 * ref[:, 9:] + 2e-3 * scale)
    assert np.all(np.abs(mean[cells] - mref) <= 2e-2 * scale)
    assert np.median(ref[:, 9]) > 0  # the probe does spread the outputs


def test_rate_zero_gives_zero_spread_and_the_plain_forward(cavity_pop):
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 16))
    mom, f, theta = _case("full", pop)
    ok = pop.counts >= 4
    s, _ = _net("full", 4)
    _scalers(s, f[ok])
    md, td = torch.from_numpy(mom).cuda(), torch.from_numpy(pop.tau).cuda()
    sens, mean, fl = s.sensitivity(md, td, n_passes=4, rate=0.0, seed=1)
    x, _ = s.features(md, td)
    t = s.forward(x, standardized=False)[:, :9].double()
    torch.cuda.synchronize()
    okd = torch.from_numpy(ok).cuda()
    assert torch.all(sens[okd] == 0)
    itc = 1 / td
    fac = torch.cat([itc[:, None].expand(-1, 6), (itc / md[:, 4].sqrt())[:, None].expand(-1, 3)], 1)
    assert torch.equal(mean[okd], (t * fac)[okd])


def test_sensitivity_argument_errors():
    s, _ = _net("lite", 1)
    mom = torch.zeros((4, api.NMOM), dtype=torch.float64, device="cuda")
    tau = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(api.FPError):
        s.sensitivity(mom, tau)  # a LITE network reads LITE vectors
    lite = torch.zeros((4, api.NLITE), dtype=torch.float64, device="cuda")
    with pytest.raises(api.FPError):
        s.sensitivity(lite, tau, rate=1.0)
    with pytest.raises(api.FPError):
        s.sensitivity(lite, tau, n_passes=0)
