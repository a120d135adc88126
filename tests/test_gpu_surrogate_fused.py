"""The learned closure's fused kernel (inputs, network, coefficients, checks
and fallback list in one tcgen05 kernel) against its parts run one by one:
fp_surrogate_features / fp_surrogate_lite_features, fp_mlp_forward on their
output and the documented epilogue arithmetic.

Both paths form the same BF16 inputs and run the same network code, so the
predictions agree bit for bit, and so do the coefficients of every cell the
network serves (C = t / tau and G = t / (tau sqrt(theta)), scaled in FP32
and widened exactly).  The energy flag is compared away from its threshold
(the residual is summed in FP32 by the kernel); cells the fused kernel lists
must carry the exact closure of the oracle.
"""

import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_15622_gb300 import api, surrogate as S
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu

W = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_15622_gb300", "weights")
PRE = api.FLAG_FEW | api.FLAG_SINGULAR | api.FLAG_NONFINITE


def _scaled(v, tau, theta):
    """The coefficients from FP32 predictions as the epilogue forms them."""
    t32 = tau.astype(np.float32)
    itc = np.float32(1.0) / t32
    ig = itc / np.sqrt(np.where(theta > 0, theta, 1.0).astype(np.float32))
    y = np.empty((v.shape[0], 9))
    y[:, :6] = (v[:, :6] * itc[:, None]).astype(np.float64)
    y[:, 6:] = (v[:, 6:9] * ig[:, None]).astype(np.float64)
    return y


def _cells(pop, idx):
    sub = pop.subset(idx)
    m = O.moments(sub.v64, sub.offsets)
    return sub, m


@pytest.mark.parametrize("n", [None, 1, 127, 129, 300, 5000])
def test_fused_full_closure_equals_its_parts(cavity_pop, n):
    s = S.Surrogate.load(os.path.join(W, "surrogate_full.fpw"))
    idx = np.arange(cavity_pop.n_cells) if n is None else np.arange(n) % cavity_pop.n_cells
    pop, m = _cells(cavity_pop, idx)
    mom, tau = torch.from_numpy(m).cuda(), torch.from_numpy(pop.tau).cuda()
    x, fl0 = s.features(mom, tau)
    v = s.forward(x, standardized=False)
    y, fl = s.closure(mom, tau)
    _, _, aux = api.fp_surrogate_training_rows(mom, tau, targets=False, raw=False)
    torch.cuda.synchronize()
    v, fl0, y, fl, aux = (t.cpu().numpy() for t in (v, fl0, y, fl, aux))
    nc = len(idx)
    prm = api.default_params()
    fb = (fl & api.FLAG_FALLBACK) != 0
    # the inputs' flags are carried; precondition and range failures fall back
    assert np.all((fl & api.FLAG_RANGE) == (fl0 & api.FLAG_RANGE))
    assert np.all(fb[(fl0 & (PRE | api.FLAG_RANGE)) != 0])
    # energy residual of the predicted drift, in FP64 from the FP32 pieces
    u, b, s4 = aux[:, :6].astype(np.float64), aux[:, 6:9].astype(np.float64), aux[:, 9].astype(np.float64)
    vv = v[:, :9].astype(np.float64)
    cu = vv[:, 0] * u[:, 0] + 2 * vv[:, 1] * u[:, 1] + 2 * vv[:, 2] * u[:, 2] + vv[:, 3] * u[:, 3] \
        + 2 * vv[:, 4] * u[:, 4] + vv[:, 5] * u[:, 5]
    e = 1 + (cu + (vv[:, 6:9] * b).sum(1) - s.eps2_hat * s4) / 3
    clear = np.abs(np.abs(e) - prm.surr_energy_tol) > 1e-4
    served = ((fl0 & (PRE | api.FLAG_RANGE)) == 0) & np.isfinite(vv).all(1)
    want_fb = ~served | (np.abs(e) > prm.surr_energy_tol)
    np.testing.assert_array_equal(fb[clear], want_fb[clear])
    assert np.all(((fl & api.FLAG_ENERGY) != 0)[clear & served] == (np.abs(e) > prm.surr_energy_tol)[clear & served])
    # the cells the network serves: its predictions, scaled, bit for bit
    keep = ~fb
    if keep.any():
        np.testing.assert_array_equal(y[keep], _scaled(v, pop.tau, m[:, O.M_THETA])[keep])
        assert np.all(fl[keep] == 0)
    # the listed cells: the oracle's exact closure
    if fb.any():
        yr, flr = O.closure(m, pop.tau)
        den = np.maximum(np.linalg.norm(yr[fb], axis=1), 1e-300)
        assert (np.linalg.norm(y[fb] - yr[fb], axis=1) / den).max() <= 1e-10
        assert np.all((fl[fb] & api.FALLBACK_FLAGS) == flr[fb])
    assert nc == len(fl)


def test_fused_full_closure_on_degenerate_cells():
    """Too few particles, theta = 0, a NaN moment and tau = 0 go to the
    exact closure's own answers (the linear drift for the first, the
    flagged zero-temperature and non-finite cells as the exact closure
    leaves them), next to ordinary cells in the same tile."""
    s = S.Surrogate.load(os.path.join(W, "surrogate_full.fpw"))
    pop = P.couette()
    sub = pop.subset(np.arange(200))
    m = O.moments(sub.v64, sub.offsets)
    tau = sub.tau.copy()
    m[3, O.M_N] = 2
    m[7, O.M_THETA] = 0.0
    m[11, O.M_W + 2] = np.nan
    tau[13] = 0.0
    mom, taud = torch.from_numpy(m).cuda(), torch.from_numpy(tau).cuda()
    y, fl = s.closure(mom, taud)
    torch.cuda.synchronize()
    y, fl = y.cpu().numpy(), fl.cpu().numpy()
    yr, flr = O.closure(m, tau)
    for c in (3, 7, 11, 13):
        assert fl[c] & api.FLAG_FALLBACK
        assert (fl[c] & api.FALLBACK_FLAGS) == flr[c]
        np.testing.assert_array_equal(np.isfinite(y[c]), np.isfinite(yr[c]))
        ok = np.isfinite(yr[c])
        np.testing.assert_allclose(y[c][ok], yr[c][ok], rtol=1e-10, atol=0)
    assert fl[3] & api.FLAG_FEW and fl[7] & api.FLAG_SINGULAR
    assert fl[11] & api.FLAG_NONFINITE and fl[13] & api.FLAG_NONFINITE


@pytest.mark.parametrize("n", [None, 1, 129, 5000])
def test_fused_lite_closure_equals_its_parts(cavity_pop, n):
    s = S.Surrogate.load(os.path.join(W, "surrogate_lite.fpw"))
    idx = np.arange(cavity_pop.n_cells) if n is None else np.arange(n) % cavity_pop.n_cells
    pop = cavity_pop.subset(idx)
    vd, offd = torch.from_numpy(pop.v64).cuda(), torch.from_numpy(pop.offsets).cuda()
    tau = torch.from_numpy(pop.tau).cuda()
    lite = api.fp_moments_lite(vd, offd)
    x, fl0 = s.lite_features(lite, tau)
    v = s.forward(x, standardized=False)
    y, fl = s.closure_lite(lite, tau)
    torch.cuda.synchronize()
    v, fl0, y, fl, lt = (t.cpu().numpy() for t in (v, fl0, y, fl, lite))
    np.testing.assert_array_equal(fl & ~api.FLAG_NONFINITE, fl0 & ~api.FLAG_NONFINITE)
    drift = (fl & PRE) != 0
    assert np.all(drift[(fl0 & PRE) != 0])
    np.testing.assert_array_equal(drift, ((fl0 & PRE) != 0) | ~np.isfinite(v[:, :9]).all(1))
    keep = ~drift
    np.testing.assert_array_equal(y[keep], _scaled(v, pop.tau, lt[:, 4])[keep])
    lin = np.zeros((drift.sum(), 9))
    lin[:, [0, 3, 5]] = (-1.0 / pop.tau[drift])[:, None]
    np.testing.assert_array_equal(y[drift], lin)


@pytest.mark.parametrize("n_cells", [1, 37, 2000, 16384])
def test_fallback_equals_exact_solve_bitwise(cavity_pop, n_cells):
    """An energy tolerance of zero sends every cell to the fallback.  The
    listed cells must carry exactly what fp_closure_solve gives for the same
    moments: short lists take the half-warp solve, the 16384-cell list the
    one-thread-per-cell one."""
    s = S.Surrogate.load(os.path.join(W, "surrogate_full.fpw"))
    pop = cavity_pop.subset(np.arange(n_cells))
    m = O.moments(pop.v64, pop.offsets)
    m[::7, O.M_N] = 2  # a few cells the exact closure flags itself
    mom, tau = torch.from_numpy(m).cuda(), torch.from_numpy(pop.tau).cuda()
    prm = api.default_params(eps2_hat=s.eps2_hat, surr_energy_tol=0.0)
    y, fl = s.closure(mom, tau, params=prm)
    ye, fle = api.fp_closure_solve(mom, tau, params=prm, prec="fp64")
    torch.cuda.synchronize()
    y, fl, ye, fle = (t.cpu().numpy() for t in (y, fl, ye, fle))
    assert np.all(fl & api.FLAG_FALLBACK)
    np.testing.assert_array_equal(fl & api.FALLBACK_FLAGS, fle)
    np.testing.assert_array_equal(y.view(np.int64), ye.view(np.int64))
