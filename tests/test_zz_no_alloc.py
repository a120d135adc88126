"""fp_closure_exact_static -- the exact closure for callers that may not
allocate device memory (its scratch is an array built into the library).

Checked through the C ABI on two calls in a row: a full cavity population
(16384 cells) first, then a small population of edge cells -- empty,
single-particle, too-few, identical particles (theta = 0), a NaN velocity, a
20000-particle cell and ragged sizes -- whose slots the first call filled with
other moments, so that a cell the gather failed to overwrite would show as a
stale result.  Each call is compared with fp_closure_exact (scratch from the
caller; same kernels, so the results are identical in practice, and must
agree to the closure tests' tolerances: 1e-10 relative for FP64 moments, 1e-4
for FP32 moments) and with the CPU oracle (flags equal outside the
near-threshold band, unflagged cells within the same tolerances, flagged
cells exactly the linear drift).
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_15622_gb300 import api
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _edge_cells():
    rng = np.random.default_rng(41)
    sizes = [0, 1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 0, 63, 64, 65, 100, 0, 20000, 255, 256, 257,
             10, 10, 0, 0]
    parts = [rng.standard_normal((3, s)) * rng.uniform(0.3, 3) + rng.uniform(-5, 5, (3, 1)) for s in sizes]
    parts[25][:] = 2.5  # theta = 0
    parts[26][1, 3] = np.nan
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    v = np.ascontiguousarray(np.concatenate(parts, axis=1))
    return P.Population("edge", v, offs, rng.uniform(0.5, 2.0, len(sizes)))


def _check(pop, prec):
    vh = pop.v64 if prec == "fp64" else pop.v32
    v, off, tau = _dev(vh), _dev(pop.offsets), _dev(pop.tau)
    y_static, f_static = api.fp_closure_exact_static(v, off, tau, prec=prec)
    _, y_ref, f_ref = api.fp_closure_exact(v, off, tau, prec=prec, want_moments=False)
    torch.cuda.synchronize()
    ys, fs = y_static.cpu().numpy(), f_static.cpu().numpy()
    # against the entry point that takes its scratch from the caller
    assert np.array_equal(fs, f_ref.cpu().numpy())
    yr = y_ref.cpu().numpy()
    live = fs == 0
    err = np.linalg.norm(ys[live] - yr[live], axis=1) / np.linalg.norm(yr[live], axis=1)
    assert err.size == 0 or err.max() <= TOL[prec], err.max()
    np.testing.assert_array_equal(ys[~live], yr[~live])
    # against the oracle
    m = O.moments(vh.astype(np.float64), pop.offsets)
    y, fl, cond, mp = O.closure(m, pop.tau, want_cond=True)
    floor = O.DEFAULT_PIVOT_RTOL if prec == "fp64" else api.FP32_PIVOT_FLOOR
    near = (mp > O.DEFAULT_PIVOT_RTOL / 10) & (mp < 10 * floor)
    np.testing.assert_array_equal(fs[~near], fl[~near])
    ok = (fl == 0) & (fs == 0) & (cond <= 1e8)
    assert ok.sum() > 0
    e = np.linalg.norm(ys[ok] - y[ok], axis=1) / np.linalg.norm(y[ok], axis=1)
    assert e.max() <= TOL[prec], e.max()
    bad = (fl != 0) & ~near
    np.testing.assert_array_equal(ys[bad], y[bad])
    return fs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_matches_workspace_path_and_oracle_on_two_calls(prec):
    _check(P.cavity(seed=12), prec)
    fs = _check(_edge_cells(), prec)
    # the edge cells kept their own flags, not the first call's moments
    assert fs[0] & api.FLAG_FEW and fs[1] & api.FLAG_FEW
    assert fs[25] & api.FLAG_SINGULAR and fs[26] & api.FLAG_NONFINITE


def test_static_scratch_rejects_too_many_cells():
    n = api.STATIC_MAX_CELLS + 1
    v = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    off = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    tau = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(api.FPError, match="FP_STATIC_MAX_CELLS"):
        api.fp_closure_exact_static(v, off, tau)
