"""fp_step_host (host-resident step, chunked copy/compute pipeline) against
the separate device-side calls on the whole population.

Cells are independent and every chunk runs the same kernels on its slice,
so with FP64 velocities and moments the results are bit-identical to the
unchunked calls.  With FP32 moments the per-cell sums of the tiled gather
may be blocked differently when the launch starts at another cell, so
coefficients and velocities agree to the FP32-moment tolerance instead.
"""

import os

import numpy as np
import pytest
import torch

from paper_2606_15622_gb300 import api
from paper_2606_15622_gb300 import populations as P
from paper_2606_15622_gb300 import surrogate as S

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_15622_gb300",
                       "weights", "surrogate_full.fpw")


def _reference(pop, v, prec, sur, dt, seed, step):
    dev = v.device
    off, tau = torch.from_numpy(pop.offsets).to(dev), torch.from_numpy(pop.tau).to(dev)
    mom, y, fl = api.fp_closure_exact(v, off, tau, prec=prec)
    m6 = torch.empty(pop.n_cells, dtype=torch.float64, device=dev)
    api.fp_moments(v, off, prec=prec, m6_out=m6)  # the pipeline's update reads the particles once
    lu = torch.empty(api.lu_doubles(pop.n_cells), dtype=torch.float64, device=dev)
    api.fp_closure_solve(mom, tau, prec=prec, lu_out=lu)  # the factors the pipeline's adjoint reuses
    fl_v = fl.clone()
    v_out = torch.empty_like(v)
    api.fp_velocity_update(v, off, mom, y, tau, fl_v, dt, seed=seed, step=step, v_out=v_out, m6=m6)
    ys, fls = sur.closure(mom, tau, prec=prec)
    gY = torch.ones_like(y)
    gm, gv = api.fp_closure_backward(v, off, tau, mom, y, fl, gY, lu=lu)
    torch.cuda.synchronize()
    return dict(coeffs=y, flags=fl_v, v_out=v_out, coeffs_s=ys, flags_s=fls, grad_m=gm, grad_v=gv)


def _pipeline(pop, vh, prec, sur, dt, seed, step, n_chunks):
    hs = api.HostStep(pop.n_cells, pop.n_particles, dtype=vh.dtype, surrogate=sur, adjoint=True)
    h_off = torch.from_numpy(pop.offsets).pin_memory()
    h_tau = torch.from_numpy(pop.tau).pin_memory()
    h_out = torch.empty_like(vh).pin_memory()
    h_y = torch.empty((pop.n_cells, 9), dtype=torch.float64).pin_memory()
    h_fl = torch.empty(pop.n_cells, dtype=torch.int32).pin_memory()
    hs(vh, h_off, h_tau, h_out, h_y, h_fl, dt, prec=prec, seed=seed, step=step, n_chunks=n_chunks)
    torch.cuda.synchronize()
    res = dict(coeffs=h_y, flags=h_fl, v_out=h_out, coeffs_s=hs.coeffs_s.cpu(), flags_s=hs.flags_s.cpu(),
               grad_m=hs.grad_moments.cpu(), grad_v=hs.grad_v.cpu())
    hs.close()
    return res


@pytest.mark.parametrize("n_chunks", [1, 7])
def test_fp64_pipeline_is_bit_identical(cavity_pop, n_chunks):
    pop = cavity_pop
    sur = S.Surrogate.load(WEIGHTS)
    vh = torch.from_numpy(pop.v64).pin_memory()
    ref = _reference(pop, vh.cuda(), "fp64", sur, 0.2, 5, 3)
    got = _pipeline(pop, vh, "fp64", sur, 0.2, 5, 3, n_chunks)
    for k in ref:
        assert torch.equal(got[k], ref[k].cpu()), k


def test_fp32_pipeline_matches_separate_calls():
    pop = P.cylinder(nx=128, ny=64, target_particles=750_000)
    sur = S.Surrogate.load(WEIGHTS)
    vh = torch.from_numpy(pop.v32).pin_memory()
    ref = _reference(pop, vh.cuda(), "fp32", sur, 0.1, 9, 1)
    got = _pipeline(pop, vh, "fp32", sur, 0.1, 9, 1, 6)
    same = (got["flags"] == ref["flags"].cpu()).numpy()
    assert same.mean() > 0.999
    ok = same & (got["flags"].numpy() == 0)
    y, yr = got["coeffs"].numpy()[ok], ref["coeffs"].cpu().numpy()[ok]
    assert np.all(np.abs(y - yr) <= 1e-5 * np.abs(yr).max(axis=1, keepdims=True))
    cell_of = np.repeat(np.arange(pop.n_cells), pop.counts)
    okp = ok[cell_of]
    scale = np.sqrt(np.maximum(pop.v32.astype(np.float64).var(axis=1), 1e-30))[:, None]
    dv = np.abs(got["v_out"].numpy()[:, okp] - ref["v_out"].cpu().numpy()[:, okp]) / scale
    assert dv.max() <= 1e-4


def test_argument_errors(cavity_pop):
    pop = cavity_pop
    hs = api.HostStep(pop.n_cells, pop.n_particles, dtype=torch.float32)
    h = dict(h_v=torch.from_numpy(pop.v32), h_offsets=torch.from_numpy(pop.offsets),
             h_tau=torch.from_numpy(pop.tau), h_v_out=torch.empty((3, pop.n_particles), dtype=torch.float32),
             h_coeffs=torch.empty((pop.n_cells, 9), dtype=torch.float64),
             h_flags=torch.empty(pop.n_cells, dtype=torch.int32))
    with pytest.raises(api.FPError):
        hs(**h, dt=0.1, n_chunks=0)
    with pytest.raises(api.FPError):
        hs(**h, dt=0.1, n_chunks=65)
    bad = dict(h)
    off = torch.from_numpy(pop.offsets.copy())
    off[-1] += 1  # offsets not ending at n_particles
    bad["h_offsets"] = off
    with pytest.raises(api.FPError):
        hs(**bad, dt=0.1)
    hs.close()
