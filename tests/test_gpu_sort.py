"""GPU cell sort and collision step against the oracle.

The sort is integer work: the permutation, the offsets and the gathered
velocities are compared bit for bit with the oracle's stable sort.  The
collision step runs the same kernels as the separate calls on the sorted
particles, so with the exact closure it equals them bit for bit; the LITE
step's update is compared with the oracle's update (FP32 tolerances of the
velocity tests) on the same coefficients.
"""

import os

import numpy as np
import pytest
import torch

import oracle as O
from oracle import lite as L
from paper_2606_15622_gb300 import api, surrogate as S
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu


def _gpu_sort(cell_of, n_cells, v=None):
    c = torch.from_numpy(cell_of.astype(np.int32)).cuda()
    vd = None if v is None else torch.from_numpy(v).cuda()
    perm, off, vs = api.fp_sort_by_cell(c, n_cells, v=vd)
    torch.cuda.synchronize()
    return perm.cpu().numpy(), off.cpu().numpy(), None if vs is None else vs.cpu().numpy()


@pytest.mark.parametrize("n,n_cells", [(0, 5), (1, 1), (2047, 1), (2048, 255), (2049, 256), (5000, 257),
                                       (100_000, 65535), (300_001, 131072), (250_000, 1 << 20)])
def test_sort_matches_oracle(n, n_cells):
    rng = np.random.default_rng(n + n_cells)
    cell_of = rng.integers(-3, n_cells + 3, size=n)  # a few indices outside the cells
    v = rng.standard_normal((3, n)).astype(np.float32)
    perm, off, vs = _gpu_sort(cell_of, n_cells, v)
    pr, offr = O.sort_by_cell(cell_of, n_cells)
    np.testing.assert_array_equal(perm, pr)
    np.testing.assert_array_equal(off, offr)
    np.testing.assert_array_equal(vs, v[:, pr])


def test_sort_nearly_sorted_and_many_equal_keys():
    """A sorted population with 3 % of particles moved to a neighbouring
    cell (a step of particle motion), and one cell holding 40 % of all
    particles (equal keys across many tiles keep their order)."""
    pop = P.cavity(seed=6)
    cell_of = np.repeat(np.arange(pop.n_cells), pop.counts)
    rng = np.random.default_rng(1)
    moved = rng.random(cell_of.size) < 0.03
    cell_of = np.where(moved, np.clip(cell_of + rng.integers(-1, 2, cell_of.size), 0, pop.n_cells - 1), cell_of)
    cell_of[rng.random(cell_of.size) < 0.4] = 77
    perm, off, vs = _gpu_sort(cell_of, pop.n_cells, pop.v64)
    pr, offr = O.sort_by_cell(cell_of, pop.n_cells)
    np.testing.assert_array_equal(perm, pr)
    np.testing.assert_array_equal(off, offr)
    np.testing.assert_array_equal(vs, pop.v64[:, pr])


def test_sort_full_size_cylinder_shuffled():
    pop = P.cylinder()
    cell_of = np.repeat(np.arange(pop.n_cells), pop.counts)
    rng = np.random.default_rng(2)
    shuffle = rng.permutation(cell_of.size)
    perm, off, _ = _gpu_sort(cell_of[shuffle], pop.n_cells)
    pr, offr = O.sort_by_cell(cell_of[shuffle], pop.n_cells)
    np.testing.assert_array_equal(off, pop.offsets)
    np.testing.assert_array_equal(off, offr)
    np.testing.assert_array_equal(perm, pr)


def _shuffled(pop, seed, outside=0.01):
    """The population in random order, some particles given no cell."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(pop.n_particles)
    cell_of = np.repeat(np.arange(pop.n_cells), pop.counts)[order]
    gone = rng.random(cell_of.size) < outside
    cell_of = np.where(gone, -1, cell_of)
    return cell_of.astype(np.int32), order


@pytest.mark.parametrize("vdtype,prec", [("f64", "fp64"), ("f32", "fp32")])
def test_exact_collision_step_equals_separate_calls(cavity_pop, vdtype, prec):
    pop = cavity_pop
    cell_of, order = _shuffled(pop, 3)
    v = (pop.v64 if vdtype == "f64" else pop.v32)[:, order].copy()
    vd = torch.from_numpy(v).cuda()
    cd = torch.from_numpy(cell_of).cuda()
    tau = torch.from_numpy(pop.tau).cuda()
    v_out, perm, off, y, fl = api.fp_collision_step(cd, vd, pop.n_cells, tau, 0.2, prec=prec, seed=11, step=4)
    # the separate calls on the sorted particles
    perm_r, off_r, vs = api.fp_sort_by_cell(cd, pop.n_cells, v=vd)
    m6 = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    mom = api.fp_moments(vs, off_r, prec=prec, m6_out=m6)
    yr, flr = api.fp_closure_solve(mom, tau, prec=prec)
    vr = torch.empty_like(vs)
    api.fp_velocity_update(vs, off_r, mom, yr, tau, flr, 0.2, seed=11, step=4, v_out=vr, m6=m6)
    torch.cuda.synchronize()
    assert torch.equal(perm, perm_r) and torch.equal(off, off_r)
    assert torch.equal(y, yr) and torch.equal(fl, flr)
    inside = int(off[-1])
    assert inside < pop.n_particles  # some particles are in no cell
    assert torch.equal(v_out[:, :inside], vr[:, :inside])
    assert torch.equal(v_out[:, inside:], vs[:, inside:])  # copied unchanged
    # the sorted order is the oracle's
    pr, offr = O.sort_by_cell(cell_of, pop.n_cells)
    np.testing.assert_array_equal(perm.cpu().numpy(), pr)
    np.testing.assert_array_equal(off.cpu().numpy(), offr)


def _lite_net():
    from oracle import mlp as M
    s = S.Surrogate(eps2_hat=1e-3, seed=5, features="lite")
    prm = M.init_params(5)
    s.set_params(prm["W"], prm["b"])
    s.x_mu[:16] = torch.tensor([60.0, 1.5, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 3.0, 1.0])
    s.x_sigma[:16] = torch.tensor([30.0, 0.6, 0.3, 0.3, 0.3, 0.2, 0.1, 0.1, 0.2, 0.1, 0.2, 0.2, 0.2, 0.2, 3.0, 0.3])
    s.y_mu[:9] = torch.tensor([-1.0, 0, 0, -1.0, 0, -1.0, 0, 0, 0])
    s.y_sigma[:9] = 0.05
    s._net = None
    return s


@pytest.mark.parametrize("vdtype", ["f64", "f32"])
def test_lite_velocity_update_matches_oracle(couette_pop, vdtype):
    """The update from LITE vectors (alpha summed over the particles) on the
    oracle's LITE moments and exact coefficients, against the oracle's
    update; the oracle reads U, theta and b_i, given here through third
    moments whose sums u_ikk are b_i."""
    pop = couette_pop
    v = pop.v64 if vdtype == "f64" else pop.v32.astype(np.float64)
    lite = L.lite_moments(v, pop.offsets)
    mom = O.moments(v, pop.offsets)
    y, fl = O.closure(mom, pop.tau)
    full = np.zeros_like(mom)
    full[:, :O.M_U3] = lite[:, :O.M_U3]
    full[:, O.M_U3:O.M_U3 + 3] = lite[:, L.L_B:L.L_B + 3]
    vref, aref, fref = O.velocity_update(v, pop.offsets, full, y, pop.tau, fl, 0.3, seed=7, step=2)
    vd = torch.from_numpy(pop.v64 if vdtype == "f64" else pop.v32).cuda()
    alpha = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    fld = torch.from_numpy(fl.astype(np.int32)).cuda()
    vo, _, _ = api.fp_velocity_update_lite(vd, torch.from_numpy(pop.offsets).cuda(), torch.from_numpy(lite).cuda(),
                                           torch.from_numpy(y).cuda(), torch.from_numpy(pop.tau).cuda(), fld, 0.3,
                                           seed=7, step=2, alpha_out=alpha, v_out=torch.empty_like(vd))
    torch.cuda.synchronize()
    cell_of = np.repeat(np.arange(pop.n_cells), pop.counts)
    scale = np.abs(vref) + np.sqrt(np.maximum(lite[cell_of, L.L_THETA], 0))[None, :]
    tol = 2e-6 if vdtype == "f64" else 6e-6  # FP32 normals on the GPU; FP32 arithmetic for FP32 velocities
    assert np.max(np.abs(vo.cpu().numpy() - vref) / scale) <= tol
    np.testing.assert_array_equal(fld.cpu().numpy(), fref)
    ok = (fref & (O.FALLBACK_FLAGS | O.FLAG_ALPHA)) == 0
    np.testing.assert_allclose(alpha.cpu().numpy()[ok], aref[ok], rtol=1e-12 if vdtype == "f64" else 1e-5)


def test_lite_collision_step_equals_separate_calls(couette_pop):
    """LITE step: sort, LITE moments, the learned closure on them, the update
    with alpha from a pass over the particles; the same as the separate
    calls on the sorted particles, bit for bit."""
    pop = couette_pop
    cell_of, order = _shuffled(pop, 5, outside=0.002)
    v = pop.v32[:, order].copy()
    s = _lite_net()
    vd, cd = torch.from_numpy(v).cuda(), torch.from_numpy(cell_of).cuda()
    tau = torch.from_numpy(pop.tau).cuda()
    lite = torch.empty((pop.n_cells, api.NLITE), dtype=torch.float64, device="cuda")
    v_out, perm, off, y, fl = api.fp_collision_step(cd, vd, pop.n_cells, tau, 0.3, net_lite=s.net(), seed=7, step=2,
                                                    moments_out=lite)
    perm_r, off_r, vs = api.fp_sort_by_cell(cd, pop.n_cells, v=vd)
    lr = api.fp_moments_lite(vs, off_r)
    yr, flr = s.closure_lite(lr, tau)
    vr = torch.empty_like(vs)
    api.fp_velocity_update_lite(vs, off_r, lr, yr, tau, flr, 0.3, seed=7, step=2, v_out=vr)
    torch.cuda.synchronize()
    assert torch.equal(perm, perm_r) and torch.equal(off, off_r) and torch.equal(lite, lr)
    assert torch.equal(y, yr) and torch.equal(fl, flr)
    inside = int(off[-1])
    assert torch.equal(v_out[:, :inside], vr[:, :inside])
    assert torch.equal(v_out[:, inside:], vs[:, inside:])


def test_collision_step_argument_errors():
    c = torch.zeros(10, dtype=torch.int32, device="cuda")
    v = torch.zeros((3, 10), dtype=torch.float32, device="cuda")
    tau = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(api.FPError):
        api.fp_collision_step(c, v, 2, tau, -1.0)
    with pytest.raises(api.FPError):
        api.fp_collision_step(c, v, 2, tau, 0.1, workspace=torch.empty(8, dtype=torch.uint8, device="cuda"))
    with pytest.raises(api.FPError):
        api.fp_sort_by_cell(c.long(), 2)


def test_sort_and_step_degenerate_sizes():
    """No particles; no cells (every particle outside); one cell."""
    tau1 = torch.ones(1, dtype=torch.float64, device="cuda")
    # no particles
    c = torch.zeros(0, dtype=torch.int32, device="cuda")
    v = torch.zeros((3, 0), dtype=torch.float32, device="cuda")
    perm, off, vs = api.fp_sort_by_cell(c, 3, v=v)
    assert perm.numel() == 0 and off.cpu().tolist() == [0, 0, 0, 0]
    tau3 = torch.ones(3, dtype=torch.float64, device="cuda")
    v_out, perm, off, y, fl = api.fp_collision_step(c, v, 3, tau3, 0.1)
    torch.cuda.synchronize()
    assert off.cpu().tolist() == [0, 0, 0, 0] and torch.all((fl & api.FLAG_FEW) != 0)
    # no cells: every particle is outside and comes back unchanged
    rng = np.random.default_rng(3)
    vv = torch.from_numpy(rng.standard_normal((3, 50)).astype(np.float32)).cuda()
    cc = torch.from_numpy(rng.integers(0, 5, 50).astype(np.int32)).cuda()
    v_out, perm, off, y, fl = api.fp_collision_step(cc, vv, 0, tau1[:0], 0.1)
    torch.cuda.synchronize()
    assert off.cpu().tolist() == [0]
    assert torch.equal(v_out, vv[:, perm.long()])
    np.testing.assert_array_equal(perm.cpu().numpy(), np.arange(50))
    # one cell: the sort keeps the input order
    c1 = torch.zeros(40, dtype=torch.int32, device="cuda")
    v1 = torch.from_numpy(rng.standard_normal((3, 40))).cuda()
    perm, off, vs = api.fp_sort_by_cell(c1, 1, v=v1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(perm.cpu().numpy(), np.arange(40))
    assert off.cpu().tolist() == [0, 40] and torch.equal(vs, v1)


def test_sort_rejects_too_many_cells():
    """2^31 cells: the binding refuses the short offsets array, and the
    library itself answers FP_ERR_UNSUPPORTED before touching any buffer."""
    import ctypes
    c = torch.zeros(4, dtype=torch.int32, device="cuda")
    off = torch.empty(1, dtype=torch.int64, device="cuda")
    perm = torch.empty(4, dtype=torch.int32, device="cuda")
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(api.FPError):
        api.fp_sort_by_cell(c, 2 ** 31, offsets_out=off, workspace=ws)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = api.lib().fp_sort_by_cell(ptr(c), 4, 2 ** 31, None, 0, None, ptr(perm), ptr(off), ptr(ws), ws.numel(),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == api.FP_ERR_UNSUPPORTED


def test_collision_steps_full_size_cylinder():
    """The cylinder population at full size (12M particles, 3 % moved to a
    neighbouring cell, in the previous step's order): both collision steps
    equal their separate calls bit for bit; the sort equals the oracle's."""
    pop = P.cylinder()
    cell_sorted = np.repeat(np.arange(pop.n_cells), pop.counts)
    rng = np.random.default_rng(17)
    moved = rng.random(pop.n_particles) < 0.03
    cell_of = np.where(moved, np.clip(cell_sorted + rng.integers(-1, 2, pop.n_particles), 0, pop.n_cells - 1),
                       cell_sorted).astype(np.int32)
    vd, cd = torch.from_numpy(pop.v32).cuda(), torch.from_numpy(cell_of).cuda()
    tau = torch.from_numpy(pop.tau).cuda()
    perm_r, off_r, vs = api.fp_sort_by_cell(cd, pop.n_cells, v=vd)
    pr, offr = O.sort_by_cell(cell_of, pop.n_cells)
    np.testing.assert_array_equal(perm_r.cpu().numpy(), pr)
    np.testing.assert_array_equal(off_r.cpu().numpy(), offr)
    # exact
    v_out, perm, off, y, fl = api.fp_collision_step(cd, vd, pop.n_cells, tau, 0.1, prec="fp32", seed=3, step=9)
    m6 = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    mom = api.fp_moments(vs, off_r, prec="fp32", m6_out=m6)
    yr, flr = api.fp_closure_solve(mom, tau, prec="fp32")
    vr = torch.empty_like(vs)
    api.fp_velocity_update(vs, off_r, mom, yr, tau, flr, 0.1, seed=3, step=9, v_out=vr, m6=m6)
    torch.cuda.synchronize()
    assert torch.equal(perm, perm_r) and torch.equal(y, yr) and torch.equal(fl, flr) and torch.equal(v_out, vr)
    # learned closure on LITE inputs
    s = S.Surrogate.load(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                      "paper_2606_15622_gb300", "weights", "surrogate_lite.fpw"))
    v_out, perm, off, y, fl = api.fp_collision_step(cd, vd, pop.n_cells, tau, 0.1, net_lite=s.net(), seed=3, step=9)
    lr = api.fp_moments_lite(vs, off_r)
    yr, flr = s.closure_lite(lr, tau)
    vr = torch.empty_like(vs)
    api.fp_velocity_update_lite(vs, off_r, lr, yr, tau, flr, 0.1, seed=3, step=9, v_out=vr)
    torch.cuda.synchronize()
    assert torch.equal(y, yr) and torch.equal(fl, flr) and torch.equal(v_out, vr)
