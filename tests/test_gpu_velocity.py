"""GPU parity of fp_velocity_update (through the C ABI) against the oracle's
update (Eqs. update_vel, update_N, update_alpha).

Tolerances: FP64 velocities with given variates agree to 1e-12 relative;
FP32 velocities are updated in FP32, so each component carries a few ulps of
|v| plus the FP32 rounding of the cell constants: |dv| <= 4e-6 (|v| +
sqrt(theta)).  Philox variates: the GPU maps the same 32-bit words to normals
in FP32 (a fitted quantile, |dxi| <= 1.3e-6 over all inputs), the oracle in
FP64, so xi differs by <= ~3e-7 relative.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_15622_gb300 import api
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle_state(pop, vdtype, eps2_hat=O.DEFAULT_EPS2_HAT):
    v = pop.v64 if vdtype == "f64" else pop.v32.astype(np.float64)
    m = O.moments(v, pop.offsets)
    y, fl = O.closure(m, pop.tau, eps2_hat=eps2_hat)
    return v, m, y, fl


def _gpu_update(pop, vdtype, m, y, fl, dt, xi=None, seed=0, step=0, eps2_hat=O.DEFAULT_EPS2_HAT, one_pass=False):
    v = _dev(pop.v64 if vdtype == "f64" else pop.v32)
    x = None if xi is None else _dev(xi.astype(np.float64 if vdtype == "f64" else np.float32))
    alpha = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    flags = _dev(fl.astype(np.int32))
    api.fp_velocity_update(v, _dev(pop.offsets), _dev(m), _dev(y), _dev(pop.tau), flags, dt,
                           params=api.default_params(eps2_hat=eps2_hat), xi=x, seed=seed, step=step, alpha_out=alpha,
                           m6=_dev(O.speed_moment6(pop.v64 if vdtype == "f64" else pop.v32, pop.offsets))
                           if one_pass else None)
    torch.cuda.synchronize()
    return v.cpu().numpy().astype(np.float64), alpha.cpu().numpy(), flags.cpu().numpy()


def _check(pop, vref, aref, fref, vg, ag, fg, vdtype, m, noise_tol=0.0):
    np.testing.assert_array_equal(fg, fref)
    fin = np.isfinite(vref)
    assert np.array_equal(fin, np.isfinite(vg))
    cell_of = np.repeat(np.arange(pop.n_cells), pop.counts)
    scale = np.abs(vref) + np.sqrt(np.maximum(m[cell_of, 4], 0))[None, :]
    tol = (1e-12 if vdtype == "f64" else 4e-6) + noise_tol
    err = np.abs(vg - vref)[fin] / scale[fin]
    assert err.max() <= tol, f"max velocity err {err.max():.3e}"
    aok = np.isfinite(aref)
    atol = 1e-12 if vdtype == "f64" else 2e-6
    assert np.abs(ag[aok] - aref[aok]).max() <= atol + noise_tol


@pytest.mark.parametrize("one_pass", [False, True])
@pytest.mark.parametrize("vdtype", ["f64", "f32"])
@pytest.mark.parametrize("dt", [0.05, 0.7])
def test_update_with_given_variates(cavity_pop, vdtype, dt, one_pass):
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 5))
    v, m, y, fl = _oracle_state(pop, vdtype, eps2_hat=1e-2)
    xi = np.random.default_rng(1).standard_normal((3, pop.n_particles))
    if vdtype == "f32":
        xi = xi.astype(np.float32).astype(np.float64)
    vref, aref, fref = O.velocity_update(v, pop.offsets, m, y, pop.tau, fl, dt, eps2_hat=1e-2, xi=xi)
    vg, ag, fg = _gpu_update(pop, vdtype, m, y, fl, dt, xi=xi, eps2_hat=1e-2, one_pass=one_pass)
    _check(pop, vref, aref, fref, vg, ag, fg, vdtype, m)


@pytest.mark.parametrize("one_pass", [False, True])
@pytest.mark.parametrize("vdtype", ["f64", "f32"])
def test_update_with_philox_variates(couette_pop, vdtype, one_pass):
    pop = couette_pop
    v, m, y, fl = _oracle_state(pop, vdtype)
    vref, aref, fref = O.velocity_update(v, pop.offsets, m, y, pop.tau, fl, 0.3, seed=2024, step=17)
    vg, ag, fg = _gpu_update(pop, vdtype, m, y, fl, 0.3, seed=2024, step=17, one_pass=one_pass)
    _check(pop, vref, aref, fref, vg, ag, fg, vdtype, m, noise_tol=2e-6)


def test_cylinder_full_size_pipeline_sampled():
    """Full-size launch: FP64 closure then FP64 update of all 131072 cells on
    the GPU; the oracle recomputes a seeded sample of cells from the same
    input velocities (moments, closure and update of its own)."""
    pop = P.cylinder()
    v = _dev(pop.v64)
    off, tau = _dev(pop.offsets), _dev(pop.tau)
    mom, y, fl = api.fp_closure_exact(v, off, tau, prec="fp64")
    m6 = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    api.fp_moments(v, off, prec="fp64", m6_out=m6)  # one-pass update: <|c|^6> from the gather
    alpha = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    api.fp_velocity_update(v, off, mom, y, tau, fl, 0.2, seed=7, step=3, alpha_out=alpha, m6=m6)
    torch.cuda.synchronize()
    vg, ag, fg = v.cpu().numpy(), alpha.cpu().numpy(), fl.cpu().numpy()
    rng = np.random.default_rng(5)
    cells = np.sort(rng.choice(pop.n_cells, 1500, replace=False))
    sub = pop.subset(cells)
    m = O.moments(sub.v64, sub.offsets)
    yr, flr = O.closure(m, sub.tau)
    # the oracle's counter is the particle's global index: rebuild the
    # sample's variates with the same counters
    idx = np.concatenate([np.arange(pop.offsets[c], pop.offsets[c + 1]) for c in cells])
    xi = np.concatenate([O.normals(1, 7, 3, first_index=int(i)) for i in idx], axis=1)
    vref, aref, fref = O.velocity_update(sub.v64, sub.offsets, m, yr, sub.tau, flr, 0.2, xi=xi)
    ok = fref == fg[cells]
    assert ok.mean() > 0.99
    cell_of = np.repeat(np.arange(sub.n_cells), sub.counts)
    okp = ok[cell_of]
    scale = np.abs(vref) + np.sqrt(np.maximum(m[cell_of, 4], 0))[None, :]
    err = np.abs(vg[:, idx] - vref)[:, okp] / scale[:, okp]
    assert err.max() <= 1e-6, err.max()  # FP32 inverse distribution on the GPU (noise terms)
    assert np.abs(ag[cells][ok] - aref[ok]).max() <= 1e-9


def test_linear_cells_alpha_flag_and_momentum():
    pop = P.maxwellian_cells([0, 3, 40, 60, 50], theta=[1.0, 1.0, 2.0, 0.5, 1.0], tau=[1, 1, 0.5, 2.0, 1.0], seed=9)
    v, m, y, fl = _oracle_state(pop, "f64")
    y = y.copy()
    y[4, 0] = np.nan  # a non-finite coefficient: alpha^2 is NaN -> FP_FLAG_ALPHA
    xi = np.zeros((3, pop.n_particles))
    vref, aref, fref = O.velocity_update(v, pop.offsets, m, y, pop.tau, fl, 0.4, xi=xi)
    vg, ag, fg = _gpu_update(pop, "f64", m, y, fl, 0.4, xi=xi)
    assert fref[1] & api.FLAG_FEW and fref[4] & api.FLAG_ALPHA
    np.testing.assert_array_equal(fg, fref)
    np.testing.assert_allclose(ag, aref, rtol=1e-12)
    # without noise the cell mean velocity stays U (momentum of the drift)
    for c in (2, 3):
        s = slice(pop.offsets[c], pop.offsets[c + 1])
        np.testing.assert_allclose(vg[:, s].mean(1), m[c, 1:4], atol=1e-12)


def test_argument_errors():
    v = torch.zeros((3, 4), dtype=torch.float32, device="cuda")
    off = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    mom = torch.zeros((1, 30), dtype=torch.float64, device="cuda")
    y = torch.zeros((1, 9), dtype=torch.float64, device="cuda")
    tau = torch.ones(1, dtype=torch.float64, device="cuda")
    fl = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(api.FPError):
        api.fp_velocity_update(v, off, mom, y, tau, fl, -1.0)
    with pytest.raises(api.FPError):
        api.fp_velocity_update(v, off, mom, y, tau, fl, 0.1, xi=torch.zeros((3, 4), dtype=torch.float64, device="cuda"))
    big = torch.zeros(15, dtype=torch.float32, device="cuda")
    with pytest.raises(api.FPError):  # v_out overlapping v without being v
        api.fp_velocity_update(big[:12].view(3, 4), off, mom, y, tau, fl, 0.1, v_out=big[3:].view(3, 4))


@pytest.mark.parametrize("vdtype", ["f64", "f32"])
def test_out_of_place_matches_in_place(cavity_pop, vdtype):
    """Writing M^{n+1} to a separate array gives the in-place result bit for
    bit and leaves M^n untouched."""
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 3))
    _, m, y, fl = _oracle_state(pop, vdtype)
    v0 = _dev(pop.v64 if vdtype == "f64" else pop.v32)
    off, mom, yd, tau = _dev(pop.offsets), _dev(m), _dev(y), _dev(pop.tau)
    v_in = v0.clone()
    f_in = _dev(fl.astype(np.int32))
    a_in = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    api.fp_velocity_update(v_in, off, mom, yd, tau, f_in, 0.3, seed=11, step=2, alpha_out=a_in)
    v_src, v_dst = v0.clone(), torch.full_like(v0, float("nan"))
    f_out = _dev(fl.astype(np.int32))
    a_out = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    api.fp_velocity_update(v_src, off, mom, yd, tau, f_out, 0.3, seed=11, step=2, alpha_out=a_out, v_out=v_dst)
    torch.cuda.synchronize()
    assert torch.equal(v_dst, v_in)
    assert torch.equal(v_src, v0)
    assert torch.equal(f_out, f_in) and torch.equal(a_out, a_in)


@pytest.mark.parametrize("vdtype", ["f64", "f32"])
def test_split_update_with_particle_offset_equals_whole(cavity_pop, vdtype):
    """The update of two cell ranges, each on its own particle slice with
    fp_params.particle_offset = the slice's first global particle, equals the
    update of the whole population bit for bit (the sharded multi-GPU run)."""
    from paper_2606_15622_gb300 import shard as SH
    pop = cavity_pop
    v = pop.v64 if vdtype == "f64" else pop.v32
    mom = O.moments(v.astype(np.float64), pop.offsets)
    y, fl = O.closure(mom, pop.tau)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    whole = dev(v)
    fw = dev(fl.astype(np.int32))
    api.fp_velocity_update(whole, dev(pop.offsets), dev(mom), dev(y), dev(pop.tau), fw, 0.25, seed=31, step=6)
    pieces = []
    for rank in range(2):
        c0, c1, p0, p1 = SH.shard_bounds(pop.offsets, 2, rank)
        part = dev(v[:, p0:p1])
        fp = dev(fl[c0:c1].astype(np.int32))
        prm = api.default_params(particle_offset=p0)
        api.fp_velocity_update(part, dev(pop.offsets[c0:c1 + 1] - p0), dev(mom[c0:c1]), dev(y[c0:c1]),
                               dev(pop.tau[c0:c1]), fp, 0.25, params=prm, seed=31, step=6)
        pieces.append((part, fp))
    torch.cuda.synchronize()
    assert torch.equal(torch.cat([q[0] for q in pieces], dim=1), whole)
    assert torch.equal(torch.cat([q[1] for q in pieces]), fw)


def test_update_normals_are_the_quantiles_of_the_philox_words():
    """The update's own variates, read out exactly: every cell flagged linear
    (no drift), every velocity at U = 0 in FP64 storage, so M^{n+1} = nz xi
    with nz = sqrt(theta (1 - a^2)) and one rounding.  Against the oracle's
    quantile (an FP64 inversion of Phi) of the same Philox words: 3M variates,
    about 6000 of them in the kernel's tail branch (|xi| > 3.1)."""
    n_cells, ppc, dt = 256, 4096, 0.5
    n_p = n_cells * ppc
    off = np.arange(n_cells + 1, dtype=np.int64) * ppc
    mom = np.zeros((n_cells, api.NMOM))
    mom[:, 0] = ppc
    mom[:, 4] = 1.0  # theta
    flags = _dev(np.full(n_cells, api.FLAG_FEW, dtype=np.int32))
    v = torch.zeros((3, n_p), dtype=torch.float64, device="cuda")
    api.fp_velocity_update(v, _dev(off), _dev(mom), _dev(np.zeros((n_cells, 9))), _dev(np.ones(n_cells)), flags, dt,
                           seed=99, step=4)
    a = np.exp(-dt)
    xi_gpu = (v.cpu().numpy() / np.sqrt((1 - a) * (1 + a))).astype(np.float32).astype(np.float64)
    xi = O.normals(n_p, 99, 4)
    err = np.abs(xi_gpu - xi)
    assert err.max() <= 1.5e-6, err.max()
    assert (err / np.abs(xi)).max() <= 4e-7
    tail = np.abs(xi) > 3.1
    assert tail.sum() > 3000
    assert err[tail].max() <= 1.5e-6
    np.testing.assert_array_equal(flags.cpu().numpy(), api.FLAG_FEW)
