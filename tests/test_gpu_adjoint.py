"""GPU adjoint (fp_closure_backward via the C ABI and torch.autograd) against
the oracle's complex-step gradient and against central finite differences of
the GPU forward in float64 (64 random cells, step 1e-6)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_15622_gb300 import api, autograd
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def small_cells():
    """Cavity-like cells with 8..14 particles (the oracle's velocity gradient
    is O(N^2) per cell)."""
    return P.cavity(seed=31, nx=12, ny=12, mean_ppc=11, ppc_range=(8, 14))


def _forward(pop, prec="fp64", vdtype="f64"):
    v = _dev(pop.v64 if vdtype == "f64" else pop.v32)
    off, tau = _dev(pop.offsets), _dev(pop.tau)
    mom, y, fl = api.fp_closure_exact(v, off, tau, prec=prec)
    return v, off, tau, mom, y, fl


def test_moment_gradient_matches_oracle(cavity_pop):
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 41))
    v, off, tau, mom, y, fl = _forward(pop)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((pop.n_cells, 9))
    gin = rng.standard_normal((pop.n_cells, 30)) * 0.1
    gm, _ = api.fp_closure_backward(v, off, tau, mom, y, fl, _dev(g), grad_moments_in=_dev(gin), want_grad_v=False)
    torch.cuda.synchronize()
    m = O.moments(pop.v64, pop.offsets)
    gref, _ = O.closure_backward(pop.v64, pop.offsets, pop.tau, m, g, grad_moments_in=gin, want_grad_v=False)
    _, _, cond, _ = O.closure(m, pop.tau, want_cond=True)
    gm = gm.cpu().numpy()
    ok = cond < 1e6
    err = np.linalg.norm(gm - gref, axis=1) / np.linalg.norm(gref, axis=1)
    assert ok.mean() > 0.9
    assert err[ok].max() < 1e-9, err[ok].max()


@pytest.mark.parametrize("vdtype,tol", [("f64", 1e-9), ("f32", 2e-4)])
def test_velocity_gradient_matches_oracle(small_cells, vdtype, tol):
    pop = small_cells.subset(np.arange(0, small_cells.n_cells, 2))
    prec = "fp64" if vdtype == "f64" else "fp32"
    v, off, tau, mom, y, fl = _forward(pop, prec, vdtype)
    rng = np.random.default_rng(4)
    g = rng.standard_normal((pop.n_cells, 9))
    gm, gv = api.fp_closure_backward(v, off, tau, mom, y, fl, _dev(g))
    torch.cuda.synchronize()
    vv = pop.v64 if vdtype == "f64" else pop.v32.astype(np.float64)
    m = O.moments(vv, pop.offsets)
    yr, flr, cond, _ = O.closure(m, pop.tau, want_cond=True)
    gref_m, gref_v = O.closure_backward(vv, pop.offsets, pop.tau, m, g)
    ok = (flr == 0) & (fl.cpu().numpy() == flr) & (cond < 1e5)
    assert ok.mean() > 0.8
    gv = gv.cpu().numpy().astype(np.float64)
    for c in np.nonzero(ok)[0]:
        s = slice(pop.offsets[c], pop.offsets[c + 1])
        ref = gref_v[:, s]
        assert np.linalg.norm(gv[:, s] - ref) <= tol * np.linalg.norm(ref) + 1e-300, c


def test_central_differences_on_64_random_cells(cavity_pop):
    """L = sum_c gY_c . Y_c; FD of the GPU FP64 forward along random
    directions, in the moments and in the particle velocities."""
    rng = np.random.default_rng(8)
    cells = np.sort(rng.choice(cavity_pop.n_cells, 64, replace=False))
    pop = cavity_pop.subset(cells)
    v, off, tau, mom, y, fl = _forward(pop)
    g = _dev(rng.standard_normal((pop.n_cells, 9)))
    gm, gv = api.fp_closure_backward(v, off, tau, mom, y, fl, g)
    h = 1e-6

    def L_m(mm):
        yy, _ = api.fp_closure_solve(mm, tau, prec="fp64")
        return float((g * yy).sum())

    def L_v(vv):
        _, yy, _ = api.fp_closure_exact(vv, off, tau, prec="fp64")
        return float((g * yy).sum())

    for trial in range(3):
        dm = _dev(rng.standard_normal((pop.n_cells, 30)) * np.abs(mom.cpu().numpy()).clip(1e-3))
        dm[:, :4] = 0  # N and U: no closure dependence
        fd = (L_m(mom + h * dm) - L_m(mom - h * dm)) / (2 * h)
        an = float((gm * dm).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (fd, an)
        dv = _dev(rng.standard_normal(pop.v64.shape))
        fd = (L_v(v + h * dv) - L_v(v - h * dv)) / (2 * h)
        an = float((gv * dv).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (fd, an)


def test_autograd_function_and_flagged_cells(small_cells):
    pop = small_cells.subset(np.arange(0, 40))
    v = _dev(pop.v64).requires_grad_(True)
    off, tau = _dev(pop.offsets), _dev(pop.tau)
    mom, y, fl = autograd.closure(v, off, tau)
    # a loss on both outputs: coefficients and the temperature moment
    loss = (y ** 2).sum() + mom[:, 4].sum()
    loss.backward()
    gY = (2 * y).detach()
    gin = torch.zeros_like(mom)
    gin[:, 4] = 1
    _, gv = api.fp_closure_backward(v.detach(), off, tau, mom.detach(), y.detach(), fl, gY, grad_moments_in=gin)
    torch.cuda.synchronize()
    assert torch.allclose(v.grad, gv, rtol=1e-12, atol=1e-14)
    # moments-only function
    m = mom.detach().clone().requires_grad_(True)
    yy = autograd.closure_from_moments(m, tau)
    (yy * gY).sum().backward()
    gm, _ = api.fp_closure_backward(v.detach(), off, tau, mom.detach(), y.detach(), fl, gY, want_grad_v=False)
    assert torch.allclose(m.grad, gm, rtol=1e-12, atol=1e-14)
    # flagged cells: no closure gradient
    flagged = (fl & api.FALLBACK_FLAGS) != 0
    fl2 = fl.clone()
    fl2[:5] |= api.FLAG_FEW
    gm2, _ = api.fp_closure_backward(v.detach(), off, tau, mom.detach(), y.detach(), fl2, gY, want_grad_v=False)
    assert torch.all(gm2[:5] == 0)
    assert not flagged[:5].all()


def _lu_row(lu, c):
    """The FP_LU_STRIDE entries of cell c (tiles of 32 cells, entries 32 apart)."""
    base = (c // 32) * 32 * api.LU_STRIDE + c % 32
    return lu[base + 32 * np.arange(api.LU_STRIDE)]


def _unpack_lu(row):
    """(P, L, U) with P A = L U from one cell's stored entries."""
    M = row[:81].reshape(9, 9)
    L = np.tril(M, -1) + np.eye(9)
    U = np.triu(M, 1) + np.diag(1.0 / np.diag(M))  # the diagonal holds 1 / pivot
    perm = int(np.frombuffer(row[81:82].tobytes(), dtype=np.uint64)[0])
    P = np.eye(9)
    for k in range(9):  # the swaps of the elimination, in order
        b = (perm >> (4 * k)) & 15
        P[[k, b]] = P[[b, k]]
    return P, L, U


def test_stored_factors_reproduce_the_oracle_matrix(cavity_pop):
    """The factors fp_closure_solve keeps satisfy P A = L U for the oracle's
    assembled A (relative to max |A|), with |L| <= 1 (partial pivoting)."""
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 97))
    v, off, tau, mom, y, fl = _forward(pop)
    lu = torch.full((api.lu_doubles(pop.n_cells),), np.nan, dtype=torch.float64, device="cuda")
    y2, fl2 = api.fp_closure_solve(mom, tau, prec="fp64", lu_out=lu)
    torch.cuda.synchronize()
    assert torch.equal(y2, y) and torch.equal(fl2, fl)
    m, lu = mom.cpu().numpy(), lu.cpu().numpy()
    checked = 0
    for c in np.flatnonzero(fl.cpu().numpy() == 0):
        A, _ = O.assemble(m[c], pop.tau[c])
        Pm, L, U = _unpack_lu(_lu_row(lu, c))
        assert np.abs(np.tril(L, -1)).max() <= 1.0
        assert np.abs(Pm @ A - L @ U).max() <= 1e-13 * np.abs(A).max() * 9
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("vdtype", ["f64", "f32"])
def test_backward_with_stored_factors_matches_recomputation(cavity_pop, vdtype):
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 7))
    prec = "fp64" if vdtype == "f64" else "fp32"
    v, off, tau, mom, y, fl = _forward(pop, prec, vdtype)
    lu = torch.empty(api.lu_doubles(pop.n_cells), dtype=torch.float64, device="cuda")
    api.fp_closure_solve(mom, tau, prec=prec, lu_out=lu)
    g = _dev(np.random.default_rng(12).standard_normal((pop.n_cells, 9)))
    gm0, gv0 = api.fp_closure_backward(v, off, tau, mom, y, fl, g)
    gm1, gv1 = api.fp_closure_backward(v, off, tau, mom, y, fl, g, lu=lu)
    torch.cuda.synchronize()
    _, _, cond, _ = O.closure(mom.cpu().numpy(), pop.tau, want_cond=True)
    ok = torch.from_numpy((cond < 1e6) & (fl.cpu().numpy() == 0)).cuda()
    assert ok.float().mean() > 0.9
    rel = (gm1 - gm0).norm(dim=1) / gm0.norm(dim=1).clamp_min(1e-300)
    assert rel[ok].max().item() < 1e-9
    # flagged cells carry only grad_moments_in (zero here) in both
    assert torch.equal(gm1[fl != 0], gm0[fl != 0])
    cell_of = torch.repeat_interleave(torch.arange(pop.n_cells, device="cuda"), _dev(pop.counts))
    okp = ok[cell_of]
    scale = gv0.abs().max()
    tol = 1e-9 if vdtype == "f64" else 1e-4
    assert ((gv1 - gv0).abs()[:, okp].max() / scale).item() < tol
