"""GPU high-order diagnostics and coefficient under-relaxation (through the C
ABI) against the oracle's definitions."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_15622_gb300 import api
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("with_rho", [False, True])
def test_diagnostics_match_oracle(cavity_pop, with_rho):
    pop = cavity_pop.subset(np.arange(0, cavity_pop.n_cells, 7))
    v = torch.from_numpy(pop.v64).cuda()
    off = torch.from_numpy(pop.offsets).cuda()
    m6 = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    mom = api.fp_moments(v, off, prec="fp64", m6_out=m6)
    rho = torch.from_numpy(pop.counts * 0.37 + 1.0).cuda() if with_rho else None
    d = api.fp_diagnostics(mom, m6, rho=rho, theta_inf=1.1, rho_inf=50.0, dg_inf=0.01)
    torch.cuda.synchronize()
    ref = O.diagnostics(mom.cpu().numpy(), m6.cpu().numpy(), rho=None if rho is None else rho.cpu().numpy(),
                        theta_inf=1.1, rho_inf=50.0, dg_inf=0.01)
    got = d.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    scale = np.maximum(np.abs(ref), 1.0)
    assert np.all(np.abs(got - ref)[ok] <= 1e-12 * scale[ok])


def test_diagnostics_edge_cells():
    pop = P.maxwellian_cells([0, 1, 2, 500], theta=[1.0, 1.0, 1.0, 2.0], seed=4)
    v = torch.from_numpy(pop.v64).cuda()
    off = torch.from_numpy(pop.offsets).cuda()
    m6 = torch.empty(pop.n_cells, dtype=torch.float64, device="cuda")
    mom = api.fp_moments(v, off, prec="fp64", m6_out=m6)
    d = api.fp_diagnostics(mom, m6).cpu().numpy()
    assert np.isnan(d[0]).all() and np.isnan(d[1]).all()  # N < 2
    assert np.isfinite(d[3]).all() and d[3, 8] >= 0


def test_relaxation_matches_oracle():
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal((1000, 9)), rng.standard_normal((1000, 9))
    ya, yb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    api.fp_coeffs_relax(ya, yb, 0.2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(yb.cpu().numpy(), O.coeffs_relax(a, b, 0.2), rtol=0, atol=1e-15)
    with pytest.raises(api.FPError):
        api.fp_coeffs_relax(ya, yb, 1.5)
