"""fp_closure_exact_static -- the exact closure for callers that may not
allocate device memory (its scratch is an array built into the library).

Checked through the C ABI against fp_closure_exact (which takes its scratch
from the caller) on two calls in a row, the second on a different, smaller
population so that anything left in the shared array by the first call would
show.  Both paths run the same kernels on the same inputs, so the results
must agree to the parity tolerances of the closure tests (1e-10 relative for
FP64 moments, 1e-4 for FP32 moments); in practice they are identical.
"""

import numpy as np
import pytest
import torch

from paper_2606_15622_gb300 import api
from paper_2606_15622_gb300 import populations as P

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _compare(pop, prec):
    v = _dev(pop.v64 if prec == "fp64" else pop.v32)
    off, tau = _dev(pop.offsets), _dev(pop.tau)
    y_static, f_static = api.fp_closure_exact_static(v, off, tau, prec=prec)
    _, y_ref, f_ref = api.fp_closure_exact(v, off, tau, prec=prec, want_moments=False)
    torch.cuda.synchronize()
    assert torch.equal(f_static, f_ref)
    ys, yr = y_static.cpu().numpy(), y_ref.cpu().numpy()
    err = np.linalg.norm(ys - yr, axis=1) / np.linalg.norm(yr, axis=1)
    assert err.max() <= TOL[prec], err.max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_matches_workspace_path_on_two_calls(prec):
    first = P.cavity(seed=12)                       # 16384 cells
    second = P.couette(seed=13)                     # 400 cells
    _compare(first, prec)
    _compare(second, prec)


def test_static_scratch_rejects_too_many_cells():
    n = api.STATIC_MAX_CELLS + 1
    v = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    off = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    tau = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(api.FPError, match="FP_STATIC_MAX_CELLS"):
        api.fp_closure_exact_static(v, off, tau)
