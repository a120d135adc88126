"""The bounded mbarrier wait gives up: a wait on a barrier that nothing
completes returns after its limit and reports it (no spin, no fault), and
the context stays usable."""

import pytest
import torch

from paper_2606_15622_gb300 import api

pytestmark = pytest.mark.gpu


def test_wait_on_an_incomplete_barrier_gives_up_after_its_limit():
    status, waited = api.fp_selftest_wait_timeout(1_000_000)  # 1 ms
    assert status == 0
    assert 1_000_000 <= waited < 200_000_000
    with pytest.raises(api.FPError):
        api.fp_selftest_wait_timeout(0)
    x = torch.arange(8, device="cuda", dtype=torch.float64)
    assert float(x.sum().item()) == 28.0  # the context still works
