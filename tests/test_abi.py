"""The C ABI library builds, loads without a GPU, and exports every entry
point that include/*.h declares (no compute call is made here)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(fp_\w+)\s*\(", txt, flags=re.M))
    return names


def test_header_declares_the_four_calls():
    names = _declared()
    assert "fp_closure_exact" in names and "fp_workspace_bytes" in names


def test_library_exports_every_declared_symbol():
    from paper_2606_15622_gb300 import api
    L = ctypes.CDLL(api.library_path()) if os.path.exists(api.library_path()) else api.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2606_15622_gb300 import api
    assert _declared() <= set(api.SIGNATURES)


def test_host_only_calls_work_without_gpu():
    from paper_2606_15622_gb300 import api
    L = api.lib()
    assert L.fp_version() >= 100
    assert L.fp_status_string(-1) == b"invalid argument"
    p = api.default_params()
    assert p.min_particles == 4 and p.pivot_rtol == 1e-13
    assert api.workspace_bytes(1000, 5000, "fp32") == 256 * ((1000 * 30 * 8 + 255) // 256)
    assert api.workspace_bytes(1000, 5000, "fp32", moments_out_given=True) == 0


def test_binding_checks_tensor_arguments_before_the_abi():
    """The C ABI takes plain pointers, so the binding refuses host tensors,
    wrong dtypes and too-short arrays before anything reaches the library."""
    import torch

    from paper_2606_15622_gb300 import api
    with pytest.raises(api.FPError, match="CUDA tensors"):
        api.fp_moments(torch.zeros((3, 8)), torch.zeros(3, dtype=torch.int64), moments_out=torch.zeros((2, 30)))
    assert api._nv(torch.zeros((3, 7))) == 7 and api._nv(torch.zeros(21, dtype=torch.float64)) == 7
    for bad in (torch.zeros((4, 7)), torch.zeros(20), torch.zeros((3, 7), dtype=torch.float16)):
        with pytest.raises(api.FPError):
            api._nv(bad)
    api._want(None, "x", torch.float64, 10)
    api._want(torch.zeros(10, dtype=torch.float64), "x", torch.float64, 10)
    with pytest.raises(api.FPError, match="must be torch.float64"):
        api._want(torch.zeros(10, dtype=torch.float32), "x", torch.float64, 10)
    with pytest.raises(api.FPError, match="at least 11"):
        api._want(torch.zeros(10, dtype=torch.float64), "x", torch.float64, 11)
    api._want_cells(4, torch.zeros(5, dtype=torch.int64), torch.zeros(4, dtype=torch.float64),
                    torch.zeros((4, api.NMOM), dtype=torch.float64), torch.zeros((4, 9), dtype=torch.float64),
                    torch.zeros(4, dtype=torch.int32))
    with pytest.raises(api.FPError, match="offsets"):
        api._want_cells(4, offsets=torch.zeros(5, dtype=torch.int32))
    with pytest.raises(api.FPError, match="moments"):
        api._want_cells(4, moments=torch.zeros((4, api.NLITE), dtype=torch.float64))
    api._want_cells(4, moments=torch.zeros((4, api.NLITE), dtype=torch.float64), stride=api.NLITE)


def test_train_step_refuses_bad_arguments_on_the_host():
    """fp_surrogate_train_step validates its arguments before any launch (no
    GPU needed): network shape, parameter count, step number, null arrays,
    alignment and workspace size; an empty batch is a no-op."""
    from paper_2606_15622_gb300 import api
    L = api.lib()
    net = api.FpMlp()
    for l in range(5):
        net.W[l] = 0x1000 * (l + 1)
        net.b[l] = 0x10000 + 0x1000 * l
    net.x_mu = net.x_sigma = net.y_mu = net.y_sigma = net.x_min = net.x_max = 0x20000
    net.in_dim, net.hidden, net.depth, net.out_dim, net.eps2_hat = 32, 128, 4, 16, 1e-3
    npar = int(L.fp_mlp_param_count())
    w = (ctypes.c_float * 9)(*([1.0] * 9))
    fake = 0x40000  # never dereferenced: every call below fails (or returns) before a launch
    n = 1000
    need = int(L.fp_surrogate_train_step_workspace_bytes(n))
    assert need > 0 and int(L.fp_surrogate_train_step_workspace_bytes(0)) == 0

    def call(n=n, npar=npar, t=1, x=fake, ws=fake, ws_bytes=need, net=net):
        return L.fp_surrogate_train_step(ctypes.byref(net), x, fake, fake, n, w, 0.1, 1.0, 1.0 / max(n, 1), fake,
                                         fake, fake, fake, npar, 1e-3, 0.9, 0.999, 1e-8, t, None, fake, ws,
                                         ws_bytes, None)

    assert call(npar=npar - 1) == api.FP_ERR_ARG
    assert call(t=0) == api.FP_ERR_ARG
    assert call(n=-1) == api.FP_ERR_ARG
    assert call(n=0) == api.FP_OK
    assert call(x=None) == api.FP_ERR_ARG
    assert call(x=fake + 8) == api.FP_ERR_ARG           # x must be 16-byte aligned
    assert call(ws_bytes=need - 1) == api.FP_ERR_WORKSPACE
    assert call(ws=fake + 64) == api.FP_ERR_ARG         # workspace must be 256-byte aligned
    bad = api.FpMlp.from_buffer_copy(net)
    bad.hidden = 64
    assert call(net=bad) == api.FP_ERR_UNSUPPORTED
