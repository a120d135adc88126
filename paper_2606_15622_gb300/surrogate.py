"""The learned closure: network container, training on exact-closure data,
and the surrogate call (paper Sec. 4: phases 1-3; Alg. 2).

Every numerical step of training and inference runs in libfpclosure's
kernels (features, fused BF16 MLP forward, loss + gradient, BF16 backward
GEMMs, Adam, exact fallback); torch provides device memory, the data
shuffling and the scaler statistics of the training set.

Two input sets share the network shape (inputs padded to 32):
  "full": the 25 normalised high-order moments (u/theta, u3/theta^1.5,
          w/theta^2, z/theta^2.5) of the full moment vector;
  "lite": the 16 low-order inputs rho, T, U, Pi, q, DM2, nu of the LITE
          moment vector (fp_moments_lite; Sec. 4, Phase 1-2 item 1 and
          Phase 3 item 2).
Both predict the same dimensionless targets (tau C, tau sqrt(theta) G).

Weight file (little-endian): magic b"FPCW", u32 version, u32 dims (32, 128,
4, 16), f64 eps2_hat, u64 training seed, [version 2: u32 input set, 0 full,
1 lite], then FP32 arrays: the flat parameters (fp_mlp_param_count), x_mu,
x_sigma, x_min, x_max [32], y_mu, y_sigma [16].  Version 1 files hold a
full-input network.
"""

from __future__ import annotations

import ctypes
import io
import os
import struct
import time

import numpy as np
import torch

from . import api

IN, HID, OUT, DEPTH, NFEAT, NOUT = 32, 128, 16, 4, 25, 9
NFEAT_LITE = 16
FEATURE_SETS = {"full": (0, NFEAT), "lite": (1, NFEAT_LITE)}
MAGIC = b"FPCW"
VERSION = 2


FpMlp = api.FpMlp


def _lib():
    return api.lib()


def param_count() -> int:
    return int(_lib().fp_mlp_param_count())


def param_offset(which: int, layer: int) -> int:
    return int(_lib().fp_mlp_param_offset(which, layer))


def saved_rows(a):
    """A saved-activation buffer of fp_mlp_forward ([4][128 / b][n][b]: b = 8
    for H, 4 for Z) as [4][n][128]."""
    d, kb, n, b = a.shape
    return a.permute(0, 2, 1, 3).reshape(d, n, kb * b)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Surrogate:
    """Parameters (FP32 master + BF16 shadow), scalers and the fp_mlp view."""

    def __init__(self, device="cuda", eps2_hat=1e-3, seed=0, features="full"):
        if features not in FEATURE_SETS:
            raise api.FPError(f"unknown input set {features!r}")
        self.features_set = features
        self.nfeat = FEATURE_SETS[features][1]
        self.device = torch.device(device)
        self.eps2_hat = float(eps2_hat)
        self.seed = int(seed)
        n = param_count()
        self.params = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.shadow = torch.zeros(n, dtype=torch.bfloat16, device=self.device)
        self.x_mu = torch.zeros(IN, dtype=torch.float32, device=self.device)
        self.x_sigma = torch.ones(IN, dtype=torch.float32, device=self.device)
        self.x_min = torch.full((IN,), -3e38, dtype=torch.float32, device=self.device)
        self.x_max = torch.full((IN,), 3e38, dtype=torch.float32, device=self.device)
        self.y_mu = torch.zeros(OUT, dtype=torch.float32, device=self.device)
        self.y_sigma = torch.ones(OUT, dtype=torch.float32, device=self.device)
        self._net = None

    # ---- parameters ----------------------------------------------------
    def layer_views(self):
        dims = [(HID, IN), (HID, HID), (HID, HID), (HID, HID), (OUT, HID)]
        W = [self.params[param_offset(0, l):param_offset(0, l) + o * i].view(o, i) for l, (o, i) in enumerate(dims)]
        b = [self.params[param_offset(1, l):param_offset(1, l) + o] for l, (o, _) in enumerate(dims)]
        return W, b

    def init_params(self, seed=None):
        """He-style init (uniform scaled 1/sqrt(fan_in)); padded inputs and
        outputs are zero."""
        g = torch.Generator(device="cpu").manual_seed(self.seed if seed is None else seed)
        W, b = self.layer_views()
        for l, w in enumerate(W):
            fan_in = w.shape[1] if l > 0 else self.nfeat
            w.copy_((torch.rand(w.shape, generator=g) * 2 - 1) * np.sqrt(3.0 / fan_in))
            b[l].zero_()
        W[0][:, self.nfeat:] = 0
        W[4][NOUT:, :] = 0
        self.sync_shadow()

    def set_params(self, Ws, bs):
        W, b = self.layer_views()
        for l in range(5):
            W[l].copy_(torch.as_tensor(np.asarray(Ws[l]), dtype=torch.float32))
            b[l].copy_(torch.as_tensor(np.asarray(bs[l]), dtype=torch.float32))
        self.sync_shadow()

    def sync_shadow(self):
        self.shadow.copy_(self.params.to(torch.bfloat16))
        self._net = None

    def net(self) -> FpMlp:
        if self._net is None:
            m = FpMlp()
            for l in range(5):
                m.W[l] = self.shadow.data_ptr() + 2 * param_offset(0, l)
                m.b[l] = self.params.data_ptr() + 4 * param_offset(1, l)
            m.x_mu, m.x_sigma = self.x_mu.data_ptr(), self.x_sigma.data_ptr()
            m.y_mu, m.y_sigma = self.y_mu.data_ptr(), self.y_sigma.data_ptr()
            m.x_min, m.x_max = self.x_min.data_ptr(), self.x_max.data_ptr()
            m.in_dim, m.hidden, m.depth, m.out_dim = IN, HID, DEPTH, OUT
            m.eps2_hat = self.eps2_hat
            self._net = m
        return self._net

    # ---- kernels -------------------------------------------------------
    def _want(self, features):
        if self.features_set != features:
            raise api.FPError(f"this network reads the {self.features_set!r} inputs, not {features!r}")

    def features(self, moments, tau, params=None, x_out=None, flags_out=None, stream=None):
        self._want("full")
        n = moments.shape[0]
        x = x_out if x_out is not None else torch.empty((n, IN), dtype=torch.bfloat16, device=self.device)
        fl = flags_out if flags_out is not None else torch.empty(n, dtype=torch.int32, device=self.device)
        api._need_cuda(moments, tau, x, fl)
        api._want_cells(n, None, tau, moments, None, fl)
        api._want(x, "x_out", torch.bfloat16, n * IN)
        p = params if params is not None else api.default_params(eps2_hat=self.eps2_hat)
        rc = _lib().fp_surrogate_features(ctypes.byref(self.net()), _p(moments), n, _p(tau), ctypes.byref(p),
                                          _p(x), _p(fl), api._stream(stream))
        api._check(rc, "fp_surrogate_features")
        return x, fl

    def forward(self, x, standardized=True, save=False, out=None, stream=None):
        n = x.shape[0]
        o = out if out is not None else torch.empty((n, OUT), dtype=torch.float32, device=self.device)
        h = z = None
        if save:  # column-block-major (see saved_rows)
            h = torch.empty((DEPTH, HID // 8, n, 8), dtype=torch.bfloat16, device=self.device)
            z = torch.empty((DEPTH, HID // 4, n, 4), dtype=torch.float32, device=self.device)
        api._need_cuda(x, o)
        api._want(x, "x", torch.bfloat16, n * IN)
        api._want(o, "out", torch.float32, n * OUT)
        rc = _lib().fp_mlp_forward(ctypes.byref(self.net()), _p(x), n, int(bool(standardized)), _p(o), _p(h), _p(z),
                                   api._stream(stream))
        api._check(rc, "fp_mlp_forward")
        return (o, h, z) if save else o

    def closure(self, moments, tau, params=None, prec="fp64", coeffs_out=None, flags_out=None, workspace=None,
                stream=None):
        """The surrogate closure with exact fallback -> (coeffs, flags)."""
        self._want("full")
        n = moments.shape[0]
        y = coeffs_out if coeffs_out is not None else torch.empty((n, 9), dtype=torch.float64, device=self.device)
        fl = flags_out if flags_out is not None else torch.empty(n, dtype=torch.int32, device=self.device)
        need = int(_lib().fp_surrogate_workspace_bytes(n))
        ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=self.device)
        api._need_cuda(moments, tau, y, fl, ws)
        api._want_cells(n, None, tau, moments, y, fl)
        p = params if params is not None else api.default_params(eps2_hat=self.eps2_hat)
        rc = _lib().fp_closure_surrogate(ctypes.byref(self.net()), _p(moments), n, _p(tau), ctypes.byref(p),
                                         api._PREC.get(prec, prec), _p(y), _p(fl), _p(ws), ws.numel(),
                                         api._stream(stream))
        api._check(rc, "fp_closure_surrogate")
        return y, fl

    def lite_features(self, lite, tau, params=None, x_out=None, flags_out=None, stream=None):
        """Standardised BF16 inputs [n, 32] and flags from LITE vectors."""
        self._want("lite")
        n = lite.shape[0]
        x = x_out if x_out is not None else torch.empty((n, IN), dtype=torch.bfloat16, device=self.device)
        fl = flags_out if flags_out is not None else torch.empty(n, dtype=torch.int32, device=self.device)
        api._need_cuda(lite, tau, x, fl)
        api._want_cells(n, None, tau, lite, None, fl, stride=api.NLITE)
        api._want(x, "x_out", torch.bfloat16, n * IN)
        p = params if params is not None else api.default_params(eps2_hat=self.eps2_hat)
        rc = _lib().fp_surrogate_lite_features(ctypes.byref(self.net()), _p(lite), n, _p(tau), ctypes.byref(p),
                                               _p(x), _p(fl), api._stream(stream))
        api._check(rc, "fp_surrogate_lite_features")
        return x, fl

    def closure_lite(self, lite, tau, params=None, coeffs_out=None, flags_out=None, workspace=None, stream=None):
        """The learned closure on LITE vectors -> (coeffs, flags); cells it
        cannot serve take the linear drift -I/tau."""
        self._want("lite")
        n = lite.shape[0]
        y = coeffs_out if coeffs_out is not None else torch.empty((n, 9), dtype=torch.float64, device=self.device)
        fl = flags_out if flags_out is not None else torch.empty(n, dtype=torch.int32, device=self.device)
        need = int(_lib().fp_surrogate_lite_workspace_bytes(n))
        ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=self.device)
        api._need_cuda(lite, tau, y, fl, ws)
        api._want_cells(n, None, tau, lite, y, fl, stride=api.NLITE)
        p = params if params is not None else api.default_params(eps2_hat=self.eps2_hat)
        rc = _lib().fp_closure_surrogate_lite(ctypes.byref(self.net()), _p(lite), n, _p(tau), ctypes.byref(p),
                                              _p(y), _p(fl), _p(ws), ws.numel(), api._stream(stream))
        api._check(rc, "fp_closure_surrogate_lite")
        return y, fl

    def sensitivity(self, moments, tau, n_passes=50, rate=0.2, seed=0, params=None, sens_out=None, mean_out=None,
                    flags_out=None, workspace=None, stream=None):
        """The heuristic coefficient-sensitivity probe (dropout at inference,
        n_passes forward passes) -> (sens [n, 11]: sigma of the nine
        coefficients, sigma_Stress, sigma_Heat; mean coefficients [n, 9];
        input flags).  moments: full vectors [n, 30] or LITE vectors [n, 14],
        as the network's input set requires."""
        n = moments.shape[0]
        stride = api.NMOM if self.features_set == "full" else api.NLITE
        if moments.shape[1] != stride:
            raise api.FPError(f"a {self.features_set!r} network reads [n, {stride}] moment vectors")
        dev = self.device
        sens = sens_out if sens_out is not None else torch.empty((n, api.NSENS), dtype=torch.float64, device=dev)
        mean = mean_out if mean_out is not None else torch.empty((n, 9), dtype=torch.float64, device=dev)
        fl = flags_out if flags_out is not None else torch.empty(n, dtype=torch.int32, device=dev)
        need = int(_lib().fp_surrogate_sensitivity_workspace_bytes(n))
        ws = workspace if workspace is not None else torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        api._need_cuda(moments, tau, sens, mean, fl, ws)
        api._want_cells(n, None, tau, moments, mean, fl, stride=stride)
        api._want(sens, "sens_out", torch.float64, n * api.NSENS)
        p = params if params is not None else api.default_params(eps2_hat=self.eps2_hat)
        rc = _lib().fp_surrogate_sensitivity(ctypes.byref(self.net()), _p(moments), stride, n, _p(tau),
                                             ctypes.byref(p), int(n_passes), float(rate), int(seed), _p(sens),
                                             _p(mean), _p(fl), _p(ws), ws.numel(), api._stream(stream))
        api._check(rc, "fp_surrogate_sensitivity")
        return sens, mean, fl

    # ---- persistence ---------------------------------------------------
    def save(self, path):
        buf = io.BytesIO()
        buf.write(MAGIC)
        buf.write(struct.pack("<IIIIIdQ", VERSION, IN, HID, DEPTH, OUT, self.eps2_hat, self.seed))
        buf.write(struct.pack("<I", FEATURE_SETS[self.features_set][0]))
        for t in (self.params, self.x_mu, self.x_sigma, self.x_min, self.x_max, self.y_mu, self.y_sigma):
            buf.write(t.detach().cpu().numpy().astype("<f4").tobytes())
        tmp = path + ".tmp"
        with open(tmp, "wb") as f:
            f.write(buf.getvalue())
        os.replace(tmp, path)

    @classmethod
    def load(cls, path, device="cuda"):
        raw = open(path, "rb").read()
        if raw[:4] != MAGIC:
            raise api.FPError(f"{path}: not a weight file")
        ver, i, h, d, o, eps2_hat, seed = struct.unpack("<IIIIIdQ", raw[4:4 + 36])
        if ver not in (1, 2) or (i, h, d, o) != (IN, HID, DEPTH, OUT):
            raise api.FPError(f"{path}: unsupported version/shape")
        pos0, features = 40, "full"
        if ver == 2:
            (fid,) = struct.unpack("<I", raw[40:44])
            names = {v[0]: k for k, v in FEATURE_SETS.items()}
            if fid not in names:
                raise api.FPError(f"{path}: unknown input set {fid}")
            pos0, features = 44, names[fid]
        s = cls(device=device, eps2_hat=eps2_hat, seed=seed, features=features)
        arr = np.frombuffer(raw[pos0:], dtype="<f4")
        n = param_count()
        parts = [n, IN, IN, IN, IN, OUT, OUT]
        if arr.size != sum(parts):
            raise api.FPError(f"{path}: truncated")
        pos = 0
        for t, k in zip((s.params, s.x_mu, s.x_sigma, s.x_min, s.x_max, s.y_mu, s.y_sigma), parts):
            t.copy_(torch.from_numpy(arr[pos:pos + k].copy()))
            pos += k
        s.sync_shadow()
        return s


# ---------------------------------------------------------------------------
# training data and training
# ---------------------------------------------------------------------------
def dimensionless(coeffs, mom, tau):
    """Dimensionless coefficients (tau C, tau sqrt(theta) G) [n, 9] of `coeffs`,
    from the library's kernel (FP32 values, returned as float64)."""
    _, t, _ = api.fp_surrogate_training_rows(mom, tau, coeffs=coeffs, raw=False, aux=False)
    return t[:, :NOUT].double()


def aux_moments(mom, tau):
    """(u^_ij (6), b^_i (3), s4^) [n, 10] normalised moments of the full
    moment vectors, from the library's kernel (FP32, returned as float64)."""
    _, _, x = api.fp_surrogate_training_rows(mom, tau, raw=False, targets=False)
    return x[:, :10].double()


def error_report(s: "Surrogate", mom, tau, y_exact, flags_exact, eps2_hat, params=None, lite=None):
    """Error of the learned closure against the exact closure's coefficients on
    the same cells (dimensionless, ||dY|| / ||Y|| per cell, over the cells the
    exact closure does not flag):
      network   the network's prediction for every such cell (before fallback)
      closure   the learned closure's output (after its fallback: cells it
                flags are re-solved exactly, or take the linear drift on LITE
                inputs)
    plus |e| of the energy residual e = 1 + (sum C^_ij u^_ij + sum G^_i b^_i -
    eps^2 s4^) / 3 of both (0 for the exact closure), the flag rates, and the
    linear drift's error for scale.  `lite` selects LITE inputs."""
    p = params if params is not None else api.default_params(eps2_hat=eps2_hat)
    if lite is not None:
        x, fl_in = s.lite_features(lite, tau, params=p)
        y_s, fl_s = s.closure_lite(lite, tau, params=p)
        fb = (fl_s & api.FALLBACK_FLAGS) != 0
    else:
        x, fl_in = s.features(mom, tau, params=p)
        y_s, fl_s = s.closure(mom, tau, params=p)
        fb = (fl_s & api.FLAG_FALLBACK) != 0
    t_net = s.forward(x, standardized=False)[:, :NOUT].double()
    t_ex = dimensionless(y_exact, mom, tau)
    t_cl = dimensionless(y_s, mom, tau)
    ax = aux_moments(mom, tau)
    ok = (flags_exact == 0) & torch.isfinite(t_ex).all(1)
    mult = torch.tensor([1, 2, 2, 1, 2, 1], dtype=torch.float64, device=t_ex.device)

    def energy(t):
        return 1 + ((t[:, :6] * ax[:, :6] * mult).sum(1) + (t[:, 6:] * ax[:, 6:9]).sum(1) - eps2_hat * ax[:, 9]) / 3

    def stats(x):
        x = x[torch.isfinite(x)].float().cpu()
        if x.numel() == 0:
            return None
        return {"median": float(x.median()), "p95": float(torch.quantile(x, 0.95)),
                "p99": float(torch.quantile(x, 0.99)), "max": float(x.max())}

    nrm = t_ex.norm(dim=1)
    rel_net = ((t_net - t_ex).norm(dim=1) / nrm)[ok]
    rel_cl = ((t_cl - t_ex).norm(dim=1) / nrm)[ok]
    lin = torch.zeros_like(t_ex)
    lin[:, [0, 3, 5]] = -1.0
    rel_lin = ((lin - t_ex).norm(dim=1) / nrm)[ok]
    kept = ok & ~fb
    return {
        "cells": int(ok.numel()), "cells_compared": int(ok.sum()), "inputs": s.features_set,
        "fallback_rate": float(fb.double().mean()),
        "range_flag_rate": float(((fl_s & api.FLAG_RANGE) != 0).double().mean()),
        "energy_flag_rate": float(((fl_s & api.FLAG_ENERGY) != 0).double().mean()),
        "rel_err_network_before_fallback": stats(rel_net),
        "rel_err_closure_after_fallback": stats(rel_cl),
        "rel_err_network_on_kept_cells": stats(((t_cl - t_ex).norm(dim=1) / nrm)[kept]),
        "energy_residual_abs_network": stats(energy(t_net)[ok].abs()),
        "energy_residual_abs_closure": stats(energy(t_cl)[ok].abs()),
        "rel_err_linear_closure": stats(rel_lin),
    }


class TrainingSet:
    """Cells labelled by the exact FP64 GPU closure.  Everything the training
    reads comes from the library's kernels (fp_surrogate_training_rows): the
    unstandardised inputs of the chosen set (statistics for the scalers),
    the dimensionless targets, and the aux moments (always from the full
    moment vector: the energy term of the loss needs s4).  The network's
    inputs themselves are made by the inference kernels (fp_surrogate_features
    / fp_surrogate_lite_features) once the scalers are set (`inputs`), so
    training and inference see the same BF16 inputs.  Cells the exact closure
    flags, and coefficients beyond 1e6 in magnitude (dimensionless), are
    dropped."""

    def __init__(self, pop, eps2_hat=1e-3, device="cuda", chunk=262144, features="full"):
        dev = torch.device(device)
        prm = api.default_params(eps2_hat=eps2_hat)
        raws, targs, auxs, srcs, taus = [], [], [], [], []
        n_cells = pop.n_cells
        for c0 in range(0, n_cells, chunk):
            c1 = min(n_cells, c0 + chunk)
            a, b = int(pop.offsets[c0]), int(pop.offsets[c1])
            v = torch.from_numpy(np.ascontiguousarray(pop.v64[:, a:b])).to(dev)
            off = torch.from_numpy(pop.offsets[c0:c1 + 1] - a).to(dev)
            tau = torch.from_numpy(pop.tau[c0:c1]).to(dev)
            mom, y, fl = api.fp_closure_exact(v, off, tau, params=prm, prec="fp64")
            lite = api.fp_moments_lite(v, off) if features != "full" else None
            r, t, x = api.fp_surrogate_training_rows(mom, tau, coeffs=y, lite=lite, lite_inputs=features != "full")
            rfull = r if features == "full" else api.fp_surrogate_training_rows(mom, tau, aux=False, targets=False)[0]
            keep = ((fl == 0) & torch.isfinite(t).all(1) & (t.abs() <= 1e6).all(1) & torch.isfinite(r).all(1)
                    & torch.isfinite(rfull).all(1))
            nf = FEATURE_SETS[features][1]
            raws.append(r[keep, :nf])
            targs.append(t[keep, :NOUT])
            auxs.append(x[keep])
            srcs.append((mom if features == "full" else lite)[keep])
            taus.append(tau[keep])
        self.f = torch.cat(raws)
        self.t = torch.cat(targs)
        self.aux = torch.cat(auxs)
        self.src = torch.cat(srcs)  # moment (or LITE) vectors of the kept cells
        self.tau = torch.cat(taus)
        self.features = features
        self.eps2_hat = eps2_hat

    def __len__(self):
        return self.f.shape[0]

    def inputs(self, s: "Surrogate"):
        """The BF16 standardised inputs [n, 32] made by the inference kernel
        with s's scalers."""
        n = len(self)
        x = torch.empty((n, IN), dtype=torch.bfloat16, device=self.f.device)
        step = 1 << 20
        for c0 in range(0, n, step):
            c1 = min(n, c0 + step)
            if self.features == "full":
                s.features(self.src[c0:c1], self.tau[c0:c1], x_out=x[c0:c1])
            else:
                s.lite_features(self.src[c0:c1], self.tau[c0:c1], x_out=x[c0:c1])
        return x


def fit_scalers(s: Surrogate, ts: TrainingSet):
    if ts.f.shape[1] != s.nfeat:
        raise api.FPError("training inputs and network input set differ")
    f, t = ts.f.double(), ts.t.double()
    nf = s.nfeat
    mu = f.mean(0)
    sd = f.std(0).clamp_min(1e-6)
    s.x_mu[:nf] = mu.float()
    s.x_sigma[:nf] = sd.float()
    s.x_min[:nf] = f.min(0).values.float()
    s.x_max[:nf] = f.max(0).values.float()
    s.x_mu[nf:] = 0
    s.x_sigma[nf:] = 1
    s.x_min[nf:] = -1
    s.x_max[nf:] = 1
    s.y_mu[:NOUT] = t.mean(0).float()
    s.y_sigma[:NOUT] = t.std(0).clamp_min(1e-6).float()
    s.y_mu[NOUT:] = 0
    s.y_sigma[NOUT:] = 1
    s._net = None


class Trainer:
    """Adam on the loss of fp_surrogate_loss, every step in the library's
    kernels; returns the per-epoch mean losses."""

    def __init__(self, s: Surrogate, batch=8192, lr=1e-3, w_gamma=2.0, lam_drift=0.1, lam_energy=1.0,
                 fused=True):
        self.s = s
        self.fused = fused  # one fp_surrogate_train_step call, else the four calls it fuses
        self.batch = batch
        self.lr = lr
        self.w = np.array([1.0] * 6 + [w_gamma] * 3, dtype=np.float32)  # Gamma block weighted up (q-weighting)
        self.lam_drift = lam_drift
        self.lam_energy = lam_energy
        n = param_count()
        dev = s.device
        self.grads = torch.zeros(n, dtype=torch.float32, device=dev)
        self.m = torch.zeros(n, dtype=torch.float32, device=dev)
        self.v = torch.zeros(n, dtype=torch.float32, device=dev)
        self.t = 0
        B = batch
        self.dout = torch.empty((B, OUT), dtype=torch.float32, device=dev)
        self.dout_bf = torch.empty((B, OUT), dtype=torch.bfloat16, device=dev)
        self.loss_acc = torch.zeros(1, dtype=torch.float32, device=dev)
        self.ws = torch.empty(int(_lib().fp_mlp_backward_workspace_bytes(B)), dtype=torch.uint8, device=dev)
        self.ws_step = torch.empty(int(_lib().fp_surrogate_train_step_workspace_bytes(B)), dtype=torch.uint8,
                                   device=dev)
        self.wbuf = (ctypes.c_float * 9)(*self.w.tolist())

    def step(self, x, t, aux, scale):
        s = self.s
        L = _lib()
        n = x.shape[0]
        if self.fused:
            ws = self.ws_step
            if n > self.batch:
                ws = torch.empty(int(L.fp_surrogate_train_step_workspace_bytes(n)), dtype=torch.uint8,
                                 device=s.device)
            self.t += 1
            rc = L.fp_surrogate_train_step(ctypes.byref(s.net()), _p(x), _p(t), _p(aux), n, self.wbuf,
                                           self.lam_drift, self.lam_energy, scale, _p(s.params), _p(self.grads),
                                           _p(self.m), _p(self.v), s.params.numel(), self.lr, 0.9, 0.999, 1e-8,
                                           self.t, _p(s.shadow), _p(self.loss_acc), _p(ws), ws.numel(),
                                           api._stream(None))
            api._check(rc, "fp_surrogate_train_step")
            return
        out, h, z = s.forward(x, standardized=True, save=True)
        wbuf = (ctypes.c_float * 9)(*self.w.tolist())
        rc = L.fp_surrogate_loss(_p(out), _p(t), _p(aux), _p(s.y_mu), _p(s.y_sigma), n, wbuf, self.lam_drift,
                                 self.lam_energy, s.eps2_hat, scale, _p(self.dout), _p(self.dout_bf),
                                 _p(self.loss_acc), api._stream(None))
        api._check(rc, "fp_surrogate_loss")
        rc = L.fp_mlp_backward(ctypes.byref(s.net()), _p(x), _p(h), _p(z), _p(self.dout_bf), _p(self.dout), n,
                               _p(self.grads), _p(self.ws), self.ws.numel(), api._stream(None))
        api._check(rc, "fp_mlp_backward")
        self.t += 1
        rc = L.fp_adam_step(_p(s.params), _p(self.grads), _p(self.m), _p(self.v), s.params.numel(), self.lr, 0.9,
                            0.999, 1e-8, self.t, _p(s.shadow), api._stream(None))
        api._check(rc, "fp_adam_step")

    def fit(self, ts: TrainingSet, epochs=10, seed=0, log=None, lr_decay=0.85):
        s = self.s
        x_all = ts.inputs(s)
        n = len(ts)
        gen = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        for ep in range(epochs):
            perm = torch.randperm(n, generator=gen).to(s.device)
            self.loss_acc.zero_()
            t0 = time.time()
            nb = 0
            for b0 in range(0, n - self.batch + 1, self.batch):
                idx = perm[b0:b0 + self.batch]
                self.step(x_all[idx].contiguous(), ts.t[idx].contiguous(), ts.aux[idx].contiguous(), 1.0 / self.batch)
                nb += 1
            torch.cuda.synchronize()
            mean_loss = float(self.loss_acc.item()) / max(1, nb * self.batch)
            hist.append(mean_loss)
            if log:
                log(f"epoch {ep}: loss {mean_loss:.5f} ({time.time() - t0:.1f} s, {nb} steps)")
            self.lr *= lr_decay
        return hist
