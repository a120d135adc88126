"""CPU FP64 oracle of the cubic Fokker-Planck closure -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py`` (with their worker processes) may import this
package.  The product path (the CUDA library and
its Python binding) never does, and this package imports nothing from it.

The arithmetic lives in ``fp_oracle.c`` / ``closure_core.h`` (plain C99,
compiled here with gcc on first use); this file only marshals numpy arrays.
``mlp.py`` holds the numpy reference of the surrogate network.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

NMOM = 30
FLAG_FEW, FLAG_SINGULAR, FLAG_NONFINITE, FLAG_ALPHA = 1, 2, 4, 64
FALLBACK_FLAGS = FLAG_FEW | FLAG_SINGULAR | FLAG_NONFINITE

# slots of the moment vector
M_N, M_U, M_THETA, M_U2, M_U3, M_W, M_Z = 0, 1, 4, 5, 11, 21, 27
SYM2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
SYM3 = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2),
        (1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2)]

DEFAULT_EPS2_HAT = 1e-3
DEFAULT_MIN_PARTICLES = 4
DEFAULT_PIVOT_RTOL = 1e-13

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C99, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liboracle.so")
    srcs = [os.path.join(_HERE, "fp_oracle.c"), os.path.join(_HERE, "closure_core.h")]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", "-o", tmp, srcs[0], "-lm"])
    os.replace(tmp, out)
    return out


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            lp = ctypes.POINTER(ctypes.c_int64)
            up = ctypes.POINTER(ctypes.c_uint32)
            i64, d, i32, u64 = ctypes.c_int64, ctypes.c_double, ctypes.c_int32, ctypes.c_uint64
            L.oracle_moments.argtypes = [dp, i64, lp, i64, dp]
            L.oracle_assemble.argtypes = [dp, d, d, dp, dp]
            L.oracle_solve.argtypes = [dp, dp, d, dp]
            L.oracle_closure.argtypes = [dp, dp, i64, d, i32, d, dp, ip, dp, dp]
            L.oracle_closure_jacobian.argtypes = [dp, d, d, i32, d, dp]
            L.oracle_closure_backward.argtypes = [dp, i64, lp, i64, dp, d, i32, d, dp, dp, dp, dp, dp]
            L.oracle_philox4x32_10.argtypes = [up, up, up]
            L.oracle_philox4x32_10.restype = None
            L.oracle_normals.argtypes = [i64, i64, u64, u64, dp]
            L.oracle_velocity_update.argtypes = [dp, i64, lp, i64, dp, dp, dp, d, d, dp, u64, u64, dp, ip]
            _LIB = L
    return _LIB


def _p(a, ct=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def moments(v, offsets):
    """Per-cell central moments [n_cells, 30] of SoA velocities v [3, n_p]."""
    v = _f64(v)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n_cells = offsets.size - 1
    out = np.zeros((n_cells, NMOM))
    lib().oracle_moments(_p(v), v.shape[1], _p(offsets, ctypes.c_int64), n_cells, _p(out))
    return out


def speed_moment6(v, offsets):
    """<|c|^6> per cell, c = v - U (the cell mean): the sixth central moment
    of the peculiar speed, which the cell average <N.N> of Eq. update_alpha
    contains once N (Eq. update_N, cubic in c) is expanded.  Plain definition:
    mean over the cell's particles of (c.c)^3, in FP64 (empty cells: 0)."""
    v = _f64(v)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    out = np.zeros(offsets.size - 1)
    for k in range(offsets.size - 1):
        a, b = offsets[k], offsets[k + 1]
        if b > a:
            c = v[:, a:b] - v[:, a:b].mean(axis=1, keepdims=True)
            out[k] = np.mean(np.sum(c * c, axis=0) ** 3)
    return out


NDIAG = 12


def sort_by_cell(cell_of, n_cells):
    """The cell sort of Alg. 1 / Alg. 2 (particles ordered by cell index),
    stable: (perm, offsets) with perm[i] the input index of the particle at
    sorted position i and offsets[c] the first sorted position of cell c
    (c = 0..n_cells).  Indices outside [0, n_cells) count as n_cells: those
    particles follow the last cell and belong to none."""
    cell_of = np.asarray(cell_of, dtype=np.int64)
    key = np.where((cell_of >= 0) & (cell_of < n_cells), cell_of, n_cells)
    perm = np.argsort(key, kind="stable")
    offsets = np.searchsorted(key[perm], np.arange(n_cells + 1), side="left")
    return perm.astype(np.int64), offsets.astype(np.int64)


def diagnostics(m, m6, rho=None, theta_inf=1.0, rho_inf=1.0, dg_inf=0.0):
    """Per-cell high-order diagnostics and covariance entropy proxies
    [n_cells, 12], written out from their definitions (the cavity study's
    normalised R_ij = <c_i c_j c_k c_k>, Delta_4 = <(c_k c_k)^2> - 15 theta^2,
    DM6 = <(c_k c_k)^3>; the cylinder audit's Eqs. cyl_theta_def,
    cyl_entropy_eq, cyl_DG, cyl_entropy_kinG and D_q = |q_hat|^2 / 5 with
    q_hat = <c |c|^2> / (2 theta^1.5)).  Invalid cells (N < 2, theta <= 0,
    det Theta <= 0, rho <= 0, non-finite input): NaN."""
    m = np.atleast_2d(_f64(m))
    m6 = np.atleast_1d(_f64(m6))
    n = m.shape[0]
    out = np.full((n, NDIAG), np.nan)
    for k in range(n):
        th = m[k, M_THETA]
        Theta = np.array([[m[k, M_U2 + SYM2.index(tuple(sorted((i, j))))] for j in range(3)] for i in range(3)])
        d = m[k, M_N] if rho is None else rho[k]
        det = np.linalg.det(Theta)
        if not (m[k, M_N] >= 2 and th > 0 and det > 0 and d > 0 and np.all(np.isfinite(m[k])) and np.isfinite(m6[k])):
            continue
        W = m[k, M_W:M_W + 6]
        out[k, 0:6] = W / th ** 2
        out[k, 6] = (W[0] + W[3] + W[5]) / th ** 2 - 15.0
        out[k, 7] = m6[k] / th ** 3
        dg = -0.5 * np.log(np.linalg.det(Theta / th))
        out[k, 8] = dg
        u3 = m[k, M_U3:M_U3 + 10]
        b = np.array([sum(u3[SYM3.index(tuple(sorted((i, j, j))))] for j in range(3)) for i in range(3)])
        qhat = b / (2.0 * th ** 1.5)
        out[k, 9] = qhat @ qhat / 5.0
        ds_eq = 1.5 * np.log(th / theta_inf) - np.log(d / rho_inf)
        out[k, 10] = ds_eq
        out[k, 11] = ds_eq - (dg - dg_inf)
    return out


def coeffs_relax(y_new, y_prev, w):
    """Temporal under-relaxation of the coefficient field (the cylinder
    deployment's w = 0.2): w y_new + (1 - w) y_prev."""
    return w * _f64(y_new) + (1.0 - w) * _f64(y_prev)


def assemble(m, tau, eps2_hat=DEFAULT_EPS2_HAT):
    """The 9x9 matrix and right-hand side of one cell."""
    m = _f64(m)
    A = np.zeros(81)
    r = np.zeros(9)
    lib().oracle_assemble(_p(m), float(tau), float(eps2_hat), _p(A), _p(r))
    return A.reshape(9, 9), r


def solve(A, r, pivot_rtol=DEFAULT_PIVOT_RTOL):
    """Solve one 9x9 system by the oracle's elimination -> (y, flag)."""
    y = np.zeros(9)
    f = lib().oracle_solve(_p(_f64(A).reshape(81)), _p(_f64(r)), float(pivot_rtol), _p(y))
    return y, f


def closure(mom, tau, eps2_hat=DEFAULT_EPS2_HAT, min_particles=DEFAULT_MIN_PARTICLES,
            pivot_rtol=DEFAULT_PIVOT_RTOL, want_cond=False):
    """Coefficients [n_cells, 9], flags [n_cells] (and cond, min pivot ratio)."""
    mom = _f64(mom).reshape(-1, NMOM)
    tau = _f64(tau)
    n = mom.shape[0]
    Y = np.zeros((n, 9))
    fl = np.zeros(n, dtype=np.int32)
    cond = np.zeros(n) if want_cond else None
    mp = np.zeros(n) if want_cond else None
    lib().oracle_closure(_p(mom), _p(tau), n, float(eps2_hat), int(min_particles), float(pivot_rtol),
                         _p(Y), _p(fl, ctypes.c_int32), _p(cond), _p(mp))
    if want_cond:
        return Y, fl, cond, mp
    return Y, fl


def closure_jacobian(m, tau, eps2_hat=DEFAULT_EPS2_HAT, min_particles=DEFAULT_MIN_PARTICLES,
                     pivot_rtol=DEFAULT_PIVOT_RTOL):
    J = np.zeros(9 * NMOM)
    lib().oracle_closure_jacobian(_p(_f64(m)), float(tau), float(eps2_hat), int(min_particles),
                                  float(pivot_rtol), _p(J))
    return J.reshape(9, NMOM)


def closure_backward(v, offsets, tau, mom, grad_coeffs, grad_moments_in=None,
                     eps2_hat=DEFAULT_EPS2_HAT, min_particles=DEFAULT_MIN_PARTICLES,
                     pivot_rtol=DEFAULT_PIVOT_RTOL, want_grad_v=True):
    v = _f64(v)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n_cells = offsets.size - 1
    gm = np.zeros((n_cells, NMOM))
    gv = np.zeros_like(v) if want_grad_v else None
    gin = None if grad_moments_in is None else _f64(grad_moments_in)
    lib().oracle_closure_backward(_p(v), v.shape[1], _p(offsets, ctypes.c_int64), n_cells, _p(_f64(tau)),
                                  float(eps2_hat), int(min_particles), float(pivot_rtol), _p(_f64(mom)),
                                  _p(_f64(grad_coeffs)), _p(gin), _p(gm), _p(gv))
    return gm, gv


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def normals(n, seed, step, first_index=0):
    xi = np.zeros((3, n))
    lib().oracle_normals(int(n), int(first_index), int(seed), int(step), _p(xi))
    return xi


def velocity_update(v, offsets, mom, coeffs, tau, flags, dt, eps2_hat=DEFAULT_EPS2_HAT,
                    xi=None, seed=0, step=0):
    """Returns (v_new [3, n_p], alpha [n_cells], flags_out [n_cells])."""
    v = _f64(v).copy()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n_cells = offsets.size - 1
    alpha = np.zeros(n_cells)
    fl = np.ascontiguousarray(flags, dtype=np.int32).copy()
    lib().oracle_velocity_update(_p(v), v.shape[1], _p(offsets, ctypes.c_int64), n_cells, _p(_f64(mom)),
                                 _p(_f64(coeffs)), _p(_f64(tau)), float(dt), float(eps2_hat),
                                 _p(None if xi is None else _f64(xi)), int(seed), int(step),
                                 _p(alpha), _p(fl, ctypes.c_int32))
    return v, alpha, fl
