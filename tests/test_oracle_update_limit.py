"""Pins of the oracle's Eq. update_N that do not restate it (Sec. 3.8-3.10).

With the noise switched off (xi = 0) and the coefficients of the exact
closure, the update of Eq. update_vel is a consistent one-step scheme for the
drift of the cubic model, so as dt -> 0:

  (i)  (M^{n+1} - M^n) / dt -> A(M'), the cubic drift of Eq. cubic_drift
       evaluated straight from the coefficients Y: C M' + G (|M'|^2 - 3 theta)
       - eps^2 (M' |M'|^2 - b).  No N appears in the test: N = A + M'/tau is
       what the update must have built for this limit to hold (the +I/tau of
       Eq. update_N undoes the exp(-dt/tau) relaxation of the OU part).
  (ii) the cell's central moments change at the Maxwell-molecule production
       rates the closure is built to match: the second moments at -(2/tau) u_ij
       (drift only; the diffusion's +(2 theta/tau) delta_ij comes from the noise,
       and the two together give the stress relaxation -(2/tau)(u - theta I)),
       and <c_i |c|^2> at -(4/(3 tau)) b_i (the diffusion adds nothing to it).

Both limits are approached at O(dt), and alpha = 1 + O(dt^2): the exact
closure conserves energy, so the unscaled step already keeps the expected
energy to first order.  (A slip that breaks <M'.N> = 0 is first-order
compensated by alpha in the particle rates, but shows in alpha - 1 = O(dt).)

(iii) For unflagged cells given the linear model's coefficients (C = -I/tau,
       G = 0, eps = 0) the cubic update must reduce to the exact
       Ornstein-Uhlenbeck transition of the linear Fokker-Planck model
       (Eq. linear_drift with the diffusion of Sec. 3.8), at any dt.

A mutation test compiles copies of the oracle with the plausible slips in
Eq. update_N -- the +delta_ij/tau dropped, the sign of the G term flipped, b
replaced by q/rho = b/2 -- and checks that these pins reject every one of them.
"""

import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2606_15622_gb300 import populations as P

EPS2_HAT = 0.05  # large enough that the eps^2 terms of Eq. update_N matter


def _cells():
    # non-Maxwellian cells (Grad-13 perturbed and bimodal): G and the third
    # moments are far from zero, so every term of the drift is exercised
    cav = P.cavity(seed=5, nx=16, ny=16, mean_ppc=120, ppc_range=(80, 200))
    return cav.subset(np.arange(0, cav.n_cells, 9))


def _sym(y):
    return np.array([[y[O.SYM2.index(tuple(sorted((i, j))))] for j in range(3)] for i in range(3)])


def _bvec(m):
    u3 = m[O.M_U3:O.M_U3 + 10]
    return np.array([sum(u3[O.SYM3.index(tuple(sorted((i, j, j))))] for j in range(3)) for i in range(3)])


def _drift(c, m, y, tau):
    """Eq. cubic_drift at the peculiar velocities c [3, n] from Y alone."""
    th = m[O.M_THETA]
    e2 = EPS2_HAT / (tau * th)
    C, G, b = _sym(y[:6]), y[6:9], _bvec(m)
    r2 = (c * c).sum(0)
    return C @ c + G[:, None] * (r2 - 3 * th) - e2 * (c * r2 - b[:, None])


def _update(pop, m, y, fl, dt, update=None):
    xi = np.zeros_like(pop.v64)
    if update is None:
        vn, alpha, _ = O.velocity_update(pop.v64, pop.offsets, m, y, pop.tau, fl, dt, eps2_hat=EPS2_HAT, xi=xi)
    else:
        vn, alpha = update(pop.v64, pop.offsets, m, y, pop.tau, fl, dt, xi)
    return vn, alpha


def _limit_errors(pop, update=None):
    """Per dt: the largest relative deviation of (i) the particle rates from
    A(M') and (ii) the moment rates from the production rates, over cells."""
    m = O.moments(pop.v64, pop.offsets)
    y, fl = O.closure(m, pop.tau, eps2_hat=EPS2_HAT)
    live = np.flatnonzero(fl == 0)
    assert live.size >= 20
    out = {}
    for dt in (1e-4, 1e-5):
        vn, alpha = _update(pop, m, y, fl, dt, update)
        m1 = O.moments(vn, pop.offsets)
        e_part, e_u2, e_b = 0.0, 0.0, 0.0
        for k in live:
            s = slice(pop.offsets[k], pop.offsets[k + 1])
            c = pop.v64[:, s] - m[k, O.M_U:O.M_U + 3, None]
            A = _drift(c, m[k], y[k], pop.tau[k])
            rate = (vn[:, s] - pop.v64[:, s]) / dt
            e_part = max(e_part, np.abs(rate - A).max() / np.abs(A).max())
            tau, th = pop.tau[k], m[k, O.M_THETA]
            du2 = (m1[k, O.M_U2:O.M_U2 + 6] - m[k, O.M_U2:O.M_U2 + 6]) / dt
            want_u2 = -(2.0 / tau) * m[k, O.M_U2:O.M_U2 + 6]
            e_u2 = max(e_u2, np.abs(du2 - want_u2).max() / (th / tau))
            db = (_bvec(m1[k]) - _bvec(m[k])) / dt
            want_b = -(4.0 / (3.0 * tau)) * _bvec(m[k])
            e_b = max(e_b, np.abs(db - want_b).max() / (th ** 1.5 / tau))
        out[dt] = (e_part, e_u2, e_b, np.abs(alpha[live] - 1).max())
    return out


def test_update_converges_to_the_cubic_drift_and_its_production_rates():
    errs = _limit_errors(_cells())
    for dt, (e_part, e_u2, e_b, da) in errs.items():
        # first-order convergence: the deviation is a modest multiple of dt
        assert e_part < 50 * dt, (dt, e_part)
        assert e_u2 < 50 * dt, (dt, e_u2)
        assert e_b < 50 * dt, (dt, e_b)
        assert da < 1e3 * dt * dt, (dt, da)  # alpha - 1 = O(dt^2): <M'.N> = 0
    # and it is O(dt), not a floor: ten times smaller step, about ten times closer
    (p4, u4, b4, _), (p5, u5, b5, _) = errs[1e-4], errs[1e-5]
    assert p5 < 0.2 * p4 and u5 < 0.2 * u4 and b5 < 0.2 * b4


def _ou_error(update=None):
    """Largest deviation of the cubic update, fed the linear model's
    coefficients on unflagged cells, from the exact OU transition."""
    pop = _cells()
    m = O.moments(pop.v64, pop.offsets)
    y = np.zeros((pop.n_cells, 9))
    y[:, [0, 3, 5]] = -1.0 / pop.tau[:, None]
    fl = np.zeros(pop.n_cells, dtype=np.int32)
    xi = np.random.default_rng(8).standard_normal(pop.v64.shape)
    dt = 0.4
    if update is None:
        vn, alpha, _ = O.velocity_update(pop.v64, pop.offsets, m, y, pop.tau, fl, dt, eps2_hat=0.0, xi=xi)
    else:
        vn, alpha = update(pop.v64, pop.offsets, m, y, pop.tau, fl, dt, xi, eps2_hat=0.0)
    err = np.abs(alpha - 1).max()
    for k in range(pop.n_cells):
        s = slice(pop.offsets[k], pop.offsets[k + 1])
        a = np.exp(-dt / pop.tau[k])
        U = m[k, O.M_U:O.M_U + 3, None]
        ou = (pop.v64[:, s] - U) * a + np.sqrt(m[k, O.M_THETA] * (1 - a * a)) * xi[:, s] + U
        err = max(err, np.abs(vn[:, s] - ou).max() / np.sqrt(m[k, O.M_THETA]))
    return err


def test_linear_coefficients_give_the_exact_ou_step():
    assert _ou_error() < 1e-12


def test_diffusion_completes_the_stress_relaxation():
    """Adding the noise's expected contribution (2 theta/tau) dt delta_ij in
    closed form to the drift-only second-moment rate gives the
    Maxwell-molecule stress relaxation -(2/tau)(u_ij - theta delta_ij); the
    same noise leaves the energy unchanged (the trace of the rate is 0)."""
    pop = _cells()
    m = O.moments(pop.v64, pop.offsets)
    y, fl = O.closure(m, pop.tau, eps2_hat=EPS2_HAT)
    dt = 1e-5
    vn, _ = _update(pop, m, y, fl, dt)
    m1 = O.moments(vn, pop.offsets)
    diag = np.array([1, 0, 0, 1, 0, 1], dtype=np.float64)
    for k in np.flatnonzero(fl == 0):
        tau, th = pop.tau[k], m[k, O.M_THETA]
        a = np.exp(-dt / tau)
        # expected second-moment increase from xi: theta (1 - a^2) per component
        noise = th * (1 - a * a) * diag
        rate = (m1[k, O.M_U2:O.M_U2 + 6] + noise - m[k, O.M_U2:O.M_U2 + 6]) / dt
        want = -(2.0 / tau) * (m[k, O.M_U2:O.M_U2 + 6] - th * diag)
        assert np.abs(rate - want).max() < 50 * dt * th / tau
        assert abs(rate[0] + rate[3] + rate[5]) < 50 * dt * th / tau


# ---- mutation test: the pins reject plausible slips in Eq. update_N ----------

# each slip is a textual substitution in the oracle's velocity update
SLIPS = {
    # Eq. update_N without the +delta_ij/tau
    "dropped_identity_over_tau": (r"Cm\[i\]\[j\] = Y\[SYM2\[i\]\[j\]\] \+ \(i == j \? 1\.0 / tc : 0\.0\);",
                                  "Cm[i][j] = Y[SYM2[i][j]];"),
    # the G term with the opposite sign
    "flipped_gamma_sign": (r"\+ G\[i\] \* \(m2 - 3\.0 \* th\)", "- G[i] * (m2 - 3.0 * th)"),
    # q_i / rho = b_i / 2 in place of 2 q_i / rho = b_i
    "half_b": (r"b\[i\] = m\[M_U3 \+ SYM3\[i\]\[0\]\[0\]\] \+ m\[M_U3 \+ SYM3\[i\]\[1\]\[1\]\] \+ m\[M_U3 \+ SYM3\[i\]\[2\]\[2\]\];",
               "b[i] = 0.5 * (m[M_U3 + SYM3[i][0][0]] + m[M_U3 + SYM3[i][1][1]] + m[M_U3 + SYM3[i][2][2]]);"),
}


def _mutant(tmp_path, name, pattern, repl):
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
    src = open(os.path.join(here, "fp_oracle.c")).read()
    start = src.index("int oracle_velocity_update(")
    head, body = src[:start], src[start:]
    body2, n = re.subn(pattern, repl, body, count=1)
    assert n == 1, f"slip {name} does not apply"
    d = tmp_path / name
    d.mkdir()
    (d / "fp_oracle.c").write_text(head + body2)
    shutil.copy(os.path.join(here, "closure_core.h"), d / "closure_core.h")
    so = d / "libmut.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                           "-o", str(so), str(d / "fp_oracle.c"), "-lm"])
    L = ctypes.CDLL(str(so))
    dp, ip, lp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    L.oracle_velocity_update.argtypes = [dp, ctypes.c_int64, lp, ctypes.c_int64, dp, dp, dp, ctypes.c_double,
                                         ctypes.c_double, dp, ctypes.c_uint64, ctypes.c_uint64, dp, ip]

    def update(v, offsets, m, y, tau, fl, dt, xi, eps2_hat=EPS2_HAT):
        v = np.ascontiguousarray(v, dtype=np.float64).copy()
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        alpha = np.zeros(offsets.size - 1)
        f = np.ascontiguousarray(fl, dtype=np.int32).copy()
        L.oracle_velocity_update(O._p(v), v.shape[1], O._p(offsets, ctypes.c_int64), offsets.size - 1,
                                 O._p(O._f64(m)), O._p(O._f64(y)), O._p(O._f64(tau)), float(dt), float(eps2_hat),
                                 O._p(O._f64(xi)), 0, 0, O._p(alpha), O._p(f, ctypes.c_int32))
        return v, alpha

    return update


@pytest.mark.slow
@pytest.mark.parametrize("slip", sorted(SLIPS))
def test_pins_reject_slips_in_update_N(tmp_path, slip):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    update = _mutant(tmp_path, slip, *SLIPS[slip])
    errs = _limit_errors(_cells(), update)
    dt = 1e-5
    e_part, e_u2, e_b, da = errs[dt]
    ou = _ou_error(update)
    # the unmodified oracle passes all of these bounds (tests above); each slip breaks one
    caught = [e_part >= 50 * dt, e_u2 >= 50 * dt, e_b >= 50 * dt, da >= 1e3 * dt * dt, ou >= 1e-12]
    assert any(caught), (slip, errs, ou)
