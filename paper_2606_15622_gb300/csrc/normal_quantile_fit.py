"""Coefficients of the update kernel's standard normal quantile (velocity.cu,
normal_quantile), fitted here from the mathematics, and an exhaustive check of
the kernel's FP32 evaluation.

The kernel maps a 32-bit Philox word w to u = (k + 1/2) 2^-23, k = w >> 9,
and returns z = Phi^-1(u) = sqrt(2) erfinv(x) with x = 2u - 1 =
(2k + 1 - 2^23) 2^-23 (exact in FP32), in the form of Giles' erfinv
approximation (M. Giles, "Approximating the erfinv function", GPU Computing
Gems Jade Edition, 2011): with lg = log2(1 - x^2),
    z = x P(lg - c_P)            for lg >= -8   (99.8 % of the words)
    z = x Q(sqrt(-lg) - c_Q)     otherwise,
P of degree 9 and Q of degree 8.  Both are fitted on all 2^23 inputs to the
quotient z / x, with z from scipy's ndtri in FP64, minimising the maximum
relative error by Lawson's iteratively reweighted least squares.

The check evaluates the kernel's arithmetic in FP32 for every k (1 - x^2 by
one fused multiply-add, Horner's rule in fused multiply-adds, the square root
correctly rounded) with lg the correctly rounded log2, and again with lg
moved by the error bound of the hardware approximation (lg2.approx.f32:
2^-22.6 absolute for 1 - x^2 in [1/2, 1], else 2 ulps), and prints the
largest absolute and relative errors of z and the coefficients as C++.

    python normal_quantile_fit.py        (a minute or two, ~3 GB of memory)
"""

import numpy as np
from scipy.special import ndtri

SPLIT = -8.0          # lg at the switch between P and Q
C_P, DEG_P = -4.0, 9  # P's expansion point (centre of [-8, 0]) and degree
C_Q, DEG_Q = 3.75, 8  # Q's expansion point (within [sqrt(8), sqrt(22.x)]) and degree


def _f32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def _fma32(a, b, c):
    # a * b is exact in FP64 for FP32 a, b; the sum is then rounded to FP32
    return _f32(a * b + c)


def _horner32(coef, v):
    r = np.full_like(v, _f32(coef[-1]))
    for a in coef[-2::-1]:
        r = _fma32(r, v, _f32(a))
    return r


def lawson_fit(var, target, deg, centre, iters=30):
    """Polynomial in (var - centre) of degree `deg` with the smallest maximum
    relative error found by Lawson's reweighting of least squares."""
    V = np.vander(var - centre, deg + 1, increasing=True)
    scale = np.abs(V).max(axis=0)
    Vs = V / scale
    rel = 1.0 / np.abs(target)
    w = np.full(var.size, 1.0 / var.size)
    best = (np.inf, None)
    for _ in range(iters):
        sw = np.sqrt(w) * rel
        a, *_ = np.linalg.lstsq(Vs * sw[:, None], target * sw, rcond=None)
        e = np.abs(Vs @ a - target) * rel
        if e.max() < best[0]:
            best = (e.max(), a / scale)
        w = w * e
        w /= w.sum()
    return best


def main():
    k = np.arange(1 << 23, dtype=np.int64)
    m = 2 * k + 1 - (1 << 23)
    x = m * 2.0 ** -23                      # exact in FP32
    z = ndtri((k + 0.5) * 2.0 ** -23)
    t = _fma32(-x, x, 1.0)                  # 1 - x^2, one rounding
    lg = np.log2(t)
    cen = lg >= SPLIT
    g = z / x
    err_p, P = lawson_fit(lg[cen], g[cen], DEG_P, C_P)
    err_q, Q = lawson_fit(np.sqrt(-lg[~cen]), g[~cen], DEG_Q, C_Q)
    print(f"fit: max relative error of P {err_p:.2e}, of Q {err_q:.2e}; {np.mean(~cen):.2%} of the words take Q")
    P32, Q32 = _f32(P), _f32(Q)

    def kernel(lg_used):
        lg32 = _f32(lg_used)
        zp = _f32(x * _horner32(P32, _f32(lg32 - C_P)))
        s = _f32(np.sqrt(_f32(-np.minimum(lg32, 0.0))))
        zq = _f32(x * _horner32(Q32, _f32(s - C_Q)))
        return np.where(t >= 2.0 ** SPLIT, zp, zq)

    ulp = np.spacing(np.abs(lg).astype(np.float32)).astype(np.float64)
    bound = np.where(t >= 0.5, 2.0 ** -22.6, 2.0 * ulp)
    for name, lg_used in (("correctly rounded log2", lg), ("log2 low by its bound", lg - bound),
                          ("log2 high by its bound", lg + bound)):
        ae = np.abs(kernel(lg_used) - z)
        print(f"FP32 evaluation, {name}: max |dz| {ae.max():.2e} (P branch {ae[cen].max():.2e}, "
              f"Q branch {ae[~cen].max():.2e}), max |dz|/|z| {np.max(ae / np.abs(z)):.2e}")

    def cxx(name, c):
        body = ", ".join(f"{float(v):.9e}f" for v in c)
        return f"constexpr float {name}[{len(c)}] = {{{body}}};"
    print(cxx("kQuantileP", P32))
    print(cxx("kQuantileQ", Q32))


if __name__ == "__main__":
    main()
