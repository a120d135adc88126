"""The update kernel's normal quantile (velocity.cu, normal_quantile) on the
CPU: its coefficients are read from the CUDA source and its FP32 arithmetic
is evaluated in numpy (FP32 rounding after every operation, fused
multiply-adds rounded once, the logarithm correctly rounded), on the Philox
words of the oracle's generator, and compared with the oracle's FP64 inverse
of Phi for the same words.  An edited coefficient, a wrong branch point or a
wrong expansion point fails here without a GPU; the exhaustive error analysis
over all 2^23 words is csrc/normal_quantile_fit.py's."""

import os
import re

import numpy as np

import oracle as O
from oracle import mlp as OM

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_15622_gb300", "csrc",
                   "velocity.cu")


def _horner_coefficients(name):
    """Coefficients of the Horner array `name` (leading first in the
    source), constant term first."""
    src = open(SRC).read()
    body = re.search(r"constexpr float " + name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
    coef = re.findall(r"([-+0-9.e]+)f", body)
    return [np.float32(c) for c in reversed(coef)]


def _f32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def _horner32(coef, v):
    r = np.full_like(v, float(coef[-1]))
    for c in coef[-2::-1]:
        r = _f32(r * v + float(c))  # exact product of two FP32 values, one rounding
    return r


def _kernel_quantile(w):
    P, Q = _horner_coefficients("kQuantileP"), _horner_coefficients("kQuantileQ")
    assert len(P) == 10 and len(Q) == 9
    m = ((w >> 9).astype(np.int64) << 1) + 1 - (1 << 23)
    x = m * 2.0 ** -23
    t = _f32(1.0 - x * x)
    lg = _f32(np.log2(t))
    zp = _f32(x * _horner32(P, _f32(lg + 4.0)))
    zq = _f32(x * _horner32(Q, _f32(_f32(np.sqrt(-np.minimum(lg, 0.0))) - 3.75)))
    return np.where(t >= 2.0 ** -8, zp, zq)


def test_kernel_quantile_matches_the_oracle_inverse():
    n, seed, step = 200_000, 4242, 9  # n particles: 3n words, 3n / 4 Philox blocks
    nb = 3 * n // 4
    ctr = np.zeros((nb, 4), dtype=np.uint64)
    b = np.arange(nb, dtype=np.uint64)
    ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3] = b & 0xFFFFFFFF, b >> 32, step, 0
    words = OM.philox4x32_10(ctr, (seed & 0xFFFFFFFF, seed >> 32)).reshape(-1)  # the stream, word j of block j // 4
    xi = O.normals(n, seed, step)  # [3, n], the oracle's FP64 quantiles of words 3p + k
    for k in range(3):
        z = _kernel_quantile(words[3 * np.arange(n) + k].astype(np.uint64))
        err = np.abs(z - xi[k])
        assert err.max() <= 1.0e-6, (k, err.max())
        assert (err / np.abs(xi[k])).max() <= 3.0e-7


def test_kernel_quantile_extremes_and_symmetry():
    # the smallest and largest words of each branch, and words around the switch
    k = np.array([0, 1, 2, 1000, 8191, 8192, 8193, (1 << 22) - 1, 1 << 22, (1 << 23) - 8193, (1 << 23) - 1],
                 dtype=np.int64)
    w = (k << 9).astype(np.uint64)
    z = _kernel_quantile(w)
    from scipy.special import ndtri
    exact = ndtri((k + 0.5) * 2.0 ** -23)
    assert np.abs(z - exact).max() <= 1.0e-6
    z_mirror = _kernel_quantile((((1 << 23) - 1 - k) << 9).astype(np.uint64))
    np.testing.assert_array_equal(z_mirror, -z)
