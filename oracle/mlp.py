"""Reference of the learned closure -- TEST INFRASTRUCTURE (see oracle/__init__).

Plain numpy, written from the definitions:
  * features: the 25 moments of w = c / sqrt(theta) (u_ij / theta,
    u_ijk / theta^1.5, w_ij / theta^2, z_i / theta^2.5), standardised, zero
    padded to 32;
  * network: Linear(32, 128) -> SiLU -> 3 x [Linear(128, 128) -> SiLU] ->
    Linear(128, 16), of which the first 9 outputs are used;
  * targets: the dimensionless coefficients (tau C_ij, tau sqrt(theta) G_i),
    standardised -- the cubic-FP system of Eq. system9x9 is invariant under
    the scaling c -> c / sqrt(theta), C -> tau C, G -> tau sqrt(theta) G,
    eps^2 -> tau theta eps^2, so these depend on the features (and eps2_hat)
    only;
  * the training loss per cell: weighted standardised coefficient MSE, the
    mean square of the drift difference the coefficients induce over the
    cell's velocity distribution (a quadratic form in the coefficient error
    with moment weights), and the square of the energy residual of the
    predicted drift;
  * Adam (Kingma & Ba, 2015).
`bf16=True` reproduces the GPU's rounding points: BF16 inputs, weights and
hidden activations, FP32 accumulation (here FP64 sums rounded to FP32).
"""

from __future__ import annotations

import numpy as np

IN, HID, OUT, DEPTH = 32, 128, 16, 4
NFEAT, NOUT = 25, 9
M_THETA, M_U2, M_U3, M_W, M_Z = 4, 5, 11, 21, 27
SYM2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
SYM3 = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2),
        (1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2)]


def bf16_round(x):
    """Round-to-nearest-even to bfloat16, returned as float32 values."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(x), x, out)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def raw_features(mom):
    """The 25 normalised moments of each cell: [n_cells, 25] (FP64)."""
    mom = np.asarray(mom, dtype=np.float64)
    th = mom[:, M_THETA:M_THETA + 1]
    f = np.empty((mom.shape[0], NFEAT))
    f[:, 0:6] = mom[:, M_U2:M_U2 + 6] / th
    f[:, 6:16] = mom[:, M_U3:M_U3 + 10] / th ** 1.5
    f[:, 16:22] = mom[:, M_W:M_W + 6] / th ** 2
    f[:, 22:25] = mom[:, M_Z:M_Z + 3] / th ** 2.5
    return f


def targets(coeffs, mom, tau):
    """Dimensionless coefficients (tau C, tau sqrt(theta) G): [n, 9]."""
    th = np.asarray(mom)[:, M_THETA]
    t = np.empty((coeffs.shape[0], NOUT))
    t[:, :6] = coeffs[:, :6] * tau[:, None]
    t[:, 6:] = coeffs[:, 6:] * (tau * np.sqrt(th))[:, None]
    return t


def coeffs_from_targets(t, mom, tau):
    th = np.asarray(mom)[:, M_THETA]
    y = np.empty_like(t)
    y[:, :6] = t[:, :6] / tau[:, None]
    y[:, 6:] = t[:, 6:] / (tau * np.sqrt(th))[:, None]
    return y


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    dims = [(HID, IN), (HID, HID), (HID, HID), (HID, HID), (OUT, HID)]
    W, b = [], []
    for (o, i) in dims:
        W.append(rng.standard_normal((o, i)) * np.sqrt(1.0 / i))
        b.append(np.zeros(o))
    W[0][:, NFEAT:] = 0.0
    W[-1][NOUT:, :] = 0.0
    return {"W": W, "b": b}


def forward(params, x, bf16=False, keep=False):
    """x [n, 32] standardised features -> out [n, 16] (and the cache)."""
    W, b = params["W"], params["b"]
    h = bf16_round(x).astype(np.float64) if bf16 else np.asarray(x, dtype=np.float64)
    hs, zs = [h], []
    for l in range(5):
        Wl = bf16_round(W[l]).astype(np.float64) if bf16 else W[l]
        z = h @ Wl.T + b[l]
        if bf16:
            z = z.astype(np.float32).astype(np.float64)
        zs.append(z)
        if l < 4:
            h = silu(z)
            if bf16:
                h = bf16_round(h).astype(np.float64)
            hs.append(h)
        else:
            h = z
    if keep:
        return h, (hs, zs)
    return h


def backward(params, cache, dout):
    """FP64 reverse mode of forward(): returns (dW list, db list, dx)."""
    W = params["W"]
    hs, zs = cache
    dW, db = [None] * 5, [None] * 5
    g = np.asarray(dout, dtype=np.float64)
    for l in range(4, -1, -1):
        dW[l] = g.T @ hs[l]
        db[l] = g.sum(axis=0)
        dh = g @ W[l]
        if l > 0:
            g = dh * silu_grad(zs[l - 1])
        else:
            g = dh
    return dW, db, g


def drift_matrix(mom):
    """Per-cell quadratic form Q (9x9) with <|dA|^2> tau^2 / theta =
    d^T Q d for the dimensionless coefficient error d = (dC_hat, dG_hat):
      dA_i = dC_ij c_j + dG_i (|c|^2 - 3 theta)
      <|dA|^2> = dC_ij dC_ik u_jk + 2 dC_ij dG_i b_j + |dG|^2 (s4 - 9 theta^2)
    written in the normalised moments (u_hat, b_hat, s4_hat)."""
    n = mom.shape[0]
    f = raw_features(mom)
    uh = np.zeros((n, 3, 3))
    for a, (i, j) in enumerate(SYM2):
        uh[:, i, j] = uh[:, j, i] = f[:, a]
    u3 = {idx: f[:, 6 + a] for a, idx in enumerate(SYM3)}
    bh = np.stack([sum(u3[tuple(sorted((i, k, k)))] for k in range(3)) for i in range(3)], axis=1)
    s4h = f[:, 16] + f[:, 19] + f[:, 21]
    # expand d -> (dC full 3x3, dG)
    E = np.zeros((9, 3, 3))  # E[a] = d(dC)/d(d_a)
    for a, (i, j) in enumerate(SYM2):
        E[a, i, j] = E[a, j, i] = 1.0
    Q = np.zeros((n, 9, 9))
    for a in range(6):
        for c in range(6):
            # sum_ijk E[a]_ij E[c]_ik u_jk
            Q[:, a, c] = np.einsum("ij,ik,njk->n", E[a], E[c], uh)
    for a in range(6):
        for i in range(3):
            # 2 dC_ij dG_i b_j, split symmetrically
            v = np.einsum("j,nj->n", E[a][i], bh)
            Q[:, a, 6 + i] += v
            Q[:, 6 + i, a] += v
    for i in range(3):
        Q[:, 6 + i, 6 + i] = s4h - 9.0
    return Q


def energy_residual(t, mom, eps2_hat):
    """e = 1 + (sum_ij C_hat_ij u_hat_ij + sum_i G_hat_i b_hat_i
    - eps2_hat s4_hat) / 3; zero for the exact closure (trace of the stress
    rows of Eq. system9x9)."""
    f = raw_features(mom)
    mult = np.array([1, 2, 2, 1, 2, 1], dtype=np.float64)
    cu = (t[:, :6] * f[:, :6] * mult).sum(1)
    u3 = {idx: f[:, 6 + a] for a, idx in enumerate(SYM3)}
    bh = np.stack([sum(u3[tuple(sorted((i, k, k)))] for k in range(3)) for i in range(3)], axis=1)
    gb = (t[:, 6:9] * bh).sum(1)
    s4h = f[:, 16] + f[:, 19] + f[:, 21]
    return 1.0 + (cu + gb - eps2_hat * s4h) / 3.0


def loss(out, t_true, mom, y_mu, y_sigma, eps2_hat, w_coef, lam_drift, lam_energy):
    """Mean over cells of
      sum_a w_a (out_a - (t_a - mu_a)/sigma_a)^2
      + lam_drift d^T Q d + lam_energy e^2,  d = t_pred - t_true."""
    o = out[:, :NOUT]
    z = (t_true - y_mu) / y_sigma
    t_pred = y_mu + y_sigma * o
    d = t_pred - t_true
    Q = drift_matrix(mom)
    e = energy_residual(t_pred, mom, eps2_hat)
    per = (w_coef * (o - z) ** 2).sum(1) + lam_drift * np.einsum("na,nab,nb->n", d, Q, d) + lam_energy * e ** 2
    return per.mean()


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step t >= 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------
# heuristic coefficient-sensitivity probe (the cylinder study's dropout probe)
# ---------------------------------------------------------------------------
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) on many counters at
    once: ctr [..., 4] uint32, key (k0, k1) -> [..., 4] uint32.  Each round
    multiplies words 0 and 2 by the Philox constants (64-bit products), mixes
    the high halves with words 1, 3 and the round key, and bumps the key by
    the Weyl constants."""
    x = np.asarray(ctr, dtype=np.uint64) & 0xFFFFFFFF
    x0, x1, x2, x3 = x[..., 0], x[..., 1], x[..., 2], x[..., 3]
    k0, k1 = np.uint64(key[0] & 0xFFFFFFFF), np.uint64(key[1] & 0xFFFFFFFF)
    mask = np.uint64(0xFFFFFFFF)
    for _ in range(10):
        p0 = np.uint64(PHILOX_M0) * x0
        p1 = np.uint64(PHILOX_M1) * x2
        x0, x1, x2, x3 = ((p1 >> np.uint64(32)) ^ x1 ^ k0) & mask, p1 & mask, \
                         ((p0 >> np.uint64(32)) ^ x3 ^ k1) & mask, p0 & mask
        k0 = (k0 + np.uint64(PHILOX_W0)) & mask
        k1 = (k1 + np.uint64(PHILOX_W1)) & mask
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def dropout_scales(cells, k, seed, rate):
    """Dropout factors of pass k for the given cell indices: [4 layers][n][128],
    0 for a dropped activation, 1/(1 - rate) (FP32) for a kept one.  Unit j of
    hidden layer l of cell r uses word j % 4 of Philox4x32-10 (key = seed) on
    counter (r lo, r hi, k, 32 l + j / 4); u = (floor(w / 2^8) + 1) 2^-24 and
    the unit is dropped when u <= rate (rate rounded to FP32)."""
    cells = np.asarray(cells, dtype=np.int64)
    n = cells.size
    ctr = np.zeros((4, n, 32, 4), dtype=np.uint64)
    ctr[..., 0] = (cells & 0xFFFFFFFF)[None, :, None]
    ctr[..., 1] = (cells >> 32)[None, :, None]
    ctr[..., 2] = k
    ctr[..., 3] = 32 * np.arange(4)[:, None, None] + np.arange(32)[None, None, :]
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, seed >> 32)).reshape(4, n, 128)
    u = ((w >> 8).astype(np.float64) + 1.0) * 2.0 ** -24
    keep_scale = float(np.float32(1.0 / (1.0 - rate)))
    return np.where(u <= float(np.float32(rate)), 0.0, keep_scale)


def forward_dropout(params, x, scales, bf16=True):
    """forward() with each hidden activation multiplied by its dropout factor
    (scales [4][n][128]) after the SiLU and before the BF16 rounding."""
    W, b = params["W"], params["b"]
    h = bf16_round(x).astype(np.float64) if bf16 else np.asarray(x, dtype=np.float64)
    for l in range(5):
        Wl = bf16_round(W[l]).astype(np.float64) if bf16 else W[l]
        z = h @ Wl.T + b[l]
        if bf16:
            z = z.astype(np.float32).astype(np.float64)
        if l < 4:
            h = silu(z) * scales[l]
            if bf16:
                h = bf16_round(h).astype(np.float64)
        else:
            h = z
    return h


def sensitivity(params, x, y_mu, y_sigma, tau, theta, cells, n_passes, rate, seed):
    """The probe: n_passes dropout forward passes of the standardised inputs
    x [n][32]; per cell sigma_i (1/N) of each physical coefficient (outputs
    un-standardised to (tau C, tau sqrt(theta) Gamma), divided by tau and
    tau sqrt(theta)), sigma_Stress = |sigma_C|, sigma_Heat = |sigma_Gamma|:
    [n][11]; and the mean coefficients [n][9]."""
    ys = []
    for k in range(n_passes):
        out = forward_dropout(params, x, dropout_scales(cells, k, seed, rate))[:, :NOUT]
        ys.append(out * np.asarray(y_sigma[:NOUT], np.float64) + np.asarray(y_mu[:NOUT], np.float64))
    ys = np.stack(ys)                                    # [passes][n][9]
    f = np.empty((x.shape[0], NOUT))
    f[:, :6] = 1.0 / np.asarray(tau)[:, None]
    f[:, 6:] = 1.0 / (np.asarray(tau) * np.sqrt(theta))[:, None]
    sig = ys.std(axis=0) * f                              # numpy std: 1/N
    out = np.empty((x.shape[0], 11))
    out[:, :9] = sig
    out[:, 9] = np.sqrt((sig[:, :6] ** 2).sum(1))
    out[:, 10] = np.sqrt((sig[:, 6:] ** 2).sum(1))
    return out, ys.mean(axis=0) * f
