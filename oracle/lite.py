"""CPU FP64 oracle of the LITE path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py`` may import this module.  Plain numpy, one cell at a time.

The LITE moment pass (Sec. 4, Phase 3 item 2) computes only the moments up
to the heat flux that the network's 16 inputs need (Sec. 4, Phase 1-2
item 1: rho, T, U (3), Pi (6), q (3), DM2, nu).  Readings of the paper's
names, per cell with c = v - U the peculiar velocity:
  rho  = N, the particle count (proportional to density at fixed cell
         volume and particle weight);
  T    = theta = <c.c> / 3;
  Pi   = u - theta I, u_ij = <c_i c_j> (deviatoric stress per unit mass);
  q_i  = <c_i |c|^2> / 2 (heat flux per unit mass);
  DM2  = det u (determinant of the second-moment tensor);
  nu   = 1 / tau (collision frequency).
"""

from __future__ import annotations

import numpy as np

NLITE = 14
NFEAT_LITE = 16
# slots of the LITE moment vector
L_N, L_U, L_THETA, L_U2, L_B = 0, 1, 4, 5, 11
SYM2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def lite_moments(v, offsets):
    """LITE moment vectors [n_cells, 14]: N, U (3), theta, u_ij (6, order
    11,12,13,22,23,33), b_i = <c_i |c|^2> (3); empty cells are all zero."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    offsets = np.asarray(offsets, dtype=np.int64)
    n_cells = offsets.size - 1
    out = np.zeros((n_cells, NLITE))
    for k in range(n_cells):
        a, b = offsets[k], offsets[k + 1]
        if b <= a:
            continue
        vk = v[:, a:b]
        U = vk.mean(axis=1)
        c = vk - U[:, None]
        c2 = np.sum(c * c, axis=0)
        out[k, L_N] = b - a
        out[k, L_U:L_U + 3] = U
        out[k, L_THETA] = c2.mean() / 3.0
        for s, (i, j) in enumerate(SYM2):
            out[k, L_U2 + s] = np.mean(c[i] * c[j])
        for i in range(3):
            out[k, L_B + i] = np.mean(c[i] * c2)
    return out


def second_moment_tensor(lite_row):
    """u_ij of one LITE vector as a symmetric 3x3 matrix."""
    u = np.empty((3, 3))
    for s, (i, j) in enumerate(SYM2):
        u[i, j] = u[j, i] = lite_row[L_U2 + s]
    return u


def lite_features(lite, tau):
    """The 16 network inputs [n, 16] (rho, T, U, Pi, q, DM2, nu), in the
    order of Sec. 4's input list; DM2 by cofactor expansion along row 1."""
    lite = np.atleast_2d(np.asarray(lite, dtype=np.float64))
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    f = np.empty((lite.shape[0], NFEAT_LITE))
    for k in range(lite.shape[0]):
        m = lite[k]
        th = m[L_THETA]
        u = second_moment_tensor(m)
        f[k, 0] = m[L_N]
        f[k, 1] = th
        f[k, 2:5] = m[L_U:L_U + 3]
        pi = u - th * np.eye(3)
        f[k, 5:11] = [pi[i, j] for (i, j) in SYM2]
        f[k, 11:14] = 0.5 * m[L_B:L_B + 3]
        f[k, 14] = (u[0, 0] * (u[1, 1] * u[2, 2] - u[1, 2] * u[2, 1])
                    - u[0, 1] * (u[1, 0] * u[2, 2] - u[1, 2] * u[2, 0])
                    + u[0, 2] * (u[1, 0] * u[2, 1] - u[1, 1] * u[2, 0]))
        f[k, 15] = 1.0 / tau[k]
    return f
