"""Seeded synthetic particle populations for the cubic Fokker-Planck closure.

This module only draws inputs: particle velocities sorted by cell, the CSR
cell offsets and the per-cell collision time tau.  It holds none of the
closure's arithmetic (no moments, no matrix, no solve) and imports nothing
from the rest of the package, so the CUDA path, the CPU oracle, the tests and
the benchmark can all draw identical inputs from it.

Units are dimensionless: free-stream temperature theta_inf = 1, number
density n_inf = 1, molecular mass 1.  For Maxwell molecules the viscosity is
proportional to temperature, so tau = 2 mu / p (Eq. tau, Sec. 3.3) reduces to
tau_ref / n with tau_ref = 1.

The three shapes stand in for the paper's flows (Couette, Sec. 5.1; lid-driven
cavity, Sec. 5.2; hypersonic cylinder, Sec. 6), whose particle data are not
available; see the recipe of each generator.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = 5.0 / 3.0


@dataclass
class Population:
    """Particles sorted by cell (SoA velocities) plus per-cell inputs."""

    name: str
    v64: np.ndarray  # (3, n_particles) float64, C-contiguous SoA
    offsets: np.ndarray  # (n_cells + 1,) int64, offsets[0] = 0, offsets[-1] = n_particles
    tau: np.ndarray  # (n_cells,) float64
    meta: dict = field(default_factory=dict)
    _v32: np.ndarray | None = None

    @property
    def n_cells(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_particles(self) -> int:
        return int(self.v64.shape[1])

    @property
    def counts(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def v32(self) -> np.ndarray:
        """The same velocities rounded to float32 (SoA, contiguous)."""
        if self._v32 is None:
            self._v32 = np.ascontiguousarray(self.v64.astype(np.float32))
        return self._v32

    def subset(self, cells) -> "Population":
        """A population holding only the given cells (in the given order)."""
        cells = np.asarray(cells, dtype=np.int64)
        cnt = self.counts[cells]
        offs = np.zeros(len(cells) + 1, dtype=np.int64)
        np.cumsum(cnt, out=offs[1:])
        idx = np.concatenate([np.arange(self.offsets[c], self.offsets[c + 1]) for c in cells]) \
            if len(cells) else np.zeros(0, dtype=np.int64)
        v = np.ascontiguousarray(self.v64[:, idx])
        return Population(f"{self.name}[subset]", v, offs, self.tau[cells].copy(), dict(self.meta))


def _assemble(name, per_cell_v, tau, meta) -> Population:
    counts = np.array([v.shape[1] for v in per_cell_v], dtype=np.int64)
    offs = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=offs[1:])
    v = np.ascontiguousarray(np.concatenate(per_cell_v, axis=1)) if len(per_cell_v) else np.zeros((3, 0))
    return Population(name, v.astype(np.float64), offs, np.asarray(tau, dtype=np.float64), meta)


def from_counts(name, counts, draw, tau, meta=None) -> Population:
    """Build a population from per-cell counts and a vectorised drawer.

    ``draw(cell_ids)`` returns a (3, len(cell_ids)) array of velocities for a
    flat array of particle -> cell ids (sorted by cell).
    """
    counts = np.asarray(counts, dtype=np.int64)
    offs = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=offs[1:])
    cell_of = np.repeat(np.arange(len(counts), dtype=np.int64), counts)
    v = np.ascontiguousarray(draw(cell_of), dtype=np.float64)
    return Population(name, v, offs, np.asarray(tau, dtype=np.float64), meta or {})


# --------------------------------------------------------------------------
# Couette-like: 20 x 20 cells, exactly 100 particles per cell, Maxwellian.
# --------------------------------------------------------------------------
def couette(seed: int = 1, nx: int = 20, ny: int = 20, ppc: int = 100) -> Population:
    """Maxwellian cells with seeded density n ~ U[0.8, 1.2], temperature
    theta ~ U[0.8, 1.2] and mean u_x linear in the wall-normal index from
    -0.5 to 0.5 (Couette shear, Sec. 5.1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_cells = nx * ny
    dens = rng.uniform(0.8, 1.2, n_cells)
    theta = rng.uniform(0.8, 1.2, n_cells)
    iy = np.arange(n_cells) // nx
    ux = -0.5 + iy / max(ny - 1, 1)
    mean = np.stack([ux, np.zeros(n_cells), np.zeros(n_cells)])
    counts = np.full(n_cells, ppc, dtype=np.int64)

    def draw(cell_of):
        z = rng.standard_normal((3, cell_of.size))
        return mean[:, cell_of] + np.sqrt(theta[cell_of]) * z

    return from_counts("couette_20x20_ppc100", counts, draw, 1.0 / dens,
                       {"theta": theta, "density": dens, "mean": mean, "shape": (ny, nx)})


# --------------------------------------------------------------------------
# Cavity-like: 128 x 128 cells, Poisson(50) clipped to [8, 400].
# --------------------------------------------------------------------------
def _grad13_batch(rng, counts, pihat, qhat, bimodal, delta, e_dir, cmax=3.0):
    """Normalised velocities c_hat for many cells at once, in cell order.

    Non-bimodal cells: rejection sampling from the Grad-13 density
    f_M [1 + pihat_ij c_i c_j / 2 + qhat_i c_i (c^2/5 - 1)] with 1 + phi
    truncated at 0 and clipped at its bound over |c_hat| <= cmax (so the far
    tails are those of f_M scaled by that bound).
    Bimodal cells: a 50/50 mixture of unit Maxwellians at +/- delta e_dir.
    Candidates are over-drawn per cell and the first ``counts[c]`` accepted
    ones are kept; cells left short are topped up in further rounds.
    """
    counts = np.asarray(counts, dtype=np.int64)
    n_cells = counts.size
    need = counts.copy()
    parts_cell, parts_c, parts_rank = [], [], []
    filled = np.zeros(n_cells, dtype=np.int64)
    bound_all = 1.0 + 0.5 * np.abs(pihat).sum((1, 2)) * cmax ** 2 + \
        np.linalg.norm(qhat, axis=1) * cmax * (cmax ** 2 / 5.0 + 1.0)
    todo = np.nonzero(need > 0)[0]
    p00, p11, p22 = pihat[:, 0, 0], pihat[:, 1, 1], pihat[:, 2, 2]
    p01, p02, p12 = pihat[:, 0, 1], pihat[:, 0, 2], pihat[:, 1, 2]
    while todo.size:
        reps = np.ceil(1.3 * need[todo] * np.where(bimodal[todo], 1.0, bound_all[todo])).astype(np.int64) + 8
        cell = np.repeat(todo, reps)
        m = cell.size
        c = rng.standard_normal((3, m))
        c0, c1, c2_ = c[0], c[1], c[2]
        csq = c0 * c0 + c1 * c1 + c2_ * c2_
        quad = p00[cell] * c0 * c0 + p11[cell] * c1 * c1 + p22[cell] * c2_ * c2_ + \
            2.0 * (p01[cell] * c0 * c1 + p02[cell] * c0 * c2_ + p12[cell] * c1 * c2_)
        qc = qhat[cell, 0] * c0 + qhat[cell, 1] * c1 + qhat[cell, 2] * c2_
        phi = 0.5 * quad + qc * (csq / 5.0 - 1.0)
        bound = bound_all[cell]
        acc = rng.uniform(size=m) * bound < np.clip(1.0 + phi, 0.0, bound)
        bi = bimodal[cell]
        sign = np.where(rng.uniform(size=m) < 0.5, 1.0, -1.0)
        shift = (delta[cell] * sign)[None, :] * e_dir[cell].T
        c = np.where(bi[None, :], rng.standard_normal((3, m)) + shift, c)
        acc |= bi
        cell_a = cell[acc]
        c_a = c[:, acc]
        # rank of each accepted candidate within its cell (cell is sorted)
        first = np.searchsorted(cell_a, cell_a, side="left")
        rank = np.arange(cell_a.size) - first + filled[cell_a]
        keep = rank < counts[cell_a]
        parts_cell.append(cell_a[keep])
        parts_c.append(c_a[:, keep])
        parts_rank.append(rank[keep])
        np.add.at(filled, cell_a[keep], 1)
        need = counts - filled
        todo = np.nonzero(need > 0)[0]
    cell = np.concatenate(parts_cell)
    rank = np.concatenate(parts_rank)
    c = np.concatenate(parts_c, axis=1)
    order = np.lexsort((rank, cell))
    return c[:, order]


def _random_grad13_params(rng, n):
    a = rng.uniform(-0.3, 0.3, (n, 3, 3))
    pihat = 0.5 * (a + a.transpose(0, 2, 1))
    pihat -= np.trace(pihat, axis1=1, axis2=2)[:, None, None] / 3.0 * np.eye(3)[None]
    pihat = np.clip(pihat, -0.3, 0.3)
    qd = rng.standard_normal((n, 3))
    qd /= np.linalg.norm(qd, axis=1, keepdims=True)
    qhat = qd * rng.uniform(0.0, 0.2, (n, 1))
    ed = rng.standard_normal((n, 3))
    ed /= np.linalg.norm(ed, axis=1, keepdims=True)
    delta = rng.uniform(0.5, 1.5, n)
    return pihat, qhat, ed, delta


def cavity(seed: int = 2, nx: int = 128, ny: int = 128, mean_ppc: float = 50.0,
           ppc_range=(8, 400), bimodal_fraction: float = 0.10) -> Population:
    """Lid-driven-cavity-shaped population (Sec. 5.2).

    * ppc = clip(Poisson(50), 8, 400);
    * theta(x, y) = 1 + 2 g(x, y) with g a smooth bump in [0, 1] (ratio 3);
    * u_x lid-like near the top row plus a weak recirculation;
    * velocities from a Grad-13 perturbed Maxwellian with seeded stress
      |pi_ij| <= 0.3 p and normalised heat flux |q| / (p sqrt(theta)) <= 0.2,
      and in 10 % of the cells a 50/50 mixture of two Maxwellians at
      +/- Delta e, Delta ~ U[0.5, 1.5] sqrt(theta).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_cells = nx * ny
    ix = np.arange(n_cells) % nx
    iy = np.arange(n_cells) // nx
    xs = (ix + 0.5) / nx
    ys = (iy + 0.5) / ny
    g = np.exp(-((xs - 0.7) ** 2 + (ys - 0.75) ** 2) / (2 * 0.18 ** 2))
    theta = 1.0 + 2.0 * g
    dens = 1.0 + 0.2 * np.sin(np.pi * xs) * np.cos(np.pi * ys)
    ux = ys ** 6 - 0.15 * np.sin(np.pi * ys) * np.sin(np.pi * xs)
    uy = 0.15 * np.sin(2 * np.pi * xs) * np.sin(np.pi * ys)
    counts = np.clip(rng.poisson(mean_ppc, n_cells), ppc_range[0], ppc_range[1]).astype(np.int64)
    bimodal = rng.uniform(size=n_cells) < bimodal_fraction
    pihat, qhat, e_dir, delta = _random_grad13_params(rng, n_cells)
    ch = _grad13_batch(rng, counts, pihat, qhat, bimodal, delta, e_dir)
    cell_of = np.repeat(np.arange(n_cells), counts)
    v = np.sqrt(theta[cell_of])[None, :] * ch
    v[0] += ux[cell_of]
    v[1] += uy[cell_of]
    offs = np.zeros(n_cells + 1, dtype=np.int64)
    np.cumsum(counts, out=offs[1:])
    return Population("cavity_128x128_poisson50", np.ascontiguousarray(v), offs, 1.0 / dens,
                      {"theta": theta, "density": dens, "bimodal": bimodal, "shape": (ny, nx)})


# --------------------------------------------------------------------------
# Hypersonic-cylinder-like: 512 x 256 cells, log-normal ppc, ~12M particles.
# --------------------------------------------------------------------------
def cylinder(seed: int = 3, nx: int = 512, ny: int = 256, target_particles: int = 12_000_000,
             sigma: float = 0.55, kappa: float = 0.6, ppc_range=(2, 2000)) -> Population:
    """Mach-10 cylinder-shaped population (Sec. 6).

    Free stream u_x = 10 sqrt(gamma) (Mach 10, gamma = 5/3), theta = 1, n = 1.
    A cylinder of radius 28 cells sits at 3/4 of the x-extent.  Ahead of it a
    bow-shaped post-shock layer carries n up to 5x, theta up to 40x and a
    decelerated flow; its outer three cells (the shock itself) hold a
    mixture of the cold free-stream beam and the hot post-shock Maxwellian.
    The cells touching the wall hold a half-range Maxwellian at
    theta_wall = 2.5 (500 K / 200 K) leaving the wall; the wake is rarefied.
    ppc = clip(round(LogNormal(ln m, sigma) * n^kappa), 2, 2000) with the
    median m tuned so the total is close to ``target_particles``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_cells = nx * ny
    ix = np.arange(n_cells) % nx
    iy = np.arange(n_cells) // nx
    cx, cy, R = 0.75 * nx, 0.5 * ny, 28.0
    dx = ix + 0.5 - cx
    dy = iy + 0.5 - cy
    r = np.hypot(dx, dy)
    phi = np.arctan2(np.abs(dy), -dx)  # 0 = straight upstream
    u_inf = 10.0 * np.sqrt(GAMMA)
    r_shock = R + 10.0 + 30.0 * phi ** 2
    strength = np.clip(np.cos(np.minimum(phi, np.pi / 2)) ** 2, 0.05, 1.0)
    kind = np.zeros(n_cells, dtype=np.int8)  # 0 free stream, 1 post-shock, 2 shock, 3 wall, 4 wake, 5 body
    post = (r >= R) & (r < r_shock) & (phi < 1.9)
    shock = (r >= r_shock) & (r < r_shock + 3.0) & (phi < 1.9)
    wall = (r >= R) & (r < R + 1.5)
    wake = (dx > 0) & (np.abs(dy) < R + 0.4 * dx) & (r >= R) & ~post & ~shock
    body = r < R
    kind[post] = 1
    kind[shock] = 2
    kind[wake] = 4
    kind[wall] = 3
    kind[body] = 5
    # post-shock profile: 1 at the wall, 0 at the shock
    h = np.clip((r_shock - r) / np.maximum(r_shock - R, 1.0), 0.0, 1.0)
    dens = np.ones(n_cells)
    theta = np.ones(n_cells)
    ux = np.full(n_cells, u_inf)
    uy = np.zeros(n_cells)
    s = strength
    dens[post] = 1.0 + 4.0 * s[post] * (0.6 + 0.4 * h[post])
    theta[post] = 1.0 + 39.0 * s[post] * (0.7 + 0.3 * h[post])
    ux[post] = u_inf * (1.0 - 0.85 * s[post] * (0.3 + 0.7 * h[post]))
    uy[post] = 0.25 * u_inf * np.sign(dy[post]) * np.sin(phi[post]) * (1.0 - h[post])
    dens[shock] = 1.0 + 2.0 * s[shock]
    theta[shock] = 1.0 + 20.0 * s[shock]
    ux[shock] = u_inf * (1.0 - 0.4 * s[shock])
    dens[wall] = 3.0
    theta[wall] = 2.5
    ux[wall] = 0.0
    dens[wake] = 0.25
    theta[wake] = 3.0
    ux[wake] = 0.2 * u_inf
    dens[body] = 0.05
    theta[body] = 2.5
    ux[body] = 0.0
    z = rng.standard_normal(n_cells)
    base = np.exp(sigma * z) * dens ** kappa
    med = target_particles / base.sum()
    counts = np.clip(np.rint(med * base), ppc_range[0], ppc_range[1]).astype(np.int64)
    # shock cells: fraction of particles from the upstream beam
    beam_frac = np.where(kind == 2, 0.5, 0.0)
    # post-shock state used by the shock mixture
    th_post = 1.0 + 39.0 * s * 0.7
    ux_post = u_inf * (1.0 - 0.85 * s * 0.3)
    nxw = np.where(r > 0, dx / np.maximum(r, 1e-12), 1.0)
    nyw = np.where(r > 0, dy / np.maximum(r, 1e-12), 0.0)

    def draw(cell_of):
        m = cell_of.size
        zz = rng.standard_normal((3, m))
        th = theta[cell_of].copy()
        u0 = ux[cell_of].copy()
        u1 = uy[cell_of].copy()
        k = kind[cell_of]
        sh = k == 2
        pick_beam = sh & (rng.uniform(size=m) < beam_frac[cell_of])
        hot = sh & ~pick_beam
        th[pick_beam] = 1.0
        u0[pick_beam] = u_inf
        th[hot] = th_post[cell_of[hot]]
        u0[hot] = ux_post[cell_of[hot]]
        v = np.sqrt(th)[None, :] * zz
        v[0] += u0
        v[1] += u1
        wl = k == 3
        if wl.any():
            nxc, nyc = nxw[cell_of[wl]], nyw[cell_of[wl]]
            vn = v[0, wl] * nxc + v[1, wl] * nyc
            flip = vn < 0.0  # reflect into the outward half range
            v0 = v[0, wl] - 2.0 * flip * vn * nxc
            v1 = v[1, wl] - 2.0 * flip * vn * nyc
            v[0, wl] = v0
            v[1, wl] = v1
        return v

    return from_counts("cylinder_512x256_mach10", counts, draw, 1.0 / dens,
                       {"theta": theta, "density": dens, "kind": kind, "shape": (ny, nx)})


def maxwellian_cells(counts, theta=1.0, mean=(0.0, 0.0, 0.0), tau=1.0, seed: int = 0,
                     name="maxwellian") -> Population:
    """Cells of plain Maxwellian velocities (for tests of closed forms)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = np.asarray(counts, dtype=np.int64)
    n_cells = counts.size
    th = np.broadcast_to(np.asarray(theta, dtype=np.float64), (n_cells,))
    mu = np.broadcast_to(np.asarray(mean, dtype=np.float64).reshape(-1, 1) if np.ndim(mean) == 1
                         else np.asarray(mean, dtype=np.float64), (3, n_cells))
    tu = np.broadcast_to(np.asarray(tau, dtype=np.float64), (n_cells,)).copy()

    def draw(cell_of):
        z = rng.standard_normal((3, cell_of.size))
        return mu[:, cell_of] + np.sqrt(th[cell_of]) * z

    return from_counts(name, counts, draw, tu, {"theta": np.array(th)})


def integer_cells(counts, lo=-3, hi=3, tau=1.0, seed: int = 0) -> Population:
    """Cells of small-integer velocities (exact in binary; for brute force)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = np.asarray(counts, dtype=np.int64)
    tu = np.broadcast_to(np.asarray(tau, dtype=np.float64), (counts.size,)).copy()

    def draw(cell_of):
        return rng.integers(lo, hi + 1, size=(3, cell_of.size)).astype(np.float64)

    return from_counts("integer", counts, draw, tu)


def concat(pops, name="concat") -> Population:
    """The cells of several populations one after another."""
    counts = np.concatenate([p.counts for p in pops])
    offs = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=offs[1:])
    v = np.ascontiguousarray(np.concatenate([p.v64 for p in pops], axis=1))
    return Population(name, v, offs, np.concatenate([p.tau for p in pops]))


def _cylinder_cells(n_cells: int, seed: int) -> Population:
    """n_cells cells drawn at random from cylinder-like populations of fresh
    seeds (the Mach-10 flow's free stream, shock layer, wall and wake cells
    in their proportions)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts, left, k = [], n_cells, 0
    while left > 0:
        cyl = cylinder(seed=1000003 * (seed + 1) + k)
        take = min(left, cyl.n_cells // 2)
        parts.append(cyl.subset(np.sort(rng.choice(cyl.n_cells, take, replace=False))))
        left -= take
        k += 1
    return concat(parts) if len(parts) > 1 else parts[0]


def training_cells(n_cells: int, seed: int, cylinder_fraction: float = 0.0) -> Population:
    """Cells drawn from the Couette-like and cavity-like distributions (half
    each of the remainder): Maxwellian cells with 100 particles, and Grad-13 /
    bimodal cells with Poisson(50) particles clipped to [8, 400] and theta in
    [1, 3]; with cylinder_fraction > 0, that fraction of the cells comes from
    cylinder-like populations of fresh seeds."""
    n_cyl = int(round(cylinder_fraction * n_cells))
    if n_cyl > 0:
        rest = training_cells(n_cells - n_cyl, seed) if n_cells > n_cyl else None
        cyl = _cylinder_cells(n_cyl, seed)
        out = concat([rest, cyl]) if rest is not None else cyl
        out.name = f"training_{n_cells}_cyl{cylinder_fraction:g}"
        return out
    n_a = n_cells // 2
    n_b = n_cells - n_a
    rng = np.random.Generator(np.random.PCG64(seed))
    dens_a = rng.uniform(0.8, 1.2, n_a)
    th_a = rng.uniform(0.8, 1.2, n_a)
    ux_a = rng.uniform(-0.5, 0.5, n_a)
    cnt_b = np.clip(rng.poisson(50.0, n_b), 8, 400).astype(np.int64)
    th_b = 1.0 + 2.0 * rng.uniform(0.0, 1.0, n_b)
    dens_b = 1.0 + 0.2 * rng.uniform(-1.0, 1.0, n_b)
    bimodal = rng.uniform(size=n_b) < 0.10
    pihat, qhat, e_dir, delta = _random_grad13_params(rng, n_b)
    counts = np.concatenate([np.full(n_a, 100, dtype=np.int64), cnt_b])
    tau = 1.0 / np.concatenate([dens_a, dens_b])
    offs = np.zeros(n_cells + 1, dtype=np.int64)
    np.cumsum(counts, out=offs[1:])
    v = np.empty((3, int(offs[-1])))
    cell_a = np.repeat(np.arange(n_a), 100)
    v[:, : 100 * n_a] = np.sqrt(th_a[cell_a])[None, :] * rng.standard_normal((3, 100 * n_a))
    v[0, : 100 * n_a] += ux_a[cell_a]
    ch = _grad13_batch(rng, cnt_b, pihat, qhat, bimodal, delta, e_dir)
    cell_b = np.repeat(np.arange(n_b), cnt_b)
    v[:, 100 * n_a:] = np.sqrt(th_b[cell_b])[None, :] * ch
    return Population(f"training_{n_cells}", np.ascontiguousarray(v), offs, tau,
                      {"theta": np.concatenate([th_a, th_b])})


CONFIGS = {
    "couette": couette,
    "cavity": cavity,
    "cylinder": cylinder,
}


def make(name: str, seed: int | None = None, **kw) -> Population:
    fn = CONFIGS[name]
    return fn(**kw) if seed is None else fn(seed=seed, **kw)
