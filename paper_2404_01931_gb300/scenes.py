"""Seeded synthetic FLIP scenes (inputs only; none of the method's arithmetic).

A scene is a set of fluid cells on an ``nx x ny x nz`` MAC grid of spacing ``dx``
(domain ``[0, n*dx)`` per axis, y is up) plus the particles seeded in them.

Seeding follows the jittered-grid scheme of the paper (Section 3.1.2, Fig. 3):
every fluid cell is split into ``density**3`` sub-cells ("density 2" = 8 sub-cells
per cell) and each sub-cell receives one particle at a uniformly random position
inside it.  A cell is fluid when its centre lies inside the scene's region (the
sharp level-set region of Section 3.1.2).  Initial velocities are zero unless a
constant velocity is given.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
64-bit output for counter ``c`` under seed ``s`` is the SplitMix64 finaliser
applied to ``s*G + (c+1)*G`` (``G = 0x9E3779B97F4A7C15``, arithmetic mod 2**64),
and a uniform double in [0, 1) is its top 53 bits times 2**-53.  The counter of
sub-cell ``s`` of cell ``c`` on axis ``a`` is ``(c*density**3 + s)*3 + a``, with
``c`` the x-fastest linear cell index.  Positions are computed in float64 and
rounded to float32 once; both the CUDA path and the oracle receive those float32
arrays.

Scenes named after the paper's benchmarks (Table 1): ``dam_break`` (fluid block
against the x=0 wall), ``double_dam_break`` (two blocks against the opposite x
walls), ``water_drop`` (a free sphere falling to the floor) and ``pool_drop`` (a
pool plus a falling sphere).  The paper names the scenes but gives no geometry;
the shapes used here are the synthetic stand-ins this project measures on.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 output number ``counter`` of the stream started at ``seed*G``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * _G + (counter.astype(np.uint64) + np.uint64(1)) * _G
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(counter: np.ndarray, seed: int) -> np.ndarray:
    """Uniform float64 in [0, 1) from the top 53 bits of ``splitmix64``."""
    return (splitmix64(counter, seed) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Scene:
    """Particles (float32 SoA, seeding order) and the grid they live on."""

    n: tuple  # (nx, ny, nz)
    dx: float
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    fluid_mask: np.ndarray  # bool, shape (nz, ny, nx): the seeded cells
    name: str = ""

    @property
    def n_particles(self) -> int:
        return int(self.x.shape[0])

    def arrays(self):
        return self.x, self.y, self.z, self.u, self.v, self.w


def cell_centres(n, dx):
    """Cell-centre coordinates as three (nz, ny, nx) float64 arrays."""
    nx, ny, nz = n
    cz, cy, cx = np.meshgrid((np.arange(nz) + 0.5) * dx, (np.arange(ny) + 0.5) * dx,
                             (np.arange(nx) + 0.5) * dx, indexing="ij")
    return cx, cy, cz


def seed_mask(mask: np.ndarray, dx: float, density: int = 2, seed: int = 0,
              velocity=(0.0, 0.0, 0.0), name: str = "", chunk_cells: int = 1 << 20) -> Scene:
    """Jittered seeding of every True cell of ``mask`` (shape (nz, ny, nx))."""
    mask = np.ascontiguousarray(mask, dtype=bool)
    nz, ny, nx = mask.shape
    cells = np.flatnonzero(mask.ravel()).astype(np.int64)
    d = int(density)
    sub = d ** 3
    s = np.arange(sub, dtype=np.int64)
    sx, sy, sz = s % d, (s // d) % d, s // (d * d)
    npart = cells.size * sub
    out = [np.empty(npart, np.float32) for _ in range(3)]
    for c0 in range(0, cells.size, chunk_cells):
        cc = cells[c0:c0 + chunk_cells]
        ci = cc % nx
        cj = (cc // nx) % ny
        ck = cc // (nx * ny)
        base = (cc[:, None] * sub + s[None, :]) * 3
        for a, (idx, so) in enumerate(((ci, sx), (cj, sy), (ck, sz))):
            r = uniform01(base + a, seed)
            pos = (idx[:, None].astype(np.float64) + (so[None, :] + r) / d) * dx
            out[a][c0 * sub:(c0 + cc.size) * sub] = pos.astype(np.float32).ravel()
    vel = [np.full(npart, np.float32(velocity[a]), np.float32) for a in range(3)]
    return Scene((nx, ny, nz), float(dx), out[0], out[1], out[2], vel[0], vel[1], vel[2],
                 mask, name)


def dam_break(n: int, frac_x: float = 0.25, frac_y: float = 0.5, density: int = 2,
              seed: int = 0) -> Scene:
    """Fluid block ``x < frac_x, y < frac_y`` over the full z extent of an n^3 box."""
    dx = 1.0 / n
    cx, cy, _ = cell_centres((n, n, n), dx)
    mask = (cx < frac_x) & (cy < frac_y)
    return seed_mask(mask, dx, density, seed, name=f"dam_break_{n}")


def pool_drop(n: int, depth: float = 0.3, centre=(0.5, 0.7, 0.5), radius: float = 0.15,
              density: int = 2, seed: int = 0) -> Scene:
    """Pool ``y < depth`` plus a sphere of fluid (the "water drop" benchmark shape)."""
    dx = 1.0 / n
    cx, cy, cz = cell_centres((n, n, n), dx)
    sphere = (cx - centre[0]) ** 2 + (cy - centre[1]) ** 2 + (cz - centre[2]) ** 2 < radius ** 2
    mask = (cy < depth) | sphere
    return seed_mask(mask, dx, density, seed, name=f"pool_drop_{n}")


def double_dam_break(n: int, frac_x: float = 0.2, frac_y: float = 0.5, density: int = 2,
                     seed: int = 0) -> Scene:
    """Two fluid blocks ``x < frac_x`` and ``x > 1 - frac_x`` (``y < frac_y``, full z)."""
    dx = 1.0 / n
    cx, cy, _ = cell_centres((n, n, n), dx)
    mask = ((cx < frac_x) | (cx > 1.0 - frac_x)) & (cy < frac_y)
    return seed_mask(mask, dx, density, seed, name=f"double_dam_break_{n}")


def water_drop(n: int, centre=(0.5, 0.6, 0.5), radius: float = 0.2, density: int = 2,
               seed: int = 0) -> Scene:
    """A sphere of fluid at rest, free to fall onto the floor."""
    dx = 1.0 / n
    cx, cy, cz = cell_centres((n, n, n), dx)
    mask = (cx - centre[0]) ** 2 + (cy - centre[1]) ** 2 + (cz - centre[2]) ** 2 < radius ** 2
    return seed_mask(mask, dx, density, seed, name=f"water_drop_{n}")


def layer(n, height_cells: int, density: int = 2, seed: int = 0) -> Scene:
    """Full-width fluid layer of ``height_cells`` cells resting on the floor."""
    if np.isscalar(n):
        n = (n, n, n)
    nx, ny, nz = n
    mask = np.zeros((nz, ny, nx), bool)
    mask[:, :height_cells, :] = True
    return seed_mask(mask, 1.0 / max(n), density, seed, name=f"layer_{height_cells}")


def box(n, lo, hi, density: int = 2, seed: int = 0, velocity=(0.0, 0.0, 0.0),
        dx: float | None = None) -> Scene:
    """Cells whose centre lies in the axis-aligned box [lo, hi)."""
    if np.isscalar(n):
        n = (n, n, n)
    dx = 1.0 / max(n) if dx is None else dx
    cx, cy, cz = cell_centres(n, dx)
    mask = ((cx >= lo[0]) & (cx < hi[0]) & (cy >= lo[1]) & (cy < hi[1])
            & (cz >= lo[2]) & (cz < hi[2]))
    return seed_mask(mask, dx, density, seed, velocity=velocity, name="box")


def random_mask(n, fill: float, seed: int) -> np.ndarray:
    """Random cell mask (shape (nz, ny, nx)) with at least one air cell."""
    if np.isscalar(n):
        n = (n, n, n)
    nx, ny, nz = n
    c = np.arange(nx * ny * nz, dtype=np.int64)
    m = (uniform01(c, seed + 7919) < fill).reshape(nz, ny, nx)
    m.flat[int(splitmix64(np.array([1]), seed)[0] % np.uint64(m.size))] = False
    return m


def random_velocities(scene: Scene, scale: float, seed: int) -> Scene:
    """Same scene with i.i.d. uniform velocities in [-scale, scale)."""
    np_ = scene.n_particles
    c = np.arange(np_, dtype=np.int64) * 3
    vel = [((uniform01(c + a, seed + 104729) * 2.0 - 1.0) * scale).astype(np.float32)
           for a in range(3)]
    return Scene(scene.n, scene.dx, scene.x, scene.y, scene.z, vel[0], vel[1], vel[2],
                 scene.fluid_mask, scene.name)


def batch_scenes(count: int, edges=(32, 48, 64, 80, 96), frac_range=(0.2, 0.5),
                 density: int = 2, seed: int = 0):
    """Independent dam-break scenes of uneven size (grid edge and fluid fraction by seed).

    Scene ``s`` takes its edge from ``edges`` and a fluid fraction ``f`` uniform in
    ``frac_range``; the block is ``x < sqrt(f), y < sqrt(f)`` over the full z extent.
    """
    out = []
    for s in range(count):
        r = uniform01(np.array([2 * s, 2 * s + 1], dtype=np.int64), seed + 15485863)
        n = int(edges[int(r[0] * len(edges)) % len(edges)])
        f = frac_range[0] + (frac_range[1] - frac_range[0]) * r[1]
        side = float(np.sqrt(f))
        out.append(dam_break(n, side, side, density, seed + s))
    return out


def corner_field_sphere(n, h: float, centre, radius: float, noise: float = 0.0,
                        seed: int = 0) -> np.ndarray:
    """Float32 corner field (shape (nz+1, ny+1, nx+1)) of a sphere's distance function
    |x - centre| - radius sampled at h*(i,j,k), plus uniform noise in [-noise, noise)
    from the counter-based generator (a meshing input, not a simulation)."""
    if np.isscalar(n):
        n = (n, n, n)
    g = [np.arange(n[a] + 1) * h for a in range(3)]
    Z, Y, X = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    phi = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2) - radius
    if noise:
        c = np.arange(phi.size, dtype=np.int64)
        phi = phi + ((uniform01(c, seed + 31337) * 2.0 - 1.0) * noise).reshape(phi.shape)
    return phi.astype(np.float32)


def corner_field_random(n, seed: int, bias: float = 0.0, closed: bool = True) -> np.ndarray:
    """Float32 corner field of i.i.d. uniform values in [-1 + bias, 1 + bias); with
    ``closed`` the corners on the box boundary are set to 1 (outside)."""
    if np.isscalar(n):
        n = (n, n, n)
    shape = (n[2] + 1, n[1] + 1, n[0] + 1)
    c = np.arange(int(np.prod(shape)), dtype=np.int64)
    phi = (uniform01(c, seed + 271828) * 2.0 - 1.0 + bias).reshape(shape)
    if closed:
        phi[0], phi[-1], phi[:, 0], phi[:, -1], phi[:, :, 0], phi[:, :, -1] = (1.0,) * 6
    return phi.astype(np.float32)
