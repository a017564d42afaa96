"""Seeded synthetic particle sets shaped like the paper's workloads.

This module only draws coordinates and parameters; it holds none of the
search or density arithmetic, so the oracle and the CUDA path can both be fed
from it.  The paper's own inputs (the Poiseuille set-up of its ref. [40], the
circle set of Table 1) are not available; these stand in for them:

  lattice sets   -- particles on a regular lattice of spacing dx (the paper's
                    particle spacing Delta s, with h = 1.2 dx as in the text under
                    Eq. 3), each coordinate jittered by U(-j dx, +j dx);
  random sets    -- uniform random particles in the unit square / cube, the set-up
                    of Table 2;
  circle pairs   -- a centre particle and particles on a circle of radius
                    kh (1 +- dR), the set-up behind Table 1 / Fig. 9.

Every generator takes an explicit seed and uses numpy's PCG64.  Sizes:

  C1  2D, 100 x 100 lattice in the unit square, dx = 0.01, jitter 0.1 dx,
      h = 1.2 dx, kh = 2h (10,000 particles)                         seed 1
  C2  3D, 100^3 lattice in the unit cube, dx = 0.01, jitter 0.1 dx,
      h = 1.3 dx, kh = 2.6 dx (1,000,000 particles)                  seed 2
  C3  3D, 200^3 lattice (dx = 1/200) filling the lower half of a 1 x 1 x 2
      box, 5 % of the particles moved to a uniform spray in z in (1, 2],
      jitter 0.2 dx, h = 1.5 dx, kh = 3 dx (8,000,000 particles)     seed 3
  C4  256 independent 3D systems, N log-uniform in [2e3, 2e5], per-system
      dx in [0.005, 0.02], h/dx in [1.2, 1.5], kh = 2h, jitter 0.1 dx seed 4
  C5  Poisson request stream (mean 200 req/s), 70 % 3D / 30 % 2D, N
      log-uniform in [1e3, 2e6], dx = 1/ceil(N^(1/d)), h/dx in [1.2, 1.5] seed 5
"""
from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class ParticleSet:
    """Coordinates (N x dim, float64, row-major) and the search parameters."""
    xyz: np.ndarray
    h: float
    kh: float
    dx: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.xyz.shape[0]

    @property
    def dim(self):
        return self.xyz.shape[1]


def lattice(shape, dx, jitter=0.0, seed=0, origin=0.0, count=None):
    """Lattice points (i + 0.5) dx (+ origin), x fastest, with each coordinate
    jittered by U(-jitter dx, +jitter dx).  ``shape`` is (nx, ny) or
    (nx, ny, nz).  ``count`` truncates to the first ``count`` points."""
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    axes = [(np.arange(s, dtype=np.float64) + 0.5) * dx for s in shape]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    xyz = np.stack([g.reshape(-1) for g in grids], axis=1)
    if count is not None:
        xyz = xyz[:count]
    xyz = xyz + origin
    if jitter:
        rng = np.random.default_rng(seed)
        xyz = xyz + rng.uniform(-jitter * dx, jitter * dx, size=xyz.shape)
    return np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, dim)


def c1_2d_10k(seed=1, side=100):
    dx = 1.0 / side
    h = 1.2 * dx
    xyz = lattice((side, side), dx, 0.1, seed)
    return ParticleSet(xyz, h, 2.0 * h, dx, "2d_10k_lattice")


def c2_3d_1m(seed=2, side=100):
    """The 3D jittered-lattice workload; ``side`` = 100 gives 1,000,000 particles
    (smaller sides give the same shape at a size the oracle finishes quickly)."""
    dx = 0.01
    h = 1.3 * dx
    xyz = lattice((side, side, side), dx, 0.1, seed)
    return ParticleSet(xyz, h, 2.0 * h, dx, "3d_%d_lattice" % side ** 3)


def c3_3d_dambreak(seed=3, side=200, spray=0.05):
    """Block filling z in [0, 1] of a 1 x 1 x 2 box with a sparse spray above.
    ``side`` = 200 gives 8,000,000 particles."""
    dx = 1.0 / side
    h = 1.5 * dx
    rng = np.random.default_rng(seed)
    xyz = lattice((side, side, side), dx, 0.0)
    xyz = xyz + rng.uniform(-0.2 * dx, 0.2 * dx, size=xyz.shape)
    n = xyz.shape[0]
    nspray = int(round(spray * n))
    idx = rng.choice(n, size=nspray, replace=False)
    spray_xyz = rng.uniform(0.0, 1.0, size=(nspray, 3))
    spray_xyz[:, 2] = 2.0 - rng.uniform(0.0, 1.0, size=nspray)  # (1, 2]
    xyz[idx] = spray_xyz
    return ParticleSet(np.ascontiguousarray(xyz), h, 2.0 * h, dx, "3d_%d_dambreak" % n)


def _system(rng, n, dim, dx, hr, jitter=0.1):
    side = int(math.ceil(n ** (1.0 / dim)))
    xyz = lattice((side,) * dim, dx, 0.0, count=n)
    xyz = xyz + rng.uniform(-jitter * dx, jitter * dx, size=xyz.shape)
    h = hr * dx
    return ParticleSet(np.ascontiguousarray(xyz), h, 2.0 * h, dx)


def c4_batched(seed=4, nsys=256, nmin=2000, nmax=200000):
    """256 independent 3D systems of uneven sizes."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(nsys):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        dx = rng.uniform(0.005, 0.02)
        hr = rng.uniform(1.2, 1.5)
        ps = _system(rng, n, 3, dx, hr)
        ps.name = "batch_sys%d" % s
        out.append(ps)
    return out


@dataclass
class Request:
    t_arrival: float
    pset: ParticleSet


def c5_request_stream(seed=5, count=2200, rate=200.0, nmin=1000, nmax=2000000, frac3d=0.7,
                      materialise=True):
    """Poisson stream of search-plus-density requests.  With ``materialise`` False
    only the request shapes are drawn (coordinates are drawn on demand by
    :func:`materialise_request`)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += rng.exponential(1.0 / rate)
        dim = 3 if rng.uniform() < frac3d else 2
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        hr = rng.uniform(1.2, 1.5)
        sub_seed = int(rng.integers(0, 2 ** 62))
        spec = dict(dim=dim, n=n, hr=hr, seed=sub_seed)
        ps = materialise_request(spec) if materialise else None
        out.append((t, spec, ps))
    return out


def materialise_request(spec):
    dim, n = spec["dim"], spec["n"]
    dx = 1.0 / math.ceil(n ** (1.0 / dim))
    rng = np.random.default_rng(spec["seed"])
    ps = _system(rng, n, dim, dx, spec["hr"])
    ps.name = "req_%dd_%d" % (dim, n)
    return ps


def random_uniform(n, dim, seed=0, extent=1.0):
    """Uniform random particles in [0, extent]^dim (the Table 2 set-up)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, extent, size=(n, dim))


def circle_pairs(kh, dR, count, dim=2, seed=0, center=(0.5, 0.5, 0.5)):
    """A centre particle plus ``count`` particles at distance kh (1 + s dR)
    with random sign s and random direction (the Table 1 / Fig. 9 set-up
    with the circle radius taken as the search radius)."""
    rng = np.random.default_rng(seed)
    c = np.asarray(center[:dim], dtype=np.float64)
    if dim == 2:
        th = rng.uniform(0, 2 * math.pi, size=count)
        u = np.stack([np.cos(th), np.sin(th)], axis=1)
    else:
        v = rng.normal(size=(count, 3))
        u = v / np.linalg.norm(v, axis=1, keepdims=True)
    s = rng.choice([-1.0, 1.0], size=count)
    r = kh * (1.0 + s * dR)
    pts = c + u * r[:, None]
    return np.ascontiguousarray(np.vstack([c[None, :], pts]))


def face_set(kh, dim=3, seed=0, reps=4):
    """Particles placed on multiples of kh from the box corner (where cell faces
    fall) and nudged by a few units in the last place either way, plus the box
    corners, so binning sees coordinates on and beside every face."""
    rng = np.random.default_rng(seed)
    base = []
    k = np.arange(0, 4, dtype=np.float64)
    grid = np.stack(np.meshgrid(*([k] * dim), indexing="ij"), axis=-1).reshape(-1, dim) * kh
    for _ in range(reps):
        ulps = rng.integers(-3, 4, size=grid.shape)
        base.append(grid + ulps * np.spacing(np.maximum(grid, kh)))
    pts = np.vstack(base + [grid])
    pts = pts + 1.0  # keep away from zero so nudges are relative
    return np.ascontiguousarray(pts)


def exact_lattice(side, dim, dx):
    """Unjittered lattice with spacing dx starting at dx (power-of-two dx gives
    exactly representable coordinates and exact squared distances)."""
    return lattice((side,) * dim, dx, 0.0, origin=0.5 * dx)
