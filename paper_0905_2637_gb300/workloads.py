"""Seeded synthetic inputs shaped like the paper's vortex-blob workloads.

This module holds input recipes only -- no part of the FMM's arithmetic -- and
is the one piece shared by the FP64 oracle's tests and the CUDA path's tests
and benchmark.  All randomness comes from ``numpy.random.default_rng(seed)``
(PCG64), so both sides read identical bits.

The paper's own test case is a lattice of Gaussian blobs carrying a smooth
vorticity field in a square domain (Sec. 7.1), plus uniform random points in a
square (Fig. 5).  The recipes below follow that shape:

* ``uniform``   -- x, y ~ U(0, 1), gamma ~ U(-1, 1) (10,000 blobs, sigma 0.005,
                   L = 4, p = 12, FP64 storage).
* ``lattice``   -- 1024 x 1024 jittered lattice, h = 1/1024, jitter U(-h/4, h/4),
                   gamma = h^2 exp(-|x - (1/2, 1/2)|^2 / 0.01), sigma = 1.5 h,
                   L = 8, p = 17.
* ``clustered`` -- 2^24 blobs from a mixture of 8 isotropic Gaussians (centres
                   U(0.2, 0.8)^2, std 0.02, equal weights), gamma ~ N(0, 1)/N,
                   sigma = 0.002, L = 10, p = 17, FP32 storage.
* ``batch``     -- 512 instances, N log-uniform in [1e3, 2^18], uniform points,
                   gamma ~ U(-1, 1), sigma = 0.5 / sqrt(N), p in {8, 12, 17}.
* ``lamb_oseen``-- the Sec. 7.1 initial condition: a lattice with h / sigma = 0.8
                   carrying the Gaussian vorticity of Eq. 16.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

UNIT_DOMAIN = (0.0, 0.0, 1.0)


@dataclasses.dataclass
class Workload:
    name: str
    x: np.ndarray
    y: np.ndarray
    gamma: np.ndarray
    sigma: float
    domain: tuple
    L: int
    p: int
    dtype: str  # "f64" or "f32": storage type of x, y, gamma, u, v

    @property
    def n(self) -> int:
        return int(self.x.size)

    def as_f64(self):
        return (self.x.astype(np.float64), self.y.astype(np.float64),
                self.gamma.astype(np.float64))


def _store(dtype, *arrays):
    if dtype == "f32":
        return tuple(np.ascontiguousarray(a, dtype=np.float32) for a in arrays)
    return tuple(np.ascontiguousarray(a, dtype=np.float64) for a in arrays)


def uniform(n=10_000, seed=1, sigma=0.005, L=4, p=12, dtype="f64", name="uniform-10k"):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, n)
    y = rng.uniform(0.0, 1.0, n)
    g = rng.uniform(-1.0, 1.0, n)
    x, y, g = _store(dtype, x, y, g)
    return Workload(name, x, y, g, sigma, UNIT_DOMAIN, L, p, dtype)


def lattice(side=1024, seed=1, L=8, p=17, dtype="f64", name="lattice-1M"):
    rng = np.random.default_rng(seed)
    h = 1.0 / side
    i = np.arange(side, dtype=np.float64)
    gx, gy = np.meshgrid(i, i, indexing="xy")
    x = (gx.ravel() + 0.5) * h + rng.uniform(-0.25 * h, 0.25 * h, side * side)
    y = (gy.ravel() + 0.5) * h + rng.uniform(-0.25 * h, 0.25 * h, side * side)
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    g = h * h * np.exp(-r2 / 0.01)
    x, y, g = _store(dtype, x, y, g)
    return Workload(name, x, y, g, 1.5 * h, UNIT_DOMAIN, L, p, dtype)


def clustered(n=1 << 24, seed=1, L=10, p=17, sigma=0.002, dtype="f32", name="clustered-16M"):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, (8, 2))
    comp = rng.integers(0, 8, n)
    pts = centres[comp] + 0.02 * rng.standard_normal((n, 2))
    np.clip(pts, 0.0, 1.0, out=pts)
    g = rng.standard_normal(n) / n
    x, y, g = _store(dtype, pts[:, 0], pts[:, 1], g)
    return Workload(name, x, y, g, sigma, UNIT_DOMAIN, L, p, dtype)


def clustered_scaled(shrink_levels=3, seed=1, dtype="f32"):
    """The clustered workload with 4^-k of the blobs on a tree k levels
    shallower: the same expected blobs per leaf and the same leaf-occupancy
    profile, so the same per-blob work."""
    n = (1 << 24) >> (2 * shrink_levels)
    return clustered(n=n, seed=seed, L=10 - shrink_levels, dtype=dtype,
                     name=f"clustered-{n}-L{10 - shrink_levels}")


def lamb_oseen(sigma=0.02, half_width=0.5, core=0.1, gamma0=1.0, L=4, p=17, dtype="f64"):
    """Sec. 7.1 test case: lattice with h / sigma = 0.8, strengths from the
    Lamb-Oseen vorticity (Eq. 16) with 4 nu t = core^2, gamma_i = omega h^2."""
    h = 0.8 * sigma
    m = int(math.floor(half_width / h))
    c = (np.arange(-m, m + 1, dtype=np.float64)) * h
    gx, gy = np.meshgrid(c, c, indexing="xy")
    x, y = gx.ravel(), gy.ravel()
    four_nu_t = core * core
    omega = gamma0 / (math.pi * four_nu_t) * np.exp(-(x * x + y * y) / four_nu_t)
    g = omega * h * h
    x, y, g = _store(dtype, x, y, g)
    dom = (-half_width - h, -half_width - h, 2 * (half_width + h))
    return Workload("lamb-oseen", x, y, g, sigma, dom, L, p, dtype)


def lamb_oseen_paper(dtype="f32"):
    """The Sec. 7.1 test case at the paper's size: an 875 x 875 lattice
    (765,625 blobs) with sigma = 0.02 and h = 0.8 sigma, L = 10, p = 17; the
    paper leaves Gamma_0, nu and t open, taken here as Gamma_0 = 1 and
    4 nu t = 1."""
    w = lamb_oseen(sigma=0.02, half_width=7.0, core=1.0, gamma0=1.0, L=10, p=17, dtype=dtype)
    w.name = "lamb-oseen-765k"
    return w


def batch(n_inst=512, seed=1, dtype="f64", n_min=1_000, n_max=262_144):
    """Independent uniform instances of uneven size (log-uniform N)."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_inst))).astype(np.int64)
    orders = rng.choice(np.array([8, 12, 17]), n_inst)
    out = []
    for i in range(n_inst):
        r = np.random.default_rng(seed * 1000 + i)
        n = int(sizes[i])
        x = r.uniform(0.0, 1.0, n)
        y = r.uniform(0.0, 1.0, n)
        g = r.uniform(-1.0, 1.0, n)
        x, y, g = _store(dtype, x, y, g)
        out.append(Workload(f"batch-{i}", x, y, g, 0.5 / math.sqrt(n), UNIT_DOMAIN, -1,
                            int(orders[i]), dtype))
    return out


def laplace_uniform(n=1 << 20, seed=1, L=8, p=17, dtype="f64", name="laplace-1M"):
    """The second kernel's workload: n charges q ~ U(-1, 1) uniform on the
    unit square (the paper's "square domain" points), 16 per leaf at L = 8.
    sigma is unused by the logarithmic kernel."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, n)
    y = rng.uniform(0.0, 1.0, n)
    q = rng.uniform(-1.0, 1.0, n)
    x, y, q = _store(dtype, x, y, q)
    return Workload(name, x, y, q, 1.0, UNIT_DOMAIN, L, p, dtype)


def tiny(n, seed, L=3, p=10, sigma=None, dtype="f64", clustered_frac=0.0):
    """Small random cases for property sweeps: uniform points, optionally with a
    fraction packed into one tight clump (ragged, very uneven leaves)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, n)
    y = rng.uniform(0.0, 1.0, n)
    k = int(clustered_frac * n)
    if k:
        c = rng.uniform(0.3, 0.7, 2)
        x[:k] = np.clip(c[0] + 0.01 * rng.standard_normal(k), 0.0, 1.0)
        y[:k] = np.clip(c[1] + 0.01 * rng.standard_normal(k), 0.0, 1.0)
    g = rng.uniform(-1.0, 1.0, n)
    if sigma is None:
        sigma = 0.25 / (1 << L)
    x, y, g = _store(dtype, x, y, g)
    return Workload(f"tiny-{n}-{seed}", x, y, g, sigma, UNIT_DOMAIN, L, p, dtype)


def sample_targets(n, count, seed=7):
    """Seeded sample of target indices (sorted, without repetition)."""
    rng = np.random.default_rng(seed)
    count = min(count, n)
    return np.sort(rng.choice(n, count, replace=False)).astype(np.int64)


# ---------------------------------------------------------------------------
# Three dimensions (the octree extension): point charges in the unit cube.
# ---------------------------------------------------------------------------
UNIT_CUBE = (0.0, 0.0, 0.0, 1.0)


@dataclasses.dataclass
class Workload3D:
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    q: np.ndarray
    domain: tuple
    L: int
    p: int
    dtype: str

    @property
    def n(self) -> int:
        return int(self.x.size)

    def as_f64(self):
        return tuple(a.astype(np.float64) for a in (self.x, self.y, self.z, self.q))


def uniform3d(n=1 << 21, seed=1, L=5, p=8, dtype="f32", name="uniform3d-2M"):
    """x, y, z ~ U(0, 1), q ~ U(-1, 1) / n: 64 charges per leaf at L = 5."""
    rng = np.random.default_rng(seed)
    x, y, z = rng.uniform(0.0, 1.0, (3, n))
    q = rng.uniform(-1.0, 1.0, n) / n
    return Workload3D(name, *_store(dtype, x, y, z, q), UNIT_CUBE, L, p, dtype)


def clustered3d(n=1 << 21, seed=1, L=6, p=8, dtype="f32", k=8, std=0.04, name="clustered3d-2M"):
    """A mixture of k isotropic Gaussians (centres U(0.2, 0.8)^3, equal
    weights), clipped to the cube; q ~ N(0, 1) / n."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, (k, 3))
    comp = rng.integers(0, k, n)
    pts = np.clip(centres[comp] + std * rng.standard_normal((n, 3)), 0.0, 1.0)
    q = rng.standard_normal(n) / n
    return Workload3D(name, *_store(dtype, pts[:, 0], pts[:, 1], pts[:, 2], q), UNIT_CUBE, L, p,
                      dtype)


def tiny3d(n, seed, L=3, p=8, dtype="f64", clustered_frac=0.0):
    """Small 3D inputs for the parity tests: uniform charges, a fraction of
    them in one tight cluster (hot leaves next to empty ones)."""
    rng = np.random.default_rng(seed)
    x, y, z = rng.uniform(0.0, 1.0, (3, n))
    k = int(n * clustered_frac)
    if k:
        c = rng.uniform(0.2, 0.8, 3)
        pts = np.clip(c + 0.02 * rng.standard_normal((k, 3)), 0.0, 1.0)
        x[:k], y[:k], z[:k] = pts.T
    q = rng.uniform(-1.0, 1.0, n)
    return Workload3D(f"tiny3d-{n}", *_store(dtype, x, y, z, q), UNIT_CUBE, L, p, dtype)
