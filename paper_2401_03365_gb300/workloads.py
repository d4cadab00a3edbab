"""Seeded synthetic point clouds shaped like the paper's inputs.

The paper evaluates MLS on normalised polygonal models sampled with additive
Gaussian noise (Sec. 3.2) and times a 25M-point scan (Sec. 3.3 tables).  Those
models and that scan are not available, so these generators stand in for them:
analytic surfaces at unit scale, sampled at random, with noise and outliers.

This module holds no part of the MLS method: it only draws points.  Both the
CUDA path and the FP64 oracle are fed from here, which is the only code the
two sides share.  Every array is float32 (the method's input precision) and
every draw comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Cloud", "sphere", "torus", "heightfield", "bumpy_sphere", "batch_clouds",
    "make", "CONFIGS",
]


@dataclass
class Cloud:
    """A point cloud plus the parameters the workload fixes for it."""
    name: str
    xyz: np.ndarray                 # (N, 3) float32, row i = point i
    k: int                          # neighbours per point (self included)
    degree: int = 2                 # height-polynomial degree
    precision: str = "mixed"        # "fp32" | "mixed" | "fp64"
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def sphere(n: int = 20_000, seed: int = 1, sigma: float = 0.01, k: int = 20) -> Cloud:
    """Unit sphere, directions uniform, radial Gaussian noise of std ``sigma``."""
    rng = np.random.default_rng(seed)
    u = _unit_vectors(rng, n)
    rad = 1.0 + sigma * rng.standard_normal(n)
    xyz = (u * rad[:, None]).astype(np.float32)
    return Cloud("sphere", xyz, k, 2, "mixed", {"sigma": sigma, "radius": 1.0, "seed": seed})


def torus(n: int = 2_000_000, seed: int = 2, R: float = 1.0, r: float = 0.3,
          sigma: float = 0.005, outlier_frac: float = 0.01, k: int = 32) -> Cloud:
    """Torus (major radius R, tube radius r) sampled uniformly by area, displaced
    along the surface normal by N(0, sigma^2), plus a fraction of points drawn
    uniformly in the clean torus's bounding box.  Rows are shuffled."""
    rng = np.random.default_rng(seed)
    n_out = int(round(n * outlier_frac))
    n_surf = n - n_out
    # area element on the torus is proportional to (R + r cos v): accept the tube
    # angle v with probability (1 + (r/R) cos v) / (1 + r/R)
    vs = []
    got = 0
    while got < n_surf:
        m = int((n_surf - got) * 1.4) + 1024
        v = rng.uniform(0.0, 2 * math.pi, m)
        keep = rng.uniform(0.0, 1.0, m) < (1.0 + (r / R) * np.cos(v)) / (1.0 + r / R)
        v = v[keep]
        vs.append(v)
        got += v.size
    v = np.concatenate(vs)[:n_surf]
    u = rng.uniform(0.0, 2 * math.pi, n_surf)
    nrm = np.stack([np.cos(v) * np.cos(u), np.cos(v) * np.sin(u), np.sin(v)], axis=1)
    ring = np.stack([R * np.cos(u), R * np.sin(u), np.zeros_like(u)], axis=1)
    surf = ring + r * nrm + sigma * rng.standard_normal(n_surf)[:, None] * nrm
    lo = np.array([-(R + r), -(R + r), -r])
    hi = -lo
    out = lo + (hi - lo) * rng.uniform(0.0, 1.0, (n_out, 3))
    xyz = np.concatenate([surf, out], axis=0)
    xyz = xyz[rng.permutation(n)].astype(np.float32)
    return Cloud("torus", xyz, k, 2, "mixed",
                 {"R": R, "r": r, "sigma": sigma, "outlier_frac": outlier_frac, "seed": seed})


def heightfield(n: int = 50_000_000, seed: int = 3, sigma: float = 0.002, k: int = 64,
                n_waves: int = 8, chunk: int = 5_000_000) -> Cloud:
    """z = sum of ``n_waves`` random sinusoids over [0,1]^2.  x is drawn with a
    density proportional to 1 + 9x (a 10x ramp across the domain), y uniformly,
    and z gets N(0, sigma^2) noise."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.01, 0.05, n_waves)
    fmag = rng.uniform(1.0, 6.0, n_waves)
    fang = rng.uniform(0.0, 2 * math.pi, n_waves)
    freq = np.stack([fmag * np.cos(fang), fmag * np.sin(fang)], axis=1)
    phase = rng.uniform(0.0, 2 * math.pi, n_waves)
    xyz = np.empty((n, 3), np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        uu = rng.uniform(0.0, 1.0, m)
        x = (-1.0 + np.sqrt(1.0 + 99.0 * uu)) / 9.0     # inverse CDF of (1+9x)/5.5
        y = rng.uniform(0.0, 1.0, m)
        z = np.zeros(m)
        for a, f, p in zip(amp, freq, phase):
            z += a * np.sin(2 * math.pi * (f[0] * x + f[1] * y) + p)
        z += sigma * rng.standard_normal(m)
        xyz[s:s + m, 0] = x
        xyz[s:s + m, 1] = y
        xyz[s:s + m, 2] = z
    return Cloud("heightfield", xyz, k, 2, "mixed",
                 {"sigma": sigma, "amp": amp, "freq": freq, "phase": phase, "seed": seed})


def bumpy_radius(u: np.ndarray, centres: np.ndarray, amps: np.ndarray, widths: np.ndarray) -> np.ndarray:
    """rho(u) = 1 + sum_m a_m exp(-(1 - <u, c_m>) / s_m^2) for unit directions u."""
    dots = u @ centres.T
    return 1.0 + (amps[None, :] * np.exp(-(1.0 - dots) / (widths[None, :] ** 2))).sum(axis=1)


def bumpy_sphere(n: int = 1_000_000, seed: int = 5, n_bumps: int = 64, sigma: float = 0.005,
                 k: int = 32) -> Cloud:
    """Sphere with Gaussian bumps: x = (rho(u) + N(0, sigma^2)) u, u uniform on S^2."""
    rng = np.random.default_rng(seed)
    centres = _unit_vectors(rng, n_bumps)
    amps = rng.uniform(-0.05, 0.05, n_bumps)
    widths = rng.uniform(0.15, 0.35, n_bumps)
    u = _unit_vectors(rng, n)
    rho = np.empty(n)
    for s in range(0, n, 1 << 18):
        rho[s:s + (1 << 18)] = bumpy_radius(u[s:s + (1 << 18)], centres, amps, widths)
    xyz = ((rho + sigma * rng.standard_normal(n))[:, None] * u).astype(np.float32)
    return Cloud("bumpy_sphere", xyz, k, 2, "fp32",
                 {"centres": centres, "amps": amps, "widths": widths, "sigma": sigma, "seed": seed})


def _superquadric_point(eta, om, a, e1, e2):
    def spow(t, e):
        return np.sign(t) * np.abs(t) ** e
    ce, se = np.cos(eta), np.sin(eta)
    co, so = np.cos(om), np.sin(om)
    return np.stack([a[0] * spow(ce, e1) * spow(co, e2),
                     a[1] * spow(ce, e1) * spow(so, e2),
                     a[2] * spow(se, e1)], axis=-1)


def _area_uniform_superquadric(rng, n, a, e1, e2):
    """Parametric samples (eta, omega) accepted with probability proportional to
    the surface area element |dS/deta x dS/domega| (finite differences), which
    makes the accepted points area-uniform up to the clipped density peaks."""
    def area_elem(eta, om):
        d = 1e-4
        p_e = (_superquadric_point(eta + d, om, a, e1, e2) - _superquadric_point(eta - d, om, a, e1, e2)) / (2 * d)
        p_o = (_superquadric_point(eta, om + d, a, e1, e2) - _superquadric_point(eta, om - d, a, e1, e2)) / (2 * d)
        return np.linalg.norm(np.cross(p_e, p_o), axis=-1)
    probe_e = rng.uniform(-math.pi / 2, math.pi / 2, 4096)
    probe_o = rng.uniform(-math.pi, math.pi, 4096)
    cap = np.quantile(area_elem(probe_e, probe_o), 0.98)
    out, got = [], 0
    while got < n:
        m = max(2 * (n - got), 1024)
        eta = rng.uniform(-math.pi / 2, math.pi / 2, m)
        om = rng.uniform(-math.pi, math.pi, m)
        acc = rng.uniform(0.0, 1.0, m) * cap < np.minimum(area_elem(eta, om), cap)
        pts = _superquadric_point(eta[acc], om[acc], a, e1, e2)
        out.append(pts)
        got += pts.shape[0]
    return np.concatenate(out)[:n]


def _batch_draws(rng, n_min: int, n_max: int, size_scale: float):
    n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * size_scale))
    return max(n, 64), int(rng.choice([16, 32, 64]))


def batch_cloud_size(b: int, seed0: int = 4, n_min: int = 1_000, n_max: int = 500_000,
                     size_scale: float = 1.0) -> tuple[int, int]:
    """(points, k) of cloud b of batch_clouds, without generating it."""
    return _batch_draws(np.random.default_rng(seed0 + b), n_min, n_max, size_scale)


def batch_cloud(b: int, seed0: int = 4, n_min: int = 1_000, n_max: int = 500_000, noise_frac: float = 0.003,
                size_scale: float = 1.0) -> Cloud:
    """Cloud b of batch_clouds (same arguments) alone."""
    return _batch_cloud(b, seed0, n_min, n_max, noise_frac, size_scale)


def _batch_cloud(b: int, seed0: int, n_min: int, n_max: int, noise_frac: float, size_scale: float) -> Cloud:
    rng = np.random.default_rng(seed0 + b)
    n, k = _batch_draws(rng, n_min, n_max, size_scale)
    a = rng.uniform(0.2, 1.0, 3)
    if b % 2 == 0:
        e1 = e2 = 1.0                               # ellipsoid
    else:
        e1, e2 = rng.uniform(0.3, 2.0, 2)
    pts = _area_uniform_superquadric(rng, n, a, e1, e2)
    diag = float(np.linalg.norm(pts.max(0) - pts.min(0)))
    pts = pts + noise_frac * diag * rng.standard_normal(pts.shape)
    return Cloud(f"quadric{b}", pts.astype(np.float32), min(k, n), 2, "mixed",
                 {"semi_axes": a, "eps": (e1, e2), "seed": seed0 + b})


def batch_clouds(n_clouds: int = 256, seed0: int = 4, n_min: int = 1_000, n_max: int = 500_000,
                 noise_frac: float = 0.003, size_scale: float = 1.0, workers: int = 1) -> list[Cloud]:
    """Clouds of uneven size: half ellipsoids, half superquadrics (semi-axes
    U(0.2, 1), exponents U(0.3, 2)); size log-uniform in [n_min, n_max] (times
    ``size_scale``); k drawn from {16, 32, 64}; isotropic noise of
    ``noise_frac`` times the cloud's bounding-box diagonal.  Cloud b uses seed
    ``seed0 + b`` alone, so ``workers`` > 1 (a spawned process pool, safe
    after CUDA has started) gives the same clouds faster."""
    args = [(b, seed0, n_min, n_max, noise_frac, size_scale) for b in range(n_clouds)]
    if workers > 1 and n_clouds > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, n_clouds)) as pool:
            return pool.starmap(_batch_cloud, args, chunksize=1)
    return [_batch_cloud(*a) for a in args]


# Single-cloud workloads by name (the batched one is batch_clouds).
CONFIGS = {
    "sphere20k_k20": lambda **kw: sphere(**kw),
    "torus2m_k32": lambda **kw: torus(**kw),
    "heightfield50m_k64": lambda **kw: heightfield(**kw),
    "bumpy1m_k32": lambda **kw: bumpy_sphere(**kw),
}


def make(name: str, **kw) -> Cloud:
    return CONFIGS[name](**kw)
