"""Denoising quality against the neighbourhood radius (the shape of Sec. 3.3's
study, Tables 1-6, on analytic surfaces instead of the paper's models).

For a surface with a closed-form distance (unit sphere, torus R = 1, r = 0.3)
sampled area-uniformly and displaced by Gaussian noise of standard deviation
sigma along random directions, the radius-R projection (the paper's own
neighbourhood and outlier rule) is run for a sweep of R; the deviation of the
kept points from the exact surface (mean, standard deviation, min, max) is
reported beside the noisy input's, with the fraction of points removed as
outliers.  Everything runs through libmls on the GPU.

    python -m paper_2401_03365_gb300.denoise_study [--n 200000] [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch


def sphere_points(n: int, sigma: float, seed: int):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    noise = rng.standard_normal((n, 3)) * sigma
    return (u + noise).astype(np.float32)


def sphere_distance(p: np.ndarray) -> np.ndarray:
    return np.abs(np.linalg.norm(p.astype(np.float64), axis=1) - 1.0)


def torus_points(n: int, sigma: float, seed: int, R: float = 1.0, r: float = 0.3):
    rng = np.random.default_rng(seed)
    out = []
    while sum(len(o) for o in out) < n:
        m = 2 * n
        u = rng.uniform(0, 2 * math.pi, m)
        v = rng.uniform(0, 2 * math.pi, m)
        keep = rng.uniform(0, 1, m) < (R + r * np.cos(v)) / (R + r)      # area-uniform
        u, v = u[keep], v[keep]
        out.append(np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], 1))
    p = np.concatenate(out)[:n]
    p = p + rng.standard_normal(p.shape) * sigma
    return p.astype(np.float32)


def torus_distance(p: np.ndarray, R: float = 1.0, r: float = 0.3) -> np.ndarray:
    p = p.astype(np.float64)
    rho = np.hypot(p[:, 0], p[:, 1])
    return np.abs(np.hypot(rho - R, p[:, 2]) - r)


SURFACES = {"sphere": (sphere_points, sphere_distance), "torus": (torus_points, torus_distance)}


def stats(d: np.ndarray) -> dict:
    if d.size == 0:
        return {"mean": None, "std": None, "min": None, "max": None}
    return {"mean": float(d.mean()), "std": float(d.std()), "min": float(d.min()), "max": float(d.max())}


def run(n: int = 200_000, surfaces=("sphere", "torus"), sigmas=(0.002, 0.005, 0.01),
        radii=(0.005, 0.01, 0.015, 0.02, 0.03, 0.04), seed: int = 7, device="cuda") -> list[dict]:
    from .mls import project_radius
    rows = []
    for surf in surfaces:
        gen, dist = SURFACES[surf]
        for si, sigma in enumerate(sigmas):
            pts = gen(n, sigma, seed + si)
            before = stats(dist(pts))
            x = torch.from_numpy(pts).to(device)
            for R in radii:
                try:
                    res = project_radius(x, R, h=R, degree=2, precision="mixed", min_neighbors=3)
                except RuntimeError as e:          # a neighbourhood above the row capacity
                    rows.append({"surface": surf, "sigma": sigma, "R": R, "error": str(e).split(":")[0]})
                    continue
                kept = res.kept.shape[0]
                after = stats(dist(res.xyz.cpu().numpy()))
                rows.append({"surface": surf, "n": n, "sigma": sigma, "R": R, "before": before, "after": after,
                             "removed_frac": 1.0 - kept / n})
    return rows


def table(rows: list[dict]) -> str:
    lines = ["| surface | sigma | R | mean before | mean after | std after | max after | removed |",
             "|---|---:|---:|---:|---:|---:|---:|---:|"]
    for r in rows:
        if "error" in r:
            lines.append(f"| {r['surface']} | {r['sigma']} | {r['R']} | - | {r['error']} | | | |")
            continue
        a, b = r["after"], r["before"]
        fmt = (lambda v: "-" if v is None else f"{v:.2e}")
        lines.append(f"| {r['surface']} | {r['sigma']} | {r['R']} | {b['mean']:.2e} | {fmt(a['mean'])} | "
                     f"{fmt(a['std'])} | {fmt(a['max'])} | {100 * r['removed_frac']:.1f} % |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    from . import build
    build.build()
    rows = run(n=args.n)
    print(table(rows))
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
