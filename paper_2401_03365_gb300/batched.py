"""Batched MLS projection of many clouds in one persistent launch.

    bp = BatchedProjector.from_clouds([xyz0, xyz1, ...], ks=[16, 32, ...])
    bp.tune()                      # autotuned launch shape (cached on disk)
    bp.capture()                   # CUDA graph of the whole batched projection
    bp.replay()                    # one graph launch per call
    bp.out_xyz, bp.out_normal, bp.out_status      # (total, 3), (total, 3), (total,)

Per cloud, the neighbour rows come from mls_build_grid + mls_knn and h from
mls_mean_knn_dist (h = 2 x mean neighbour distance) unless given.  Every step
runs in libmls; this module sequences the C-ABI calls and keeps the autotuner's
cache (a JSON file: launch shape per device, degree, precision, k mix and
size class).
"""
from __future__ import annotations

import json
import math
import os
from collections import Counter

import torch

from . import capi


def default_cache_path() -> str:
    return os.environ.get("MLS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mls_gb300", "autotune.json"))


def tune_key(device_name: str, degree: int, precision: str, ks, total: int) -> str:
    """Cache key: the device, the fit, the mix of k (as fractions rounded to
    0.1) and the total size class (power of two)."""
    cnt = Counter(int(k) for k in ks)
    mix = ",".join(f"{k}:{round(c / len(ks), 1)}" for k, c in sorted(cnt.items()))
    return f"{device_name}|deg{degree}|{precision}|k[{mix}]|2^{max(0, math.ceil(math.log2(max(total, 1))))}"


class TuneCache:
    """JSON file of key -> {"shape": [lanes, threads, rounds], "ms": t}."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self.data = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, key):
        e = self.data.get(key)
        if not e or len(e.get("shape", ())) != 3:
            return None
        return tuple(int(v) for v in e["shape"])

    def put(self, key, shape, ms):
        self.data[key] = {"shape": [int(v) for v in shape], "ms": float(ms)}
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def neighbours(xyz: torch.Tensor, k: int):
    """(rows (n, k) int32, grid order (n,) int32, h) of one cloud."""
    grid = capi.mls_build_grid(xyz, 0.0, k)
    try:
        idx, _ = capi.mls_knn(grid, k)
        order = capi.mls_grid_order(grid).clone()
        h = 2.0 * float(capi.mls_mean_knn_dist(xyz, idx).item())
    finally:
        torch.cuda.current_stream().synchronize()
        grid.close()
    return idx, order, h


class BatchedProjector:
    """Inputs, outputs and the mls_batch handle of one batch of clouds."""

    def __init__(self, xyz, idx, order, h, offsets, ks, degree: int = 2, precision: str = "mixed"):
        self.batch = capi.mls_batch_create(offsets, ks)
        self.xyz, self.idx, self.order, self.h = xyz, idx, order, h
        self.degree, self.precision = degree, precision
        self.out_xyz = torch.empty_like(xyz)
        self.out_normal = torch.empty_like(xyz)
        self.out_status = torch.empty(xyz.shape[0], dtype=torch.uint8, device=xyz.device)
        self.tuned = None

    @classmethod
    def from_clouds(cls, clouds, ks, hs=None, degree: int = 2, precision: str = "mixed"):
        """clouds: list of (n_c, 3) float32 CUDA tensors; ks: per-cloud k;
        hs: per-cloud bandwidths (None: 2 x mean kNN distance)."""
        rows, orders, hh, offsets = [], [], [], [0]
        for c, (x, k) in enumerate(zip(clouds, ks)):
            idx, order, h = neighbours(x, int(k))
            rows.append(idx.reshape(-1))
            orders.append(order)
            hh.append(h if hs is None else float(hs[c]))
            offsets.append(offsets[-1] + x.shape[0])
        dev = clouds[0].device
        xyz = torch.cat(clouds).contiguous()
        idx = torch.cat(rows).contiguous()
        order = torch.cat(orders).contiguous()
        h = torch.tensor(hh, dtype=torch.float32, device=dev)
        return cls(xyz, idx, order, h, offsets, ks, degree, precision)

    def run(self, stream=None):
        return capi.mls_project_batched(self.batch, self.xyz, self.idx, self.h, self.degree, self.precision,
                                        order=self.order, out_xyz=self.out_xyz, out_normal=self.out_normal,
                                        out_status=self.out_status, stream=stream)

    def tune(self, cache: TuneCache | None = None, reps: int = 3, retune: bool = False):
        """Launch shape from the cache, or from the autotuner (then cached)."""
        cache = cache if cache is not None else TuneCache()
        key = tune_key(torch.cuda.get_device_name(self.xyz.device), self.degree, self.precision,
                       self.batch.ks, self.batch.total)
        shape = None if retune else cache.get(key)
        if shape is not None:
            capi.mls_batch_set_shape(self.batch, *shape)
            self.tuned = {"shape": shape, "source": "cache", "key": key}
        else:
            shape, table = capi.mls_batch_autotune(self.batch, self.xyz, self.idx, self.h, self.degree,
                                                   self.precision, order=self.order, out_xyz=self.out_xyz,
                                                   out_normal=self.out_normal, out_status=self.out_status,
                                                   reps=reps)
            best = min(t[3] for t in table)
            cache.put(key, shape, best)
            self.tuned = {"shape": shape, "source": "autotune", "key": key, "table": table}
        return self.tuned

    def capture(self):
        capi.mls_batch_capture(self.batch, self.xyz, self.idx, self.h, self.degree, self.precision,
                               order=self.order, out_xyz=self.out_xyz, out_normal=self.out_normal,
                               out_status=self.out_status)

    def replay(self, stream=None):
        capi.mls_batch_replay(self.batch, stream)

    def cloud(self, c: int):
        """Slices (xyz', normal, status) of cloud c."""
        a, b = self.batch.offsets[c], self.batch.offsets[c + 1]
        return self.out_xyz[a:b], self.out_normal[a:b], self.out_status[a:b]

    def close(self):
        self.batch.close()
