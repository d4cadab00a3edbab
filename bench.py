"""Benchmark of the MLS projection hot path on one or more GPUs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: 2,000,000-point torus (R = 1, r = 0.3, normal noise 0.005, 1 %
uniform outliers), k = 32, degree-2 polynomial, mixed precision.  One step is
one pass of the whole hot path over the cloud: grid build, exact kNN, the MLS
projection and its backward with a fixed cotangent (through the C ABI of
libmls, inputs resident in HBM).  L2 is
flushed (a 256 MB write) before every timed step, outside the timed events.

With N > 1 (torchrun) every rank projects its own cloud (seed 2 + rank): the
points are independent problems, so there is no data-path collective; the
step time is the maximum over ranks.  `--impl reference` times the FP64 CPU
oracle on the host cores instead (rank 0 only).

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLS-projected points/sec at k=32 (fwd and fwd+bwd), % FP32 roofline, vs plain FP64"
WORKLOAD = ("torus2m_k32: 2,000,000 points on a torus (R=1, r=0.3) with normal noise sigma=0.005 "
            "and 1% uniform outliers in its bounding box; k=32, Gaussian h = 2 x mean kNN distance, "
            "degree-2 polynomial, FP32 moments with FP64 eigen/6x6 solves where ill-conditioned")
N_POINTS = 2_000_000
K = 32

# Algorithmic work per point of the degree-2 projection, counted from the
# oracle's operation list (FMA = 2 flops): forward pass A 17, pass B 18,
# pass C 62 flops per neighbour; per point the 3x3 Jacobi (3 sweeps), the 6x6
# Cholesky with two solves and one refinement, q and p' (645).  The adjoint
# (oracle adjoint_point) recomputes the forward and adds per neighbour 190
# (height-fit reverse 106, covariance 43, centroid 17, weights 18, gather 6)
# and per point 307 (the solve for z 150, the eigenvector derivative 116,
# ofs and the rest 41).
# The timed step saves the forward's fit state for the adjoint: the
# projection then also solves for A^-1 e_0 (two 6x6 triangular solves, 72),
# and the adjoint's own work is the 190 per neighbour and, per point, the 307
# with the z solve (150) replaced by z = a0-bar A^-1 e_0 (6): 163.
FLOPS_PER_NEIGHBOUR = 97
FLOPS_PER_POINT = 645
STATE_FLOPS_PER_POINT = 72
BWD_FLOPS_PER_NEIGHBOUR = 97 + 190
BWD_FLOPS_PER_POINT = 645 + 307
BWD_STATE_FLOPS_PER_NEIGHBOUR = 190
BWD_STATE_FLOPS_PER_POINT = 307 - 150 + 6


def proj_flops(k, state=False):
    return FLOPS_PER_NEIGHBOUR * k + FLOPS_PER_POINT + (STATE_FLOPS_PER_POINT if state else 0)


def bwd_flops(k, state=False):
    if state:
        return BWD_STATE_FLOPS_PER_NEIGHBOUR * k + BWD_STATE_FLOPS_PER_POINT
    return BWD_FLOPS_PER_NEIGHBOUR * k + BWD_FLOPS_PER_POINT


# The kNN's algorithmic HBM bytes per query: read its float4, write its row
# of sorted positions (k int32).
def knn_bytes(k):
    return 16 + 4 * k


GRID_BYTES_PER_POINT = 12 + 16 + 8 + 4

# Measured per-query figures of the kNN's two kernels (k_knn_chain +
# k_knn_sparse, one ncu capture on the 1,000,000-point torus, k = 32):
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) and warp
# instructions (smsp__inst_executed.sum), each divided by the point count;
# valid only while the kernel sources they were taken on are unchanged
# (SHA-256 of each file).
KNN_MEASURED = {
    "traffic_bytes_per_query": 202.2,
    "warp_inst_per_query": 1916.8,
    "sources": {
        "paper_2401_03365_gb300/csrc/knn_search.cuh": "099d6dc317972f78b50cf17229b5ec1e84de938d472e928d351505d9238b5ee9",
        "paper_2401_03365_gb300/csrc/knn.cu": "ad1382bae4762e19f8d9c33ebd51971c9fb2e239bbb303fd01147bf1f4891d35",
        "paper_2401_03365_gb300/csrc/grid.cuh": "560013b7ab7f99966e1993aaaeb0c1a1733ec5389faaaa2bc0604f6aafc0ffcc",
        "paper_2401_03365_gb300/csrc/common.cuh": "9d6ac0dc2ad528cdc5d1d35b34889db2a24ebc7196733e8c248a68ed29f7d816",
    },
}


def knn_measured(field, n_points):
    """The measured figure for n_points queries, or None when unmeasured or
    stale."""
    import hashlib
    v = KNN_MEASURED.get(field)
    if v is None or not KNN_MEASURED["sources"]:
        return None
    for rel, digest in KNN_MEASURED["sources"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return v * n_points


def device_sms(dev):
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def load_peaks(sms):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = {"hbm_gbs": 6800.0, "source": "fallback"}
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        peaks.update(p)
        peaks["source"] = "measured"
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32: SMs (read from the device) x 128 FP32 lanes x 2 flops (FMA) x
    # the maximum SM clock; instruction issue: SMs x 4 schedulers x 1 warp
    # instruction per cycle x the clock
    peaks["sms"] = sms
    peaks["fp32_tflops"] = sms * 128 * 2 * sm_max * 1e6 / 1e12
    peaks["issue_ginst_per_mhz"] = sms * 4 * 1e6 / 1e9
    return peaks


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons.  Started before the
    warm-up (the tool's own start-up then falls outside the timed region);
    the summary keeps the samples read inside the timed window."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []             # (host time, csv line)
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 10.0 and self.proc.poll() is None:
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, t_begin, t_end):
        self.window = (t_begin, t_end)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        lines = self.lines
        if self.window is not None:
            a, b = self.window
            inside = [x for x in lines if a <= x[0] <= b]
            # a timed region shorter than the sampling period: the samples next to it
            lines = inside or [x for x in lines if a - 0.25 <= x[0] <= b + 0.25]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seeds(rank):
    """(cloud seed, cotangent seed) of a rank: every rank projects its own
    cloud, so the N-GPU job is N independent problems (weak scaling)."""
    return 2 + rank, 11 + rank


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of per-rank timings over all ranks (the job's
    time is the slowest rank's); identity without a process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(world, points_per_rank, ms):
    """Points per second of the whole job: all ranks' points over the
    slowest rank's time."""
    return world * points_per_rank / (ms * 1e-3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2401_03365_gb300 import build, capi, workloads

    world, rank, local = dist_setup(args)
    n_pts = args.points
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    dev = torch.device("cuda", local)
    sms = device_sms(dev)
    cloud_seed, cot_seed = rank_seeds(rank)
    cloud = workloads.torus(n=n_pts, seed=cloud_seed, k=K)
    x = torch.from_numpy(cloud.xyz).to(dev)
    stream = torch.cuda.current_stream()

    idx = torch.empty((n_pts, K), dtype=torch.int32, device=dev)
    pos = torch.empty((n_pts, K), dtype=torch.int32, device=dev)
    out_xyz = torch.empty_like(x)
    out_n = torch.empty_like(x)
    out_st = torch.empty(n_pts, dtype=torch.uint8, device=dev)
    grad = torch.empty_like(x)
    grad_h = torch.empty(1, dtype=torch.float32, device=dev)
    fit_state = torch.empty((capi.FIT_STATE_FLOATS, n_pts), dtype=torch.float32, device=dev)
    bucket_off = torch.empty(n_pts + 1, dtype=torch.int32, device=dev)
    gen = torch.Generator(device=dev).manual_seed(cot_seed)
    gp = torch.randn((n_pts, 3), generator=gen, device=dev)          # cotangent of the points
    gn = 0.1 * torch.randn((n_pts, 3), generator=gen, device=dev)    # cotangent of the normals
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # bandwidth of the workload: 2 x mean kNN distance, from the GPU kNN
    grid = capi.mls_build_grid(x, 0.0, K)
    capi.mls_knn(grid, K, out_idx=idx)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())

    # one step: grid build, kNN (rows of sorted positions) and the projection
    # saving the fit state, pipelined in one call (the projection of the
    # points the kNN's first pass finished runs beside its second pass, and
    # the adjoint's bucket offsets are counted beside its tail), and the
    # adjoint from the state with a fixed cotangent, all in the grid's order.
    # split=True makes the kNN and the projection two calls and lets the
    # adjoint count its own offsets, for the per-stage times.
    def step(xin, ev=None, before_forward_out=None, after_forward=None, before_backward=None, split=False):
        nonlocal grid
        if ev: ev[0].record(stream)
        grid = capi.mls_build_grid(xin, 0.0, K, grid=grid)
        if ev: ev[1].record(stream)
        if split:
            capi.mls_knn_sorted(grid, K, out_pos=pos)
            if ev: ev[2].record(stream)
            if before_forward_out: before_forward_out()
            capi.mls_project_sorted(grid, pos, h, 2, "mixed", out_xyz=out_xyz, out_normal=out_n,
                                    out_status=out_st, with_state=True, out_state=fit_state)
        else:
            if before_forward_out: before_forward_out()
            capi.mls_knn_project_sorted(grid, K, h, 2, "mixed", out_pos=pos, out_xyz=out_xyz, out_normal=out_n,
                                        out_status=out_st, with_state=True, out_state=fit_state,
                                        out_offsets=bucket_off)
            if ev: ev[2].record(stream)
        if ev: ev[3].record(stream)
        if after_forward: after_forward()
        if before_backward: before_backward()
        capi.mls_project_backward_sorted(grid, pos, h, gp, gn, 2, "mixed", out_grad_xyz=grad, out_grad_h=grad_h,
                                         state=fit_state, offsets=None if split else bucket_off)
        if ev: ev[4].record(stream)

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        for _ in range(args.warmup):
            step(x)
        torch.cuda.synchronize()
        launches0 = capi.mls_kernel_launches()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_begin = time.time()
        t0 = time.perf_counter()
        for s in range(args.steps):
            flush.zero_()
            step(x, events[s])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clocks.mark(t_begin, time.time())
    if world > 1:
        dist.barrier()
    launches = capi.mls_kernel_launches() - launches0
    deferred = capi.mls_knn_deferred(grid)
    stage = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in events])  # ms
    build_ms, knn_proj_ms, _, bwd_ms = (float(v) for v in stage.mean(0))
    step_ms, fwd_ms, wall_ms = max_over_ranks([stage.sum(1).mean(), stage[:, :3].sum(1).mean(),
                                               wall * 1e3 / args.steps], dev)
    # the same steps with the kNN and the projection as two calls: their own
    # times (the kNN's roofline, the projection's FP32 fraction)
    split_events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for s in range(args.steps):
        flush.zero_()
        step(x, split_events[s], split=True)
    torch.cuda.synchronize()
    split_stage = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in split_events])
    _, knn_ms, proj_ms, _ = (float(v) for v in split_stage.mean(0))
    value = job_throughput(world, n_pts, step_ms)
    # end to end through the public API with host buffers: every step copies
    # its points in from pinned memory, runs the four calls, and copies the
    # projected points, normals, status and gradient back.  The copies run on
    # two side streams, ordered by events: the next step's points go into the
    # other of two device buffers while this step computes, the projected
    # points, normals and status go back while the adjoint runs, the gradient
    # while the next step runs.  One timed region over all the steps, from the
    # first copy in to the last copy out (the L2 flush between steps included).
    host_in = torch.from_numpy(cloud.xyz).pin_memory()
    host_xyz = torch.empty((n_pts, 3), dtype=torch.float32).pin_memory()
    host_n = torch.empty((n_pts, 3), dtype=torch.float32).pin_memory()
    host_st = torch.empty(n_pts, dtype=torch.uint8).pin_memory()
    host_g = torch.empty((n_pts, 3), dtype=torch.float32).pin_memory()
    x_bufs = [torch.empty_like(x), torch.empty_like(x)]
    copy_in = torch.cuda.Stream(device=dev)
    copy_out = torch.cuda.Stream(device=dev)

    def e2e_run(n_steps):
        in_ready = [torch.cuda.Event(), torch.cuda.Event()]
        step_done = [None] * n_steps
        fwd_copied = [None] * n_steps
        grad_copied = [None] * n_steps
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        copy_in.wait_event(start)
        with torch.cuda.stream(copy_in):
            x_bufs[0].copy_(host_in, non_blocking=True)
        in_ready[0].record(copy_in)
        for s in range(n_steps):
            if s > 0:
                flush.zero_()
            stream.wait_event(in_ready[s % 2])
            if s + 1 < n_steps:
                if s > 0:                   # the other buffer is free once the previous step is done
                    copy_in.wait_event(step_done[s - 1])
                with torch.cuda.stream(copy_in):
                    x_bufs[(s + 1) % 2].copy_(host_in, non_blocking=True)
                in_ready[(s + 1) % 2].record(copy_in)

            def wait_fwd_copy(s=s):
                if s > 0: stream.wait_event(fwd_copied[s - 1])

            def copy_fwd(s=s):
                ev = torch.cuda.Event()
                ev.record(stream)
                copy_out.wait_event(ev)
                with torch.cuda.stream(copy_out):
                    host_xyz.copy_(out_xyz, non_blocking=True)
                    host_n.copy_(out_n, non_blocking=True)
                    host_st.copy_(out_st, non_blocking=True)
                fwd_copied[s] = torch.cuda.Event()
                fwd_copied[s].record(copy_out)

            def wait_grad_copy(s=s):
                if s > 0: stream.wait_event(grad_copied[s - 1])

            step(x_bufs[s % 2], before_forward_out=wait_fwd_copy, after_forward=copy_fwd,
                 before_backward=wait_grad_copy)
            step_done[s] = torch.cuda.Event()
            step_done[s].record(stream)
            copy_out.wait_event(step_done[s])
            with torch.cuda.stream(copy_out):
                host_g.copy_(grad, non_blocking=True)
            grad_copied[s] = torch.cuda.Event()
            grad_copied[s].record(copy_out)
        stream.wait_event(grad_copied[n_steps - 1])
        end.record(stream)
        end.synchronize()
        return start.elapsed_time(end) / n_steps

    e2e_run(2)                                  # warms the copy path
    e2e_ms = [e2e_run(min(max(args.steps, 3), 10))]
    (e2e_step_ms,) = max_over_ranks([float(np.mean(e2e_ms))], dev)
    e2e_value = job_throughput(world, n_pts, e2e_step_ms)

    # the form with the weights about q (Sec. 1.4, Eq. 1), same rows and h
    grid = capi.mls_build_grid(x, 0.0, K, grid=grid)
    capi.mls_knn(grid, K, out_idx=idx)
    order = capi.mls_grid_order(grid)
    lv = [torch.empty_like(x), torch.empty_like(x), torch.empty(n_pts, dtype=torch.uint8, device=dev)]
    for _ in range(2):
        capi.mls_project_levin(x, idx, h, 2, "mixed", max_iter=32, tol=1e-6, order=order, out_xyz=lv[0], out_normal=lv[1],
                               out_status=lv[2])
    lv_ms = []
    for _ in range(5):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        capi.mls_project_levin(x, idx, h, 2, "mixed", max_iter=32, tol=1e-6, order=order, out_xyz=lv[0], out_normal=lv[1],
                               out_status=lv[2])
        b.record(stream)
        b.synchronize()
        lv_ms.append(a.elapsed_time(b))
    lv_not_conv = float(((lv[2] & 8) != 0).float().mean().item())

    # the paper's own neighbourhood: every point within R (about 32 on the
    # torus surface), the projection over those rows, the outliers dropped
    R_ball = 0.008
    rd_ms = []
    for rep in range(4):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        off_r, rows_r, _ = capi.mls_radius_neighbors(grid, R_ball)
        _, _, st_r = capi.mls_project_rows(x, off_r, rows_r, R_ball, 2, "mixed", 3, order=order)
        kept_r = capi.mls_compact(st_r, capi.MLS_PT_OUTLIER)
        b.record(stream)
        b.synchronize()
        if rep:
            rd_ms.append(a.elapsed_time(b))
    rd_mean_nb = float(off_r[-1].item()) / n_pts
    rd_kept = int(kept_r.shape[0])

    # the kNN and the projection in one pass (rows kept on chip, not
    # written), on the same grid and h, against the timed step's two passes
    fz = [torch.empty_like(x), torch.empty_like(x), torch.empty(n_pts, dtype=torch.uint8, device=dev)]
    for _ in range(2):
        capi.mls_knn_project(grid, K, h, 2, "mixed", out_xyz=fz[0], out_normal=fz[1], out_status=fz[2])
    fz_ms = []
    for _ in range(5):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        capi.mls_knn_project(grid, K, h, 2, "mixed", out_xyz=fz[0], out_normal=fz[1], out_status=fz[2])
        b.record(stream)
        b.synchronize()
        fz_ms.append(a.elapsed_time(b))
    grid.close()
    del pos
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return None

    peaks = load_peaks(sms)
    clk = clocks.summary()
    mhz = clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    kernels = stage_kernels(n_pts, K, build_ms, knn_ms, proj_ms, bwd_ms, peaks, mhz)
    kernels["knn_project_pipelined"] = {
        "ms": knn_proj_ms, "calls": "mls_knn_project_sorted (the timed step's kNN and projection in one call)",
        "two_calls_ms": knn_ms + proj_ms,
        "note": "knn and project above are the same work as two calls (mls_knn_sorted, mls_project_sorted), timed "
                "in as many extra steps right after the timed ones; the pipelined call overlaps the projection of "
                "the points the kNN's first pass finished with its second (sparse) pass"}
    roofline = dict(kernels["knn"]["roofline_hbm"])
    roofline["issue"] = kernels["knn"]["roofline_issue"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "points/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if n_pts == N_POINTS else
                   WORKLOAD.replace("2,000,000", f"{n_pts:,}").replace("torus2m", "torus") + " (profiling size)",
                   "points_per_gpu": n_pts, "k": K, "degree": 2, "precision": "mixed",
                   "h": h, "step": ("grid build + exact kNN (rows by sorted position) and MLS projection saving "
                                    "the fit state, pipelined in one call, + the adjoint from that state, in the "
                                    "grid's order (fwd+bwd)"),
                   "l2": "flushed before every step (256 MB write, outside the timed events)",
                   "parallelism": f"independent clouds per GPU x{world}"},
        "fwd": {"value": job_throughput(world, n_pts, fwd_ms), "unit": "points/s", "ms_per_step": fwd_ms,
                "step": "grid build + exact kNN + MLS projection"},
        "wall": {"ms_per_step": wall_ms, "value": job_throughput(world, n_pts, wall_ms), "unit": "points/s",
                 "note": ("host clock around the timed loop / steps: adds to the events the L2 flush, the "
                          "Python launch of each step's calls and the host side of mls_build_grid's one "
                          "stream synchronisation (its level sizes are read back)")},
        "roofline": roofline,
        "kernels": kernels,
        "knn_deferred_frac": deferred / n_pts,
        "levin": {"ms": float(np.median(lv_ms)), "points_per_s": n_pts / (float(np.median(lv_ms)) * 1e-3),
                  "step": "mls_project_levin (weights about q, fixed point from q = r, tol 1e-6 h, <= 32 passes), "
                          "mixed, degree 2, same rows and h",
                  "not_converged_frac": lv_not_conv},
        "radius": {"ms": float(np.median(rd_ms)), "points_per_s": n_pts / (float(np.median(rd_ms)) * 1e-3),
                   "step": f"mls_radius_count + mls_radius_rows + mls_project_rows + mls_compact, R = h = {R_ball}, "
                           "mixed, degree 2, outliers (< 3 neighbours) dropped; on the already built grid",
                   "mean_neighbours": rd_mean_nb, "kept": rd_kept},
        "fused": {"ms": float(np.median(fz_ms)), "points_per_s": n_pts / (float(np.median(fz_ms)) * 1e-3),
                  "two_pass_ms": knn_ms + proj_ms,
                  "step": "mls_knn_project: exact kNN + MLS projection in one pass (each warp projects its last 32 "
                          "queries from an L2-resident row buffer; rows not written), mixed, degree 2, same grid "
                          "and h; two_pass_ms = mls_knn_sorted + mls_project_sorted as separate calls"},
        "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": n_pts * 12,
                "d2h_bytes_per_step": n_pts * (12 + 12 + 1 + 12)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s_timed_region": wall,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cloud.xyz, h, args.cpu_sample)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(cloud.xyz, h, args.cpu_sample)
    del cloud, x, idx, out_xyz, out_n, out_st, grad, gp, gn
    torch.cuda.empty_cache()
    if world == 1:
        line["sphere20k_k20"] = run_latency(args, dev)
    if world == 1 and not args.no_scan:
        line["scan50m_k64"] = run_scan(args, dev, peaks, flush)
    if world == 1 and not args.no_differentiable:
        line["bumpy1m_k32"] = run_differentiable(args, dev, peaks, flush)
    if world == 1 and not args.no_batched:
        line["batched"] = run_batched(args, dev)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return line


def stage_kernels(n, k, build_ms, knn_ms, proj_ms, bwd_ms, peaks, mhz):
    """Per-stage times and roofline fractions of one step over n points."""
    knn_gbs = n * knn_bytes(k) / (knn_ms * 1e-3) / 1e9
    proj_tf = n * proj_flops(k, state=True) / (proj_ms * 1e-3) / 1e12
    bwd_tf = n * bwd_flops(k, state=True) / (bwd_ms * 1e-3) / 1e12
    inst = knn_measured("warp_inst_per_query", n) if k == K else None
    issue_peak = peaks["issue_ginst_per_mhz"] * mhz          # G warp instructions / s
    issue = {"bound": "issue", "unit": "G warp-inst/s", "peak": issue_peak,
             "peak_source": f"derived: {peaks['sms']} SM x 4 schedulers x 1 inst/cycle x {mhz:.0f} MHz "
                            "(median SM clock sampled in the timed region)",
             "warp_inst_per_query": None if inst is None else inst / n,
             "achieved": None if inst is None else inst / (knn_ms * 1e-3) / 1e9}
    issue["frac"] = None if inst is None else issue["achieved"] / issue_peak
    return {
        "grid_build": {"ms": build_ms, "calls": "mls_build_grid",
                       "achieved_gbs": n * GRID_BYTES_PER_POINT / (build_ms * 1e-3) / 1e9},
        "knn": {"ms": knn_ms, "calls": "mls_knn_sorted (k_knn_chain + k_knn_sparse)",
                "roofline_hbm": {"kernel": "mls_knn_sorted (k_knn_chain + k_knn_sparse)", "bound": "hbm",
                                 "achieved": knn_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": knn_gbs / peaks["hbm_gbs"],
                                 "traffic": knn_measured("traffic_bytes_per_query", n) if k == K else None,
                                 "peak_source": f"{peaks['source']} hbm_gbs (copy)",
                                 "algorithmic_bytes_per_point": knn_bytes(k)},
                "roofline_issue": issue},
        "project": {"ms": proj_ms, "calls": "mls_project_sorted (k_project + k_project_deferred), fit state saved", "bound": "alu",
                    "flops_per_point": proj_flops(k, state=True), "achieved_tflops": proj_tf,
                    "frac": proj_tf / peaks["fp32_tflops"]},
        "backward": {"ms": bwd_ms, "calls": "mls_project_backward_sorted from the saved fit state and the bucket offsets of the pipelined call (adjoint, bucket sums)",
                     "bound": "alu", "flops_per_point": bwd_flops(k, state=True), "achieved_tflops": bwd_tf,
                     "frac": bwd_tf / peaks["fp32_tflops"]},
        "fp32_peak_tflops": peaks["fp32_tflops"],
        "fp32_peak_source": f"derived: {peaks['sms']} SM (from the device) x 128 FP32 lanes x 2 flops x max SM clock",
    }


def _timed_stages(fns, reps, stream, flush=None):
    """Runs the stage callables in sequence `reps` times with CUDA events
    between them; returns the mean ms of each stage."""
    import torch
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)] for _ in range(reps)]
    for r in range(reps):
        if flush is not None:
            flush.zero_()
        ev[r][0].record(stream)
        for i, f in enumerate(fns):
            f()
            ev[r][i + 1].record(stream)
    torch.cuda.synchronize()
    return [float(np.mean([ev[r][i].elapsed_time(ev[r][i + 1]) for r in range(reps)])) for i in range(len(fns))]


def run_latency(args, dev):
    """The small workload (20,000 points on a noisy unit sphere, k = 20,
    mixed): the latency of one whole step (grid build + kNN + projection
    saving the fit state + adjoint from it), from CUDA events on the stream
    and from the host clock (which adds the launches and the grid build's one
    stream synchronisation); the cloud stays in L2 between steps."""
    import torch

    from paper_2401_03365_gb300 import capi, workloads
    c = workloads.sphere()
    n, k = c.n, c.k
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(c.xyz).to(dev)
    grid = capi.mls_build_grid(x, 0.0, k)
    idx, _ = capi.mls_knn(grid, k)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    del idx
    pos = torch.empty((n, k), dtype=torch.int32, device=dev)
    out = [torch.empty_like(x), torch.empty_like(x), torch.empty(n, dtype=torch.uint8, device=dev)]
    fit_state = torch.empty((capi.FIT_STATE_FLOATS, n), dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev).manual_seed(5)
    gp = torch.randn(n, 3, device=dev, generator=gen)
    gn = 0.1 * torch.randn(n, 3, device=dev, generator=gen)
    grad = torch.empty_like(x)
    grad_h = torch.empty(1, dtype=torch.float32, device=dev)
    state = {"grid": grid}

    def step(ev=None):
        if ev: ev[0].record(stream)
        state["grid"] = capi.mls_build_grid(x, 0.0, k, grid=state["grid"])
        if ev: ev[1].record(stream)
        capi.mls_knn_sorted(state["grid"], k, out_pos=pos)
        if ev: ev[2].record(stream)
        capi.mls_project_sorted(state["grid"], pos, h, 2, "mixed", out_xyz=out[0], out_normal=out[1],
                                out_status=out[2], with_state=True, out_state=fit_state)
        if ev: ev[3].record(stream)
        capi.mls_project_backward_sorted(state["grid"], pos, h, gp, gn, 2, "mixed", out_grad_xyz=grad,
                                         out_grad_h=grad_h, state=fit_state)
        if ev: ev[4].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    steps = max(args.steps, 20)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
    wall = []
    for s in range(steps):
        t0 = time.perf_counter()
        step(evs[s])
        evs[s][4].synchronize()
        wall.append((time.perf_counter() - t0) * 1e3)
    stage = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in evs])
    state["grid"].close()
    ms = float(np.median(stage.sum(1)))
    return {"workload": "sphere20k_k20: 20,000 points on a unit sphere, radial noise 0.01, k=20, h = 2 x mean kNN "
                        "distance, degree 2, mixed",
            "ms_per_step": ms, "value": n / (ms * 1e-3), "unit": "points/s", "steps": steps,
            "host_ms_per_step": float(np.median(wall)),
            "stages_ms": {name: float(np.median(stage[:, i])) for i, name in
                          enumerate(("grid_build", "knn", "project", "backward"))},
            "step": "grid build + exact kNN + projection (fit state saved) + adjoint from it, one step at a time "
                    "(median over the steps); host_ms_per_step: host clock from the first call to the step's end",
            "l2": "the cloud stays in L2 (20,000 points): a latency figure"}


def run_scan(args, dev, peaks, flush):
    """The scan-scale workload: 50M points on the height field of 8 random
    sinusoids over [0,1]^2 with a 10x sampling-density ramp, noise 0.002,
    k = 64, mixed precision; one forward step = grid build + exact kNN + the
    projection in the grid's order."""
    import torch

    from paper_2401_03365_gb300 import capi, workloads
    t0 = time.perf_counter()
    c = workloads.heightfield()
    t_gen = time.perf_counter() - t0
    n, k = c.n, c.k
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(c.xyz).to(dev)
    grid = capi.mls_build_grid(x, 0.0, k)
    idx, _ = capi.mls_knn(grid, k)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    del idx
    pos = torch.empty((n, k), dtype=torch.int32, device=dev)
    out = [torch.empty_like(x), torch.empty_like(x), torch.empty(n, dtype=torch.uint8, device=dev)]
    state = {"grid": grid}

    def build():
        state["grid"] = capi.mls_build_grid(x, 0.0, k, grid=state["grid"])

    def knn():
        capi.mls_knn_sorted(state["grid"], k, out_pos=pos)

    def project():
        capi.mls_project_sorted(state["grid"], pos, h, 2, "mixed", out_xyz=out[0], out_normal=out[1],
                                out_status=out[2])

    steps = max(3, min(args.steps, 5))
    _timed_stages([build, knn, project], args.warmup, stream)
    build_ms, knn_ms, proj_ms = _timed_stages([build, knn, project], steps, stream)
    deferred = capi.mls_knn_deferred(state["grid"])
    regular = float(((out[2] & 3) == 0).float().mean().item())
    state["grid"].close()
    step_ms = build_ms + knn_ms + proj_ms
    kernels = stage_kernels(n, k, build_ms, knn_ms, proj_ms, float("nan"), peaks,
                            float(peaks.get("sm_max_mhz", 2070.0)))
    kernels.pop("backward")
    line = {"workload": ("heightfield50m_k64: 50,000,000 points on z = sum of 8 random sinusoids over [0,1]^2, "
                         "density ramp 1+9x, noise 0.002, k=64, h = 2 x mean kNN distance, degree 2, mixed"),
            "value": n / (step_ms * 1e-3), "unit": "points/s", "ms_per_step": step_ms, "steps": steps,
            "step": "grid build + exact kNN (rows by sorted position) + MLS projection in the grid's order",
            "l2": "inputs far larger than L2 (0.6 GB of points, 12.8 GB of rows); no flush",
            "h": h, "regular_frac": regular, "knn_deferred_frac": deferred / n, "kernels": kernels,
            "setup_s": {"generate": t_gen}}
    del x, pos, out
    torch.cuda.empty_cache()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_scan(c.xyz, k, h)
    return line


def cpu_baseline_scan(xyz, k, h, sub=5_000_000, sample=20_000):
    """The oracle on a bounded sample of the 50M-point cloud: its k-d tree
    over a seeded 5M-point subset (time scaled to the whole cloud by n log n)
    and the kNN + FP64 projection of 20,000 sampled queries against it (time
    per query scaled to every point)."""
    import oracle
    n = xyz.shape[0]
    rng = np.random.default_rng(77)
    part = np.ascontiguousarray(xyz[np.sort(rng.choice(n, sub, replace=False))])
    t0 = time.perf_counter()
    oracle.knn_kdtree(part, k, queries=np.zeros(0, np.int64))
    t_build = time.perf_counter() - t0
    q = np.sort(rng.choice(sub, sample, replace=False))
    t0 = time.perf_counter()
    rows, _ = oracle.knn_kdtree(part, k, queries=q)
    t_knn = time.perf_counter() - t0 - t_build
    t0 = time.perf_counter()
    oracle.project(part, rows, h, 2, queries=q)
    t_proj = time.perf_counter() - t0
    t_full = t_build * (n * np.log2(n)) / (sub * np.log2(sub)) + (t_knn + t_proj) * n / sample
    return {"value": n / t_full, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": (f"k-d tree over a seeded {sub:,}-point subset ({t_build:.1f} s, scaled by n log n to the "
                       f"{n:,} points) + kNN ({t_knn:.2f} s) and FP64 projection ({t_proj:.2f} s) of {sample:,} "
                       f"sampled queries, scaled to every point"),
            "seconds": t_build + t_knn + t_proj}


def run_differentiable(args, dev, peaks, flush):
    """The differentiable workload: 1M points on a sphere with 64 Gaussian
    bumps, k = 32, FP32 forward and backward of the loss
    L = sum_i (|p'_i| - rho(p'_i / |p'_i|))^2 (the squared radial residual of
    every projected point to the analytic surface) with respect to the
    coordinates and h, through the autograd Function.  One step = grid build
    + kNN + projection + loss + backward (the adjoint kernels and the loss's
    own gradient)."""
    import torch

    from paper_2401_03365_gb300 import capi, mls, workloads
    c = workloads.bumpy_sphere()
    n, k = c.n, c.k
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(c.xyz).to(dev)
    centres = torch.as_tensor(c.meta["centres"], dtype=torch.float32, device=dev)
    amps = torch.as_tensor(c.meta["amps"], dtype=torch.float32, device=dev)
    widths = torch.as_tensor(c.meta["widths"], dtype=torch.float32, device=dev)
    grid = capi.mls_build_grid(x, 0.0, k)
    idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    pos = torch.empty((n, k), dtype=torch.int32, device=dev)
    capi.mls_knn(grid, k, out_idx=idx)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    state = {"grid": grid}

    def loss_of(p):
        r = p.norm(dim=1)
        u = p / r[:, None]
        rho = 1.0 + (amps[None, :] * torch.exp(-(1.0 - u @ centres.T) / widths[None, :] ** 2)).sum(1)
        return ((r - rho) ** 2).sum()

    def build():
        state["grid"] = capi.mls_build_grid(x, 0.0, k, grid=state["grid"])

    def knn():
        capi.mls_knn_sorted(state["grid"], k, out_pos=pos)

    def fwd():
        state["xg"] = x.detach().requires_grad_(True)
        state["h"] = torch.tensor(h, dtype=torch.float32, device=dev, requires_grad=True)
        order = capi.mls_grid_order(state["grid"])
        out, _, _ = mls.project_differentiable(state["xg"], idx, state["h"], 2, "fp32", order=order,
                                               grid=state["grid"], pos=pos)
        state["loss"] = loss_of(out)

    def bwd():
        state["loss"].backward()

    steps = max(args.steps, 5)
    _timed_stages([build, knn, fwd, bwd], args.warmup, stream, flush)
    build_ms, knn_ms, fwd_ms, bwd_ms = _timed_stages([build, knn, fwd, bwd], steps, stream, flush)
    gx = state["xg"].grad
    finite = bool(torch.isfinite(gx).all().item()) and bool(torch.isfinite(state["h"].grad).all().item())
    state["grid"].close()
    step_ms = build_ms + knn_ms + fwd_ms + bwd_ms
    kernels = stage_kernels(n, k, build_ms, knn_ms, fwd_ms, bwd_ms, peaks, float(peaks.get("sm_max_mhz", 2070.0)))
    kernels["project"]["calls"] += " + the loss (torch ops)"
    kernels["backward"]["calls"] += " + the loss's gradient (torch autograd)"
    line = {"workload": ("bumpy1m_k32: 1,000,000 points on a sphere with 64 Gaussian bumps, noise 0.005, k=32, "
                         "h = 2 x mean kNN distance, degree 2, FP32; loss sum (|p'| - rho(p'/|p'|))^2"),
            "value": n / (step_ms * 1e-3), "unit": "points/s", "ms_per_step": step_ms, "steps": steps,
            "step": "grid build + kNN + projection (autograd Function) + loss + backward to xyz and h",
            "l2": "flushed before every step (256 MB write, outside the timed events)",
            "h": h, "gradients_finite": finite, "kernels": kernels}
    del x, idx, pos, state
    torch.cuda.empty_cache()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_differentiable(c, h)
    return line


def cpu_baseline_differentiable(c, h, sample=20_000):
    """The oracle on a bounded sample of the bumpy-sphere workload: its k-d
    tree over the whole cloud, then kNN, FP64 projection and FP64 adjoint of
    a seeded 20,000-point sample (with the loss's cotangent at the oracle's
    own outputs), scaled to every point."""
    import oracle
    from paper_2401_03365_gb300 import workloads
    n, k = c.n, c.k
    rng = np.random.default_rng(78)
    q = np.sort(rng.choice(n, sample, replace=False))
    t0 = time.perf_counter()
    oracle.knn_kdtree(c.xyz, k, queries=np.zeros(0, np.int64))
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    rows, _ = oracle.knn_kdtree(c.xyz, k, queries=q)
    o_xyz, _, _, _ = oracle.project(c.xyz, rows, h, 2, queries=q)
    # the cotangent's radial part 2 (|p'| - rho) p' / |p'| (only timed: the
    # oracle's cost does not depend on the cotangent's values)
    r = np.linalg.norm(o_xyz, axis=1)
    rho = workloads.bumpy_radius(o_xyz / r[:, None], c.meta["centres"], c.meta["amps"], c.meta["widths"])
    gp = np.zeros((n, 3))
    gp[q] = (2.0 * (r - rho) / r)[:, None] * o_xyz
    oracle.project_grad(c.xyz, rows, h, 2, gp, queries=q)
    t_sample = time.perf_counter() - t0 - t_build
    t_full = t_build + t_sample * n / sample
    return {"value": n / t_full, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": (f"k-d tree over all {n:,} points ({t_build:.2f} s) + kNN, FP64 projection, loss cotangent "
                       f"and FP64 adjoint of a seeded {sample:,}-point sample ({t_sample:.2f} s), scaled to every "
                       "point"),
            "seconds": t_build + t_sample}


def run_batched(args, dev):
    """The batched form on 256 clouds (ellipsoids and superquadrics, sizes
    log-uniform in 1e3..5e5, k in {16, 32, 64}): one graph replay of the
    autotuned persistent mixed-precision launch against 256 per-cloud launches
    of the plain FP64 projection, on the same rows and h."""
    import torch

    from paper_2401_03365_gb300 import capi, workloads
    from paper_2401_03365_gb300.batched import BatchedProjector, TuneCache

    t0 = time.perf_counter()
    clouds = workloads.batch_clouds(workers=min(os.cpu_count() or 1, 16))
    t_gen = time.perf_counter() - t0
    xs = [torch.from_numpy(c.xyz).to(dev) for c in clouds]
    bp = BatchedProjector.from_clouds(xs, [c.k for c in clouds])
    total = bp.batch.total
    import tempfile
    cache = TuneCache(os.path.join(tempfile.gettempdir(), "mls_autotune_bench.json"))
    tuned = bp.tune(cache=cache, reps=2, retune=True)
    bp.capture()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        bp.replay()
    torch.cuda.synchronize()
    steps = max(args.steps, 5)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(steps):
        bp.replay()
    ev[1].record(stream)
    torch.cuda.synchronize()
    batched_ms = ev[0].elapsed_time(ev[1]) / steps

    # the plain FP64 form, one launch per cloud, into its own outputs
    f_xyz = torch.empty_like(bp.xyz)
    f_n = torch.empty_like(bp.xyz)
    f_st = torch.empty(total, dtype=torch.uint8, device=dev)
    views = []
    for c, cl in enumerate(clouds):
        a, e = bp.batch.offsets[c], bp.batch.offsets[c + 1]
        views.append((bp.xyz[a:e], bp.idx[bp.batch.idx_offset(c):bp.batch.idx_offset(c + 1)].view(e - a, cl.k),
                      float(bp.h[c].item()), bp.order[a:e], f_xyz[a:e], f_n[a:e], f_st[a:e]))

    def fp64_pass():
        for x, idx, h, order, ox, on, os_ in views:
            capi.mls_project(x, idx, h, 2, "fp64", order=order, out_xyz=ox, out_normal=on, out_status=os_)

    fp64_pass()
    torch.cuda.synchronize()
    reps = 2
    ev[0].record(stream)
    for _ in range(reps):
        fp64_pass()
    ev[1].record(stream)
    torch.cuda.synchronize()
    fp64_ms = ev[0].elapsed_time(ev[1]) / reps

    # accuracy of the batched mixed form against the FP64 form, per cloud in
    # units of its bounding-box diagonal, on points both call regular
    devs = []
    for c in range(len(clouds)):
        a, e = bp.batch.offsets[c], bp.batch.offsets[c + 1]
        x = bp.xyz[a:e]
        diag = float((x.max(0).values - x.min(0).values).norm())
        ok = ((bp.out_status[a:e] & 3) == 0) & ((f_st[a:e] & 3) == 0)
        d = ((bp.out_xyz[a:e] - f_xyz[a:e]).double().norm(dim=1) / diag)[ok]
        devs.append(d)
    devs = torch.cat(devs)
    acc = {"max": float(devs.max()), "p99_99": float(torch.quantile(devs[:: max(1, devs.numel() // 1_000_000)],
                                                                     0.9999)),
           "frac_within_1e-5": float((devs <= 1e-5).double().mean())}
    ks = [c.k for c in clouds]
    out = {
        "workload": (f"batch256: {len(clouds)} clouds, {total:,} points, k=16/32/64 on {ks.count(16)}/"
                     f"{ks.count(32)}/{ks.count(64)} clouds, degree 2, per-cloud h = 2 x mean kNN distance"),
        "value": total / (batched_ms * 1e-3), "unit": "points/s", "ms": batched_ms,
        "form": "one CUDA-graph replay: memset + float4 pack + persistent kernel, mixed precision",
        "shape": {"lanes_per_point": tuned["shape"][0], "threads": tuned["shape"][1],
                  "rounds": tuned["shape"][2]},
        "autotune_ms": {f"{g}x{t}x{r}": round(ms, 4) for g, t, r, ms in tuned["table"]},
        "fp64_per_cloud": {"value": total / (fp64_ms * 1e-3), "unit": "points/s", "ms": fp64_ms,
                           "form": f"{len(clouds)} mls_project launches, precision fp64"},
        "speedup_vs_fp64_per_cloud": fp64_ms / batched_ms,
        "deviation_from_fp64_in_diag": acc,
        "setup_s": {"generate": t_gen},
    }
    bp.close()
    return out


def cpu_baseline(xyz, h, sample):
    """The FP64 oracle as it stands, single-threaded on this host: k-d tree over
    the whole cloud, then kNN, projection and adjoint of a seeded sample of
    points; the per-point time is extrapolated to the full cloud."""
    import oracle
    n = xyz.shape[0]
    rng = np.random.default_rng(123)
    q = np.sort(rng.choice(n, sample, replace=False))
    gp = rng.standard_normal((n, 3))
    gn = 0.1 * rng.standard_normal((n, 3))
    t0 = time.perf_counter()
    oracle.knn_kdtree(xyz, K, queries=np.zeros(0, np.int64))
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    rows, _ = oracle.knn_kdtree(xyz, K, queries=q)
    oracle.project(xyz, rows, h, 2, queries=q)
    oracle.project_grad(xyz, rows, h, 2, gp, gn, queries=q)
    t_sample = time.perf_counter() - t0 - t_build
    t_full = t_build + t_sample * n / sample
    return {"value": n / t_full, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": (f"k-d tree build over all {n} points ({t_build:.2f} s) + kNN, FP64 projection and FP64 "
                       f"adjoint of a seeded sample of {sample} points ({t_sample:.2f} s), extrapolated to the "
                       f"full cloud"),
            "seconds": t_build + t_sample}


def _oracle_chunk(xyz, h, queries, seed):
    """One worker of the all-cores baseline: the oracle's own k-d tree over
    the whole cloud, then kNN, projection and adjoint of its queries."""
    import oracle
    n = xyz.shape[0]
    rng = np.random.default_rng(seed)
    gp = rng.standard_normal((n, 3))
    gn = 0.1 * rng.standard_normal((n, 3))
    t0 = time.perf_counter()
    oracle.knn_kdtree(xyz, K, queries=np.zeros(0, np.int64))
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    rows, _ = oracle.knn_kdtree(xyz, K, queries=queries)
    oracle.project(xyz, rows, h, 2, queries=queries)
    oracle.project_grad(xyz, rows, h, 2, gp, gn, queries=queries)
    return t_build, time.perf_counter() - t0


def cpu_baseline_all_cores(xyz, h, sample):
    """The same single-threaded oracle in one process per host core, each on
    its share of the sample (the per-point loop of Algorithm 1 split over
    cores); the full cloud's time is the tree build plus each core's share of
    the points at the measured per-point time."""
    import multiprocessing as mp
    n = xyz.shape[0]
    cores = max(1, os.cpu_count() or 1)
    rng = np.random.default_rng(123)
    q = np.sort(rng.choice(n, sample, replace=False))
    parts = np.array_split(q, cores)
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_chunk, [(xyz, h, p, 7 + i) for i, p in enumerate(parts)])
    wall = time.perf_counter() - t0
    build = max(r[0] for r in res)
    per_point = sum(r[1] for r in res) / sample          # seconds of one core per point
    t_full = build + per_point * n / cores
    return {"value": n / t_full, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": (f"{cores} processes, each: k-d tree over all {n} points + kNN, FP64 projection and FP64 "
                       f"adjoint of its share of a {sample}-point sample; full cloud extrapolated as build + "
                       f"n / cores x the per-point time"), "seconds": wall}


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return None
    from paper_2401_03365_gb300 import workloads
    cloud = workloads.torus(n=N_POINTS, seed=2, k=K)
    import oracle
    # the bandwidth as the oracle defines it, from a seeded sample of its rows
    rng = np.random.default_rng(5)
    q = np.sort(rng.choice(N_POINTS, 20_000, replace=False))
    rows, _ = oracle.knn_kdtree(cloud.xyz, K, queries=q)
    xd = cloud.xyz.astype(np.float64)
    d = np.linalg.norm(xd[rows] - xd[q][:, None, :], axis=2)
    h = float(np.float32(2.0 * d[rows != q[:, None]].mean()))
    for _ in range(args.warmup):
        cpu_baseline(cloud.xyz, h, 1_000)
    times = []
    measured = []
    info = None
    for _ in range(args.steps):
        info = cpu_baseline(cloud.xyz, h, args.ref_sample)
        times.append(N_POINTS / info["value"])
        measured.append(info["seconds"])
    step_s = float(np.mean(times))
    value = N_POINTS / step_s
    return {
        "metric": METRIC, "impl": "reference", "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_gpu": N_POINTS, "k": K, "degree": 2,
                   "step": "oracle: k-d tree + kNN + FP64 projection + FP64 adjoint, sampled and extrapolated"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle", "sample": info["sample"]},
        "measured_s_per_sampled_step": float(np.mean(measured)),
        "ms_per_step_is": ("the full cloud's time extrapolated from each step's sample (tree over all points, "
                           f"{args.ref_sample:,} queries); the sampled step itself took measured_s_per_sampled_step"),
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample", type=int, default=300_000,
                    help="sampled queries of the cpu_baseline leg (about 10 s of oracle work)")
    ap.add_argument("--ref-sample", type=int, default=100_000,
                    help="sampled queries per step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-cloud batched measurement")
    ap.add_argument("--no-scan", action="store_true", help="skip the 50M-point height-field measurement")
    ap.add_argument("--no-differentiable", action="store_true", help="skip the 1M-point fwd+bwd loss measurement")
    ap.add_argument("--points", type=int, default=N_POINTS,
                    help="cloud size; smaller than the default only for profiling captures")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)     # at least three untimed warm-up steps
    line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
