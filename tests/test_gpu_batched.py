"""Batched projection (mls_project_batched, one persistent launch over many
clouds of uneven size and k) against the FP64 oracle cloud by cloud, for every
launch shape family; equal to mls_project at one lane per point; the captured
CUDA graph and the autotuner give the same outputs as a direct launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len, oracle_knn

pytestmark = pytest.mark.gpu

SHAPES = [(1, 128, 1), (1, 64, 4), (2, 64, 4), (4, 256, 1), (8, 128, 4), (32, 64, 1)]


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _clouds():
    """Six clouds of the batched workload's kind (ellipsoids and superquadrics,
    k in {16, 32, 64}) at test sizes, plus tiny clouds down to one point."""
    cl = workloads.batch_clouds(n_clouds=6, seed0=40, n_min=300, n_max=6000)
    rng = np.random.default_rng(41)
    xyz = [c.xyz for c in cl] + [rng.standard_normal((n, 3)).astype(np.float32) for n in (1, 2, 7)]
    ks = [c.k for c in cl] + [1, 2, 7]
    return xyz, ks


@pytest.fixture(scope="module")
def batch_case():
    """Per cloud: the oracle's rows, h, projection; plus a Morton-free random
    processing order (a permutation per cloud)."""
    xyz, ks = _clouds()
    rng = np.random.default_rng(42)
    rows, hs, outs, orders = [], [], [], []
    for x, k in zip(xyz, ks):
        idx, _ = oracle_knn(x, k)
        h = float(np.float32(2.0 * oracle.mean_knn_dist(x, idx))) if k > 1 else 1.0
        rows.append(idx)
        hs.append(h)
        outs.append(oracle.project(x, idx, h, 2))
        orders.append(rng.permutation(x.shape[0]).astype(np.int32))
    return xyz, ks, rows, hs, outs, orders


def _device_inputs(xyz, rows, hs, orders):
    x = torch.from_numpy(np.concatenate(xyz)).cuda()
    idx = torch.from_numpy(np.concatenate([r.reshape(-1) for r in rows]).astype(np.int32)).cuda()
    h = torch.tensor(hs, dtype=torch.float32, device="cuda")
    order = torch.from_numpy(np.concatenate(orders)).cuda()
    return x, idx, h, order


def _check_against_oracle(xyz, outs, offsets, g_xyz, g_n, g_st):
    for c, (x, o) in enumerate(zip(xyz, outs)):
        a, b = offsets[c], offsets[c + 1]
        if x.shape[0] < 8:          # too few points for a well-posed fit: statuses and fallbacks only
            assert np.array_equal(g_st[a:b] & 3, o[2])
            deg = (o[2] & 1) == 1
            assert np.array_equal(g_xyz[a:b][deg], x[deg])
            continue
        compare_projection(g_xyz[a:b], g_n[a:b], g_st[a:b], *o, diag_len(x), min_well_posed=0.3)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_batched_matches_oracle_per_cloud(capi, batch_case, shape, precision):
    xyz, ks, rows, hs, outs, orders = batch_case
    x, idx, h, order = _device_inputs(xyz, rows, hs, orders)
    offsets = np.concatenate([[0], np.cumsum([p.shape[0] for p in xyz])]).tolist()
    b = capi.mls_batch_create(offsets, ks)
    capi.mls_batch_set_shape(b, *shape)
    assert capi.mls_batch_get_shape(b) == shape
    g = capi.mls_project_batched(b, x, idx, h, 2, precision, order=order)
    torch.cuda.synchronize()
    _check_against_oracle(xyz, outs, offsets, *(t.cpu().numpy() for t in g))
    b.close()


def test_one_lane_per_point_equals_mls_project(capi, batch_case):
    """Same per-point arithmetic as the single-cloud kernel: bit-identical."""
    xyz, ks, rows, hs, outs, orders = batch_case
    x, idx, h, order = _device_inputs(xyz, rows, hs, orders)
    offsets = np.concatenate([[0], np.cumsum([p.shape[0] for p in xyz])]).tolist()
    b = capi.mls_batch_create(offsets, ks)
    capi.mls_batch_set_shape(b, 1, 128, 2)
    g_xyz, g_n, g_st = capi.mls_project_batched(b, x, idx, h, 2, "mixed", order=order)
    for c in range(len(xyz)):
        a, e = offsets[c], offsets[c + 1]
        xc = x[a:e].contiguous()
        ic = idx[b.idx_offset(c):b.idx_offset(c + 1)].reshape(e - a, ks[c])
        r_xyz, r_n, r_st = capi.mls_project(xc, ic, hs[c], 2, "mixed", order=order[a:e].contiguous())
        assert torch.equal(g_xyz[a:e], r_xyz)
        assert torch.equal(g_n[a:e], r_n)
        assert torch.equal(g_st[a:e], r_st)
    b.close()


@pytest.mark.parametrize("degree", [0, 1])
def test_lower_degrees(capi, batch_case, degree):
    xyz, ks, rows, hs, _, orders = batch_case
    x, idx, h, order = _device_inputs(xyz, rows, hs, orders)
    offsets = np.concatenate([[0], np.cumsum([p.shape[0] for p in xyz])]).tolist()
    b = capi.mls_batch_create(offsets, ks)
    capi.mls_batch_set_shape(b, 4, 128, 1)
    g = [t.cpu().numpy() for t in capi.mls_project_batched(b, x, idx, h, degree, "mixed", order=order)]
    outs = [oracle.project(p, r, hh, degree) for p, r, hh in zip(xyz, rows, hs)]
    _check_against_oracle(xyz, outs, offsets, *g)
    b.close()


def test_graph_replay_follows_new_point_data(capi, batch_case):
    xyz, ks, rows, hs, _, orders = batch_case
    x, idx, h, order = _device_inputs(xyz, rows, hs, orders)
    offsets = np.concatenate([[0], np.cumsum([p.shape[0] for p in xyz])]).tolist()
    b = capi.mls_batch_create(offsets, ks)
    capi.mls_batch_set_shape(b, 2, 128, 1)
    out = capi.mls_batch_capture(b, x, idx, h, 2, "mixed", order=order)
    launches = capi.mls_kernel_launches()
    for step in range(3):
        # new coordinates in the captured buffers: a rigid motion of every cloud
        th = 0.3 * (step + 1)
        R = torch.tensor([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]],
                         dtype=torch.float32, device="cuda")
        x.copy_(torch.from_numpy(np.concatenate(xyz)).cuda() @ R.T + step)
        capi.mls_batch_replay(b)
        ref = capi.mls_project_batched(b, x, idx, h, 2, "mixed", order=order)
        torch.cuda.synchronize()
        for got, want in zip(out, ref):
            assert torch.equal(got, want)
    assert capi.mls_kernel_launches() - launches == 3 * 2 + 3 * 2
    b.close()


def test_autotune_picks_a_candidate_and_leaves_its_results(capi, batch_case, tmp_path):
    from paper_2401_03365_gb300.batched import BatchedProjector, TuneCache
    xyz, ks, rows, hs, outs, orders = batch_case
    x, idx, h, order = _device_inputs(xyz, rows, hs, orders)
    offsets = np.concatenate([[0], np.cumsum([p.shape[0] for p in xyz])]).tolist()
    bp = BatchedProjector(x, idx, order, h, offsets, ks)
    cache = TuneCache(str(tmp_path / "tune.json"))
    info = bp.tune(cache=cache, reps=2)
    assert info["source"] == "autotune"
    assert len(info["table"]) == 4 * 3 * 2
    assert tuple(info["shape"]) in {t[:3] for t in info["table"]}
    assert min(t[3] for t in info["table"]) == [t[3] for t in info["table"] if t[:3] == tuple(info["shape"])][0]
    tuned = [t.clone() for t in (bp.out_xyz, bp.out_normal, bp.out_status)]
    again = bp.run()
    torch.cuda.synchronize()
    for a_, b_ in zip(tuned, again):
        assert torch.equal(a_, b_)
    _check_against_oracle(xyz, outs, offsets, *(t.cpu().numpy() for t in again))
    # a second projector of the same batch takes the shape from the cache
    bp2 = BatchedProjector(x, idx, order, h, offsets, ks)
    assert bp2.tune(cache=TuneCache(cache.path))["source"] == "cache"
    assert capi.mls_batch_get_shape(bp2.batch) == tuple(info["shape"])
    bp.close()
    bp2.close()


def test_from_clouds_uses_the_gpu_neighbours(capi):
    """The convenience path (per-cloud grid + kNN + h on the GPU) against the
    oracle on the same rows."""
    from paper_2401_03365_gb300.batched import BatchedProjector
    cl = workloads.batch_clouds(n_clouds=4, seed0=60, n_min=2000, n_max=20000)
    xs = [torch.from_numpy(c.xyz).cuda() for c in cl]
    bp = BatchedProjector.from_clouds(xs, [c.k for c in cl])
    bp.capture()
    bp.replay()
    torch.cuda.synchronize()
    for c, cloud in enumerate(cl):
        a, e = bp.batch.offsets[c], bp.batch.offsets[c + 1]
        rows = bp.idx[bp.batch.idx_offset(c):bp.batch.idx_offset(c + 1)].reshape(e - a, cloud.k).cpu().numpy()
        idx_o, _ = oracle_knn(cloud.xyz, cloud.k)
        assert np.array_equal(rows, idx_o)
        o = oracle.project(cloud.xyz, rows, float(bp.h[c].item()), 2)
        g = [t.cpu().numpy() for t in bp.cloud(c)]
        compare_projection(*g, *o, diag_len(cloud.xyz), min_well_posed=0.3)
    bp.close()


@pytest.mark.parametrize("shape", [(1, 128, 1), (2, 64, 4)])
def test_full_size_batch_clouds_sampled_against_oracle(capi, shape):
    """The largest clouds of the 256-cloud workload at full size (the two
    largest: 493k points at k = 32 and 472k at k = 16; the two largest with
    k = 64: 443k and 376k), in one batch at one and two lanes per point: the
    GPU rows of a seeded sample of 1,500 points per cloud are the oracle's
    k-d tree rows, and their projections match the oracle's."""
    from paper_2401_03365_gb300.batched import BatchedProjector
    sizes = [workloads.batch_cloud_size(b) for b in range(256)]
    big = sorted(range(256), key=lambda b: -sizes[b][0])[:2]
    big64 = sorted((b for b in range(256) if sizes[b][1] == 64), key=lambda b: -sizes[b][0])[:2]
    clouds = [workloads.batch_cloud(b) for b in big + big64]
    xs = [torch.from_numpy(c.xyz).cuda() for c in clouds]
    bp = BatchedProjector.from_clouds(xs, [c.k for c in clouds])
    capi.mls_batch_set_shape(bp.batch, *shape)
    bp.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(48)
    for c, cloud in enumerate(clouds):
        a, e = bp.batch.offsets[c], bp.batch.offsets[c + 1]
        q = np.sort(rng.choice(cloud.n, 1500, replace=False))
        rows_o, _ = oracle.knn_kdtree(cloud.xyz, cloud.k, queries=q)
        rows_g = bp.idx[bp.batch.idx_offset(c):bp.batch.idx_offset(c + 1)].reshape(e - a, cloud.k).cpu().numpy()
        assert np.array_equal(rows_g[q], rows_o)
        o = oracle.project(cloud.xyz, rows_o, float(bp.h[c].item()), 2, queries=q)
        g = [t.cpu().numpy()[q] for t in bp.cloud(c)]
        compare_projection(*g, *o, diag_len(cloud.xyz), min_well_posed=0.3)
    bp.close()
