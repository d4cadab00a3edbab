"""The sharding driver's GPU steps (GpuOps over libmls) on one rank: rows
equal to the oracle's, projection within the parity tolerances.  More
ranks run only as CPU processes here (tests/test_shard_cpu.py)."""
import numpy as np
import pytest

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len

pytestmark = pytest.mark.gpu


def test_gpu_ops_single_rank():
    from paper_2401_03365_gb300 import build, shard
    build.build()
    c = workloads.torus(n=60_000, seed=8, k=32)
    ops = shard.GpuOps()
    order = ops.morton_order(c.xyz, c.k)
    assert np.array_equal(np.sort(order), np.arange(c.n))
    rows_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = float(np.float32(2.0 * oracle.mean_knn_dist(c.xyz, rows_o)))
    ids = np.arange(c.n)
    res = shard.sharded_project(c.xyz, ids, c.k, h, ops)
    assert np.array_equal(res.rows, rows_o)
    o = oracle.project(c.xyz, rows_o, h, 2)
    compare_projection(res.xyz, res.normal, res.status, *o, diag_len(c.xyz), min_well_posed=0.3)
