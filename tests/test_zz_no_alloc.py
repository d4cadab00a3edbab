"""mls_project_noalloc: the projection for callers that cannot let the library
allocate device memory (hosts that hand out all memory from their own pool or
budget, loops where an allocation must not fail half way).  It keeps its
scratch in a fixed device array and must give what mls_project gives.

Named to be collected last: a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc(capi, x, idx, h, degree, precision, order):
    n, k = x.shape[0], idx.shape[1]
    out = torch.empty_like(x)
    nrm = torch.empty_like(x)
    st = torch.empty(n, dtype=torch.uint8, device=x.device)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = capi.lib().mls_project_noalloc(_p(x), n, _p(idx), k, float(h), degree, capi.PRECISION[precision],
                                        _p(order), _p(out), _p(nrm), _p(st), s)
    return rc, out, nrm, st


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_noalloc_matches_mls_project_on_consecutive_calls(capi, precision):
    clouds = [workloads.torus(n=150_000, seed=21), workloads.sphere(n=40_000, seed=22, k=20)]
    for c in clouds:           # two calls in a row share the scratch array
        x = torch.from_numpy(c.xyz).cuda()
        grid = capi.mls_build_grid(x, 0.0, c.k)
        idx, _ = capi.mls_knn(grid, c.k)
        order = capi.mls_grid_order(grid)
        h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
        ref_xyz, ref_n, ref_st = capi.mls_project(x, idx, h, 2, precision, order=order)
        rc, out, nrm, st = _noalloc(capi, x, idx, h, 2, precision, order)
        torch.cuda.synchronize()
        assert rc == 0, capi.mls_last_error()
        # the reference stands in for the oracle: same tolerance and mask rule
        # (here every point of the reference counts as well-posed)
        diag = np.tile([0.0, 1.0, 1.0, 1.0, 1.0], (c.n, 1))
        compare_projection(out.cpu().numpy(), nrm.cpu().numpy(), st.cpu().numpy(),
                           ref_xyz.cpu().numpy().astype(np.float64), ref_n.cpu().numpy().astype(np.float64),
                           ref_st.cpu().numpy() & 3, diag, diag_len(c.xyz))
        assert torch.equal(st, ref_st)
        grid.close()


def test_deferred_fp64_pass_is_bit_identical_to_inline(capi):
    """mls_project (mixed) finishes the points that need FP64 in a second,
    compact pass; the no-alloc form finishes them inline.  Same arithmetic:
    bit-identical outputs, and the cloud (1 % outliers) has such points."""
    c = workloads.torus(n=150_000, seed=23)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    idx, _ = capi.mls_knn(grid, c.k)
    order = capi.mls_grid_order(grid)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    for o in (order, None):
        ref_xyz, ref_n, ref_st = capi.mls_project(x, idx, h, 2, "mixed", order=o)
        rc, out, nrm, st = _noalloc(capi, x, idx, h, 2, "mixed", o)
        torch.cuda.synchronize()
        assert rc == 0, capi.mls_last_error()
        assert int(((ref_st & capi.MLS_PT_FP64_USED) != 0).sum()) > 0
        assert torch.equal(out, ref_xyz) and torch.equal(nrm, ref_n) and torch.equal(st, ref_st)
    grid.close()


def test_noalloc_rejects_clouds_beyond_its_scratch(capi):
    n = capi.MLS_NOALLOC_MAX_POINTS + 1
    x = torch.zeros((n, 3), device="cuda")
    idx = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    rc, *_ = _noalloc(capi, x, idx, 0.1, 2, "mixed", None)
    assert rc == -8
    assert "scratch" in capi.mls_last_error()


@pytest.mark.parametrize("precision", ["mixed", "fp32", "fp64"])
@pytest.mark.parametrize("degree", [0, 1, 2])
def test_noalloc_fills_its_whole_scratch(capi, degree, precision):
    """n = MLS_NOALLOC_MAX_POINTS exactly (the array filled to its last
    entry), every degree and precision: bit-identical to mls_project, and a
    successful call leaves no error message behind."""
    n = capi.MLS_NOALLOC_MAX_POINTS
    c = workloads.torus(n=n, seed=24)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, c.k)
    idx, _ = capi.mls_knn(grid, c.k)
    order = capi.mls_grid_order(grid)
    h = 2.0 * float(capi.mls_mean_knn_dist(x, idx).item())
    # a failed call first: its message must not outlive the next success
    bad, *_ = _noalloc(capi, x, idx, -1.0, degree, precision, order)
    assert bad != 0 and capi.mls_last_error()
    rc, out, nrm, st = _noalloc(capi, x, idx, h, degree, precision, order)
    assert rc == 0 and capi.mls_last_error() == ""
    ref_xyz, ref_n, ref_st = capi.mls_project(x, idx, h, degree, precision, order=order)
    torch.cuda.synchronize()
    grid.close()
    # (mixed: the deferred FP64 pass of mls_project = the inline steps here)
    assert torch.equal(out, ref_xyz) and torch.equal(nrm, ref_n) and torch.equal(st, ref_st)
