"""Argument validation and error reporting of the C ABI: every bad call
returns its status code (no fault, no abort) and leaves the context usable."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


@pytest.fixture(scope="module")
def cloud():
    rng = np.random.default_rng(0)
    return torch.from_numpy(rng.standard_normal((1000, 3)).astype(np.float32)).cuda()


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _proj(capi, xyz, idx, k, h=0.1, degree=2, precision=1, out=None):
    out = torch.empty_like(xyz) if out is None else out
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return capi.lib().mls_project(_p(xyz), xyz.shape[0], _p(idx), k, h, degree, precision, None, _p(out),
                                  None, None, s)


def test_project_argument_errors(capi, cloud):
    idx = torch.zeros((1000, 8), dtype=torch.int32, device="cuda")
    assert _proj(capi, cloud, idx, 8) == 0
    assert _proj(capi, cloud, idx, 0) == -2
    assert _proj(capi, cloud, idx, 65) == -2
    assert _proj(capi, cloud, idx, 8, degree=3) == -3
    assert _proj(capi, cloud, idx, 8, degree=-1) == -3
    for h in (0.0, -1.0, float("nan"), float("inf")):
        assert _proj(capi, cloud, idx, 8, h=h) == -1
    assert _proj(capi, cloud, idx, 8, precision=7) == -1
    assert _proj(capi, cloud, idx, 8, out=cloud) == -1            # aliasing
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert capi.lib().mls_project(None, 1000, _p(idx), 8, 0.1, 2, 1, None, _p(cloud), None, None, s) == -1
    assert capi.lib().mls_project(_p(cloud), 0, _p(idx), 8, 0.1, 2, 1, None, _p(cloud), None, None, s) == -1
    assert "degree" in capi.mls_last_error() or "null" in capi.mls_last_error() or capi.mls_last_error()
    torch.cuda.synchronize()


def test_grid_argument_errors(capi, cloud):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = ctypes.c_void_p()
    lib = capi.lib()
    assert lib.mls_build_grid(None, 10, 0.0, 8, s, ctypes.byref(h)) == -1
    assert lib.mls_build_grid(_p(cloud), 0, 0.0, 8, s, ctypes.byref(h)) == -1
    assert lib.mls_build_grid(_p(cloud), 1000, 0.0, 0, s, ctypes.byref(h)) == -2
    assert lib.mls_build_grid(_p(cloud), 1000, 0.0, 65, s, ctypes.byref(h)) == -2
    assert lib.mls_build_grid(_p(cloud), 1000, float("nan"), 8, s, ctypes.byref(h)) == -1
    assert lib.mls_build_grid(_p(cloud), 2 ** 31, 0.0, 8, s, ctypes.byref(h)) == -8
    assert h.value is None
    grid = capi.mls_build_grid(cloud, 0.0, 8)
    idx = torch.empty((1000, 8), dtype=torch.int32, device="cuda")
    assert lib.mls_knn(grid.handle, 0, _p(idx), None, s) == -2
    assert lib.mls_knn(grid.handle, 1001, _p(idx), None, s) == -2
    assert lib.mls_knn(None, 8, _p(idx), None, s) == -1
    assert lib.mls_knn(grid.handle, 8, None, None, s) == -1
    torch.cuda.synchronize()
    grid.close()
    lib.mls_grid_destroy(None)


def test_nonfinite_coordinates_rejected(capi):
    x = torch.randn(500, 3, device="cuda")
    x[123, 1] = float("nan")
    with pytest.raises(capi.MLSError) as e:
        capi.mls_build_grid(x, 0.0, 8)
    assert e.value.code == -7
    x[123, 1] = float("inf")
    with pytest.raises(capi.MLSError):
        capi.mls_build_grid(x, 0.0, 8)
    # the context is still usable
    x[123, 1] = 0.0
    g = capi.mls_build_grid(x, 0.0, 8)
    idx, _ = capi.mls_knn(g, 8)
    torch.cuda.synchronize()
    g.close()
    assert idx.shape == (500, 8)


def test_binding_type_checks(capi, cloud):
    with pytest.raises(TypeError):
        capi.mls_build_grid(cloud.double(), 0.0, 8)
    with pytest.raises(TypeError):
        capi.mls_build_grid(cloud.cpu(), 0.0, 8)
    with pytest.raises(ValueError):
        capi.mls_build_grid(cloud[:, :2].contiguous(), 0.0, 8)


def test_mean_knn_dist_matches_oracle_and_repeats_exactly(capi):
    """The bandwidth helper: the FP64 mean distance to the neighbours other
    than the point itself, summed in a fixed order (bit-identical calls)."""
    import oracle
    from paper_2401_03365_gb300 import workloads
    c = workloads.sphere(n=20_000, seed=3, k=20)
    idx_o, _ = oracle.knn_kdtree(c.xyz, c.k)
    x = torch.from_numpy(c.xyz).cuda()
    idx = torch.from_numpy(idx_o.astype(np.int32)).cuda()
    a = capi.mls_mean_knn_dist(x, idx).item()
    b = capi.mls_mean_knn_dist(x, idx).item()
    assert a == b
    ref = oracle.mean_knn_dist(c.xyz, idx_o)
    assert abs(a - ref) <= 1e-12 * ref
