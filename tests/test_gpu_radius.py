"""Radius-R neighbourhoods on the GPU (mls_radius_count / mls_radius_rows):
bit-exact CSR rows against the oracle's, including exact ties at R and
duplicates; the projection over them with the outlier rule (mls_project_rows)
element by element; the compaction that drops the outliers."""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_03365_gb300 import workloads
from tests.gpu_cases import compare_projection, diag_len, lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_2401_03365_gb300 import build, capi
    build.build()
    return capi


def _cases():
    rng = np.random.default_rng(21)
    dup = rng.uniform(0, 1, (300, 3)).astype(np.float32)
    return {
        "sphere20k": (workloads.sphere().xyz, 0.06),
        "torus100k_outliers": (workloads.torus(n=100_000, seed=12).xyz, 0.012),
        "lattice_ties": (lattice(12, 0.25), 0.25),
        "duplicates": (dup[rng.integers(0, 300, 3000)], 0.04),
        "one_point": (np.zeros((1, 3), np.float32), 0.1),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_rows_equal_the_oracle(capi, name):
    xyz, R = _cases()[name]
    off_o, rows_o = oracle.radius_neighbors(xyz, R)
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, 16)
    off, rows, keys = capi.mls_radius_neighbors(grid, R, with_key=True)
    torch.cuda.synchronize()
    grid.close()
    assert np.array_equal(off.cpu().numpy(), off_o)
    assert np.array_equal(rows.cpu().numpy(), rows_o)
    k = keys.cpu().numpy()
    i_of = np.repeat(np.arange(xyz.shape[0]), np.diff(off_o))
    d = xyz[rows_o] - xyz[i_of]
    s = d * d
    assert np.array_equal(k, (s[:, 0] + s[:, 1]) + s[:, 2])


def test_too_many_neighbours_is_reported(capi):
    xyz = np.random.default_rng(22).uniform(0, 1, (4000, 3)).astype(np.float32)
    x = torch.from_numpy(xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, 16)
    with pytest.raises(capi.MLSError) as e:
        capi.mls_radius_neighbors(grid, 0.5)
    grid.close()
    assert e.value.code == -2 and "more than 128" in str(e.value)


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_projection_over_radius_rows_and_outliers(capi, precision):
    c = workloads.torus(n=100_000, seed=12)
    R = 0.035            # about 30 neighbours on the surface, none around most outliers
    off_o, rows_o = oracle.radius_neighbors(c.xyz, R)
    h = 0.8 * R
    o_xyz, o_n, o_st, o_diag = oracle.project_rows(c.xyz, off_o, rows_o, h, 2, min_neighbors=3)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, 16)
    off, rows, _ = capi.mls_radius_neighbors(grid, R)
    order = capi.mls_grid_order(grid)
    g_xyz, g_n, g_st = capi.mls_project_rows(x, off, rows, h, 2, precision, 3, order=order)
    kept = capi.mls_compact(g_st, capi.MLS_PT_OUTLIER).cpu().numpy()
    torch.cuda.synchronize()
    grid.close()
    g_st = g_st.cpu().numpy()
    outl = (o_st & oracle.STATUS_OUTLIER) != 0
    assert 0 < outl.sum() < c.n
    assert np.array_equal((g_st & capi.MLS_PT_OUTLIER) != 0, outl)
    assert np.array_equal(g_st & 32, o_st & oracle.STATUS_DEGREE_REDUCED)
    assert np.array_equal(kept, np.nonzero(~outl)[0])
    assert np.array_equal(g_xyz.cpu().numpy()[outl], c.xyz[outl])
    keep = ~outl
    compare_projection(g_xyz.cpu().numpy()[keep], g_n.cpu().numpy()[keep], g_st[keep], o_xyz[keep], o_n[keep],
                       o_st[keep] & 3, o_diag[keep], diag_len(c.xyz), min_well_posed=0.3)


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_small_radius_lowers_the_degree_like_the_oracle(capi, precision):
    """R about twice the point spacing: two thirds of the neighbourhoods hold
    4-11 points, fitted at degree 1 or 0 (status bit 32, set exactly where the
    oracle sets it), a third 12 or more; positions and normals within the
    tolerances on well-posed points."""
    c = workloads.torus(n=100_000, seed=13)
    R = 0.02
    off_o, rows_o = oracle.radius_neighbors(c.xyz, R)
    h = R
    o_xyz, o_n, o_st, o_diag = oracle.project_rows(c.xyz, off_o, rows_o, h, 2, min_neighbors=3)
    x = torch.from_numpy(c.xyz).cuda()
    grid = capi.mls_build_grid(x, 0.0, 16)
    off, rows, _ = capi.mls_radius_neighbors(grid, R)
    order = capi.mls_grid_order(grid)
    g_xyz, g_n, g_st = capi.mls_project_rows(x, off, rows, h, 2, precision, 3, order=order)
    torch.cuda.synchronize()
    grid.close()
    g_st = g_st.cpu().numpy()
    red = (o_st & oracle.STATUS_DEGREE_REDUCED) != 0
    outl = (o_st & oracle.STATUS_OUTLIER) != 0
    assert red.mean() > 0.5 and (~red & ~outl).mean() > 0.2
    assert np.array_equal(g_st & (16 | 32), o_st & (16 | 32))
    keep = ~outl
    rep = compare_projection(g_xyz.cpu().numpy()[keep], g_n.cpu().numpy()[keep], g_st[keep], o_xyz[keep],
                             o_n[keep], o_st[keep] & 3, o_diag[keep], diag_len(c.xyz), min_well_posed=0.2)
    print(rep)
