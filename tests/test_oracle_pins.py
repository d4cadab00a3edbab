"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test ties one part of the oracle to an independent fact: brute force,
a library routine on a special case, a closed form, an invariant of the
method (Sec. 1.4, Eq. 1; Algorithm 1), or finite differences.  The mistakes
these catch include a wrong weight, a dropped centroid term, a flipped sign
in q, the wrong eigenvector, a missing or swapped monomial, a broken tie
rule, and a wrong adjoint term.
"""
import numpy as np
import pytest

import oracle
from paper_2401_03365_gb300 import workloads
from tests import golden


# --------------------------------------------------------------------------
# neighbour ranking
# --------------------------------------------------------------------------

def _numpy_key(xyz, i):
    """The ranking key with numpy float32 arithmetic (IEEE single, one rounding
    per operation, never fused)."""
    d = xyz - xyz[i]
    s = d * d
    return (s[:, 0] + s[:, 1]) + s[:, 2]


def test_knn_key_rounds_every_operation():
    rng = np.random.default_rng(0)
    p = rng.standard_normal((2000, 3)).astype(np.float32)
    q = rng.standard_normal((2000, 3)).astype(np.float32)
    ours = np.array([oracle.knn_key(p[i], q[i]) for i in range(2000)])
    d = p - q
    s = d * d
    ref = (s[:, 0] + s[:, 1]) + s[:, 2]
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))
    # the float64 value rounded once differs in some cases: the key is not that
    exact = ((p.astype(np.float64) - q) ** 2).sum(1).astype(np.float32)
    assert (exact != ref).any()


@pytest.mark.parametrize("k", [1, 5, 16])
def test_knn_brute_matches_sorting_by_key_then_index(k):
    rng = np.random.default_rng(k)
    xyz = rng.uniform(-1, 1, (300, 3)).astype(np.float32)
    xyz[50] = xyz[7]          # exact duplicates: the lower index ranks first
    xyz[51] = xyz[7]
    idx, key = oracle.knn_brute(xyz, k)
    for i in range(xyz.shape[0]):
        kk = _numpy_key(xyz, i)
        order = np.lexsort((np.arange(xyz.shape[0]), kk))[:k]
        assert np.array_equal(idx[i], order)
        assert np.array_equal(key[i], kk[order])
    assert idx[7][0] == 7 and idx[50][0] == 7 and idx[51][:3].tolist() == [7, 50, 51][:min(3, k)]


def _lattice(n_side, spacing=0.25):
    g = np.arange(n_side, dtype=np.float32) * np.float32(spacing)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


@pytest.mark.parametrize("case", ["random", "lattice", "duplicates", "clustered", "k_equals_n"])
def test_kdtree_equals_brute(case):
    rng = np.random.default_rng(11)
    k = 12
    if case == "random":
        xyz = rng.standard_normal((1500, 3)).astype(np.float32)
    elif case == "lattice":          # massive exact ties in the key
        xyz = _lattice(10)
        xyz = xyz[rng.permutation(xyz.shape[0])]
        k = 27
    elif case == "duplicates":
        base = rng.uniform(0, 1, (200, 3)).astype(np.float32)
        xyz = base[rng.integers(0, 200, 1200)]
        k = 20
    elif case == "clustered":
        xyz = np.concatenate([rng.normal(0, 1e-3, (700, 3)), rng.normal(5, 1, (300, 3))]).astype(np.float32)
    else:
        xyz = rng.standard_normal((40, 3)).astype(np.float32)
        k = 40
    ib, kb = oracle.knn_brute(xyz, k)
    ik, kk = oracle.knn_kdtree(xyz, k)
    assert np.array_equal(ib, ik)
    assert np.array_equal(kb.view(np.uint32), kk.view(np.uint32))
    # query subsets give the same rows
    q = rng.integers(0, xyz.shape[0], 50)
    iq, _ = oracle.knn_kdtree(xyz, k, queries=q)
    assert np.array_equal(iq, ib[q])


def test_mean_knn_dist_excludes_self():
    rng = np.random.default_rng(3)
    xyz = rng.standard_normal((500, 3)).astype(np.float32)
    idx, _ = oracle.knn_brute(xyz, 8)
    x = xyz.astype(np.float64)
    d = [np.linalg.norm(x[j] - x[i]) for i in range(500) for j in idx[i] if j != i]
    assert oracle.mean_knn_dist(xyz, idx) == pytest.approx(np.mean(d), rel=1e-13)


# --------------------------------------------------------------------------
# dense linear algebra
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [3, 6])
def test_jacobi_matches_eigh(m):
    rng = np.random.default_rng(m)
    for trial in range(50):
        B = rng.standard_normal((m, m))
        A = B @ B.T if trial % 2 else B + B.T
        if trial % 5 == 0:            # repeated eigenvalues
            Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
            ev = np.sort(rng.choice([1.0, 2.0], m))
            A = Q @ np.diag(ev) @ Q.T
        lam, V = oracle.jacobi_eig(A)
        ref = np.linalg.eigvalsh(A)
        scale = np.abs(ref).max()
        assert np.allclose(lam, ref, rtol=0, atol=1e-13 * scale)
        assert np.allclose(V.T @ V, np.eye(m), atol=1e-13)
        assert np.allclose(A @ V, V * lam, atol=1e-12 * scale)


def test_cholesky_solve_and_singularity():
    rng = np.random.default_rng(5)
    for m in (1, 3, 6):
        B = rng.standard_normal((m, m + 2))
        A = B @ B.T
        b = rng.standard_normal(m)
        x = oracle.cholesky_solve(A, b)
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    B = rng.standard_normal((6, 4))
    assert oracle.cholesky_solve(B @ B.T, np.ones(6)) is None      # rank 4


# --------------------------------------------------------------------------
# the projection (Sec. 1.4, Eq. 1; Algorithm 1)
# --------------------------------------------------------------------------

def _random_frame(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q[:, 0], Q[:, 1], Q[:, 2]


@pytest.mark.parametrize("degree", [0, 1, 2])
def test_plane_samples_are_fixed_points(degree):
    """Noise-free samples of a plane: the fitted plane is that plane, every
    height is zero, so each point maps to itself with the plane's normal."""
    rng = np.random.default_rng(7 + degree)
    nrm, e1, e2 = _random_frame(rng)
    uv = rng.uniform(-1, 1, (800, 2))
    xyz = (0.3 * nrm + uv[:, :1] * e1 + uv[:, 1:] * e2).astype(np.float32)
    idx, _ = oracle.knn_kdtree(xyz, 16)
    out, n_out, st, _ = oracle.project(xyz, idx, 0.15, degree)
    x = xyz.astype(np.float64)
    # the float32 inputs sit within ~1e-7 of the exact plane; the fitted plane
    # passes through them to that accuracy
    assert np.abs(out - x).max() < 5e-7
    assert np.abs(np.abs(n_out @ nrm) - 1).max() < 1e-10
    assert (st == 0).all()


def test_degree0_and_1_land_on_weighted_plane():
    """With degree 0 or 1 the fitted height at the origin is zero (in the
    eigenframe the weighted heights and first moments vanish), so p' = q: the
    point moves along n onto the plane through the weighted centroid."""
    c = workloads.sphere(n=3000, seed=21, sigma=0.02, k=16)
    idx, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = 2 * oracle.mean_knn_dist(c.xyz, idx)
    x = c.xyz.astype(np.float64)
    for degree in (0, 1):
        out, nrm, st, _ = oracle.project(c.xyz, idx, h, degree)
        for i in range(0, 3000, 97):
            nb = x[idx[i]]
            w = np.exp(-((nb - x[i]) ** 2).sum(1) / h ** 2)
            cen = (w[:, None] * nb).sum(0) / w.sum()
            assert abs(nrm[i] @ (out[i] - cen)) < 1e-13
            moved = out[i] - x[i]
            assert np.linalg.norm(moved - (moved @ nrm[i]) * nrm[i]) < 1e-13
    out2, *_ = oracle.project(c.xyz, idx, h, 2)
    assert np.abs(out2 - out).max() > 1e-4       # degree 2 does move off the plane


@pytest.mark.parametrize("degree", [0, 1, 2])
def test_fixed_frame_reproduces_polynomials(degree):
    """Over a given frame, heights sampled from any polynomial of the fitted
    degree are reproduced: a0 = g(0, 0) exactly (to FP64 rounding)."""
    rng = np.random.default_rng(30 + degree)
    h = 0.07
    for _ in range(20):
        nrm, e1, e2 = _random_frame(rng)
        q = rng.standard_normal(3)
        uv = rng.uniform(-2 * h, 2 * h, (40, 2))
        coef = rng.standard_normal(6) * np.array([0.01, 1, 1, 3, 3, 3])
        mono = np.stack([np.ones(40), uv[:, 0], uv[:, 1], uv[:, 0] ** 2, uv[:, 0] * uv[:, 1],
                         uv[:, 1] ** 2], 1)
        nb = {0: 1, 1: 3, 2: 6}[degree]
        f = mono[:, :nb] @ coef[:nb]
        P = q + uv[:, :1] * e1 + uv[:, 1:] * e2 + f[:, None] * nrm
        w = rng.uniform(0.1, 1.0, 40)
        a, cond = oracle.fit_height(P, w, nrm, e1, e2, q, h, degree)
        # the oracle's coordinates are scaled by 1/h: coefficient of a monomial
        # of total degree t is multiplied by h^t
        scale = np.array([1, h, h, h * h, h * h, h * h])[:nb]
        assert np.allclose(a[:nb], coef[:nb] * scale, rtol=1e-9, atol=1e-12)
        assert a[0] == pytest.approx(coef[0], abs=1e-13)


def test_golden_symmetric_vertex():
    g = golden.load("symmetric_vertex.txt")
    P = g["points"]
    assert np.array_equal(P[:, 2], P[:, 0] ** 2 / 2 + P[:, 1] ** 2 / 4 + P[:, 0] * P[:, 1] / 8)
    xyz = P.astype(np.float32)
    assert np.array_equal(xyz.astype(np.float64), P)
    n = xyz.shape[0]
    idx = np.tile(np.arange(n, dtype=np.int32), (n, 1))
    qi = int(g["query"])
    out, nrm, st, _ = oracle.project(xyz, idx[qi:qi + 1], g["h"], int(g["degree"]), queries=[qi])
    assert st[0] == 0
    assert np.abs(out[0] - g["expect_xyz"]).max() <= g["tol_xyz"]
    assert np.abs(nrm[0] - g["expect_normal"]).max() <= g["tol_normal"]


def _two_rings_closed_form(rho, s, delta, h):
    """Query at the origin, ring A = (+-rho,0,0),(0,+-rho,0), ring B =
    (+-s,+-s,delta).  By the D4 symmetry the weighted centroid is (0,0,zbar),
    n = e_z, q = (0,0,zbar) and the fitted quadratic is a0 + c (x^2 + y^2): a
    2 x 2 weighted least-squares problem over the three radius classes."""
    wA = np.exp(-rho ** 2 / h ** 2)
    wB = np.exp(-(2 * s * s + delta ** 2) / h ** 2)
    W = 1 + 4 * wA + 4 * wB
    zbar = 4 * wB * delta / W
    w = np.array([1.0, 4 * wA, 4 * wB])
    R2 = np.array([0.0, rho ** 2, 2 * s * s])
    f = np.array([-zbar, -zbar, delta - zbar])
    M = np.array([[w.sum(), (w * R2).sum()], [(w * R2).sum(), (w * R2 * R2).sum()]])
    rhs = np.array([(w * f).sum(), (w * R2 * f).sum()])
    a0 = np.linalg.solve(M, rhs)[0]
    return zbar + a0, zbar


def test_two_rings_closed_form():
    """Weight-, centroid- and sign-sensitive closed form."""
    rho, s, delta = 0.125, 0.125, 0.03125
    pts = [[0, 0, 0], [rho, 0, 0], [-rho, 0, 0], [0, rho, 0], [0, -rho, 0],
           [s, s, delta], [s, -s, delta], [-s, s, delta], [-s, -s, delta]]
    xyz = np.array(pts, np.float32)
    idx = np.tile(np.arange(9, dtype=np.int32), (9, 1))
    for h in (0.1, 0.2, 0.4):
        z_expect, zbar = _two_rings_closed_form(rho, s, delta, h)
        out, nrm, st, _ = oracle.project(xyz, idx[:1], h, 2, queries=[0])
        assert st[0] == 0
        assert np.abs(nrm[0] - [0, 0, 1]).max() < 1e-14
        assert np.abs(out[0, :2]).max() < 1e-15
        assert out[0, 2] == pytest.approx(z_expect, abs=1e-15)
        assert abs(z_expect - zbar) > 1e-4     # the polynomial step matters here
        out1, *_ = oracle.project(xyz, idx[:1], h, 1, queries=[0])
        assert out1[0, 2] == pytest.approx(zbar, abs=1e-15)


def test_status_degenerate_plane_and_singular_polynomial():
    # collinear points: two zero eigenvalues -> degenerate plane, p' = r
    t = np.linspace(-1, 1, 12)
    line = np.stack([t, 0.5 * t, 0 * t], 1).astype(np.float32)
    idx, _ = oracle.knn_brute(line, 12)
    out, nrm, st, _ = oracle.project(line, idx, 0.5, 2)
    assert (st == oracle.STATUS_PLANE_DEGENERATE).all()
    assert np.array_equal(out, line.astype(np.float64))
    # a planar cross (points on the u and v axes only): u*v vanishes on every
    # sample, so the degree-2 normal matrix is singular, while degree 1 is not
    a = np.array([-0.5, -0.25, 0.25, 0.5])
    cross = np.concatenate([[[0, 0, 0]], np.stack([a, 0 * a, 0 * a], 1), np.stack([0 * a, a, 0 * a], 1)])
    cross = cross.astype(np.float32)
    idx = np.tile(np.arange(9, dtype=np.int32), (9, 1))
    out, nrm, st, _ = oracle.project(cross, idx[:1], 0.5, 2, queries=[0])
    assert st[0] == oracle.STATUS_POLY_SINGULAR
    out1, _, st1, _ = oracle.project(cross, idx[:1], 0.5, 1, queries=[0])
    assert st1[0] == 0 and np.array_equal(out[0], out1[0])


def _signed_perm(rng):
    P = np.eye(3)[rng.permutation(3)]
    return P * rng.choice([-1.0, 1.0], 3)[:, None]


def test_rigid_motion_equivariance_exact():
    """Signed axis permutations and dyadic shifts are exact in float32, so the
    oracle must be equivariant to FP64 rounding: P(Rx + t) = R P(x) + t."""
    rng = np.random.default_rng(41)
    c = workloads.torus(n=4000, seed=41, k=16)
    xyz = (np.round(c.xyz.astype(np.float64) * 2 ** 16) / 2 ** 16).astype(np.float32)
    idx, _ = oracle.knn_kdtree(xyz, 16)
    h = 2 * oracle.mean_knn_dist(xyz, idx)
    out, nrm, st, diag = oracle.project(xyz, idx, h, 2)
    D = np.linalg.norm(xyz.max(0) - xyz.min(0))
    for _ in range(3):
        R = _signed_perm(rng)
        t = rng.integers(-2 ** 17, 2 ** 17, 3) / 2 ** 16
        moved = (xyz.astype(np.float64) @ R.T + t)
        assert np.array_equal(moved.astype(np.float32).astype(np.float64), moved)
        out2, nrm2, st2, _ = oracle.project(moved.astype(np.float32), idx, h, 2)
        ok = st == 0
        assert np.array_equal(st, st2)
        assert np.abs(out2[ok] - (out[ok] @ R.T + t)).max() < 1e-12 * D
        assert np.abs(np.abs((nrm[ok] @ R.T * nrm2[ok]).sum(1)) - 1).max() < 1e-9


def test_rotation_and_scale_equivariance():
    rng = np.random.default_rng(42)
    c = workloads.sphere(n=3000, seed=42, k=16)
    idx, _ = oracle.knn_kdtree(c.xyz, 16)
    h = 2 * oracle.mean_knn_dist(c.xyz, idx)
    out, nrm, st, diag = oracle.project(c.xyz, idx, h, 2)
    # general rotation: inputs round to float32, so compare at that level
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    rot = (c.xyz.astype(np.float64) @ Q.T).astype(np.float32)
    out2, *_ = oracle.project(rot, idx, h, 2)
    assert np.abs(out2 - out @ Q.T).max() < 1e-5
    # power-of-two scaling is exact: p' scales exactly with h
    out3, nrm3, st3, _ = oracle.project(c.xyz * np.float32(4.0), idx, 4 * h, 2)
    assert np.abs(out3 - 4 * out).max() < 1e-13
    assert np.abs(nrm3 - nrm).max() < 1e-12


def test_permutation_equivariance():
    rng = np.random.default_rng(43)
    c = workloads.sphere(n=2000, seed=43, k=12)
    idx, _ = oracle.knn_kdtree(c.xyz, 12)
    h = 2 * oracle.mean_knn_dist(c.xyz, idx)
    out, nrm, st, _ = oracle.project(c.xyz, idx, h, 2)
    perm = rng.permutation(2000)
    inv = np.argsort(perm)
    idx_p, _ = oracle.knn_kdtree(c.xyz[perm], 12)
    assert np.array_equal(inv[idx], idx_p[inv])          # same neighbour sets, same order
    out_p, nrm_p, st_p, _ = oracle.project(c.xyz[perm], idx_p, h, 2)
    assert np.array_equal(out_p, out[perm])


def test_denoises_and_is_nearly_idempotent():
    """The paper's quality tables (Sec. 3.3) show MLS lowers the deviation from
    the true surface; a second pass moves points far less than the first.  The
    operator weights about r and does not iterate over t, so it is a smoother
    rather than an exact projection: the second pass still removes part of the
    remaining noise (about 0.15 of the first step on this cloud).  The bound
    0.2 is this reading's; the paper gives none."""
    c = workloads.sphere()
    idx, _ = oracle.knn_kdtree(c.xyz, c.k)
    h = 2 * oracle.mean_knn_dist(c.xyz, idx)
    out, *_ = oracle.project(c.xyz, idx, h, 2)
    before = np.abs(np.linalg.norm(c.xyz.astype(np.float64), axis=1) - 1).mean()
    after = np.abs(np.linalg.norm(out, axis=1) - 1).mean()
    assert after < 0.6 * before
    p1 = out.astype(np.float32)
    idx1, _ = oracle.knn_kdtree(p1, c.k)
    out2, *_ = oracle.project(p1, idx1, h, 2)
    step1 = np.median(np.linalg.norm(out - c.xyz, axis=1))
    step2 = np.median(np.linalg.norm(out2 - p1, axis=1))
    assert step2 < 0.2 * step1


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

def _loss(xyz, idx, h, degree, gp, gn):
    out, nrm, st, _ = oracle.project(xyz, idx, h, degree)
    return (gp * out).sum() + (gn * nrm).sum(), st


@pytest.mark.parametrize("degree", [1, 2])
def test_adjoint_matches_central_differences(degree):
    rng = np.random.default_rng(50 + degree)
    c = workloads.bumpy_sphere(n=1500, seed=50, k=12)
    idx, _ = oracle.knn_kdtree(c.xyz, 12)
    h = 2 * oracle.mean_knn_dist(c.xyz, idx)
    _, _, st, diag = oracle.project(c.xyz, idx, h, degree)
    gp = rng.standard_normal((1500, 3))
    gn = rng.standard_normal((1500, 3))
    grad, gh = oracle.project_grad(c.xyz, idx, h, degree, gp, gn)
    # check a sample of coordinates; inputs are float32, so the step is taken as
    # the exact difference of the two perturbed float32 values
    checked = 0
    for p in rng.choice(1500, 25, replace=False):
        for a in range(3):
            xp = c.xyz.copy()
            xm = c.xyz.copy()
            eps = 2e-4 * h
            xp[p, a] = np.float32(c.xyz[p, a] + eps)
            xm[p, a] = np.float32(c.xyz[p, a] - eps)
            lp, stp = _loss(xp, idx, h, degree, gp, gn)
            lm, stm = _loss(xm, idx, h, degree, gp, gn)
            if not (np.array_equal(stp, st) and np.array_equal(stm, st)):
                continue
            fd = (lp - lm) / (float(xp[p, a]) - float(xm[p, a]))
            assert fd == pytest.approx(grad[p, a], rel=1e-5, abs=1e-7 * np.abs(grad).max())
            checked += 1
    assert checked > 60
    eps = 1e-5 * h
    lp, _ = _loss(c.xyz, idx, h + eps, degree, gp, gn)
    lm, _ = _loss(c.xyz, idx, h - eps, degree, gp, gn)
    assert (lp - lm) / (2 * eps) == pytest.approx(gh, rel=1e-5)


def test_adjoint_over_query_subsets_sums_to_the_whole():
    c = workloads.sphere(n=1500, seed=52, k=12)
    idx, _ = oracle.knn_kdtree(c.xyz, 12)
    rng = np.random.default_rng(53)
    gp = rng.standard_normal((1500, 3))
    g_all, h_all = oracle.project_grad(c.xyz, idx, 0.1, 2, gp)
    perm = rng.permutation(1500)
    a, b = np.sort(perm[:700]), np.sort(perm[700:])
    g_a, h_a = oracle.project_grad(c.xyz, idx[a], 0.1, 2, gp, queries=a)
    g_b, h_b = oracle.project_grad(c.xyz, idx[b], 0.1, 2, gp, queries=b)
    assert np.allclose(g_a + g_b, g_all, rtol=1e-12, atol=1e-12 * np.abs(g_all).max())
    assert h_a + h_b == pytest.approx(h_all, rel=1e-12)


def test_adjoint_term_norms():
    """grad_abs: the sum of the norms of the terms added into each gradient.
    One query alone gives each of its other neighbours exactly one term,
    so there it is that gradient's norm; over several queries it adds up
    query by query, bounds the norm of the sum, and is 0 for points in no
    row."""
    c = workloads.sphere(n=1500, seed=54, k=12)
    idx, _ = oracle.knn_kdtree(c.xyz, 12)
    rng = np.random.default_rng(55)
    gp = rng.standard_normal((1500, 3))
    gn = rng.standard_normal((1500, 3))
    i = 321
    g1, _, a1 = oracle.project_grad(c.xyz, idx[[i]], 0.1, 2, gp, gn, queries=[i], with_abs=True)
    others = idx[i][idx[i] != i]
    assert np.array_equal(a1[others], np.linalg.norm(g1[others], axis=1))
    assert a1[i] >= np.linalg.norm(g1[i])
    untouched = np.setdiff1d(np.arange(1500), idx[i])
    assert np.all(a1[untouched] == 0) and np.all(g1[untouched] == 0)
    g_all, _, a_all = oracle.project_grad(c.xyz, idx, 0.1, 2, gp, gn, with_abs=True)
    perm = rng.permutation(1500)
    a, b = np.sort(perm[:600]), np.sort(perm[600:])
    _, _, aa = oracle.project_grad(c.xyz, idx[a], 0.1, 2, gp, gn, queries=a, with_abs=True)
    _, _, ab = oracle.project_grad(c.xyz, idx[b], 0.1, 2, gp, gn, queries=b, with_abs=True)
    assert np.allclose(aa + ab, a_all, rtol=1e-12)
    assert np.all(a_all >= np.linalg.norm(g_all, axis=1) * (1 - 1e-12))
    g_plain, _ = oracle.project_grad(c.xyz, idx, 0.1, 2, gp, gn)
    assert np.array_equal(g_plain, g_all)


def test_negligible_neighbour_weights_make_a_degenerate_plane():
    """Reading R9: when every neighbour lies many h from the point, their
    Gaussian weights vanish beside the point's own and the weighted
    covariance (normalised by W) falls below 2^-40 D^2 (D the largest
    distance from the point to a row entry): the plane is degenerate and the
    point stays exactly where it is.  The same neighbours 2 h away, or at any
    distance with h far above it (every weight 1), give a regular plane."""
    rng = np.random.default_rng(17)
    h = 0.01
    for dist, hh, degenerate in ((10 * h, h, True), (2 * h, h, False), (10 * h, 1e5, False)):
        u = rng.standard_normal((15, 2))
        u *= dist / np.linalg.norm(u, axis=1, keepdims=True)
        nb = np.concatenate([u, 0.02 * dist * rng.standard_normal((15, 1))], axis=1)
        xyz = np.concatenate([np.zeros((1, 3)), nb]).astype(np.float32)
        rows = np.arange(16, dtype=np.int32)[None, :]
        out, nrm, st, diag = oracle.project(xyz, rows, hh, 0, queries=np.array([0]))
        lam_max = diag[0, 2]
        D2 = (xyz.astype(np.float64) ** 2).sum(1).max()
        if degenerate:
            assert st[0] == oracle.STATUS_PLANE_DEGENERATE
            assert lam_max <= 2.0 ** -40 * D2
            assert np.array_equal(out[0], xyz[0].astype(np.float64))
        else:
            assert st[0] & oracle.STATUS_PLANE_DEGENERATE == 0
            assert lam_max > 1e-6 * D2
            assert abs(abs(nrm[0, 2]) - 1.0) < 1e-2      # the neighbours' plane, z nearly normal
