"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exact
rational arithmetic, closed forms (polynomials the trilinear space reproduces,
TV of affine fields, the first Adam step), library routines (numpy's Philox,
scipy's k-d tree, torch.optim.Adam), central finite differences, and
constructed cases with a known answer (ties, planar fields, single points).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import gridpull as o
from paper_2308_13175_gb300 import synth


# ------------------------------------------------------------- cells
def _exact_floor(x32: np.float32, R: int) -> int:
    t = (Fraction(float(x32)) + 1) * Fraction(R, 2)
    return math.floor(t)


def test_cell_floor_is_exact():
    R = 64
    rng = np.random.default_rng(0)
    vals = list(rng.uniform(-1, 1, 2000).astype(np.float32))
    # Cell boundaries, one ulp either side, tiny values around 0 and the faces.
    for c in range(0, R + 1, 7):
        b = np.float32(-1 + 2 * c / R)
        vals += [b, np.nextafter(b, np.float32(-2)), np.nextafter(b, np.float32(2))]
    vals += [np.float32(v) for v in (0.0, -0.0, 1e-30, -1e-30, 2.0 ** -60, -(2.0 ** -60),
                                     2.0 ** -149, -(2.0 ** -149), 1.0, -1.0, 0.999999, -0.9999999)]
    x = np.array(vals, dtype=np.float32)
    pts = np.stack([x, np.roll(x, 1), np.roll(x, 2)], axis=1)
    cell, local, inside = o.cell_and_local(pts, R)
    for n in range(len(x)):
        for a in range(3):
            assert cell[n, a] == _exact_floor(pts[n, a], R), (pts[n, a], cell[n, a])
    assert np.all(local >= 0) and np.all(local < 1.0 + 1e-12)
    want_inside = np.all((cell >= 0) & (cell <= R - 1), axis=1)
    assert np.array_equal(inside, want_inside)
    # -1e-30 lies just below the plane x = 0: exact floor R/2 - 1, while a
    # float64 evaluation of (x + 1) * R/2 would round up to R/2.
    c_tiny, _, _ = o.cell_and_local(np.array([[-1e-30, 0, 0]], np.float32), R)
    assert c_tiny[0, 0] == R // 2 - 1


# ------------------------------------------------------------- Eq. 3
def _poly(coef, x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    b = np.stack([np.ones_like(X), X, Y, Z, X * Y, X * Z, Y * Z, X * Y * Z], axis=1)
    g = np.stack([coef[1] + coef[4] * Y + coef[5] * Z + coef[7] * Y * Z,
                  coef[2] + coef[4] * X + coef[6] * Z + coef[7] * X * Z,
                  coef[3] + coef[5] * X + coef[6] * Y + coef[7] * X * Y], axis=1)
    return b @ coef, g


@pytest.mark.parametrize("R", [8, 64, 256])
def test_trilinear_reproduces_eq3_polynomials(R):
    """Every polynomial of Eq. 3's form, written in world coordinates, is
    reproduced exactly (value and gradient) from its vertex values."""
    rng = np.random.default_rng(R)
    coef = rng.normal(size=8)
    q = rng.uniform(-0.999, 0.999, size=(500, 3)).astype(np.float32)
    cell, local, inside = o.cell_and_local(q, R)
    assert inside.all()
    keys = np.stack([o.vertex_key(cell + c, R) for c in o.CORNERS], axis=1)
    h = o.grid_spacing(R)
    verts = -1.0 + h * o.key_to_vertex(keys.reshape(-1), R)
    d8 = _poly(coef, verts)[0].reshape(-1, 8)
    f, g, sf, sg = o.trilinear_eval(d8, local * h, h)
    fx, gx = _poly(coef, q.astype(np.float64))
    scale = np.abs(coef).sum()
    assert np.max(np.abs(f - fx)) < 1e-9 * scale
    assert np.max(np.abs(g - gx)) < 1e-9 * scale * R


def test_trilinear_sensitivities_are_trilinear_weights():
    """df/dd_k equals the textbook weights prod(t or 1-t); they sum to 1 and
    the gradient weights sum to 0."""
    rng = np.random.default_rng(3)
    h = 2.0 / 32
    t = rng.random((200, 3))
    _, _, sf, sg = o.trilinear_eval(rng.normal(size=(200, 8)), t * h, h)
    w = np.ones((200, 8))
    for k, c in enumerate(o.CORNERS):
        for a in range(3):
            w[:, k] *= np.where(c[a] == 1, t[:, a], 1 - t[:, a])
    assert np.allclose(sf, w, atol=1e-12)
    assert np.allclose(sf.sum(1), 1.0, atol=1e-12)
    assert np.allclose(sg.sum(2), 0.0, atol=1e-9)


def test_trilinear_is_continuous_across_faces():
    R = 16
    h = o.grid_spacing(R)
    rng = np.random.default_rng(4)
    D = rng.normal(size=(R + 1) ** 3)
    # Points on the plane x = vertex 5, evaluated from the cell on each side.
    yz = rng.random((50, 2)) * 2 - 1
    c_right = np.stack([np.full(50, 5), np.floor((yz[:, 0] + 1) / h), np.floor((yz[:, 1] + 1) / h)], 1).astype(np.int64)
    c_left = c_right.copy()
    c_left[:, 0] = 4
    loc_r = np.stack([np.zeros(50), (yz[:, 0] + 1) / h - c_right[:, 1], (yz[:, 1] + 1) / h - c_right[:, 2]], 1)
    loc_l = loc_r.copy()
    loc_l[:, 0] = 1.0
    fr = o._eval_at(D, c_right, loc_r, R)[1]
    fl = o._eval_at(D, c_left, loc_l, R)[1]
    assert np.allclose(fr, fl, atol=1e-12)


# --------------------------------------------------- pull: planar field
def test_planar_field_pulls_onto_plane():
    """d = n.v - c is in Eq. 3's space, so f is the exact signed distance; a
    query q = s_k + tau n is pulled exactly onto s_k (Eq. 4), with zero
    gradient-consistency (Eq. 7) and surface (Eq. 6) terms."""
    R = 32
    rng = np.random.default_rng(5)
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    c0 = 0.1
    # Surface points on the plane n.x = c0 inside the box.
    u = rng.normal(size=3)
    u -= nrm * (u @ nrm)
    u /= np.linalg.norm(u)
    w = np.cross(nrm, u)
    ab = rng.uniform(-0.4, 0.4, size=(400, 2))
    pts = (c0 * nrm + ab[:, :1] * u + ab[:, 1:] * w).astype(np.float32)
    sets = o.band_sets(pts, R, 3, 3)
    keys = np.arange((R + 1) ** 3)
    verts = -1.0 + o.grid_spacing(R) * o.key_to_vertex(keys, R)
    D = verts @ nrm - c0
    k = rng.integers(0, len(pts), 200)
    tau = rng.uniform(-0.05, 0.05, 200)
    q = (pts[k].astype(np.float64) + tau[:, None] * nrm).astype(np.float32)
    nn = o.nearest_point(q, pts)
    res = o.query_terms(D, R, sets["pull_cells"], q, pts[nn], 1.0, 0.005)
    assert res["valid"].all()
    # The float32 query is within 1e-7 of the line s_k + tau n.
    assert np.max(np.abs(res["pulled"] - pts[nn].astype(np.float64))) < 2e-6
    assert np.max(res["l_pull"]) < 2e-6
    assert np.max(np.abs(res["l_grad"])) < 1e-12
    assert np.max(res["l_surf"]) < 1e-7
    # NN of a query straight above s_k is s_k unless another point is as close.
    d_k = np.linalg.norm(q - pts[k], axis=1)
    d_nn = np.linalg.norm(q - pts[nn], axis=1)
    assert np.all(d_nn <= d_k + 1e-12)


def test_sphere_sdf_pulls_queries_to_the_sphere():
    """Grid values of the sphere SDF |x| - r: each query is pulled to within
    the trilinear interpolation error of the exact projection onto the sphere.

    With H = 1/rho_min bounding the Hessian entries of |x| on the cell,
    |f - d| <= 3 h^2 H / 8 and |grad f - grad d| <= sqrt(3) * 2.5 h H, so
    |p - proj| <= 3 h^2 H / 8 + |f| * 2 * sqrt(3) * 2.5 h H + |f - d|."""
    R = 64
    h = o.grid_spacing(R)
    r = 0.5
    pts = synth.sphere_cloud(20000, r, seed=1)
    sets = o.band_sets(pts, R, 3, 3)
    keys = np.arange((R + 1) ** 3)
    verts = -1.0 + h * o.key_to_vertex(keys, R)
    D = np.linalg.norm(verts, axis=1) - r
    q, _ = synth.gaussian_queries(pts, 2000, 2 * h, seed=2)
    nn = o.nearest_point(q, pts)
    res = o.query_terms(D, R, sets["pull_cells"], q, pts[nn], 1.0, 0.005)
    v = res["valid"]
    q64 = q[v].astype(np.float64)
    proj = q64 / np.linalg.norm(q64, axis=1, keepdims=True) * r
    rho_min = np.linalg.norm(q64, axis=1) - math.sqrt(3) * h
    H = 1.0 / rho_min
    f = res["f"]
    interp = 3 * h * h * H / 8
    bound = interp + np.abs(f) * 2 * math.sqrt(3) * 2.5 * h * H + interp
    err = np.linalg.norm(res["pulled"] - proj, axis=1)
    assert np.all(err <= bound)
    assert err.mean() < 0.05 * h
    # |p - s| <= |p - proj| + |proj - q| + |q - s| and |q - s| <= |q - s'| for
    # s' = NN(proj), so the pull loss is bounded by the pull error plus the
    # cloud's own distance to the projection.
    s_proj = pts[o.nearest_point(proj.astype(np.float32), pts)].astype(np.float64)
    d_q = np.linalg.norm(q64 - proj, axis=1)
    bound_pull = err + 2 * d_q + np.linalg.norm(proj - s_proj, axis=1) + 1e-7
    assert np.all(res["l_pull"][v] <= bound_pull)


# ------------------------------------------------------------ Eq. 7
def test_gradient_term_identical_and_opposite():
    R = 16
    h = o.grid_spacing(R)
    a = np.array([0.3, -0.5, 0.2])
    D = np.zeros((R + 1) ** 3)
    q = np.array([[-0.5 + 0.3 * h, -0.5 + 0.4 * h, -0.5 + 0.6 * h]], np.float32)
    s = np.array([[0.5 + 0.2 * h, 0.5 + 0.7 * h, 0.5 + 0.1 * h]], np.float32)
    pull = np.arange(R ** 3)
    for sign, want in ((1.0, 0.0), (-1.0, 2.0)):
        for pt, sg in ((q, 1.0), (s, sign)):
            c, _, _ = o.cell_and_local(pt, R)
            for corner in o.CORNERS:
                key = o.vertex_key(c[0] + corner, R)
                D[key] = sg * (a @ (-1.0 + h * (c[0] + corner)))
        res = o.query_terms(D, R, pull, q, s, 1.0, 0.005)
        assert abs(res["l_grad"][0] - want) < 1e-12


# ------------------------------------------------------------ Eq. 5
def test_tv_of_affine_and_constant_fields():
    R = 12
    h = o.grid_spacing(R)
    a = np.array([0.7, -0.2, 0.4])
    keys = np.arange((R + 1) ** 3)
    ijk = o.key_to_vertex(keys, R)
    D = (-1.0 + h * ijk) @ a + 0.3
    loss, grad, tv = o.tv_term(D, R, keys)
    interior = np.all((ijk >= 2) & (ijk <= R - 2), axis=1)
    assert np.allclose(tv[np.all((ijk >= 1) & (ijk <= R - 1), axis=1)], math.sqrt(2) * h * np.linalg.norm(a), rtol=1e-12)
    assert np.max(np.abs(grad[interior])) < 1e-12
    loss0, grad0, tv0 = o.tv_term(np.full_like(D, 0.25), R, keys)
    assert loss0 == 0.0 and np.all(grad0 == 0.0)


# ------------------------------------------------- finite differences
@pytest.mark.parametrize("seed", [0, 1])
def test_full_gradient_matches_central_differences(seed):
    """dL/dD of Eq. 8 (explicit adjoints) against central differences of L."""
    R = 8
    rng = np.random.default_rng(seed)
    pts = synth.sphere_cloud(60, 0.45, seed=seed + 10)
    sets = o.band_sets(pts, R, 1, 2)
    keys = np.arange((R + 1) ** 3)
    verts = -1.0 + o.grid_spacing(R) * o.key_to_vertex(keys, R)
    D = np.linalg.norm(verts, axis=1) - 0.45 + 0.05 * rng.normal(size=len(keys))
    q, j = synth.gaussian_queries(pts, 80, 0.1, seed=seed + 20)
    s = pts[j]
    w = (1.0, 1.0, 0.3)
    res = o.step_loss_grad(D, R, sets, q, s, w)
    assert res["Bv"] > 40
    eps = 1e-6
    check = sets["required"]
    fd = np.empty(len(check))
    for n, kk in enumerate(check):
        Dp, Dm = D.copy(), D.copy()
        Dp[kk] += eps
        Dm[kk] -= eps
        lp = o.step_loss_grad(Dp, R, sets, q, s, w, with_grad=False)["loss"]
        lm = o.step_loss_grad(Dm, R, sets, q, s, w, with_grad=False)["loss"]
        fd[n] = (lp - lm) / (2 * eps)
    g = res["grad"][check]
    assert np.max(np.abs(g - fd)) < 2e-6 * np.max(np.abs(fd))
    # The per-vertex conditioning scale bounds the gradient it describes.
    assert np.all(res["abs_terms"] >= np.abs(res["grad"]) * (1 - 1e-12))
    # Vertices outside the required set get no gradient.
    other = np.setdiff1d(keys, check)
    assert np.all(res["grad"][other] == 0)


@pytest.mark.parametrize("R,npts,nq,sig,seed,noise,M", [
    (8, 60, 80, 0.1, 0, 0.05, 1), (8, 60, 80, 0.1, 1, 0.05, 1),
    (64, 5000, 30000, 0.03, 1, 0.01, 2), (64, 5000, 30000, 0.03, 2, 0.0, 2), (64, 5000, 30000, 0.03, 3, 0.05, 2)])
def test_tolerance_scale_is_bounded_on_both_sides(R, npts, nq, sig, seed, noise, M):
    """The per-vertex tolerance scale S_i (abs_terms) is pinned from below and
    from above by the plain absolute sum A_i = sum_k |c_k| of the contributions
    c_k the gradient sum adds at vertex i:  |g_i| <= A_i <= S_i <= 64 A_i.
    Measured on these cases: S_i / A_i reaches 5.9, 6.6, 25, 52 and 13 (median
    1-1.7), with kappa = |q - s| / |r| up to 87 before its cap of 64, so a
    scale inflated by a factor of two fails the bound on the exact sphere."""
    rng = np.random.default_rng(seed)
    pts = synth.sphere_cloud(npts, 0.45, seed=seed + 10)
    sets = o.band_sets(pts, R, M, M)
    keys = np.arange((R + 1) ** 3)
    verts = -1.0 + o.grid_spacing(R) * o.key_to_vertex(keys, R)
    D = np.linalg.norm(verts, axis=1) - 0.45 + noise * rng.normal(size=len(keys))
    q, j = synth.gaussian_queries(pts, nq, sig, seed=seed + 20)
    res = o.step_loss_grad(D, R, sets, q, pts[j], (1.0, 1.0, 0.005))
    S, A, g = res["abs_terms"], res["abs_contrib"], res["grad"]
    assert np.all(A >= np.abs(g) * (1 - 1e-12))
    assert np.all(S >= A * (1 - 1e-12))
    C = 64.0
    m = A > 0
    ratio = S[m] / A[m]
    print(f"tolerance scale: max S/A = {ratio.max():.3g}, kappa max = {res['kappa_max']:.3g}")
    assert ratio.max() <= C
    assert np.all(S[~m] == 0)


# ------------------------------------------------------ nearest point
def test_nearest_point_matches_kdtree_and_breaks_ties_low():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(7)
    pts = rng.uniform(-1, 1, size=(3000, 3)).astype(np.float32)
    q = rng.uniform(-1, 1, size=(500, 3)).astype(np.float32)
    nn = o.nearest_point(q, pts)
    dist, _ = cKDTree(pts.astype(np.float64)).query(q.astype(np.float64))
    mine = np.linalg.norm(q.astype(np.float64) - pts[nn].astype(np.float64), axis=1)
    assert np.allclose(mine, dist, rtol=1e-12, atol=0)
    # Ties: duplicates of a point at higher indices and a mirrored pair.
    base = np.array([[0.1, 0.2, 0.3], [0.5, 0.5, 0.5], [-0.3, 0.0, 0.25]], np.float32)
    dup = np.concatenate([base, base[::-1], base]).astype(np.float32)
    qq = np.array([[0.1, 0.2, 0.3], [0.5, 0.5, 0.5], [-0.3, 0.0, 0.25]], np.float32)
    assert list(o.nearest_point(qq, dup)) == [0, 1, 2]
    pair = np.array([[0.0, 0.0, 0.5], [0.0, 0.0, -0.5], [0.0, 0.0, 0.5]], np.float32)
    assert o.nearest_point(np.zeros((1, 3), np.float32), pair)[0] == 0
    assert o.nearest_point(np.zeros((1, 3), np.float32), pair[1:])[0] == 0


def test_knn_sigma_matches_kdtree():
    from scipy.spatial import cKDTree
    pts = synth.sphere_cloud(2000, 0.5, seed=3)
    pts = np.concatenate([pts, pts[:5]])          # some exact duplicates
    sig = o.knn_sigma(pts, 50)
    d, _ = cKDTree(pts.astype(np.float64)).query(pts.astype(np.float64), k=51)
    assert np.allclose(sig, d[:, 50], rtol=1e-12)


# ------------------------------------------------------------- bands
@pytest.mark.parametrize("M1,M2", [(2, 2), (1, 3), (3, 1)])
def test_band_of_a_single_point(M1, M2):
    R = 32
    p = np.array([[0.013, -0.021, 0.047]], np.float32)
    sets = o.band_sets(p, R, M1, M2)
    assert len(sets["occupied"]) == 1
    assert len(sets["pull_cells"]) == (2 * M1 + 1) ** 3
    n2 = 2 * M2 + 2
    assert len(sets["tv"]) == n2 ** 3
    assert len(sets["trainable"]) == (2 * max(M1, M2) + 2) ** 3
    # TV vertices plus their six-neighbourhood: a cube grown by one on each face.
    req = n2 ** 3 + 6 * n2 ** 2
    if M1 > M2:
        # corners of the bigger pull band cover the TV cube's neighbours.
        req = (2 * M1 + 2) ** 3
    assert len(sets["required"]) == req


def test_band_dense_when_negative():
    R = 8
    sets = o.band_sets(np.zeros((1, 3), np.float32), R, -1, -1)
    assert len(sets["pull_cells"]) == R ** 3
    assert len(sets["tv"]) == (R + 1) ** 3 == len(sets["trainable"]) == len(sets["required"])


# -------------------------------------------------------------- Adam
def test_adam_first_step_and_torch():
    import torch
    rng = np.random.default_rng(9)
    g = rng.normal(size=100)
    d = rng.normal(size=100)
    lr = 1e-2
    d1, m, v = o.adam(d, g, np.zeros(100), np.zeros(100), 1, lr)
    assert np.allclose(d1 - d, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    p = torch.nn.Parameter(torch.tensor(d, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    dd, mm, vv = d.copy(), np.zeros(100), np.zeros(100)
    for t in range(1, 6):
        gt = rng.normal(size=100)
        p.grad = torch.tensor(gt)
        opt.step()
        dd, mm, vv = o.adam(dd, gt, mm, vv, t, lr)
    assert np.allclose(p.detach().numpy(), dd, rtol=1e-12, atol=1e-14)


# --------------------------------------------------- counter-based RNG
def _kat():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            w = [int(x, 16) for x in line.split()]
            rows.append((w[:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert o.philox4x32(ctr, key) == want
        vec = o.philox4x32_vec(np.array([ctr[0]], np.uint64), ctr[1], ctr[2], ctr[3], key[0], key[1])
        assert [int(w[0]) for w in vec] == want


@pytest.mark.parametrize("J", [1, 2, 3, 7, 16, 1000, 4097])
def test_point_permutation_is_a_bijection(J):
    p = o.point_permutation(J, seed=11, epoch=2)
    assert np.array_equal(np.sort(p), np.arange(J))
    if J > 100:
        assert not np.array_equal(p, o.point_permutation(J, seed=11, epoch=3))


def test_sampler_draws_standard_normals():
    from scipy import stats
    pts = synth.sphere_cloud(1000, 0.5, seed=0)
    sigma = np.linspace(0.01, 0.05, 1000)
    pos = np.arange(30000)
    q, j = o.sample_queries(pts, sigma, seed=5, epoch=1, positions=pos)
    z = (q - pts[j].astype(np.float64)) / sigma[j][:, None]
    for a in range(3):
        assert stats.kstest(z[:, a], "norm").pvalue > 1e-3
    # Each point is visited Q/J times per epoch.
    assert np.all(np.bincount(j, minlength=1000) == 30)


def test_sphere_init_formula():
    R = 16
    keys = np.arange((R + 1) ** 3)
    d0 = o.sphere_init(keys, R, (0.1, 0, 0), 0.25, 0.0, 0)
    v = -1.0 + o.grid_spacing(R) * o.key_to_vertex(keys, R)
    assert np.allclose(d0, np.linalg.norm(v - [0.1, 0, 0], axis=1) - 0.25)
    d1 = o.sphere_init(keys, R, (0.1, 0, 0), 0.25, 0.1, 3)
    z = (d1 - d0) / 0.1
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1) < 0.05


# -------------------------------------------- plain torch autograd (FP64)
@pytest.mark.parametrize("M", [1, -1])
def test_oracle_matches_plain_torch_autograd(M):
    """Eq. 8 written with torch ops and differentiated by autograd agrees with
    the oracle's Eq. 3 solve and explicit adjoints."""
    import torch
    from paper_2308_13175_gb300.torch_reference import TorchStep
    R = 16
    pts = synth.sphere_cloud(300, 0.45, seed=2)
    sets = o.band_sets(pts, R, M, M)
    n = (R + 1) ** 3
    keys = np.arange(n)
    D = synth.sphere_field(synth.all_vertices(R), R, 0.45, 0.05, seed=3).astype(np.float64)
    q, j = synth.gaussian_queries(pts, 2000, 0.08, seed=4)
    s = pts[j]
    w = (1.5, 0.7, 0.2)
    ref = o.step_loss_grad(D, R, sets, q, s, w)
    pull = np.zeros(R ** 3, bool)
    pull[sets["pull_cells"]] = True
    ts = TorchStep(R, keys, np.isin(keys, sets["tv"]), np.isin(keys, sets["trainable"]), pull)
    Dt = torch.tensor(D, requires_grad=True)
    rec = torch.from_numpy(np.concatenate([q, s], axis=1))
    L, parts = ts.loss(Dt, rec, w)
    L.backward()
    assert parts["Bv"] == ref["Bv"]
    for k in ("l_pull", "l_grad", "l_surf", "l_tv", "loss"):
        assert abs(float(parts[k]) - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    g = Dt.grad.numpy()
    assert np.max(np.abs(g - ref["grad"])) <= 1e-11 * np.max(np.abs(ref["grad"]))


# ------------------------------------------------ band-sparse value store
def test_sparse_store_and_band_membership_equal_the_dense_forms():
    """The band-sparse forms the large-config tests and the CPU baseline use
    give bit-identical results to the dense forms: SparseValues over the
    required vertices in place of the (R+1)^3 array, the per-cell dilation
    test in place of the dilated cell set, and a TV subset with the full |T|
    as divisor summing to the whole."""
    R = 32
    pts = synth.sphere_cloud(400, 0.45, seed=5)
    sets = o.band_sets(pts, R, 2, 3)
    rng = np.random.default_rng(5)
    D = np.zeros((R + 1) ** 3)
    req = sets["required"]
    D[req] = np.linalg.norm(-1.0 + o.grid_spacing(R) * o.key_to_vertex(req, R), axis=1) - 0.45 \
        + 0.02 * rng.normal(size=len(req))
    all_cells = np.arange(R ** 3)
    assert np.array_equal(o.in_dilated_band(all_cells, sets["occupied"], 2, R),
                          np.isin(all_cells, sets["pull_cells"]))
    assert np.array_equal(o.in_dilated_band(all_cells, sets["occupied"], 0, R),
                          np.isin(all_cells, sets["occupied"]))
    q, j = synth.gaussian_queries(pts, 3000, 0.05, seed=6)
    w = (1.0, 1.0, 0.005)
    dense = o.step_loss_grad(D, R, sets, q, pts[j], w)
    sp = o.SparseValues(req[::-1], D[req[::-1]])
    member = lambda c: o.in_dilated_band(c, sets["occupied"], 2, R)
    sparse = o.step_loss_grad(sp, R, {"pull_cells": member, "tv": sets["tv"]}, q, pts[j], w)
    for k in ("loss", "l_pull", "l_grad", "l_surf", "l_tv", "Bv"):
        assert sparse[k] == dense[k], k
    assert np.array_equal(sparse["grad"], dense["grad"][sp.keys])
    assert np.array_equal(sparse["abs_terms"], dense["abs_terms"][sp.keys])
    assert np.all(dense["grad"][np.setdiff1d(np.arange(len(D)), req)] == 0)
    # A TV subset with the whole set's size as divisor: the two halves add up.
    T = len(sets["tv"])
    a, b = sets["tv"][: T // 3], sets["tv"][T // 3:]
    la, ga, _ = o.tv_term(sp, R, a, n_tv=T)
    lb, gbb, _ = o.tv_term(sp, R, b, n_tv=T)
    assert abs(la + lb - dense["l_tv"]) <= 1e-14 * dense["l_tv"]
    _, gfull, _ = o.tv_term(D, R, sets["tv"])
    assert np.allclose(ga + gbb, gfull[sp.keys], rtol=0, atol=1e-15 * np.abs(gfull).max())
    with pytest.raises(KeyError):
        sp.index(np.array([np.setdiff1d(np.arange(len(D)), req)[0]]))


def test_bitmap_vertex_sets_equal_the_set_form():
    """The dense-bitmap band sets equal band_sets' key-set arithmetic."""
    pts = synth.sphere_cloud(700, 0.4, seed=3)
    for R, M1, M2 in ((32, 2, 2), (32, 1, 3), (16, 0, 0), (16, 2, -1), (8, 3, 1)):
        a = o.band_sets(pts, R, M1, M2)
        b = o.band_vertex_sets_bitmap(pts, R, M1, M2)
        assert np.array_equal(a["tv"], b["tv"]) and np.array_equal(a["trainable"], b["trainable"]), (R, M1, M2)
        assert np.array_equal(a["occupied"], b["occupied"])
