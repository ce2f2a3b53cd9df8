"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Contract: integer and set results bit-exact (band sets, NN indices); floating
point within 1e-5 relative (loss terms; gradients norm-wise and per vertex
against max(|g*_i|, 1e-3 max|g*|)); Adam deltas within 1e-5 * lr.  Inputs come
from the seeded generators; expected values from the oracle only.
"""
import numpy as np
import pytest

from oracle import gridpull as o
from paper_2308_13175_gb300 import synth

from gpu_common import (REL_TOL, assert_grad_close, assert_rel, build_lib, dense_from_band, export_band,
                         have_gpu, vertex_keys)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    if not have_gpu():
        pytest.skip("no CUDA device")
    build_lib()
    from paper_2308_13175_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(gb):
    return gb.gp_create(0)


@pytest.fixture(scope="module")
def sphere5k():
    return synth.sphere_cloud(5000, 0.5, seed=0)


@pytest.fixture(scope="module")
def object100k():
    return synth.object_cloud(100_000, seed=1)


def _band(gb, ctx, pts, R, M1, M2, knn_k=50, deterministic=False):
    import torch
    return gb.gp_build_band(ctx, torch.from_numpy(np.ascontiguousarray(pts)).cuda(), R, M1, M2, knn_k,
                            deterministic=deterministic)


def _edge_points():
    return np.array([[1, 1, 1], [-1, -1, -1], [1, -1, 0.3], [-1, 0.999, -0.2], [0, 0, 0],
                     [0.0625, -0.0625, 0.5]], np.float32)


# ------------------------------------------------------------------ band
@pytest.mark.parametrize("case", [("sphere", 64, 2, 2), ("sphere", 64, 1, 3), ("sphere", 32, 3, 1),
                                  ("sphere", 16, -1, -1), ("object", 256, 2, 2), ("edge", 16, 3, 3),
                                  ("edge", 16, 0, 0)])
def test_band_sets_match_oracle(gb, ctx, sphere5k, object100k, case):
    name, R, M1, M2 = case
    pts = {"sphere": sphere5k, "object": object100k, "edge": _edge_points()}[name]
    band = _band(gb, ctx, pts, R, M1, M2, knn_k=0)
    ijk, d, fl, exists = export_band(band)
    ref = o.band_sets(pts, R, M1, M2)
    keys = vertex_keys(ijk, R)
    assert np.all(fl[~exists] == 0)
    assert np.array_equal(np.sort(keys[exists & ((fl & 1) != 0)]), ref["tv"])
    assert np.array_equal(np.sort(keys[exists & ((fl & 2) != 0)]), ref["trainable"])
    pull_v = ijk[exists & ((fl & 8) != 0)]
    assert np.array_equal(np.sort(o.cell_key(pull_v, R)), ref["pull_cells"])
    assert np.all(np.isin(ref["required"], keys[exists]))
    assert len(np.unique(keys[exists])) == int(exists.sum())
    info = band.info
    assert info["V_tv"] == len(ref["tv"]) and info["V_trainable"] == len(ref["trainable"])
    assert info["n_pull_cells"] == len(ref["pull_cells"])
    assert info["n_occupied_cells"] == len(ref["occupied"])


def test_init_sphere_matches_oracle(gb, ctx, sphere5k):
    R = 64
    band = _band(gb, ctx, sphere5k, R, 2, 2, knn_k=0)
    gb.gp_band_init_sphere(band, (0.05, -0.02, 0.1), 0.3, 0.01, seed=7)
    want_all = o.sphere_init(np.arange((R + 1) ** 3), R, (0.05, -0.02, 0.1), 0.3, 0.01, 7)
    ijk, d, fl, exists = export_band(band)
    want = want_all[vertex_keys(ijk[exists], R)]
    assert np.max(np.abs(d[exists] - want) / (1 + np.abs(want))) < 2e-6
    assert np.all(d[~exists] == 0)


# ----------------------------------------------------------------- sigma
def test_sigma_matches_oracle(gb, ctx, sphere5k, object100k):
    pts = np.concatenate([sphere5k, sphere5k[:7]])  # exact duplicates
    band = _band(gb, ctx, pts, 64, 2, 2, knn_k=50)
    sig = gb.gp_band_sigma(band).cpu().numpy()
    want = o.knn_sigma(pts, 50)
    assert np.max(np.abs(sig - want) / want) < 1e-6
    band = _band(gb, ctx, object100k, 256, 2, 2, knn_k=50)
    sig = gb.gp_band_sigma(band).cpu().numpy()
    idx = np.random.default_rng(0).choice(len(object100k), 1500, replace=False)
    want = o.knn_sigma(object100k, 50, idx=idx)
    assert np.max(np.abs(sig[idx] - want) / want) < 1e-6


def test_sigma_small_clouds(gb, ctx):
    pts = np.array([[0.1, 0.2, 0.3], [0.4, -0.1, 0.0], [0.1, 0.2, 0.3]], np.float32)
    band = _band(gb, ctx, pts, 16, 1, 1, knn_k=50)
    assert np.allclose(gb.gp_band_sigma(band).cpu().numpy(), o.knn_sigma(pts, 50), rtol=1e-6)
    band = _band(gb, ctx, pts[:1], 16, 1, 1, knn_k=50)
    assert gb.gp_band_sigma(band).cpu().numpy()[0] == 0.0


# ------------------------------------------------------------ nearest point
def _nn_gpu(gb, band, q, hint=None):
    import torch
    qt = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
    nn = torch.empty(len(q), dtype=torch.int32, device="cuda")
    rec = torch.empty((len(q), 6), dtype=torch.float32, device="cuda")
    ht = None if hint is None else torch.from_numpy(np.ascontiguousarray(hint, np.int32)).cuda()
    gb.gp_nn(band, qt, nn, rec, hint=ht)
    return nn.cpu().numpy().astype(np.int64), rec.cpu().numpy()


def test_nn_matches_bruteforce_sphere(gb, ctx, sphere5k):
    band = _band(gb, ctx, sphere5k, 64, 2, 2, knn_k=0)
    q1, _ = synth.gaussian_queries(sphere5k, 20000, 0.02, seed=3)
    q2 = np.random.default_rng(4).uniform(-1.3, 1.3, size=(3001, 3)).astype(np.float32)
    q = np.concatenate([q1, q2])
    nn, rec = _nn_gpu(gb, band, q)
    want = o.nearest_point(q, sphere5k)
    assert np.array_equal(nn, want)
    assert np.array_equal(rec[:, :3], q) and np.array_equal(rec[:, 3:], sphere5k[want])
    # Hints only seed the search: source points, random points and invalid
    # indices all give the same answer.
    _, j1 = synth.gaussian_queries(sphere5k, 20000, 0.02, seed=3)
    rng = np.random.default_rng(8)
    for hint in (np.concatenate([j1, rng.integers(0, 5000, 3001)]), rng.integers(-5, 5010, len(q))):
        nn_h, _ = _nn_gpu(gb, band, q, hint)
        assert np.array_equal(nn_h, want)


def test_nn_seeded_spatial_batch_full_size(gb, ctx, object100k):
    """The fitting step's NN configuration at the bench size: 262,144 queries
    around their source points, in spatial order, each seeded by its source
    point; 4,000 sampled queries checked by brute force."""
    R = 256
    band = _band(gb, ctx, object100k, R, 2, 2, knn_k=0)
    q, j = synth.gaussian_queries(object100k, 262_144, 0.02, seed=21)
    cell = np.floor((object100k[j].astype(np.float64) + 1) * 64).astype(np.int64)
    order = np.lexsort((cell[:, 0], cell[:, 1], cell[:, 2]))
    q, j = q[order], j[order]
    rng = np.random.default_rng(5)
    j_hint = j.copy()
    j_hint[rng.choice(len(j), 500, replace=False)] = -1       # a few unseeded queries
    nn, _ = _nn_gpu(gb, band, q, j_hint)
    sel = rng.choice(len(q), 4000, replace=False)
    assert np.array_equal(nn[sel], o.nearest_point(q[sel], object100k))
    nn_plain, _ = _nn_gpu(gb, band, q[sel])                  # per-thread search, no seed
    assert np.array_equal(nn_plain, nn[sel])


def test_nn_sorted_large_seeded_batch(gb, ctx, object100k):
    """Seeded batches of 2^20 queries or more take the radius-sorted search:
    1,100,003 queries (a ragged last block) with a few invalid seeds and a few
    non-finite queries must give, index for index, what the fused per-thread
    search gives in chunks below that size; 3,000 sampled queries are checked
    by brute force."""
    import torch
    R = 256
    band = _band(gb, ctx, object100k, R, 2, 2, knn_k=0)
    n = 1_100_003
    q, j = synth.gaussian_queries(object100k, n, 0.03, seed=22)
    cell = np.floor((object100k[j].astype(np.float64) + 1) * 64).astype(np.int64)
    order = np.lexsort((cell[:, 0], cell[:, 1], cell[:, 2]))
    q, j = q[order].copy(), j[order].copy()
    rng = np.random.default_rng(6)
    j[rng.choice(n, 700, replace=False)] = -1
    q[rng.choice(n, 5, replace=False), 1] = np.nan
    qd = torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()
    jd = torch.from_numpy(j.astype(np.int32)).cuda()
    nn_sorted = torch.empty(n, dtype=torch.int32, device="cuda")
    gb.gp_nn(band, qd, nn_sorted, None, hint=jd)
    nn_fused = torch.empty(n, dtype=torch.int32, device="cuda")
    step = (1 << 20) - 1
    for a in range(0, n, step):
        gb.gp_nn(band, qd[a:a + step], nn_fused[a:a + step], None, hint=jd[a:a + step])
    got, want = nn_sorted.cpu().numpy(), nn_fused.cpu().numpy()
    assert np.array_equal(got, want)
    assert np.all(got[np.isnan(q).any(axis=1)] == -1)
    sel = rng.choice(np.flatnonzero(np.isfinite(q).all(axis=1)), 3000, replace=False)
    assert np.array_equal(got[sel], o.nearest_point(q[sel], object100k))


def test_nn_long_cell_row(gb, ctx):
    """70,000 points on one line along x all fall in one row of search cells
    (a long row, many points per cell).  Seeded and unseeded queries around the
    line and a sphere next to it match brute force."""
    rng = np.random.default_rng(8)
    line = np.stack([rng.uniform(-0.9, 0.9, 70_000), np.full(70_000, 0.1), np.full(70_000, -0.2)], 1)
    ball = synth.sphere_cloud(3000, 0.2, seed=9) + np.array([0.0, -0.5, 0.4], np.float32)
    pts = np.concatenate([line, ball]).astype(np.float32)
    band = _band(gb, ctx, pts, 64, 1, 1, knn_k=0)
    src = rng.integers(0, len(pts), 4000)
    q = (pts[src] + rng.normal(scale=0.02, size=(4000, 3))).astype(np.float32)
    want = o.nearest_point(q, pts)
    nn_seeded, _ = _nn_gpu(gb, band, q, src.astype(np.int64))
    nn_plain, _ = _nn_gpu(gb, band, q)
    assert np.array_equal(nn_seeded, want) and np.array_equal(nn_plain, want)


def test_nn_counts_valid_records(gb, ctx, sphere5k):
    import torch
    R = 64
    band = _band(gb, ctx, sphere5k, R, 2, 2, knn_k=0)
    q1, _ = synth.gaussian_queries(sphere5k, 20000, 0.05, seed=12)
    q = np.concatenate([q1, np.random.default_rng(2).uniform(-1.2, 1.2, (5000, 3)).astype(np.float32)])
    nv = torch.zeros(1, dtype=torch.int32, device="cuda")
    rec = torch.empty((len(q), 6), dtype=torch.float32, device="cuda")
    gb.gp_nn(band, torch.from_numpy(q).cuda(), None, rec, nvalid_out=nv)
    s = sphere5k[o.nearest_point(q, sphere5k)]
    res = o.query_terms(np.zeros((R + 1) ** 3), R, o.band_sets(sphere5k, R, 2, 2)["pull_cells"], q, s, 1.0, 0.005,
                        with_grad=False)
    assert int(nv.item()) == res["Bv"]
    assert 0 < res["Bv"] < len(q)


def test_nn_non_finite_queries(gb, ctx, sphere5k):
    band = _band(gb, ctx, sphere5k, 32, 1, 1, knn_k=0)
    q = np.array([[np.nan, 0, 0], [np.inf, 0, 0], [0, -np.inf, 0.1], [1e20, 0, 0], [0.1, 0.2, 0.3],
                  [3.0, -2.5, 7.0]], np.float32)
    nn, rec = _nn_gpu(gb, band, q)
    assert list(nn[:4]) == [-1, -1, -1, -1]
    assert np.all(np.isnan(rec[:4, 3:]))
    assert np.array_equal(nn[4:], o.nearest_point(q[4:], sphere5k))


def test_nn_ties_go_to_lowest_index(gb, ctx):
    base = synth.sphere_cloud(300, 0.4, seed=5)
    pts = np.concatenate([base, base[::-1], base]).astype(np.float32)  # every point three times
    # Equidistant pair around the origin and queries sitting exactly on points.
    pair = np.array([[0.0, 0.0, 0.25], [0.0, 0.0, -0.25]], np.float32)
    pts = np.concatenate([pts, pair, pair]).astype(np.float32)
    band = _band(gb, ctx, pts, 32, 1, 1, knn_k=0)
    q = np.concatenate([base, np.zeros((1, 3), np.float32),
                        synth.gaussian_queries(base, 3000, 0.05, seed=6)[0]]).astype(np.float32)
    nn, _ = _nn_gpu(gb, band, q)
    want = o.nearest_point(q, pts)
    assert np.array_equal(nn, want)
    assert np.array_equal(nn[:300], np.arange(300))


def test_nn_matches_bruteforce_object_full_size(gb, ctx, object100k):
    """The single-object workload (100,000 points, R=256): sampled queries."""
    band = _band(gb, ctx, object100k, 256, 2, 2, knn_k=0)
    q, _ = synth.gaussian_queries(object100k, 3000, 2.0 / 256, seed=7)
    nn, _ = _nn_gpu(gb, band, q)
    assert np.array_equal(nn, o.nearest_point(q, object100k))


# ---------------------------------------------------------------- sampler
@pytest.mark.parametrize("J,Q,first,count,epoch", [(5000, 50000, 12345, 20000, 3), (5000, 50000, 0, 50000, 0),
                                                   (7, 70, 3, 61, 1)])
def test_sampler_matches_oracle(gb, ctx, sphere5k, J, Q, first, count, epoch):
    import torch
    pts = sphere5k[:J]
    band = _band(gb, ctx, pts, 32, 1, 1, knn_k=min(50, J - 1))
    q = gb.gp_sample(band, 5, epoch, Q, first, count).cpu().numpy().astype(np.float64)
    sig = o.knn_sigma(pts, min(50, J - 1))
    want, j = o.sample_queries(pts, sig, 5, epoch, np.arange(first, first + count))
    z = (want - pts[j]) / sig[j][:, None]
    bound = 2e-6 * (np.abs(pts[j]) + sig[j][:, None] * (1 + np.abs(z))) + 1e-7
    assert np.all(np.abs(q - want) <= bound)


@pytest.mark.parametrize("J,Q,first,count", [(5000, 50000, 12345, 20000), (5000, 50000, 0, 50000),
                                             (5000, 3000, 100, 2900), (7, 70, 3, 61)])
def test_sampler_spatial_order_matches_oracle(gb, ctx, sphere5k, J, Q, first, count):
    """Spatial order: the same queries (by pool position), grouped by point."""
    import torch
    pts = sphere5k[:J]
    band = _band(gb, ctx, pts, 32, 1, 1, knn_k=min(50, J - 1))
    src = torch.empty(count, dtype=torch.int32, device="cuda")
    pos = torch.empty(count, dtype=torch.int32, device="cuda")
    q = gb.gp_sample(band, 9, 2, Q, first, count, src_out=src, pos_out=pos, spatial=True)
    q = q.cpu().numpy().astype(np.float64)
    pos = pos.cpu().numpy().astype(np.int64)
    src = src.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(pos), np.arange(first, first + count))
    sig = o.knn_sigma(pts, min(50, J - 1))
    want, j = o.sample_queries(pts, sig, 9, 2, pos)
    assert np.array_equal(src, j)
    z = (want - pts[j]) / sig[j][:, None]
    bound = 2e-6 * (np.abs(pts[j]) + sig[j][:, None] * (1 + np.abs(z))) + 1e-7
    assert np.all(np.abs(q - want) <= bound)
    # Outputs of one point are adjacent, in increasing pool position, and
    # neighbours are close in space.
    starts = np.flatnonzero(np.diff(src)) + 1
    assert len(np.unique(src)) == len(starts) + 1
    same = np.diff(src) == 0
    assert np.all(np.diff(pos)[same] > 0)
    if J > 100:
        step = np.linalg.norm(np.diff(pts[src], axis=0), axis=1).mean()
        rand = np.linalg.norm(pts[src] - pts[np.random.default_rng(0).permutation(src)], axis=1).mean()
        assert step < 0.25 * rand


def test_sampler_bench_sizes(gb, ctx, object100k):
    """Single-object workload: pool of 2,000,000 queries, batches of 262,144."""
    band = _band(gb, ctx, object100k, 256, 2, 2, knn_k=50)
    Q, B = 2_000_000, 262_144
    first = 7 * B  # the ragged last batch of the epoch
    q = gb.gp_sample(band, 11, 2, Q, first, Q - first).cpu().numpy().astype(np.float64)
    sel = np.random.default_rng(1).choice(Q - first, 2000, replace=False)
    pos = first + sel
    j = o.point_permutation(len(object100k), 11, 2, pos % len(object100k))
    sig = o.knn_sigma(object100k, 50, idx=np.unique(j))
    sig_full = np.zeros(len(object100k))
    sig_full[np.unique(j)] = sig
    want, jj = o.sample_queries(object100k, sig_full, 11, 2, pos)
    assert np.array_equal(jj, j)
    z = (want - object100k[j]) / sig_full[j][:, None]
    bound = 2e-6 * (np.abs(object100k[j]) + sig_full[j][:, None] * (1 + np.abs(z))) + 1e-7
    assert np.all(np.abs(q[sel] - want) <= bound)


# ------------------------------------------------------------------- step
def _step_inputs(pts, R, M1, M2, n_queries, sigma, seed, use_nn):
    sets = o.band_sets(pts, R, M1, M2)
    q, j = synth.gaussian_queries(pts, n_queries, sigma, seed=seed)
    s = pts[o.nearest_point(q, pts)] if use_nn else pts[j]
    return sets, q, s


def _filter_ambiguous(D, R, sets, q, s):
    """Drop queries whose sign(f(s)) is decided within float32 rounding (both
    signs are valid subgradients of |f(s)| there)."""
    res = o.query_terms(D, R, sets["pull_cells"], q, s, 1.0, 0.005, with_grad=False)
    if res["Bv"] == 0:
        return q, s
    scale = 1.0 + np.max(np.abs(D))
    keep = np.ones(len(q), bool)
    v = res["valid"]
    fs = np.full(len(q), np.inf)
    fs[v] = res["fs"]
    keep &= np.abs(fs) > 1e-5 * scale
    return q[keep], s[keep]


def _run_step(gb, band, q, s, weights, flags=0, d=None):
    import torch
    rec = torch.from_numpy(np.ascontiguousarray(np.concatenate([q, s], axis=1), np.float32)).cuda()
    grad = torch.full((band.V_stored,), 7.0, dtype=torch.float32, device="cuda")
    loss = torch.zeros(8, dtype=torch.float32, device="cuda")
    gb.gp_step(band, rec, len(q), grad, loss, weights, d=d, flags=flags)
    return grad.cpu().numpy(), loss.cpu().numpy()


def _set_field(gb, band, sets, R, radius, noise, seed, center=(0.0, 0.0, 0.0)):
    """Generator values at the band's stored slots (uploaded) and, for the
    oracle, the same generator at the oracle's own required vertices."""
    import torch
    ijk, _, _, exists = export_band(band)
    vals = np.zeros(band.V_stored, np.float32)
    vals[exists] = synth.sphere_field(ijk[exists], R, radius, noise, seed, center)
    gb.gp_band_set_values(band, torch.from_numpy(vals).cuda())
    D = np.zeros((R + 1) ** 3)
    req = sets["required"]
    D[req] = synth.sphere_field(o.key_to_vertex(req, R), R, radius, noise, seed, center)
    return D, vals


def _check_step(gb, band, R, sets, q, s, weights, D, flags=0, d_override=None):
    """GPU step on the band's values (or d_override) against the oracle on D."""
    import torch
    ijk, _, _, exists = export_band(band)
    q, s = _filter_ambiguous(D, R, sets, q, s)
    sets_use = dict(sets)
    if flags & gb.GP_STEP_NO_TV:
        sets_use["tv"] = np.zeros(0, np.int64)
    ref = o.step_loss_grad(D, R, sets_use, q, s, weights)
    dt = None if d_override is None else torch.from_numpy(d_override).cuda()
    grad, loss = _run_step(gb, band, q, s, weights, flags, dt)
    assert loss[gb.GP_LOSS_BV] == ref["Bv"]
    assert loss[gb.GP_LOSS_T] == len(sets["tv"])
    for slot, key in ((gb.GP_LOSS_PULL, "l_pull"), (gb.GP_LOSS_GRAD, "l_grad"), (gb.GP_LOSS_SURF, "l_surf"),
                      (gb.GP_LOSS_TV, "l_tv"), (gb.GP_LOSS_TOTAL, "loss")):
        assert_rel(loss[slot], ref[key], what=key)
    if flags & gb.GP_STEP_LOSS_ONLY:
        assert np.all(grad == 7.0)
        return ref
    assert np.all(grad[~exists] == 0.0)
    keys = vertex_keys(ijk[exists], R)
    assert_grad_close(grad[exists], ref["grad"][keys], ref["abs_terms"][keys], what=f"step R={R} flags={flags}",
                      kappa_max=ref["kappa_max"])
    # Nothing outside the stored set receives gradient in the oracle.
    assert np.sum(np.abs(ref["grad"])) == pytest.approx(np.sum(np.abs(ref["grad"][keys])), rel=1e-12)
    return ref


def test_step_dense_sphere(gb, ctx, sphere5k):
    """Dense 64^3 grid, |x| - 0.5 + noise, 50,000 queries with their true NN."""
    R = 64
    band = _band(gb, ctx, sphere5k, R, -1, -1, knn_k=0)
    sets, q, s = _step_inputs(sphere5k, R, -1, -1, 50000, 2.0 / R, seed=2, use_nn=True)
    D, _ = _set_field(gb, band, sets, R, 0.5, 0.1, seed=1)
    _check_step(gb, band, R, sets, q, s, (1.0, 1.0, 0.005), D)


@pytest.mark.parametrize("weights", [(1.0, 1.0, 0.005), (2.0, 0.5, 0.3)])
def test_step_band_object_full_batch(gb, ctx, object100k, weights):
    """Single-object workload at full size: 256^3 band of 8^3 bricks, batch 262,144."""
    R = 256
    band = _band(gb, ctx, object100k, R, 2, 2, knn_k=0)
    c = 0.5 * (object100k.min(0) + object100k.max(0))
    sets, q, s = _step_inputs(object100k, R, 2, 2, 262_144, 2.0 / R, seed=4, use_nn=False)
    D, _ = _set_field(gb, band, sets, R, 0.3, 2e-3, seed=3, center=c)
    _check_step(gb, band, R, sets, q, s, weights, D)


def test_step_flags_and_override(gb, ctx, sphere5k):
    R = 64
    band = _band(gb, ctx, sphere5k, R, 2, 3, knn_k=0)
    sets, q, s = _step_inputs(sphere5k, R, 2, 3, 12345, 0.05, seed=10, use_nn=False)
    D, vals = _set_field(gb, band, sets, R, 0.45, 0.05, seed=9)
    w = (1.0, 1.0, 0.005)
    _check_step(gb, band, R, sets, q, s, w, D, flags=gb.GP_STEP_NO_TV)
    _check_step(gb, band, R, sets, q, s, w, D, flags=gb.GP_STEP_LOSS_ONLY)
    # Override values: the same float32 numbers on both sides.
    ov = (vals.astype(np.float64) * 1.1 + 0.01).astype(np.float32)
    D_ov = np.zeros_like(D)
    req = sets["required"]
    D_ov[req] = (D[req] * 1.1 + 0.01).astype(np.float32)
    _check_step(gb, band, R, sets, q, s, w, D_ov, d_override=ov)


def test_step_edge_cases(gb, ctx, sphere5k):
    R = 32
    band = _band(gb, ctx, sphere5k, R, 1, 1, knn_k=0)
    sets = o.band_sets(sphere5k, R, 1, 1)
    D, _ = _set_field(gb, band, sets, R, 0.4, 0.05, seed=1)
    w = (1.0, 1.0, 0.005)
    empty = np.zeros((0, 3), np.float32)
    ref = _check_step(gb, band, R, sets, empty, empty, w, D)            # B = 0: TV only
    assert ref["Bv"] == 0
    outside = np.array([[1.5, 0, 0], [0, -1.0000001, 0], [0, 0, 1.0], [0.9, 0.9, 0.9]], np.float32)
    ref = _check_step(gb, band, R, sets, outside, sphere5k[:4], w, D)   # all masked
    assert ref["Bv"] == 0
    # Queries snapped onto cell faces (one coordinate on a grid plane), among
    # them brick faces (planes 8k), near the surface so that they are valid.
    h = 2.0 / R
    rng = np.random.default_rng(3)
    base = sphere5k[rng.choice(len(sphere5k), 400, replace=False)].astype(np.float64)
    qs = base + rng.normal(scale=0.3 * h, size=base.shape)
    axis = rng.integers(0, 3, len(qs))
    plane = np.round((qs[np.arange(len(qs)), axis] + 1) / h)
    plane[::3] = np.round(plane[::3] / 8) * 8
    qs[np.arange(len(qs)), axis] = -1 + h * plane
    qs = qs.astype(np.float32)
    ss = sphere5k[o.nearest_point(qs, sphere5k)]
    ref = _check_step(gb, band, R, sets, qs, ss, w, D)
    assert ref["Bv"] > 300


def test_step_deterministic_is_bitwise_repeatable(gb, ctx, object100k):
    R = 256
    band = _band(gb, ctx, object100k, R, 2, 2, knn_k=0, deterministic=True)
    c = 0.5 * (object100k.min(0) + object100k.max(0))
    sets, q, s = _step_inputs(object100k, R, 2, 2, 100_000, 2.0 / R, seed=5, use_nn=False)
    D, _ = _set_field(gb, band, sets, R, 0.3, 0.002, seed=4, center=c)
    w = (1.0, 1.0, 0.005)
    ref = _check_step(gb, band, R, sets, q, s, w, D, flags=gb.GP_STEP_DETERMINISTIC)
    ijk, d, fl, exists = export_band(band)
    qf, sf = _filter_ambiguous(D, R, sets, q, s)
    g1, l1 = _run_step(gb, band, qf, sf, w, gb.GP_STEP_DETERMINISTIC)
    g2, l2 = _run_step(gb, band, qf, sf, w, gb.GP_STEP_DETERMINISTIC)
    assert np.array_equal(g1, g2) and np.array_equal(l1, l2)
    g3, _ = _run_step(gb, band, qf, sf, w, 0)
    keys = vertex_keys(ijk[exists], R)
    assert_grad_close(g3[exists], g1[exists].astype(np.float64), 2 * ref["abs_terms"][keys],
                      what="atomic vs deterministic")
    assert ref["Bv"] > 90_000


def _spatial_order(q, R):
    """Records sorted by the cell key of q (neighbouring records share cells,
    as in the sampler's spatial batches)."""
    cq = np.clip(np.floor((q.astype(np.float64) + 1) * R / 2).astype(np.int64), 0, R - 1)
    return np.argsort(cq[:, 0] + R * (cq[:, 1] + R * cq[:, 2]), kind="stable")


def _morton_order(s, R):
    """Records sorted by the Morton code of the cell of s, as the sampler's
    spatial batches list their source points."""
    c = np.clip(np.floor((s.astype(np.float64) + 1) * R / 2).astype(np.int64), 0, R - 1)
    code = np.zeros(len(s), np.int64)
    for b in range(11):
        for a in range(3):
            code |= ((c[:, a] >> b) & 1) << (3 * b + a)
    return np.argsort(code, kind="stable")


@pytest.mark.parametrize("form,rpt,bps", [("window", 1, 4), ("window", 2, 2), ("window_staged", 1, 2),
                                          ("window_staged", 2, 2)])
def test_step_windowed_forms_match_oracle(gb, ctx, object100k, sphere5k, form, rpt, bps):
    """The windowed query pass (a tile's in-window corner gradients summed in
    shared memory and written once; with staging, the window bricks copied in
    bulk) against the oracle: records in Morton order of their source cell
    (most cells in the window) in a batch of several tiles per block with a
    ragged last tile, the same records in random order (few in the window),
    batches shorter than a tile, tiles whose anchor record is outside the
    band or not finite, records in one cell, and a dense grid whose windows
    meet the grid boundary."""
    import torch
    f = gb.GP_QUERY_WINDOW if form == "window" else gb.GP_QUERY_WINDOW_STAGED
    R = 256
    band = _band(gb, ctx, object100k, R, 2, 2, knn_k=0)
    c = 0.5 * (object100k.min(0) + object100k.max(0))
    sets, q, s = _step_inputs(object100k, R, 2, 2, 400_123, 2.0 / R, seed=41, use_nn=False)
    D, _ = _set_field(gb, band, sets, R, 0.3, 2e-3, seed=42, center=c)
    gb.gp_band_set_query_form(band, f)
    gb.gp_band_set_query_tiles(band, rpt, bps)
    assert gb.gp_band_query_shape(band) == {"records_per_thread": rpt, "blocks_per_sm": bps, "form": f}
    order = _morton_order(s, R)
    qo, so = q[order], s[order]
    ref = _check_step(gb, band, R, sets, qo, so, (1.0, 1.0, 0.005), D)
    assert ref["Bv"] > 350_000
    _check_step(gb, band, R, sets, q[:150_000], s[:150_000], (2.0, 0.5, 0.3), D)
    for n in (1, 100, 513):
        _check_step(gb, band, R, sets, qo[:n], so[:n], (1.0, 1.0, 0.005), D)
    # Anchors outside the band (a far corner of the domain) and not finite:
    # those tiles take the direct path for every cell.
    qa, sa = qo[:2048].copy(), so[:2048].copy()
    sa[256] = (0.99, 0.99, 0.99)
    sa[512 + 256] = (np.nan, 0.0, 0.0)
    _check_step(gb, band, R, sets, qa, sa, (1.0, 1.0, 0.005), D)
    # Every record in one cell: all contributions meet on the same 8 slots.
    Rs = 64
    bs = _band(gb, ctx, sphere5k, Rs, 2, 2, knn_k=0)
    gb.gp_band_set_query_form(bs, f)
    gb.gp_band_set_query_tiles(bs, rpt, bps)
    sets_s = o.band_sets(sphere5k, Rs, 2, 2)
    Ds, _ = _set_field(gb, bs, sets_s, Rs, 0.5, 0.05, seed=43)
    h = 2.0 / Rs
    cell = np.floor((sphere5k[0].astype(np.float64) + 1) / h)
    rng = np.random.default_rng(44)
    q1 = (-1 + h * (cell + rng.uniform(0.05, 0.95, size=(3000, 3)))).astype(np.float32)
    ref = _check_step(gb, bs, Rs, sets_s, q1, np.repeat(sphere5k[:1], len(q1), axis=0), (1.0, 1.0, 0.005), Ds)
    assert ref["Bv"] > 2500
    # Dense grid: the windows of bricks on the grid boundary.
    bd = _band(gb, ctx, sphere5k, Rs, -1, -1, knn_k=0)
    gb.gp_band_set_query_form(bd, f)
    gb.gp_band_set_query_tiles(bd, rpt, bps)
    sets_d, qd, sd = _step_inputs(sphere5k, Rs, -1, -1, 30_000, 4.0 / Rs, seed=45, use_nn=True)
    Dd, _ = _set_field(gb, bd, sets_d, Rs, 0.5, 0.1, seed=46)
    od = _morton_order(sd, Rs)
    _check_step(gb, bd, Rs, sets_d, qd[od], sd[od], (1.0, 1.0, 0.005), Dd)
    # A changed form and a bad one.
    with pytest.raises(gb.GridPullError):
        gb.gp_band_set_query_form(band, 3)
    gb.gp_band_check(band)
    gb.gp_band_check(bs)
    gb.gp_band_check(bd)


@pytest.mark.parametrize("rpt,bps", [(1, 2), (1, 3), (1, 4), (2, 2), (2, 3), (2, 4)])
def test_step_tile_shapes_match_oracle(gb, ctx, object100k, rpt, bps):
    """The fused step kernel at every launch shape the autotuner can pick, on
    spatially ordered records (neighbouring threads reduce into the same
    corners) and on records in random order."""
    R = 256
    band = _band(gb, ctx, object100k, R, 2, 2, knn_k=0)
    c = 0.5 * (object100k.min(0) + object100k.max(0))
    sets, q, s = _step_inputs(object100k, R, 2, 2, 60_000, 2.0 / R, seed=11, use_nn=False)
    D, _ = _set_field(gb, band, sets, R, 0.3, 2e-3, seed=12, center=c)
    gb.gp_band_set_query_tiles(band, rpt, bps)
    order = _spatial_order(q, R)
    _check_step(gb, band, R, sets, q[order], s[order], (1.0, 1.0, 0.005), D)
    _check_step(gb, band, R, sets, q, s, (2.0, 0.5, 0.3), D)


def test_step_records_in_one_cell(gb, ctx, sphere5k):
    """Thousands of records whose q and NN(q) share one cell: every
    contribution lands on the same 8 vertices."""
    R = 64
    band = _band(gb, ctx, sphere5k, R, 2, 2, knn_k=0)
    sets = o.band_sets(sphere5k, R, 2, 2)
    D, _ = _set_field(gb, band, sets, R, 0.5, 0.05, seed=21)
    h = 2.0 / R
    p0 = sphere5k[0].astype(np.float64)
    cell = np.floor((p0 + 1) / h)
    rng = np.random.default_rng(22)
    q = (-1 + h * (cell + rng.uniform(0.05, 0.95, size=(6000, 3)))).astype(np.float32)
    s = np.repeat(sphere5k[:1], len(q), axis=0)
    ref = _check_step(gb, band, R, sets, q, s, (1.0, 1.0, 0.005), D)
    assert ref["Bv"] > 5000
    gb.gp_band_set_query_tiles(band, 2, 3)
    _check_step(gb, band, R, sets, q, s, (1.0, 1.0, 0.005), D)


def test_step_deterministic_overflow_raises_numeric(gb, ctx, sphere5k):
    """A constant field has grad f = 0, so the normal is taken against the
    1e-12 floor and a record's corner contributions reach ~1e13 (one valid
    record: B_v = 1, so the 1/B_v scaling leaves them so), beyond the
    fixed-point sums' limit of 2^42: the step raises GP_ERR_NUMERIC (read by
    gp_band_check) instead of wrapping around."""
    import torch
    R = 64
    band = _band(gb, ctx, sphere5k, R, -1, -1, knn_k=0, deterministic=True)
    gb.gp_band_set_values(band, torch.ones(band.V_stored, dtype=torch.float32, device="cuda"))
    q = (sphere5k[:1] * 1.01).astype(np.float32)
    gb.gp_band_check(band)  # clean before the step
    _, loss = _run_step(gb, band, q, sphere5k[:1], (1.0, 1.0, 0.005), gb.GP_STEP_DETERMINISTIC)
    assert loss[gb.GP_LOSS_BV] == 1
    with pytest.raises(gb.GridPullError, match="GP_ERR_NUMERIC|numeric"):
        gb.gp_band_check(band)
    gb.gp_band_check(band)  # the flag was cleared by the read


def test_autotune_picks_a_shape_and_leaves_the_band(gb, ctx, object100k):
    import torch
    R = 256
    band = _band(gb, ctx, object100k, R, 2, 2, knn_k=0)
    sets, q, s = _step_inputs(object100k, R, 2, 2, 50_000, 2.0 / R, seed=13, use_nn=False)
    c = 0.5 * (object100k.min(0) + object100k.max(0))
    D, vals = _set_field(gb, band, sets, R, 0.3, 2e-3, seed=14, center=c)
    order = _spatial_order(q, R)
    rec = torch.from_numpy(np.ascontiguousarray(np.concatenate([q[order], s[order]], axis=1), np.float32)).cuda()
    before = gb.gp_band_values(band)[0].clone()
    tune = gb.gp_band_autotune(band, rec, len(q))
    assert tune["records_per_thread"] in (1, 2) and tune["blocks_per_sm"] in (2, 3, 4)
    assert tune["form"] in (gb.GP_QUERY_DIRECT, gb.GP_QUERY_WINDOW, gb.GP_QUERY_WINDOW_STAGED)
    assert gb.gp_band_query_shape(band) == tune
    assert torch.equal(before, gb.gp_band_values(band)[0])
    _check_step(gb, band, R, sets, q[order], s[order], (1.0, 1.0, 0.005), D)
    with pytest.raises(gb.GridPullError):
        gb.gp_band_set_query_tiles(band, 3, 3)


def test_step_rejects_misaligned_buffers(gb, ctx, sphere5k):
    import torch
    band = _band(gb, ctx, sphere5k, 32, 1, 1, knn_k=0)
    rec = torch.zeros((11, 6), dtype=torch.float32, device="cuda")
    grad = torch.zeros(band.V_stored + 4, dtype=torch.float32, device="cuda")
    loss = torch.zeros(8, dtype=torch.float32, device="cuda")
    gb.gp_step(band, rec, 10, grad[4:], loss)                      # 16-byte aligned view
    with pytest.raises(gb.GridPullError):
        gb.gp_step(band, rec, 10, grad[1:], loss)                  # gradient off by 4 bytes
    with pytest.raises(gb.GridPullError):
        gb.gp_step(band, rec.view(-1)[1:], 10, grad[:band.V_stored], loss)  # records off by 4 bytes
    vals = torch.zeros(band.V_stored + 4, dtype=torch.float32, device="cuda")
    gb.gp_step(band, rec, 10, grad[4:], loss, d=vals[4:])             # 16-byte aligned values
    with pytest.raises(gb.GridPullError):
        gb.gp_step(band, rec, 10, grad[4:], loss, d=vals[1:band.V_stored + 1])  # values off by 4 bytes


def test_step_deterministic_needs_band_flag(gb, ctx, sphere5k):
    band = _band(gb, ctx, sphere5k, 32, 1, 1, knn_k=0)
    with pytest.raises(gb.GridPullError):
        _run_step(gb, band, sphere5k[:10], sphere5k[:10], (1, 1, 0.005), gb.GP_STEP_DETERMINISTIC)


# ------------------------------------------------------------------ Adam
def test_update_matches_oracle(gb, ctx, sphere5k):
    import torch
    R = 64
    band = _band(gb, ctx, sphere5k, R, 2, 2, knn_k=0)
    sets = o.band_sets(sphere5k, R, 2, 2)
    D, vals = _set_field(gb, band, sets, R, 0.5, 0.01, seed=0)
    ijk, _, fl, exists = export_band(band)
    train = exists & ((fl & 2) != 0)
    keys = vertex_keys(ijk, R)
    d0 = vals.astype(np.float64)                      # what the band holds
    assert np.array_equal(d0[train], D[keys[train]])  # the oracle sees the same trainable values
    rng = np.random.default_rng(0)
    d = d0.copy()
    m = np.zeros_like(d)
    v = np.zeros_like(d)
    m_scale = np.zeros_like(d)   # sum of |terms| of m: its float32 rounding scale
    lr = 1e-3
    for t in range(1, 4):
        g = rng.normal(scale=10.0 ** rng.uniform(-6, 0, size=len(d)), size=len(d)).astype(np.float32)
        gb.gp_update(band, torch.from_numpy(g).cuda(), lr, t)
        # The oracle takes the hyper-parameters the GPU receives: float32 values.
        d_new, m_new, v_new = o.adam(d[train], g[train].astype(np.float64), m[train], v[train], t,
                                     float(np.float32(lr)), float(np.float32(0.9)), float(np.float32(0.999)),
                                     float(np.float32(1e-8)))
        d[train], m[train], v[train] = d_new, m_new, v_new
        dg, mg, vg = [x.cpu().numpy().astype(np.float64) for x in gb.gp_band_values(band)]
        # Adam deltas within 1e-5 lr per step, plus the float32 rounding of the
        # stored values themselves (half an ulp of |d| per step).
        bound = t * (REL_TOL * lr + 2.0 ** -24 * np.abs(d[train]))
        assert np.all(np.abs((dg[train] - d0[train]) - (d[train] - d0[train])) <= bound + 2.0 ** -24 * np.abs(d0[train]))
        assert np.array_equal(dg[exists & ~train], d0[exists & ~train].astype(np.float32).astype(np.float64))
        assert np.all(mg[~train] == 0) and np.all(vg[~train] == 0)
        m_scale[train] = 0.9 * m_scale[train] + 0.1 * np.abs(g[train])
        assert np.all(np.abs(mg[train] - m[train]) <= 1e-5 * m_scale[train])
        assert np.allclose(vg[train], v[train], rtol=1e-5, atol=1e-18)


# -------------------------------------------------------------- fit step
def test_fit_steps_reduce_the_loss(gb, ctx, sphere5k):
    import torch
    from paper_2308_13175_gb300.fit import FitStep
    band = _band(gb, ctx, sphere5k, 64, -1, -1, knn_k=50)
    gb.gp_band_init_sphere(band, (0, 0, 0), 0.5, 0.1, seed=0)
    step = FitStep(band, Q=50_000, B=50_000, seed=0, lr=1e-3)
    losses = [float(step.run(t)[gb.GP_LOSS_TOTAL]) for t in range(30)]
    torch.cuda.synchronize()
    assert all(np.isfinite(losses))
    assert losses[-1] < losses[0]
    gb.gp_band_check(band)


@pytest.mark.parametrize("fused", [True, False])
def test_pipelined_steps_equal_sequential_steps(gb, ctx, sphere5k, fused):
    """FitStep.run_pipelined overlaps each next batch's sampling and nearest
    points with the current step (beside the whole fused descent, or beside
    gp_update after gp_step); with the deterministic sums it must give the
    same values, moments and loss, bit for bit, as running the steps one
    after the other - across epoch boundaries and a short last batch."""
    import torch
    from paper_2308_13175_gb300.fit import FitStep
    R = 64
    bands, fits = [], []
    for _ in range(2):
        band = _band(gb, ctx, sphere5k, R, 2, 2, knn_k=50, deterministic=True)
        gb.gp_band_init_sphere(band, (0.0, 0.0, 0.0), 0.45, 0.01, seed=5)
        bands.append(band)
        fits.append(FitStep(band, Q=40_000, B=15_000, seed=3, lr=1e-3, deterministic=True, fused=fused))
    K = 7
    for t in range(K):
        fits[0].run(t)
    fits[1].run_pipelined(0, K)
    torch.cuda.synchronize()
    for a, b in zip(gb.gp_band_values(bands[0]), gb.gp_band_values(bands[1])):
        assert torch.equal(a, b)
    assert torch.equal(fits[0].loss, fits[1].loss)
    # Two pipelined calls in a row continue where the first stopped.
    for t in range(K, K + 3):
        fits[0].run(t)
    fits[1].run_pipelined(K, 3)
    torch.cuda.synchronize()
    assert torch.equal(gb.gp_band_values(bands[0])[0], gb.gp_band_values(bands[1])[0])
    gb.gp_band_check(bands[1])


@pytest.mark.parametrize("det,form", [(False, 0), (True, 0), (False, 2)])
def test_step_update_equals_step_then_update(gb, ctx, object100k, det, form):
    """gp_step_update (query pass, then one sweep computing L_TV, adding the
    query part and applying Adam into the second value buffer) against
    gp_step then gp_update on an identical band: values, moments and loss
    slots over three steps - bit for bit with the deterministic sums."""
    import torch
    R = 256
    bands = [_band(gb, ctx, object100k, R, 2, 2, knn_k=0, deterministic=det) for _ in range(2)]
    c = 0.5 * (object100k.min(0) + object100k.max(0))
    sets, q, s = _step_inputs(object100k, R, 2, 2, 80_000, 2.0 / R, seed=31, use_nn=False)
    for band in bands:
        _set_field(gb, band, sets, R, 0.3, 2e-3, seed=32, center=c)
        gb.gp_band_set_query_form(band, form)
    if form:
        order = _morton_order(s, R)
        q, s = q[order], s[order]
    rec = torch.from_numpy(np.ascontiguousarray(np.concatenate([q, s], axis=1), np.float32)).cuda()
    flags = gb.GP_STEP_DETERMINISTIC if det else 0
    grad = torch.empty(bands[0].V_stored, dtype=torch.float32, device="cuda")
    la = torch.zeros(8, dtype=torch.float32, device="cuda")
    lb = torch.zeros(8, dtype=torch.float32, device="cuda")
    w = (1.0, 1.0, 0.005)
    d0 = gb.gp_band_values(bands[0])[0].clone()
    for t in range(1, 4):
        gb.gp_step(bands[0], rec, len(q), grad, la, w, flags=flags)
        gb.gp_update(bands[0], grad, 1e-3, t)
        gb.gp_step_update(bands[1], rec, len(q), lb, 1e-3, t, w, flags=flags)
        torch.cuda.synchronize()
        va, vb = gb.gp_band_values(bands[0]), gb.gp_band_values(bands[1])
        if det:
            assert torch.equal(la, lb)
            for x, y in zip(va, vb):
                assert torch.equal(x, y)
        else:
            for k in range(5):
                assert_rel(lb[k].item(), la[k].item(), what=f"slot {k} step {t}")
            # Float sums in different orders: moments norm-wise to 1e-5; the
            # value changes norm-wise to 1e-3 (Adam's m / sqrt(v) amplifies the
            # rounding of gradients that nearly cancel).
            for x, y, name in zip(va[1:], vb[1:], ("m", "v")):
                assert float(torch.linalg.norm(x - y)) <= 1e-5 * float(torch.linalg.norm(x)), (name, t)
            da, db = va[0] - d0, vb[0] - d0
            assert float(torch.linalg.norm(da - db)) <= 1e-3 * float(torch.linalg.norm(da)), t
    # The query gradient is left all zero; the second buffer's frozen values
    # equal the current ones.
    gb.gp_band_check(bands[1])
