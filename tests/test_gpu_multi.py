"""The many-cloud step (gp_multi_*) through the C ABI.

Each step of a multi is checked cloud by cloud: its records bit-exact against
the single-band calls (gp_sample + gp_nn on the same band, key seed + k), its
loss slots and gradient against the FP64 oracle on the band's values before the
step, and its Adam update against the oracle's Adam on the GPU's own gradient.
The clouds differ in size, resolution and band width, their batches end short
(ragged), one of them starts a new epoch at every step, and the steps cross an
epoch boundary of the others.
"""
import numpy as np
import pytest

from oracle import gridpull as o
from paper_2308_13175_gb300 import synth

from gpu_common import REL_TOL, assert_grad_close, assert_rel, build_lib, dense_from_band, export_band, have_gpu, \
    vertex_keys

pytestmark = pytest.mark.gpu

W = (1.0, 1.0, 0.005)
LR, DECAY, EVERY = 1e-3, 0.5, 2
SEED = 1234


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


# (points, R, M1, M2, Q, B): batches per epoch 3 (short last), 3 (short last), 1.
@pytest.fixture(scope="module")
def clouds():
    return [
        (synth.sphere_cloud(4000, 0.5, seed=0), 32, 2, 2, 12000, 5000),
        (synth.object_cloud(20000, seed=1), 64, 2, 2, 40000, 16384),
        (synth.superquadric_cloud(3000, seed=4), 16, 1, 1, 3000, 3000),
    ]


def _make_bands(gb, ctx, clouds):
    """Bands with a sphere start well inside every cloud (f(s) > 0 at every
    point, so no sign of |f(s)| is decided by rounding)."""
    import torch
    bands = []
    for pts, R, M1, M2, _, _ in clouds:
        band = gb.gp_build_band(ctx, torch.from_numpy(np.ascontiguousarray(pts)).cuda(), R, M1, M2, 20)
        c = 0.5 * (pts.min(0) + pts.max(0))
        rmin = float(np.min(np.linalg.norm(pts.astype(np.float64) - c, axis=1)))
        gb.gp_band_init_sphere(band, c, max(0.3 * rmin, 0.01), 1e-3, seed=7)
        bands.append(band)
    return bands


def _batch(t, Q, B):
    nb = -(-Q // B)
    epoch, b = divmod(t, nb)
    first = b * B
    return epoch, first, min(B, Q - first)


def _single_records(gb, band, k, t, Q, B, spatial):
    import torch
    epoch, first, count = _batch(t, Q, B)
    q = torch.empty((count, 3), dtype=torch.float32, device="cuda")
    src = torch.empty(count, dtype=torch.int32, device="cuda")
    rec = torch.empty((count, 6), dtype=torch.float32, device="cuda")
    gb.gp_sample(band, SEED + k, epoch, Q, first, count, q, src, spatial=spatial)
    gb.gp_nn(band, q, None, rec, hint=src)
    return rec.cpu().numpy(), src.cpu().numpy(), count


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.int32)


def _lr_at(t):
    return float(np.float32(float(np.float32(LR)) * DECAY ** (t // EVERY)))


@pytest.mark.parametrize("spatial", [False, True])
def test_multi_steps_match_single_band_calls_and_oracle(gb, ctx, clouds, spatial):
    import torch
    bands = _make_bands(gb, ctx, clouds)
    sets = [o.band_sets(pts, R, M1, M2) for pts, R, M1, M2, _, _ in clouds]
    multi = gb.gp_multi_create(ctx, bands, [c[4] for c in clouds], [c[5] for c in clouds], seed=SEED,
                               spatial=spatial)
    n = len(clouds)
    loss = torch.zeros(8 * n, dtype=torch.float32, device="cuda")
    for t in range(4):
        before = []
        for band in bands:
            ijk, d, fl, exists = export_band(band)
            _, m, v = [x.cpu().numpy().astype(np.float64) for x in gb.gp_band_values(band)]
            before.append((ijk, d.astype(np.float64), fl, exists, m, v))
        gb.gp_multi_step(multi, loss, W, lr=LR, lr_decay=DECAY, lr_every=EVERY)
        L = loss.cpu().numpy().reshape(n, 8)
        for k, ((pts, R, M1, M2, Q, B), band) in enumerate(zip(clouds, bands)):
            rec_v, src_v, grad_v = gb.gp_multi_buffers(multi, k)
            rec, src, grad = rec_v.cpu().numpy(), src_v.cpu().numpy(), grad_v.cpu().numpy()
            # Records: bit-exact against the single-band calls; NaN padding after a short batch.
            want, want_src, count = _single_records(gb, band, k, t, Q, B, spatial)
            assert np.array_equal(_bits(rec[:count]), _bits(want)), f"cloud {k} step {t}: records differ"
            assert np.array_equal(src[:count], want_src)
            assert np.all(np.isnan(rec[count:, :3])) and np.all(src[count:] == -1)
            # Loss and gradient: the oracle on the values before the step and the multi's own records.
            ijk, d0, fl, exists, m0, v0 = before[k]
            D = dense_from_band(d0, ijk, exists, R)
            ref = o.step_loss_grad(D, R, sets[k], rec[:count, :3], rec[:count, 3:], W)
            assert L[k, gb.GP_LOSS_BV] == ref["Bv"] and ref["Bv"] > 0.5 * count
            assert L[k, gb.GP_LOSS_T] == len(sets[k]["tv"])
            for slot, key in ((gb.GP_LOSS_PULL, "l_pull"), (gb.GP_LOSS_GRAD, "l_grad"),
                              (gb.GP_LOSS_SURF, "l_surf"), (gb.GP_LOSS_TV, "l_tv"), (gb.GP_LOSS_TOTAL, "loss")):
                assert_rel(L[k, slot], ref[key], what=f"cloud {k} step {t} {key}")
            assert np.min(np.abs(ref["per_query"]["fs"])) > 1e-3  # no rounding-decided sign
            keys = vertex_keys(ijk[exists], R)
            assert np.all(grad[~exists] == 0.0)
            assert_grad_close(grad[exists], ref["grad"][keys], ref["abs_terms"][keys], what=f"cloud {k} step {t}",
                              kappa_max=ref["kappa_max"])
            # Adam at step t + 1 with the scheduled rate, on the GPU's own gradient.
            _, d1, _, _ = export_band(band)
            _, m1, v1 = [x.cpu().numpy().astype(np.float64) for x in gb.gp_band_values(band)]
            train = exists & ((fl & 2) != 0)
            g = grad[train].astype(np.float64)
            dw, mw, vw = o.adam(d0[train], g, m0[train], v0[train], t + 1, _lr_at(t), float(np.float32(0.9)),
                                float(np.float32(0.999)), float(np.float32(1e-8)))
            tol = REL_TOL * _lr_at(t) + 2.0 ** -23 * np.abs(d0[train])
            assert np.all(np.abs(d1[train] - dw) <= tol), f"cloud {k} step {t}: Adam"
            assert np.array_equal(d1[exists & ~train], d0[exists & ~train].astype(np.float32))
            assert np.all(np.abs(m1[train] - mw) <= 1e-5 * (0.9 * np.abs(m0[train]) + 0.1 * np.abs(g)) + 1e-30)
            assert np.allclose(v1[train], vw, rtol=1e-5, atol=1e-18)
    info = gb.gp_multi_get_info(multi)
    assert info["step"] == 4 and info["error_bits"] == 0 and info["n"] == n
    assert info["total_B"] == sum(c[5] for c in clouds)
    assert info["V_total"] == sum(b.V_stored for b in bands)
    multi.close()


def test_multi_tiny_clouds(gb, ctx):
    """Edge sizes: a one-point cloud (sigma 0, batch of one), a seven-point cloud
    whose epochs end in a short batch (its sigma spans the cloud, so whole
    batches can fall outside the band: B_v = 0), and a 600-point cloud, in one
    multi; four steps, records bit-exact against the single-band calls and loss
    and gradient against the oracle."""
    import torch
    tiny = [
        (synth.sphere_cloud(1, 0.3, seed=11), 8, 1, 1, 1, 1),
        (synth.sphere_cloud(7, 0.4, seed=12), 16, 1, 1, 21, 8),
        (synth.sphere_cloud(600, 0.5, seed=13), 16, 2, 2, 1200, 500),
    ]
    bands = _make_bands(gb, ctx, tiny)
    sets = [o.band_sets(pts, R, M1, M2) for pts, R, M1, M2, _, _ in tiny]
    multi = gb.gp_multi_create(ctx, bands, [c[4] for c in tiny], [c[5] for c in tiny], seed=SEED)
    loss = torch.zeros(8 * len(tiny), dtype=torch.float32, device="cuda")
    for t in range(4):
        before = [export_band(b) for b in bands]
        gb.gp_multi_step(multi, loss, W, lr=LR)
        L = loss.cpu().numpy().reshape(len(tiny), 8)
        for k, ((pts, R, M1, M2, Q, B), band) in enumerate(zip(tiny, bands)):
            rec = gb.gp_multi_buffers(multi, k)[0].cpu().numpy()
            want, _, count = _single_records(gb, band, k, t, Q, B, True)
            assert np.array_equal(_bits(rec[:count]), _bits(want)), f"cloud {k} step {t}"
            assert np.all(np.isnan(rec[count:, :3]))
            ijk, d0, fl, exists = before[k]
            D = dense_from_band(d0.astype(np.float64), ijk, exists, R)
            ref = o.step_loss_grad(D, R, sets[k], rec[:count, :3], rec[:count, 3:], W)
            assert L[k, gb.GP_LOSS_BV] == ref["Bv"], f"cloud {k} step {t}"
            if k == 0:  # sigma 0: the one query is the point itself, always valid
                assert ref["Bv"] == 1
            for slot, key in ((gb.GP_LOSS_PULL, "l_pull"), (gb.GP_LOSS_TV, "l_tv"), (gb.GP_LOSS_TOTAL, "loss")):
                assert_rel(L[k, slot], ref[key], what=f"cloud {k} step {t} {key}")
            grad = gb.gp_multi_buffers(multi, k)[2].cpu().numpy()
            keys = vertex_keys(ijk[exists], R)
            assert_grad_close(grad[exists], ref["grad"][keys], ref["abs_terms"][keys], what=f"cloud {k} step {t}",
                              kappa_max=ref["kappa_max"])
    assert gb.gp_multi_get_info(multi)["error_bits"] == 0
    multi.close()


def test_multi_resume_mid_epoch(gb, ctx, clouds):
    """set_step into the middle of an epoch rebuilds that epoch's order first."""
    import torch
    bands = _make_bands(gb, ctx, clouds)
    multi = gb.gp_multi_create(ctx, bands, [c[4] for c in clouds], [c[5] for c in clouds], seed=SEED)
    loss = torch.zeros(8 * len(clouds), dtype=torch.float32, device="cuda")
    for t in (4, 5, 1):
        gb.gp_multi_set_step(multi, t)
        gb.gp_multi_step(multi, loss, W)
        for k, ((_, _, _, _, Q, B), band) in enumerate(zip(clouds, bands)):
            rec = gb.gp_multi_buffers(multi, k)[0].cpu().numpy()
            want, _, count = _single_records(gb, band, k, t, Q, B, True)
            assert np.array_equal(_bits(rec[:count]), _bits(want)), f"cloud {k} step {t}"
    assert gb.gp_multi_get_info(multi)["step"] == 2


def test_multi_autotune_keeps_state_and_graph_replay_matches_eager(gb, ctx, clouds):
    import torch
    n, K = len(clouds), 5
    Qs, Bs = [c[4] for c in clouds], [c[5] for c in clouds]
    # Eager reference run.
    bands = _make_bands(gb, ctx, clouds)
    multi = gb.gp_multi_create(ctx, bands, Qs, Bs, seed=SEED)
    loss = torch.zeros(8 * n, dtype=torch.float32, device="cuda")
    eager = []
    for _ in range(K):
        gb.gp_multi_step(multi, loss, W, lr=LR)
        eager.append(loss.cpu().numpy().reshape(n, 8).copy())
    eager_rec = [gb.gp_multi_buffers(multi, k)[0].cpu().numpy() for k in range(n)]
    multi.close()
    # Same start, autotuned, one step captured in a CUDA graph and replayed.
    bands = _make_bands(gb, ctx, clouds)
    multi = gb.gp_multi_create(ctx, bands, Qs, Bs, seed=SEED)
    d_before = [export_band(b)[1].copy() for b in bands]
    info = gb.gp_multi_autotune(multi, W)
    assert info["records_per_tile"] in (128, 256, 512)
    for key in ("blocks_per_sm_nn", "blocks_per_sm_query"):
        assert info[key] in (1, 2, 4, 8, 16)
    assert info["blocks_per_sm_tv"] in (5, 10, 15)
    assert info["step"] == 0 and info["error_bits"] == 0
    for b, d0 in zip(bands, d_before):
        assert np.array_equal(export_band(b)[1], d0)
        _, m, v = gb.gp_band_values(b)
        assert float(m.abs().max()) == 0.0 and float(v.abs().max()) == 0.0
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gb.gp_multi_step(multi, loss, W, lr=LR)
    assert gb.gp_multi_get_info(multi)["step"] == 0  # capture runs nothing
    for t in range(K):
        graph.replay()
        got = loss.cpu().numpy().reshape(n, 8)
        assert np.array_equal(got[:, gb.GP_LOSS_BV], eager[t][:, gb.GP_LOSS_BV])
        assert np.allclose(got[:, :5], eager[t][:, :5], rtol=1e-4, atol=1e-7), f"step {t}"
    assert gb.gp_multi_get_info(multi)["step"] == K
    for k in range(n):
        rec = gb.gp_multi_buffers(multi, k)[0].cpu().numpy()
        assert np.array_equal(_bits(rec), _bits(eager_rec[k]))
    del graph
    multi.close()


def test_multi_rejects_bad_input(gb, ctx, clouds):
    import torch
    pts, R, M1, M2, Q, B = clouds[0]
    tp = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    band = gb.gp_build_band(ctx, tp, R, M1, M2, 20)
    with pytest.raises(gb.GridPullError):
        gb.gp_multi_create(ctx, [band], [Q], [Q + 1])        # B > Q
    with pytest.raises(gb.GridPullError):
        gb.gp_multi_create(ctx, [band], [2 ** 31], [10])      # Q too large
    with pytest.raises(gb.GridPullError):
        gb.gp_multi_create(ctx, [band, band], [Q, Q], [B, B])  # the same band twice
    with pytest.raises(gb.GridPullError):
        gb.gp_multi_create(ctx, [gb.gp_build_band(ctx, tp, R, M1, M2, 0)], [Q], [B])  # no sigma
    with pytest.raises(gb.GridPullError):
        gb.gp_multi_create(ctx, [gb.gp_build_band(ctx, tp, R, M1, M2, 20, deterministic=True)], [Q], [B])
    multi = gb.gp_multi_create(ctx, [band], [Q], [B])
    with pytest.raises(gb.GridPullError):
        gb.gp_multi_set_step(multi, -1)
    with pytest.raises(gb.GridPullError):
        gb.gp_multi_buffers(multi, 1)
    multi.close()


def test_deterministic_multi_repeats_bitwise_and_matches_atomic(gb, ctx, clouds):
    """GP_MULTI_DETERMINISTIC: two multis over identical bands give the same
    values, moments and loss slots bit for bit after four steps (across an
    epoch boundary, spatial order, autotuned first), and agree with the
    float-atomic multi to float rounding."""
    import torch
    runs = []
    for det in (True, True, False):
        bands = _make_bands(gb, ctx, clouds)
        m = gb.gp_multi_create(ctx, bands, [c[4] for c in clouds], [c[5] for c in clouds], seed=11, spatial=True,
                               deterministic=det)
        gb.gp_multi_autotune(m, (1.0, 1.0, 0.005))
        loss = torch.zeros(8 * len(bands), dtype=torch.float32, device="cuda")
        for _ in range(4):
            gb.gp_multi_step(m, loss, (1.0, 1.0, 0.005), lr=1e-3)
        torch.cuda.synchronize()
        assert gb.gp_multi_get_info(m)["error_bits"] == 0
        runs.append(([tuple(x.clone() for x in gb.gp_band_values(b)) for b in bands], loss.clone()))
        m.close()
    (va, la), (vb, lb), (vc, lc) = runs
    assert torch.equal(la, lb)
    for a, b in zip(va, vb):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    for k in range(len(clouds)):
        for slot in (gb.GP_LOSS_TOTAL, gb.GP_LOSS_PULL, gb.GP_LOSS_GRAD, gb.GP_LOSS_SURF, gb.GP_LOSS_TV):
            assert_rel(lc[8 * k + slot].item(), la[8 * k + slot].item(), tol=1e-4, what=f"cloud {k} slot {slot}")
        # values: Adam moves each by at most about lr per step; float sums in
        # other orders can flip a near-zero gradient's step, nothing more.
        assert float((vc[k][0] - va[k][0]).abs().max()) <= 2 * 4 * 1e-3
