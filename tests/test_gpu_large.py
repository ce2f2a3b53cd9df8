"""Parity at the full sizes the benchmark runs: the superquadric union (2M
points, 512^3 band, batch 4,194,304) and the indoor scene (10M points, 1024^3
band, batch 2,097,152), through the launch configuration the bench times
(gp_nn seeded with each query's source point, which takes the sorted-search
kernel at these batch sizes; gp_step on the whole batch).

The oracle cannot evaluate a whole batch at these sizes, so it checks samples
and properties that hold at any size:
  * NN indices of 2,000 sampled queries against brute force over the whole
    cloud (on all host cores), exactly;
  * the step on a record subset (the sampled queries with their brute-force
    NN) against the oracle on a band-sparse value store: loss slots, B_v and
    the gradient at every vertex the subset touches (L_TV left out);
  * L_TV over the whole TV set (the oracle in chunks) and its gradient at
    sampled TV vertices;
  * the whole batch: B_v counted by gp_nn equals the step's, losses finite.
Values come from a closed-form field of the vertex coordinates, evaluated on
both sides; queries from the seeded generators (never from the library)."""
import os
import tempfile

import numpy as np
import pytest

from oracle import gridpull as o
from paper_2308_13175_gb300 import synth

from gpu_common import assert_grad_close, assert_rel, build_lib, export_band, have_gpu, vertex_keys

pytestmark = pytest.mark.gpu

CONFIGS = {
    "superquadric": dict(cloud=lambda: synth.superquadric_cloud(2_000_000, seed=4), R=512, B=4_194_304),
    "scene": dict(cloud=lambda: synth.room_cloud(10_000_000, seed=2), R=1024, B=2_097_152),
}
N_NN = 2000
W = (1.0, 1.0, 0.005)


def field(ijk: np.ndarray, R: int) -> np.ndarray:
    """A signed-distance-like closed form with short-range variation: the
    distance to a sphere of radius 0.35 plus 2e-3 h-scaled ripples, from the
    integer vertex coordinates (float32, as stored)."""
    h = 2.0 / R
    v = -1.0 + h * np.asarray(ijk, np.float64)
    d = np.linalg.norm(v, axis=1) - 0.35
    ripple = np.sin(37.0 * v[:, 0] + 0.5) * np.sin(41.0 * v[:, 1] + 1.0) * np.sin(43.0 * v[:, 2] + 1.5)
    return (d + 0.3 * h * ripple).astype(np.float32)


def field_store(keys: np.ndarray, R: int) -> o.SparseValues:
    keys = np.unique(np.asarray(keys, np.int64))
    return o.SparseValues(keys, field(o.key_to_vertex(keys, R), R).astype(np.float64))


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_full_size_parity(name):
    if not have_gpu():
        pytest.skip("no CUDA device")
    import torch
    from oracle.parallel import OraclePool
    build_lib()
    from paper_2308_13175_gb300 import binding as gb
    cfg = CONFIGS[name]
    R, B = cfg["R"], cfg["B"]
    h = 2.0 / R
    pts = cfg["cloud"]()
    J = len(pts)
    ctx = gb.gp_create(0)
    band = gb.gp_build_band(ctx, torch.from_numpy(pts).cuda(), R, 2, 2, 50)
    ijk, _, _, exists = export_band(band)
    vals = np.zeros(band.V_stored, np.float32)
    vals[exists] = field(ijk[exists], R)
    gb.gp_band_set_values(band, torch.from_numpy(vals).cuda())
    keys_stored = vertex_keys(ijk[exists], R)
    slots_stored = np.flatnonzero(exists)
    order = np.argsort(keys_stored)
    keys_sorted, slots_sorted = keys_stored[order], slots_stored[order]

    def slots_of(keys):
        pos = np.searchsorted(keys_sorted, keys)
        assert np.all(keys_sorted[np.minimum(pos, len(keys_sorted) - 1)] == keys)
        return slots_sorted[pos]

    # The bench's batch shape through the bench's NN launch: B queries around
    # uniformly chosen points, seeded with their source points.
    q, j = synth.gaussian_queries(pts, B, 2 * h, seed=17)
    q_t = torch.from_numpy(q).cuda()
    nn = torch.empty(B, dtype=torch.int32, device="cuda")
    rec = torch.empty((B, 6), dtype=torch.float32, device="cuda")
    nvalid = torch.zeros(1, dtype=torch.int32, device="cuda")
    gb.gp_nn(band, q_t, nn, rec, hint=torch.from_numpy(j.astype(np.int32)).cuda(), nvalid_out=nvalid)
    grad = torch.empty(band.V_stored, dtype=torch.float32, device="cuda")
    loss = torch.zeros(8, dtype=torch.float32, device="cuda")
    gb.gp_step(band, rec, B, grad, loss, W, nvalid=nvalid)
    torch.cuda.synchronize()
    lf = loss.cpu().numpy()
    assert lf[gb.GP_LOSS_BV] == float(int(nvalid.item())) > 0.5 * B
    assert np.all(np.isfinite(lf))
    nn = nn.cpu().numpy()

    # 1. NN of sampled queries against brute force over the whole cloud.
    rng = np.random.default_rng(5)
    pick = np.sort(rng.choice(B, N_NN, replace=False))
    tmp = tempfile.mkdtemp(prefix="gp_large_")
    np.save(os.path.join(tmp, "pts.npy"), pts)
    pool = OraclePool(os.path.join(tmp, "pts.npy"))
    try:
        paths = []
        for k, part in enumerate(np.array_split(q[pick], pool.cores)):
            pth = os.path.join(tmp, f"q{k}.npy")
            np.save(pth, part)
            paths.append(pth)
        nn_ref = pool.nn_indices(paths)
    finally:
        pool.close()
    assert np.array_equal(nn[pick], nn_ref), f"{np.count_nonzero(nn[pick] != nn_ref)} NN indices differ"

    # 2. The step on the sampled records against the band-sparse oracle.
    sets_v = o.band_vertex_sets_bitmap(pts, R, 2, 2)
    occ = sets_v["occupied"]
    member = lambda c: o.in_dilated_band(c, occ, 2, R, keys_sorted=True)
    qs, ss = q[pick], pts[nn_ref]
    cq, lq, inside = o.cell_and_local(qs, R)
    cq = np.clip(cq, 0, R - 1)
    cs, ls, _ = o.cell_and_local(ss, R)
    cs, _ = o.clamp_cell(cs, ls, R)
    valid = inside & member(o.cell_key(cq, R)) & member(o.cell_key(cs, R))
    touched = np.unique(np.concatenate([o.vertex_key(c[valid] + d, R) for c in (cq, cs) for d in o.CORNERS]))
    store = field_store(touched, R)
    ref = o.step_loss_grad(store, R, {"pull_cells": member, "tv": np.zeros(0, np.int64)}, qs, ss, W)
    rec_s = torch.from_numpy(np.ascontiguousarray(np.concatenate([qs, ss], axis=1), np.float32)).cuda()
    gs = torch.full((band.V_stored,), 7.0, dtype=torch.float32, device="cuda")
    ls_t = torch.zeros(8, dtype=torch.float32, device="cuda")
    gb.gp_step(band, rec_s, N_NN, gs, ls_t, W, flags=gb.GP_STEP_NO_TV)
    torch.cuda.synchronize()
    lsub = ls_t.cpu().numpy()
    assert lsub[gb.GP_LOSS_BV] == ref["Bv"] > 0.5 * N_NN
    for slot, key in ((gb.GP_LOSS_PULL, "l_pull"), (gb.GP_LOSS_GRAD, "l_grad"), (gb.GP_LOSS_SURF, "l_surf"),
                      (gb.GP_LOSS_TOTAL, "loss")):
        assert_rel(lsub[slot], ref[key], what=f"{name} {key}")
    g = gs.cpu().numpy()
    sl = slots_of(store.keys)
    assert_grad_close(g[sl], ref["grad"], ref["abs_terms"], what=f"{name} subset grad", kappa_max=ref["kappa_max"])
    others = np.ones(band.V_stored, bool)
    others[sl] = False
    assert np.all(g[others & exists] == 0.0) and np.all(g[~exists] == 0.0)

    # 3. L_TV over the whole TV set (gp_step with no records) and its gradient
    # at sampled TV vertices.
    T = sets_v["tv"]
    g0 = torch.empty(band.V_stored, dtype=torch.float32, device="cuda")
    l0 = torch.zeros(8, dtype=torch.float32, device="cuda")
    gb.gp_step(band, rec, 0, g0, l0, W)
    torch.cuda.synchronize()
    l0 = l0.cpu().numpy()
    assert l0[gb.GP_LOSS_T] == len(T)
    tv_sum = 0.0
    for part in np.array_split(T, max(1, len(T) // 2_000_000)):
        nb, ok = o.axis_neighbours(part, R)
        st = field_store(np.concatenate([part, nb[ok]]), R)
        tv_sum += o.tv_term(st, R, part, with_grad=False, n_tv=len(T))[0]
    assert_rel(l0[gb.GP_LOSS_TV], tv_sum, what=f"{name} L_TV")
    sample = np.sort(rng.choice(T, 5000, replace=False))
    nb, ok = o.axis_neighbours(sample, R)
    terms = np.intersect1d(np.unique(np.concatenate([sample, nb[ok]])), T)  # TV terms touching the sample
    nb2, ok2 = o.axis_neighbours(terms, R)
    st = field_store(np.concatenate([terms, nb2[ok2]]), R)
    _, tg, _ = o.tv_term(st, R, terms, True, n_tv=len(T))
    tabs = o.tv_term_abs(st, R, terms, n_tv=len(T))
    at = st.index(sample)
    gt = g0.cpu().numpy()[slots_of(sample)]
    assert_grad_close(gt, W[0] * tg[at], W[0] * tabs[at], what=f"{name} TV grad")
    gb.gp_band_check(band)
