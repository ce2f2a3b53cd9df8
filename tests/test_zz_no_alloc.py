"""gp_step_dense_noalloc: the query part of the step on a caller-owned dense
grid, for callers that cannot allocate device memory (its scratch is a fixed
array inside the library).  Checked through the C ABI against the float64
oracle and against gp_step on a dense band (every cell in the pull band, L_TV
left out), on two calls in a row so that the second call sees the scratch the
first one left behind; the caller's current device is unchanged by the calls.

This file is collected last on purpose: it must pass on its own in a fresh
process and after every other test."""
import numpy as np
import pytest

from oracle import gridpull as o
from paper_2308_13175_gb300 import synth

from gpu_common import assert_grad_close, assert_rel, build_lib, export_band, have_gpu, vertex_keys

pytestmark = pytest.mark.gpu


def test_dense_noalloc_matches_gp_step_twice():
    if not have_gpu():
        pytest.skip("no CUDA device")
    import torch
    build_lib()
    from paper_2308_13175_gb300 import binding as gb
    R = 64
    pts = synth.sphere_cloud(5000, 0.5, seed=0)
    ctx = gb.gp_create(0)
    band = gb.gp_build_band(ctx, torch.from_numpy(pts).cuda(), R, -1, -1, 0)
    ijk, _, _, exists = export_band(band)
    keys = vertex_keys(ijk[exists], R)
    n1 = R + 1
    dense = synth.sphere_field(synth.all_vertices(R), R, 0.5, 0.05, seed=1)
    vals = np.zeros(band.V_stored, np.float32)
    vals[exists] = dense[keys]
    gb.gp_band_set_values(band, torch.from_numpy(vals).cuda())
    d_dense = torch.from_numpy(dense).cuda()
    w = (1.0, 1.0, 0.005)
    for call, seed in enumerate((3, 4)):
        q, j = synth.gaussian_queries(pts, 30000 + 777 * call, 0.05, seed=seed)
        q[:50] = np.float32(1.5)                      # outside the domain: masked on both sides
        rec = torch.from_numpy(np.concatenate([q, pts[j]], axis=1)).cuda()
        B = len(q)
        g_band = torch.empty(band.V_stored, dtype=torch.float32, device="cuda")
        l_band = torch.zeros(8, dtype=torch.float32, device="cuda")
        gb.gp_step(band, rec, B, g_band, l_band, w, flags=gb.GP_STEP_NO_TV)
        g_na = torch.full((n1 ** 3,), 3.0, dtype=torch.float32, device="cuda")
        l_na = torch.full((8,), 3.0, dtype=torch.float32, device="cuda")
        dev_before = torch.cuda.current_device()
        gb.gp_step_dense_noalloc(ctx, R, d_dense, rec, B, g_na, l_na, w)
        assert torch.cuda.current_device() == dev_before
        torch.cuda.synchronize()
        lb, ln = l_band.cpu().numpy(), l_na.cpu().numpy()
        assert ln[gb.GP_LOSS_BV] == lb[gb.GP_LOSS_BV] == B - 50
        for slot in (gb.GP_LOSS_TOTAL, gb.GP_LOSS_PULL, gb.GP_LOSS_GRAD, gb.GP_LOSS_SURF):
            assert_rel(ln[slot], lb[slot], what=f"call {call} slot {slot}")
        gn = g_na.cpu().numpy().astype(np.float64)
        gband = g_band.cpu().numpy().astype(np.float64)
        # The float64 oracle on the same grid and records: the loss slots of
        # this entry point against it directly, not only against gp_step.
        sets = {"pull_cells": np.arange(R ** 3), "tv": np.zeros(0, np.int64)}
        ref = o.step_loss_grad(dense.astype(np.float64), R, sets, q, pts[j], w)
        assert ref["Bv"] == B - 50
        for slot, want in ((gb.GP_LOSS_TOTAL, ref["loss"]), (gb.GP_LOSS_PULL, ref["l_pull"]),
                           (gb.GP_LOSS_GRAD, ref["l_grad"]), (gb.GP_LOSS_SURF, ref["l_surf"])):
            assert_rel(ln[slot], want, what=f"call {call} slot {slot} vs oracle")
        assert_grad_close(gn[keys], ref["grad"][keys], ref["abs_terms"][keys], what=f"call {call} grad vs oracle")
        # Both GPU sides are float32 sums in different atomic orders: each may be
        # off by the tolerance times the oracle's conditioning scale of the vertex.
        assert_grad_close(gn[keys], gband[exists], 2 * ref["abs_terms"][keys], what=f"call {call} grad")
        assert np.all(gn[np.setdiff1d(np.arange(n1 ** 3), keys)] == 0)


def test_dense_noalloc_rejects_sizes_beyond_its_scratch():
    if not have_gpu():
        pytest.skip("no CUDA device")
    import torch
    build_lib()
    from paper_2308_13175_gb300 import binding as gb
    ctx = gb.gp_create(0)
    R = 8
    d = torch.zeros((R + 1) ** 3, dtype=torch.float32, device="cuda")
    loss = torch.zeros(8, dtype=torch.float32, device="cuda")
    grad = torch.zeros((R + 1) ** 3, dtype=torch.float32, device="cuda")
    big = 1_048_577
    rec = torch.zeros((big, 6), dtype=torch.float32, device="cuda")
    with pytest.raises(gb.GridPullError, match="1048576"):
        gb.gp_step_dense_noalloc(ctx, R, d, rec, big, grad, loss)
    with pytest.raises(gb.GridPullError, match="power of two"):
        gb.gp_step_dense_noalloc(ctx, 4, d, rec, 10, grad, loss)
