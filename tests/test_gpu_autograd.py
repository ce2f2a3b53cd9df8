"""The differentiation form: gp_step behind torch.autograd.Function, checked
against gp_step itself, the plain-PyTorch autograd form (float64) and central
finite differences of its own forward."""
import numpy as np
import pytest

from oracle import gridpull as o
from paper_2308_13175_gb300 import synth

from gpu_common import assert_grad_close, build_lib, export_band, have_gpu, vertex_keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not have_gpu():
        pytest.skip("no CUDA device")
    import torch
    build_lib()
    from paper_2308_13175_gb300 import binding as gb
    R = 64
    pts = synth.sphere_cloud(5000, 0.5, seed=0)
    ctx = gb.gp_create(0)
    band = gb.gp_build_band(ctx, torch.from_numpy(pts).cuda(), R, 2, 2, 0)
    ijk, _, fl, exists = export_band(band)
    vals = np.zeros(band.V_stored, np.float32)
    vals[exists] = synth.sphere_field(ijk[exists], R, 0.45, 0.03, seed=1)
    q, j = synth.gaussian_queries(pts, 40000, 0.04, seed=2)
    rec = torch.from_numpy(np.concatenate([q, pts[j]], axis=1)).cuda()
    return gb, ctx, band, R, vals, rec, pts, q, j


def test_function_matches_gp_step(setup):
    import torch
    from paper_2308_13175_gb300.autograd import gridpull_loss
    gb, ctx, band, R, vals, rec, pts, q, j = setup
    D = torch.from_numpy(vals).cuda().requires_grad_(True)
    w = (1.0, 1.0, 0.005)
    L = gridpull_loss(D, band, rec, weights=w)
    (2.0 * L).backward()
    grad = torch.empty(band.V_stored, dtype=torch.float32, device="cuda")
    loss = torch.zeros(8, dtype=torch.float32, device="cuda")
    gb.gp_step(band, rec, rec.shape[0], grad, loss, w, d=D.detach())
    assert float(L) == float(loss[gb.GP_LOSS_TOTAL])
    g1 = D.grad.cpu().numpy().astype(np.float64)
    g2 = 2.0 * grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g1 - g2) <= 1e-6 * np.linalg.norm(g2)


def test_function_matches_plain_torch_autograd(setup):
    import torch
    from paper_2308_13175_gb300.autograd import gridpull_loss
    from paper_2308_13175_gb300.torch_reference import from_band
    gb, ctx, band, R, vals, rec, pts, q, j = setup
    w = (1.0, 1.0, 0.005)
    D = torch.from_numpy(vals).cuda().requires_grad_(True)
    L = gridpull_loss(D, band, rec, weights=w)
    L.backward()
    ts = from_band(band, device="cuda", dtype=torch.float64)
    D64 = torch.from_numpy(vals.astype(np.float64)).cuda().requires_grad_(True)
    L64, parts = ts.loss(D64, rec.to(torch.float64), w)
    L64.backward()
    assert abs(float(L) - float(L64)) <= 1e-5 * abs(float(L64))
    # per-vertex scale from the oracle on the same inputs
    ijk, _, fl, exists = export_band(band)
    keys = vertex_keys(ijk[exists], R)
    Dd = np.zeros((R + 1) ** 3)
    Dd[keys] = vals[exists]
    sets = o.band_sets(pts, R, 2, 2)
    ref = o.step_loss_grad(Dd, R, sets, q, pts[j], w)
    g = D.grad.cpu().numpy().astype(np.float64)[exists]
    g64 = D64.grad.cpu().numpy()[exists]
    assert_grad_close(g, g64, ref["abs_terms"][keys], what="Function vs torch autograd")


def test_function_matches_finite_differences(setup):
    import torch
    from paper_2308_13175_gb300.autograd import gridpull_loss
    gb, ctx, band, R, vals, rec, pts, q, j = setup
    # beta = 0: |f(s)| has a kink at f(s) = 0 that a finite step straddles; its
    # gradient is checked against the oracle and the autograd form instead.
    w = (1.0, 0.0, 0.005)
    rec = rec[:2000].contiguous()  # few records: gradients well above the float32 noise of L
    D = torch.from_numpy(vals).cuda().requires_grad_(True)
    gridpull_loss(D, band, rec, weights=w).backward()
    g = D.grad.cpu().numpy().astype(np.float64)
    # well-sized gradients, away from the few largest (which sit at kinks of |r|)
    top = np.argsort(-np.abs(g))[20:32]
    eps = 1e-3
    for k in top:
        dp = vals.copy()
        dm = vals.copy()
        dp[k] += eps
        dm[k] -= eps
        with torch.no_grad():
            lp = float(gridpull_loss(torch.from_numpy(dp).cuda(), band, rec, weights=w))
            lm = float(gridpull_loss(torch.from_numpy(dm).cuda(), band, rec, weights=w))
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 5e-2 * abs(g[k]) + 1e-7, (k, fd, g[k])
