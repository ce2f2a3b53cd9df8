"""Parity of the metric kernels (through the C ABI) with the FP64 metrics oracle.

Contract: quadrature points within 1e-6 (float32 v0 + a e1 + b e2 against
float64, |x| <= 1), normals within 1e-5 and weights within 1e-5 relative on
triangles of area above 1e-6 h^2 (the float32 cross product of a sliver is
ill-conditioned); nearest terms on identical float32 inputs: the distance is
the same float64 expression on both sides, so the largest d and the fractions
below tau agree to rounding of the sums (1e-12), the means within 1e-10.
End to end (GPU quadrature against the oracle's float64 one): metrics within
1e-5 relative, F within 1e-4.  Expected values from the oracle only.
"""
import numpy as np
import pytest

from oracle import metrics as mt
from paper_2308_13175_gb300 import synth

from gpu_common import build_lib, export_band, have_gpu

pytestmark = pytest.mark.gpu

TAUS = (0.002, 0.004, 0.01)


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


def _sphere_points(n, r, seed, centre=(0.0, 0.0, 0.0)):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return (np.asarray(centre) + r * d).astype(np.float32), d.astype(np.float32)


@pytest.fixture(scope="module")
def sphere_mesh(gb, ctx):
    """Marching cubes of a sphere SDF on a dense R = 64 band (device float32)."""
    import torch
    R = 64
    pts, _ = _sphere_points(4000, 0.5, 0)
    band = gb.gp_build_band(ctx, torch.from_numpy(pts).cuda(), R, -1, -1, 0)
    ijk, _, _, exists = export_band(band)
    x = -1.0 + (2.0 / R) * ijk.astype(np.float64)
    vals = np.where(exists, np.linalg.norm(x - np.array([0.02, -0.01, 0.03]), axis=1) - 0.45, 0.0)
    gb.gp_band_set_values(band, torch.from_numpy(vals.astype(np.float32)).cuda())
    tri, _ = gb.gp_mesh_extract(band, 0.0, with_cells=False)
    band.close()
    return tri, R


@pytest.mark.parametrize("m", [1, 3, 4])
def test_quadrature_matches_oracle(gb, ctx, sphere_mesh, m):
    tri, R = sphere_mesh
    h = 2.0 / R
    p, n, w = gb.gp_mesh_quadrature(ctx, tri, m)
    p, n, w = (t.cpu().numpy().astype(np.float64) for t in (p, n, w))
    po, no, wo = mt.mesh_quadrature(tri.cpu().numpy(), m)
    assert p.shape == po.shape and len(w) == len(tri) * m * m
    np.testing.assert_allclose(p, po, rtol=0, atol=1e-6)
    ok = wo > 1e-6 * h * h
    np.testing.assert_allclose(n[ok], no[ok], rtol=0, atol=1e-5)
    np.testing.assert_allclose(w[ok], wo[ok], rtol=1e-5, atol=0)
    assert np.all(np.abs(w[~ok]) <= 2e-6 * h * h)


def test_nearest_terms_match_oracle_on_identical_inputs(gb, ctx, sphere_mesh):
    import torch
    tri, R = sphere_mesh
    p, n, w = gb.gp_mesh_quadrature(ctx, tri, 3)
    ref, ref_n = _sphere_points(30_000, 0.45, 1, centre=(0.02, -0.01, 0.03))
    ref_d, ref_nd = torch.from_numpy(ref).cuda(), torch.from_numpy(ref_n).cuda()
    ref_band = gb.gp_build_band(ctx, ref_d, R, 0, 0, 0)
    mesh_band = gb.gp_build_band(ctx, p, R, 0, 0, 0)
    acc = gb.gp_eval_nearest(ref_band, p, n, w, ref_nd, TAUS)
    comp = gb.gp_eval_nearest(mesh_band, ref_d, ref_nd, None, n, TAUS)
    P, N, W = (t.cpu().numpy() for t in (p, n, w))
    want_acc = mt.nearest_terms(P, N, W, ref, ref_n, TAUS)
    want_comp = mt.nearest_terms(ref, ref_n, None, P, N, TAUS)
    for got, want in ((acc, want_acc), (comp, want_comp)):
        for key in ("mean_d", "mean_d2", "mean_cos"):
            assert got[key] == pytest.approx(want[key], rel=1e-10), key
        assert got["max_d"] == pytest.approx(want["max_d"], rel=1e-12)
        np.testing.assert_allclose(got["below"], want["below"], rtol=1e-12, atol=1e-15)
    assert comp["W"] == len(ref)
    ref_band.close()
    mesh_band.close()


def test_surface_metrics_end_to_end(gb, ctx, sphere_mesh):
    import torch
    from paper_2308_13175_gb300 import metrics
    tri, R = sphere_mesh
    ref, ref_n = _sphere_points(50_000, 0.45, 2, centre=(0.02, -0.01, 0.03))
    got = metrics.surface_metrics(ctx, tri, torch.from_numpy(ref).cuda(), torch.from_numpy(ref_n).cuda(), TAUS)
    want = mt.surface_metrics(tri.cpu().numpy(), ref, ref_n, TAUS)
    for key in ("cd_l1", "cd_l2", "hd", "nc"):
        assert got[key] == pytest.approx(want[key], rel=1e-5), key
    for t in TAUS:
        assert got["fscore"][t] == pytest.approx(want["fscore"][t], abs=1e-4)
    # a marching-cubes sphere at R = 64 is close: CD_L1 below h / 4, NC > 0.99
    assert got["cd_l1"] < 0.25 * (2.0 / R) and got["nc"] > 0.99 and got["fscore"][0.01] > 0.99


def test_eval_edge_cases(gb, ctx):
    import ctypes
    import torch
    pts, _ = _sphere_points(500, 0.5, 3)
    band = gb.gp_build_band(ctx, torch.from_numpy(pts).cuda(), 32, 0, 0, 0)
    empty = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    res = gb.gp_eval_nearest(band, empty, taus=TAUS)
    assert res["W"] == 0 and np.isnan(res["mean_d"]) and all(np.isnan(b) for b in res["below"])
    # the cloud against itself: every distance is 0
    same = gb.gp_eval_nearest(band, torch.from_numpy(pts).cuda(), taus=TAUS)
    assert same["mean_d"] == 0 and same["max_d"] == 0 and same["below"] == [1.0, 1.0, 1.0]
    assert np.isnan(same["mean_cos"])
    lib = gb.load()
    out = (ctypes.c_double * 32)()
    tau = (ctypes.c_double * 17)(*([0.1] * 17))
    q = torch.from_numpy(pts).cuda()
    assert lib.gp_eval_nearest(band.handle, ctypes.c_void_p(q.data_ptr()), None, None, 500, None, tau, 17, out) == 1
    assert lib.gp_eval_nearest(band.handle, ctypes.c_void_p(q.data_ptr()), None, None, 500, None, tau, 1, None) == 1
    assert lib.gp_mesh_quadrature(ctx.handle, None, 4, 0, None, None, None) == 1
    band.close()
