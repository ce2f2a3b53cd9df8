"""The whole fit on the device converges to the ground-truth signed distance
near the surface.

Settings (Sec. 4 "Details"): R = 256, pull band M1 = 3, TV band M2 = 14, 50,000
queries per iteration, 1600 iterations, Adam with the rate decayed by 0.3 every
400 iterations (the rate of 1.0 read in voxel units, 1.0 h), alpha = beta = 1;
the field starts as a sphere of radius 2 h about the cloud's centre (Sec. 3).
gamma is 0.05, ten times the paper's 0.005: with every term a mean (over the
valid queries, over T), the paper's gamma leaves the queries inside the shape in
the mirrored minimum of Eq. 4 (f = +delta with grad f pointing inwards), which
pulls them onto the surface as well; measured, the field near the surface was
then 0.7-0.8 h off and L_grad 0.81.  Every step is FitStep.run: per-epoch
resampling of the query pool (10 queries per point), exact NN, the forward and
backward of Eq. 3-8, L_TV and Adam, all in the library's kernels; fit_cloud
strings them together with these defaults.

Ground truth comes from shapes with a closed-form SDF (a sphere and a torus,
points area-uniform on the surface).  Checked after the fit: values at
trainable vertices within h and 3 h of the surface match the SDF, the surface
term |f(s)| is small, the loss fell, and the marching-cubes surface of the
optimised cells has a vertex within sqrt(3) h of every ground-truth point (no
holes).  Away
from the points (beyond the reach of the queries, where only L_TV acts and the
band's frozen vertices keep the initial sign) the field can cross zero again;
those crossings are reported, not asserted.
"""
import numpy as np
import pytest

from paper_2308_13175_gb300 import synth

from gpu_common import export_band, have_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    if not have_gpu():
        pytest.skip("no CUDA device")
    from gpu_common import build_lib
    build_lib()
    from paper_2308_13175_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(gb):
    return gb.gp_create(0)


def _torus_cloud(n, R_major, r_minor, seed):
    """Area-uniform points on a torus about the z axis: the area element is
    proportional to R + r cos(v), so v is drawn by rejection."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, 2 * np.pi, 4 * n)
    v = rng.uniform(0, 2 * np.pi, 4 * n)
    keep = rng.uniform(0, R_major + r_minor, 4 * n) < R_major + r_minor * np.cos(v)
    u, v = u[keep][:n], v[keep][:n]
    ring = R_major + r_minor * np.cos(v)
    return np.stack([ring * np.cos(u), ring * np.sin(u), r_minor * np.sin(v)], axis=1).astype(np.float32)


def _shape(name):
    if name == "sphere":
        r = 0.5
        return synth.sphere_cloud(20_000, r, seed=5), (lambda x: np.linalg.norm(x, axis=1) - r)
    Rt, rt = 0.5, 0.2
    sdf = lambda x: np.sqrt((np.hypot(x[:, 0], x[:, 1]) - Rt) ** 2 + x[:, 2] ** 2) - rt
    return _torus_cloud(30_000, Rt, rt, seed=6), sdf


@pytest.mark.parametrize("name", ["sphere", "torus"])
def test_fit_converges_to_the_ground_truth_sdf(gb, ctx, name):
    import torch
    from scipy.spatial import cKDTree
    from paper_2308_13175_gb300.fit import fit_cloud
    pts, sdf = _shape(name)
    R = 256
    h = 2.0 / R
    band, first_fit = fit_cloud(ctx, torch.from_numpy(pts).cuda(), iters=1, weights=(1.0, 1.0, 0.05))
    first = float(first_fit.loss[gb.GP_LOSS_TOTAL])
    band.close()
    band, fit = fit_cloud(ctx, torch.from_numpy(pts).cuda(), R=R, M1=3, M2=14, iters=1600, batch=50_000,
                          weights=(1.0, 1.0, 0.05))
    loss = fit.loss
    torch.cuda.synchronize()
    gb.gp_band_check(band)
    loss = loss.cpu().numpy()

    ijk, d, fl, exists = export_band(band)
    trainable = (fl & 2) != 0
    x = -1.0 + h * ijk.astype(np.float64)
    g = np.where(exists, sdf(x), 0.0)
    err = {}
    for lim in (1, 3):
        m = trainable & (np.abs(g) <= lim * h)
        err[lim] = float(np.mean(np.abs(d[m] - g[m]))) / h
    far = trainable & (np.abs(g) > 3 * h)
    sign_far = float(np.mean(np.sign(d[far]) == np.sign(g[far])))

    tri, _ = gb.gp_mesh_extract(band, 0.0, with_cells=False)
    tri = tri.cpu().numpy().astype(np.float64)
    verts = np.unique(tri.reshape(-1, 3), axis=0)
    reach = cKDTree(verts).query(pts.astype(np.float64))[0] / h
    dist = np.abs(sdf(verts)) / h
    metrics = {"loss": loss[:5].round(6).tolist(), "first loss": round(first, 5),
               "mean |d - sdf| within h (h)": round(err[1], 4), "within 3h (h)": round(err[3], 4),
               "sign agreement beyond 3h": round(sign_far, 4), "triangles": len(tri),
               "points -> mesh p99 / max (h)": (round(float(np.percentile(reach, 99)), 3), round(float(reach.max()), 3)),
               "mesh vertices within 2h of the surface": round(float(np.mean(dist <= 2)), 4)}
    print(name, metrics)
    assert err[1] < 0.5 and err[3] < 1.0, metrics
    assert loss[gb.GP_LOSS_SURF] < 0.05 * h, metrics
    assert loss[gb.GP_LOSS_TOTAL] < 0.5 * first, metrics
    # A point lies in a cell that the surface crosses, and every crossing is a
    # mesh vertex on that cell's edges: with no hole, the nearest vertex is
    # within the cell's diagonal, sqrt(3) h.
    assert reach.max() < np.sqrt(3.0) and np.percentile(reach, 99) < 1.0, metrics
    band.close()


def test_trajectory_follows_the_oracle_on_the_single_sphere(gb, ctx):
    """The single-sphere configuration stepped 200 times on the device and by
    the float64 oracle from the same start: 5,000 points on a radius-0.5
    sphere, a dense 64^3 grid starting at |x| - 0.5 + N(0, 0.01) (variance
    0.01), 50,000 queries per step (the whole pool, re-drawn every step: 10 per
    point around s_j with sigma_j the 50th-neighbour distance), Adam at 1e-3,
    weights (1, 1, 0.005).  Both sides draw the same queries (Philox4x32-10 at
    the same counters) and find their nearest points exactly (the oracle by
    brute force on all host cores); the oracle carries float64 values, moments
    and sums, the device float32.  The loss curves are compared step by step:
    the first step to 1e-5 (identical inputs), the whole curve loosely (the
    float32 and float64 trajectories part slowly; reported, and held to 1%)."""
    import os
    import tempfile

    import torch
    from oracle import gridpull as o
    from oracle.parallel import OraclePool
    from paper_2308_13175_gb300.fit import FitStep
    R, Q, steps, lr = 64, 50_000, 200, 1e-3
    w = (1.0, 1.0, 0.005)
    pts = synth.sphere_cloud(5000, 0.5, seed=0)
    band = gb.gp_build_band(ctx, torch.from_numpy(pts).cuda(), R, -1, -1, 50)
    ijk, _, _, exists = export_band(band)
    n1 = R + 1
    all_keys = np.arange(n1 ** 3, dtype=np.int64)
    D0 = o.sphere_init(all_keys, R, (0.0, 0.0, 0.0), 0.5, 0.1, seed=0).astype(np.float32)
    vals = np.zeros(band.V_stored, np.float32)
    vk = ijk[exists, 0] + n1 * (ijk[exists, 1] + n1 * ijk[exists, 2])
    vals[exists] = D0[vk]
    gb.gp_band_set_values(band, torch.from_numpy(vals).cuda())
    fit = FitStep(band, Q=Q, B=Q, seed=0, weights=w, lr=lr)
    dev_loss = np.zeros((steps, 8))
    for t in range(steps):
        dev_loss[t] = fit.run(t).cpu().numpy()
    # The oracle's own run from the same (float32) start.
    D = D0.astype(np.float64)
    m = np.zeros_like(D)
    v = np.zeros_like(D)
    sig = o.knn_sigma(pts, 50)
    sets = {"pull_cells": np.arange(R ** 3, dtype=np.int64), "tv": all_keys}
    pos = np.arange(Q, dtype=np.int64)
    tmp = tempfile.mkdtemp(prefix="gp_traj_")
    np.save(os.path.join(tmp, "pts.npy"), pts)
    pool = OraclePool(os.path.join(tmp, "pts.npy"))
    ref_loss = np.zeros(steps)
    try:
        for t in range(steps):
            q, _ = o.sample_queries(pts, sig, 0, t, pos)
            q = q.astype(np.float32)
            paths = []
            for k, part in enumerate(np.array_split(q, pool.cores)):
                pth = os.path.join(tmp, f"q{k}.npy")
                np.save(pth, part)
                paths.append(pth)
            nn = pool.nn_indices(paths)
            res = o.step_loss_grad(D, R, sets, q, pts[nn], w)
            ref_loss[t] = res["loss"]
            D, m, v = o.adam(D, res["grad"], m, v, t + 1, lr)
    finally:
        pool.close()
    rel = np.abs(dev_loss[:, gb.GP_LOSS_TOTAL] - ref_loss) / np.abs(ref_loss)
    print(f"single sphere, 200 steps: loss {ref_loss[0]:.6f} -> {ref_loss[-1]:.6f} (oracle), "
          f"{dev_loss[0, 0]:.6f} -> {dev_loss[-1, 0]:.6f} (device); relative difference at step 0 "
          f"{rel[0]:.2e}, max {rel.max():.2e} (step {int(rel.argmax())}), last {rel[-1]:.2e}")
    assert rel[0] <= 1e-5
    assert rel.max() <= 1e-2
    assert ref_loss[-1] < ref_loss[0]
