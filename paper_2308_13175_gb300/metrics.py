"""Reconstruction metrics of Sec. 4 "Datasets and Metrics": CD_L1, CD_L2, HD,
NC and F-score of a triangle soup against oriented reference points.

Every stage runs in the library: gp_mesh_quadrature turns the soup into the
weighted centroids of its triangles' m^2 sub-triangles, a band over each point
set gives the exact nearest points (gp_nn), and gp_eval_nearest reduces each
direction's terms (accuracy: mesh into the reference, completeness: reference
into the mesh).  Here the two directions' means are only combined."""
from __future__ import annotations

import math

from . import binding as gb


def surface_metrics(ctx: gb.Context, tri, ref_pts, ref_nrm=None, taus=(0.002, 0.004, 0.01), m: int = 4,
                    R: int = 256) -> dict:
    """tri: (T, 3, 3) float32 device triangles; ref_pts: (N, 3) float32 device
    points in [-1, 1]^3 with unit normals ref_nrm (or None: no NC).  R is the
    grid of the point cell lists (it does not change the result)."""
    taus = tuple(float(t) for t in taus)
    nan = float("nan")
    if tri.shape[0] == 0:
        return {"cd_l1": nan, "cd_l2": nan, "hd": nan, "nc": nan, "fscore": {t: 0.0 for t in taus}, "points": 0}
    pts, nrm, w = gb.gp_mesh_quadrature(ctx, tri.reshape(-1, 9), m)
    ref_band = gb.gp_build_band(ctx, ref_pts, R, 0, 0, 0)
    mesh_band = gb.gp_build_band(ctx, pts, R, 0, 0, 0)
    try:
        acc = gb.gp_eval_nearest(ref_band, pts, nrm if ref_nrm is not None else None, w, ref_nrm, taus)
        comp = gb.gp_eval_nearest(mesh_band, ref_pts, ref_nrm, None, nrm if ref_nrm is not None else None, taus)
    finally:
        ref_band.close()
        mesh_band.close()
    f = {}
    for k, t in enumerate(taus):
        p, r = acc["below"][k], comp["below"][k]
        f[t] = 0.0 if p + r == 0 else 2 * p * r / (p + r)
    return {"cd_l1": 0.5 * (acc["mean_d"] + comp["mean_d"]), "cd_l2": 0.5 * (acc["mean_d2"] + comp["mean_d2"]),
            "hd": max(acc["max_d"], comp["max_d"]),
            "nc": 0.5 * (acc["mean_cos"] + comp["mean_cos"]) if ref_nrm is not None else nan,
            "fscore": f, "points": int(pts.shape[0]), "accuracy": acc, "completeness": comp}
