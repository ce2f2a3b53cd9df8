"""FP64 CPU oracle for the reconstruction metrics.

TEST INFRASTRUCTURE ONLY: used by the tests; never by the library.  It shares
no code with the CUDA path.

Sec. 4 "Datasets and Metrics" names the measures the paper reports: the L1 and
L2 Chamfer distances, the Hausdorff distance (HD), normal consistency (NC) and
the F-score at a distance threshold.
Their definitions (the usual ones of the works the paper follows) are written
out here for two oriented point sets A and B with weights:

* for a in A, its nearest point NN_B(a) in B (Euclidean, float64 from the
  float32 coordinates) at distance d(a);
* accuracy terms (A -> B): weighted means over A of d(a), d(a)^2,
  |n_a . n_NN_B(a)| and of [d(a) < tau]; completeness terms (B -> A) alike;
* CD_L1 = (mean_A d + mean_B d) / 2, CD_L2 = (mean_A d^2 + mean_B d^2) / 2,
  HD = max(max_A d, max_B d), NC = (mean_A |cos| + mean_B |cos|) / 2,
  F(tau) = 2 P R / (P + R) with
  precision P = mean_A [d < tau] and recall R = mean_B [d < tau] (0 when both
  are 0).

Reading: a mesh enters as the centroids of the m^2 congruent sub-triangles of
each triangle (split at m equal steps along its edges), each weighted by its
area and oriented by the triangle's unit normal, so a mean over the mesh is the
one-point quadrature of the mean over its surface and the points lie about
h / m apart (no random sampling).  A point set enters with weight 1 per point.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def subdivision_centroids(m: int) -> np.ndarray:
    """Barycentric (a, b) of the centroids of the m^2 congruent triangles that
    split a triangle at m equal steps along its edges (point v0 + a (v1 - v0)
    + b (v2 - v0)): the m (m + 1) / 2 upright ones with corners (i, j),
    (i+1, j), (i, j+1) and the m (m - 1) / 2 inverted ones with corners
    (i+1, j), (i, j+1), (i+1, j+1), in units of 1/m, for i + j < m."""
    ab = []
    for i in range(m):
        for j in range(m - i):
            ab.append(((3 * i + 1) / (3 * m), (3 * j + 1) / (3 * m)))
            if i + j < m - 1:
                ab.append(((3 * i + 2) / (3 * m), (3 * j + 2) / (3 * m)))
    return np.array(ab)


def mesh_quadrature(tri: np.ndarray, m: int = 1):
    """Points (T m^2, 3), unit normals and weights of the one-point rule on each
    of the m^2 sub-triangles of every float32 triangle (T, 3, 3), in float64:
    sub-triangle centroids, the triangle's unit normal, area / m^2 each.
    Degenerate triangles get weight 0 and a zero normal.  Point k of triangle i
    is row i m^2 + k, k in the order of subdivision_centroids."""
    t = np.asarray(tri, dtype=np.float64)
    cr = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    nrm = np.linalg.norm(cr, axis=1)
    area = 0.5 * nrm
    n = np.divide(cr, nrm[:, None], out=np.zeros_like(cr), where=nrm[:, None] > 0)
    ab = subdivision_centroids(m)
    e1, e2 = t[:, 1] - t[:, 0], t[:, 2] - t[:, 0]
    pts = t[:, None, 0] + ab[None, :, 0, None] * e1[:, None] + ab[None, :, 1, None] * e2[:, None]
    k = len(ab)
    return pts.reshape(-1, 3), np.repeat(n, k, axis=0), np.repeat(area / k, k)


def nearest_terms(a, a_nrm, a_w, b, b_nrm, taus):
    """Weighted means over A of d, d^2, |cos| and [d < tau], and the largest d
    (over points of positive weight), against B.
    a_w None = weight 1; normals None = NC not computed (NaN)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    _, j = cKDTree(b).query(a)
    diff = a - b[j]
    # the distance of the nearest point, as ((dx^2 + dy^2) + dz^2) then sqrt
    d = np.sqrt((diff[:, 0] * diff[:, 0] + diff[:, 1] * diff[:, 1]) + diff[:, 2] * diff[:, 2])
    w = np.ones(len(a)) if a_w is None else np.asarray(a_w, dtype=np.float64)
    W = w.sum()
    out = {"mean_d": float((w * d).sum() / W), "mean_d2": float((w * d * d).sum() / W),
           "max_d": float(d[w > 0].max()) if np.any(w > 0) else 0.0}
    if a_nrm is not None and b_nrm is not None:
        cos = np.abs(np.einsum("ij,ij->i", np.asarray(a_nrm, np.float64), np.asarray(b_nrm, np.float64)[j]))
        out["mean_cos"] = float((w * cos).sum() / W)
    else:
        out["mean_cos"] = float("nan")
    out["below"] = [float((w * (d < t)).sum() / W) for t in taus]
    out["d"] = d
    return out


def combine(acc: dict, comp: dict, taus) -> dict:
    """CD_L1, CD_L2, HD, NC and F(tau) from the two directions' terms."""
    f = {}
    for k, t in enumerate(taus):
        p, r = acc["below"][k], comp["below"][k]
        f[t] = 0.0 if p + r == 0 else 2 * p * r / (p + r)
    return {"cd_l1": 0.5 * (acc["mean_d"] + comp["mean_d"]), "cd_l2": 0.5 * (acc["mean_d2"] + comp["mean_d2"]),
            "hd": max(acc["max_d"], comp["max_d"]), "nc": 0.5 * (acc["mean_cos"] + comp["mean_cos"]), "fscore": f}


def surface_metrics(tri, gt_pts, gt_nrm, taus=(0.002, 0.004, 0.01), m: int = 4) -> dict:
    """Metrics of a triangle soup (sampled by mesh_quadrature with m^2 points
    per triangle) against oriented ground-truth points."""
    c, n, w = mesh_quadrature(tri, m)
    # a degenerate triangle's points still lie on the mesh: they stay targets
    # of the completeness direction, with weight 0 in the accuracy direction
    acc = nearest_terms(c, n, w, gt_pts, gt_nrm, taus)
    comp = nearest_terms(gt_pts, gt_nrm, None, c, n, taus)
    return combine(acc, comp, taus)
