"""Pins for the metrics oracle: closed forms and special cases that a dropped
term, a swapped direction or a wrong weight would break."""
import numpy as np
import pytest

from oracle import mesh as om
from oracle import metrics as mt
from oracle import gridpull as o


def _sphere_points(n, r, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return r * d, d


def test_identical_sets_are_perfect():
    p, n = _sphere_points(2000, 0.5, 0)
    acc = mt.nearest_terms(p, n, None, p, n, (0.01,))
    res = mt.combine(acc, acc, (0.01,))
    assert res["cd_l1"] == 0 and res["cd_l2"] == 0 and res["hd"] == 0
    assert res["nc"] == pytest.approx(1.0, abs=1e-15)
    assert res["fscore"][0.01] == 1.0


def test_concentric_spheres_give_the_radial_gap():
    """Points on a sphere of radius r + delta against a dense sample of radius
    r: every nearest distance is at least delta and at most
    sqrt(delta^2 + s^2), s the largest gap on the inner sphere, so CD_L1
    and HD are pinned to delta within that; normals are radial, NC near 1;
    F is 0 below delta and 1 above the bound."""
    r, delta = 0.5, 0.01
    inner, n_in = _sphere_points(200_000, r, 1)
    outer, n_out = _sphere_points(3000, r + delta, 2)
    acc = mt.nearest_terms(outer, n_out, None, inner, n_in, (0.5 * delta, 2 * delta))
    d = acc["d"]
    assert d.min() >= delta - 1e-12
    assert d.max() < 1.2 * delta
    assert acc["mean_d"] == pytest.approx(delta, rel=0.1)
    assert acc["mean_d2"] == pytest.approx(delta ** 2, rel=0.2)
    assert acc["mean_cos"] > 0.99
    assert acc["below"] == [0.0, 1.0]


def test_weights_and_normal_sign():
    a = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    b = np.array([[0.0, 0, 0.1], [1.0, 0, 0.3]])
    na = np.array([[0, 0, 1.0], [0, 0, 1.0]])
    nb = np.array([[0, 0, -1.0], [0, 1.0, 0]])           # flipped, then orthogonal
    acc = mt.nearest_terms(a, na, np.array([3.0, 1.0]), b, nb, (0.2,))
    assert acc["mean_d"] == pytest.approx((3 * 0.1 + 0.3) / 4)
    assert acc["mean_d2"] == pytest.approx((3 * 0.01 + 0.09) / 4)
    assert acc["max_d"] == pytest.approx(0.3)
    assert acc["mean_cos"] == pytest.approx(3 / 4)        # |cos| = 1 for the flipped normal, 0 orthogonal
    assert acc["below"] == [pytest.approx(3 / 4)]


def test_fscore_is_the_harmonic_mean():
    acc = {"mean_d": 0.1, "mean_d2": 0.02, "max_d": 0.3, "mean_cos": 0.9, "below": [0.5, 0.0]}
    comp = {"mean_d": 0.3, "mean_d2": 0.1, "max_d": 0.5, "mean_cos": 0.7, "below": [1.0, 0.0]}
    res = mt.combine(acc, comp, (1.0, 2.0))
    assert res["cd_l1"] == pytest.approx(0.2) and res["cd_l2"] == pytest.approx(0.06)
    assert res["hd"] == 0.5 and res["nc"] == pytest.approx(0.8)
    assert res["fscore"][1.0] == pytest.approx(2 * 0.5 / 1.5)
    assert res["fscore"][2.0] == 0.0


@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_subdivision_centroids_tile_the_triangle(m):
    """m^2 points, all inside; the mean of the centroids is the triangle's
    centroid (the rule integrates affine functions exactly)."""
    ab = mt.subdivision_centroids(m)
    assert len(ab) == m * m
    assert np.all(ab > 0) and np.all(ab.sum(axis=1) < 1)
    np.testing.assert_allclose(ab.mean(axis=0), [1 / 3, 1 / 3], atol=1e-15)
    # the mean of a^2 over the triangle is 1/6; the centroid rule drops each
    # piece's own variance of a, (1/m^2)(1/6 - 1/9), so it gives exactly
    # 1/6 - 1/(18 m^2)
    assert (ab[:, 0] ** 2).mean() == pytest.approx(1 / 6 - 1 / (18 * m * m), abs=1e-15)


def test_mesh_quadrature_integrates_the_surface():
    """Areas add up to the surface area; the area-weighted centroid of a closed
    surface's normals sums to zero; the mean distance to the sphere's centre
    approaches r at second order."""
    R, r = 32, 0.5
    n1 = R + 1
    v = -1.0 + (2.0 / R) * o.key_to_vertex(np.arange(n1 ** 3), R)
    d = np.linalg.norm(v, axis=1) - r
    tri, _ = om.marching_cubes(d, R, np.arange(R ** 3))
    c, n, w = mt.mesh_quadrature(tri, 3)
    assert len(c) == 9 * len(tri)
    assert w.sum() == pytest.approx(om.mesh_area(tri), rel=1e-12)
    np.testing.assert_allclose((w[:, None] * n).sum(axis=0), 0.0, atol=1e-12)
    # outward unit normals
    assert np.all(np.einsum("ij,ij->i", n[w > 0], c[w > 0]) > 0)
    assert abs(np.average(np.linalg.norm(c, axis=1), weights=w) - r) < (2.0 / R) ** 2


def test_surface_metrics_of_a_marching_cubes_sphere():
    """End to end: the mesh of a sphere SDF against exact sphere points is
    within the interpolation bound h^2 / (8 (r - sqrt(3) h)) plus the chord
    depth, normals agree, and everything improves with R."""
    r = 0.5
    gt, gt_n = _sphere_points(50_000, r, 3)
    prev = None
    for R in (16, 32):
        n1 = R + 1
        v = -1.0 + (2.0 / R) * o.key_to_vertex(np.arange(n1 ** 3), R)
        d = np.linalg.norm(v, axis=1) - r
        tri, _ = om.marching_cubes(d, R, np.arange(R ** 3))
        res = mt.surface_metrics(tri, gt, gt_n, taus=(0.05,))
        assert res["nc"] > 0.98 and res["fscore"][0.05] > 0.99
        if prev is not None:
            assert res["cd_l1"] < prev["cd_l1"] and res["hd"] < prev["hd"]
        prev = res
