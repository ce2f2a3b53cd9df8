"""Pins for the mesh oracle (marching cubes over the optimised cells).

Each test checks the oracle against something other than itself: the cube's
combinatorics, closed forms (a plane is reproduced exactly, a sphere's volume
and area converge at second order inside a derived shell), topology (Euler
characteristics of a sphere and a torus, closed and consistently oriented
meshes), and hand-counted cell sets.
"""

import numpy as np
import pytest

from oracle import gridpull as o
from oracle import mesh as m


def _dense_grid(R):
    n = R + 1
    return -1.0 + (2.0 / R) * o.key_to_vertex(np.arange(n ** 3), R).astype(np.float64)


def _all_cells(R):
    return np.arange(R ** 3, dtype=np.int64)


def test_edge_numbering_round_trips():
    for e in range(12):
        lo, hi = m.edge_corners(e)
        assert m.edge_id(lo, hi) == e == m.edge_id(hi, lo)
        assert sum(h - l for l, h in zip(lo, hi)) == 1


def test_face_walks_are_counter_clockwise_from_outside():
    """The cross product of consecutive steps of each walk points outwards."""
    for walk in m.face_walks():
        p = np.array(walk, dtype=float)
        centre = p.mean(axis=0)
        outward = centre - 0.5
        for k in range(4):
            a, b, c = p[k], p[(k + 1) % 4], p[(k + 2) % 4]
            assert np.dot(np.cross(b - a, c - b), outward) > 0


@pytest.mark.parametrize("k", range(8))
def test_single_corner_cases_point_to_the_positive_side(k):
    corner = o.CORNERS[k].astype(float)
    for negative_corner in (True, False):
        case = (1 << k) if negative_corner else (255 ^ (1 << k))
        tris = m.case_triangles(case)
        assert len(tris) == 1
        d = np.where(np.arange(8) == k, -1.0 if negative_corner else 1.0, 1.0 if negative_corner else -1.0)
        values = np.zeros(8)
        values[:] = d
        # one cell, R = 1: vertex keys in corner order
        dense = np.zeros(8)
        for c in range(8):
            dense[o.vertex_key(o.CORNERS[c], 1)] = values[c]
        tri, cells = m.marching_cubes(dense, 1, np.array([0]))
        assert len(tri) == 1 and cells.tolist() == [0]
        nrm = m.triangle_normals(tri)[0]
        centroid = tri[0].mean(axis=0)
        away = centroid - (-1.0 + 2.0 * corner)
        # the normal points from negative to positive: away from a lone
        # negative corner, towards a lone positive one
        assert np.dot(nrm, away) * (1 if negative_corner else -1) > 0
        # every vertex is the midpoint of an edge at that corner (t = 1/2)
        dist = np.linalg.norm(tri[0] - (-1.0 + 2.0 * corner), axis=1)
        np.testing.assert_allclose(dist, 1.0, rtol=0, atol=1e-15)


def test_every_case_covers_each_cut_edge_once():
    for case in range(256):
        neg = [(case >> k) & 1 for k in range(8)]
        cut = {e for e in range(12)
               if neg[o.vertex_key(np.array(m.edge_corners(e)[0]), 1)] != neg[o.vertex_key(np.array(m.edge_corners(e)[1]), 1)]}
        cycles = m.cell_cycles(neg)
        flat = [e for c in cycles for e in c]
        assert sorted(flat) == sorted(cut)
        assert all(len(c) >= 3 for c in cycles)
        assert len(m.case_triangles(case)) == len(cut) - 2 * len(cycles)
        assert len(m.case_triangles(case)) <= 5


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_field_mesh_is_closed_and_oriented(seed):
    """Positive on the domain boundary, random inside: the mesh is closed and
    consistently oriented, i.e. every welded edge is traversed as often in one
    direction as in the other.  (Where a cycle crosses an ambiguous face twice,
    the fans of the two cells sharing that face may both place a chord on the
    same face diagonal, so an edge can carry four triangles.)"""
    R = 8
    rng = np.random.default_rng(seed)
    ijk = o.key_to_vertex(np.arange((R + 1) ** 3), R)
    d = rng.standard_normal(len(ijk))
    on_boundary = np.any((ijk == 0) | (ijk == R), axis=1)
    d[on_boundary] = np.abs(d[on_boundary]) + 0.1
    tri, _ = m.marching_cubes(d, R, _all_cells(R))
    assert len(tri) > 50
    _, faces = m.weld(tri)
    counts = m.directed_edge_counts(faces)
    assert all(counts.get((b, a), 0) == k for (a, b), k in counts.items())
    assert m.enclosed_volume(tri) > 0


def test_planar_field_is_reproduced_exactly():
    """A linear field is interpolated exactly along every edge, so every vertex
    lies on its zero plane, every normal points along its gradient, and the
    triangles tile the plane's section of the cube: area 4 sqrt(1 + a^2 + b^2)
    for z = a x + b y + c inside the four side faces."""
    R = 16
    a, b, c = 0.23, -0.31, 0.07
    v = _dense_grid(R)
    d = v[:, 2] - a * v[:, 0] - b * v[:, 1] - c
    tri, _ = m.marching_cubes(d, R, _all_cells(R))
    p = tri.reshape(-1, 3)
    np.testing.assert_allclose(p[:, 2] - a * p[:, 0] - b * p[:, 1] - c, 0.0, atol=1e-14)
    nrm = m.triangle_normals(tri)
    grad = np.array([-a, -b, 1.0])
    area2 = np.linalg.norm(nrm, axis=1)
    keep = area2 > 1e-14
    assert np.all(nrm[keep] @ grad > 0)
    np.testing.assert_allclose(m.mesh_area(tri), 4.0 * np.sqrt(1 + a * a + b * b), rtol=1e-12)


def test_sphere_shell_topology_and_second_order_convergence():
    """Sphere SDF: the distance along an edge is convex, so each crossing lies
    inside the sphere, at most h^2 / (8 (r - sqrt(3) h)) below it; the mesh is a
    closed genus-0 surface (V - E + F = 2) and its volume and area errors fall by
    four when h halves."""
    centre, r = np.array([0.03, -0.02, 0.01]), 0.5
    errs = []
    for R in (16, 32):
        h = 2.0 / R
        v = _dense_grid(R)
        d = np.linalg.norm(v - centre, axis=1) - r
        tri, _ = m.marching_cubes(d, R, _all_cells(R))
        rad = np.linalg.norm(tri.reshape(-1, 3) - centre, axis=1)
        assert rad.max() <= r + 1e-12
        assert rad.min() >= r - h * h / (8 * (r - np.sqrt(3) * h))
        _, faces = m.weld(tri)
        counts = m.directed_edge_counts(faces)
        assert max(counts.values()) == 1 and all((b, a) in counts for (a, b) in counts)  # closed 2-manifold
        assert m.euler_characteristic(faces) == 2
        vol_err = 1 - m.enclosed_volume(tri) / (4 / 3 * np.pi * r ** 3)
        area_err = 1 - m.mesh_area(tri) / (4 * np.pi * r * r)
        assert vol_err > 0 and area_err > 0      # inscribed: smaller on both counts
        errs.append((vol_err, area_err))
    for k in range(2):
        assert 3.5 < errs[0][k] / errs[1][k] < 4.5


def test_torus_has_genus_one():
    R, Rt, rt = 32, 0.5, 0.2
    v = _dense_grid(R)
    q = np.sqrt(v[:, 0] ** 2 + v[:, 1] ** 2) - Rt
    d = np.sqrt(q * q + v[:, 2] ** 2) - rt
    tri, _ = m.marching_cubes(d, R, _all_cells(R))
    _, faces = m.weld(tri)
    assert m.euler_characteristic(faces) == 0


def test_meshed_cells_need_all_eight_corners():
    R = 8
    cell = np.array([1, 2, 3])
    corners = o.vertex_key(cell + o.CORNERS, R)
    assert m.meshed_cells(corners, R).tolist() == [o.cell_key(cell, R)]
    for k in range(8):
        assert len(m.meshed_cells(np.delete(corners, k), R)) == 0


@pytest.mark.parametrize("M", [0, 1, 2])
def test_meshed_cells_of_a_single_point_band(M):
    """One point: the trainable set is the corners of a (2M+1)^3 cube of cells,
    and exactly those cells are meshed."""
    R = 16
    p = np.array([[0.06, -0.13, 0.21]], dtype=np.float32)
    sets = o.band_sets(p, R, M, M)
    cells = m.meshed_cells(sets["trainable"], R)
    assert len(cells) == (2 * M + 1) ** 3
    np.testing.assert_array_equal(cells, np.sort(o.dilate_cells(sets["occupied"], M, R)))


def test_skipped_cells_emit_nothing_and_iso_ties_count_positive():
    R = 4
    n = R + 1
    d = np.zeros(n ** 3)
    centre = o.vertex_key(np.array([2, 2, 2]), R)
    d[centre] = -1.0
    # iso 0: only the 8 cells around the negative vertex have a negative corner
    tri, cells = m.marching_cubes(d, R, _all_cells(R), iso=0.0)
    assert len(np.unique(cells)) == 8 and len(tri) == 8
    # meshing a subset returns only triangles of that subset
    sub = _all_cells(R)[::3]
    _, cells_sub = m.marching_cubes(d, R, sub, iso=0.0)
    assert set(cells_sub.tolist()) <= set(sub.tolist())
    # a level below every value: no negative corner, no triangle
    tri, _ = m.marching_cubes(d, R, _all_cells(R), iso=-2.0)
    assert len(tri) == 0


def test_iso_level_shifts_the_surface():
    """Meshing f at level c equals meshing f - c at level 0 (to rounding)."""
    R = 16
    v = _dense_grid(R)
    d = np.linalg.norm(v, axis=1) - 0.4
    t1, c1 = m.marching_cubes(d, R, _all_cells(R), iso=0.125)
    t2, c2 = m.marching_cubes(d - 0.125, R, _all_cells(R), iso=0.0)
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_allclose(t1, t2, atol=1e-15)
