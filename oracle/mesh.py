"""FP64 CPU oracle for extracting the surface mesh from the fitted grid.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU leg; never
by the library.  It shares no code with the CUDA path.

What the paper fixes:

* Sec. 3 "Overview": the surface is the zero level set of the learned field,
  extracted with marching cubes (Lorensen and Cline, SIGGRAPH 1987);
* Sec. 3, after Eq. 8: cells that were not optimised are skipped;
* Sec. 4 "Details": meshing runs at the resolution of the grid.

Readings where the paper is silent (the CUDA path takes the same ones):

* a cell is meshed iff all 8 of its corners are trainable (optimised);
* a corner is negative iff d < iso, so d == iso counts as positive;
* an edge is cut iff its two corners differ in sign; its crossing lies at
  t = (iso - d_lo) / (d_hi - d_lo) from the edge's lower corner, at the world
  point -1 + h * (lower corner) + h * t along the edge's axis;
* topology: on each face of a cell, walked counter-clockwise as seen from
  outside the cell, every maximal run of negative corners yields one surface
  segment, from the cut edge where the walk enters the run to the cut edge
  where it leaves it.  Two negative corners on a face diagonal thus stay apart,
  and because a face's segments depend on its four corners alone, two cells
  sharing a face agree on it: the mesh is closed wherever all cells around an
  edge are meshed.  Each cut edge ends exactly one segment of a cell and starts
  exactly one, so a cell's segments chain into closed cycles;
* each cycle c0 -> c1 -> ... is started at its lowest edge id and cut into the
  fan (c0, c_k, c_{k+1}), k = 1 .. L-2; cycles go in order of their lowest edge
  id.  With the walk direction above, a triangle's normal (v1 - v0) x (v2 - v0)
  points from the negative side to the positive side.  The mesh is closed and
  consistently oriented where all cells are meshed; where a cycle crosses an
  ambiguous face twice, the fans on the two sides may share a chord on that
  face, which then carries four triangles.

Numbering: corner k = dx + 2*dy + 4*dz; the edge along axis a whose lower corner
has the other two coordinates (p, q), p on the lower-numbered of those axes, has
id 4*a + p + 2*q.
"""
from __future__ import annotations

import functools

import numpy as np

from .gridpull import CORNERS, cell_key, grid_spacing, key_to_cell, key_to_vertex, vertex_key

_OTHER_AXES = {0: (1, 2), 1: (0, 2), 2: (0, 1)}


def edge_id(c1, c2) -> int:
    """Id of the cell edge joining corners c1 and c2 (3-tuples of 0/1 that
    differ on exactly one axis)."""
    diff = [a for a in range(3) if c1[a] != c2[a]]
    assert len(diff) == 1
    a = diff[0]
    u, w = _OTHER_AXES[a]
    return 4 * a + c1[u] + 2 * c1[w]


def edge_corners(e: int):
    """Lower and upper corner (3-tuples) of edge e."""
    a, r = e // 4, e % 4
    u, w = _OTHER_AXES[a]
    lo = [0, 0, 0]
    lo[u], lo[w] = r & 1, r >> 1
    hi = list(lo)
    hi[a] = 1
    return tuple(lo), tuple(hi)


def face_walks():
    """The six faces of a cell, each as its four corners in counter-clockwise
    order seen from outside the cell (the right-hand rule about the outward
    normal).  For the face at side s of axis a, with (u, w) the cyclic pair
    after a (e_u x e_w = e_a), the order is (0,0), (1,0), (1,1), (0,1) in (u, w)
    on the + side and the reverse turn on the - side."""
    walks = []
    for a in range(3):
        u, w = (a + 1) % 3, (a + 2) % 3
        for s in (0, 1):
            uw = [(0, 0), (1, 0), (1, 1), (0, 1)] if s == 1 else [(0, 0), (0, 1), (1, 1), (1, 0)]
            walk = []
            for pu, pw in uw:
                c = [0, 0, 0]
                c[a], c[u], c[w] = s, pu, pw
                walk.append(tuple(c))
            walks.append(walk)
    return walks


def _corner_index(c) -> int:
    return c[0] + 2 * c[1] + 4 * c[2]


def cell_segments(neg) -> dict:
    """Directed surface segments of one cell: {entering edge: leaving edge}.
    neg[k] says whether corner k is negative."""
    nxt = {}
    for walk in face_walks():
        n = [bool(neg[_corner_index(c)]) for c in walk]
        entering = None
        # Start the walk just after a positive corner so that every run of
        # negative corners is seen whole.
        start = next((i for i in range(4) if not n[i]), None)
        if start is None:
            continue  # all four negative: no crossing on this face
        for step in range(1, 5):
            i0, i1 = (start + step - 1) % 4, (start + step) % 4
            if not n[i0] and n[i1]:
                entering = edge_id(walk[i0], walk[i1])
            elif n[i0] and not n[i1]:
                leaving = edge_id(walk[i0], walk[i1])
                assert entering is not None and entering not in nxt
                nxt[entering] = leaving
                entering = None
    return nxt


def cell_cycles(neg) -> list:
    """Closed cycles of cut edges of one cell, each started at its lowest edge
    id, in order of that id."""
    nxt = cell_segments(neg)
    seen, cycles = set(), []
    for e in sorted(nxt):
        if e in seen:
            continue
        cyc = [e]
        seen.add(e)
        f = nxt[e]
        while f != e:
            assert f not in seen
            cyc.append(f)
            seen.add(f)
            f = nxt[f]
        cycles.append(cyc)
    return cycles


@functools.lru_cache(maxsize=256)
def case_triangles(case: int) -> tuple:
    """Triangles (edge-id triples) of the cell whose negative corners are the
    set bits of `case`."""
    neg = [(case >> k) & 1 for k in range(8)]
    tris = []
    for cyc in cell_cycles(neg):
        for k in range(1, len(cyc) - 1):
            tris.append((cyc[0], cyc[k], cyc[k + 1]))
    return tuple(tris)


def meshed_cells(trainable_keys: np.ndarray, R: int) -> np.ndarray:
    """Cells (sorted cell keys) whose eight corners are all trainable (Sec. 3:
    cells not optimised are skipped)."""
    tk = np.unique(np.asarray(trainable_keys, dtype=np.int64))
    v = key_to_vertex(tk, R)
    cand = v[np.all(v < R, axis=1)]                     # possible lowest corners
    ok = np.ones(len(cand), dtype=bool)
    for c in CORNERS:
        ok &= np.isin(vertex_key(cand + c, R), tk)
    return np.sort(cell_key(cand[ok], R))


def marching_cubes(values: np.ndarray, R: int, cells: np.ndarray, iso: float = 0.0):
    """Triangles of the iso-surface over the given cells.

    values: dense (R+1)^3 array indexed by vertex key, widened to float64;
    cells: cell keys to mesh; iso: the level (a float32 value).
    Returns (tri, tri_cell): tri is (T, 3, 3) float64 world positions, tri_cell
    the key of each triangle's cell; cells in ascending key order, each cell's
    triangles in the order of case_triangles."""
    cells = np.sort(np.asarray(cells, dtype=np.int64))
    h = grid_spacing(R)
    iso = float(iso)
    base = key_to_cell(cells, R)                                  # (N, 3)
    d = np.stack([values[vertex_key(base + c, R)] for c in CORNERS], axis=1).astype(np.float64)
    case = np.zeros(len(cells), dtype=np.int64)
    for k in range(8):
        case |= (d[:, k] < iso).astype(np.int64) << k
    out_tri, out_cell, out_order = [], [], []
    for c in np.unique(case):
        tris = case_triangles(int(c))
        if not tris:
            continue
        sel = np.nonzero(case == c)[0]
        b, dc = base[sel].astype(np.float64), d[sel]
        for ti, tri in enumerate(tris):
            pos = np.empty((len(sel), 3, 3))
            for vi, e in enumerate(tri):
                lo, hi = edge_corners(e)
                klo, khi = _corner_index(lo), _corner_index(hi)
                t = (iso - dc[:, klo]) / (dc[:, khi] - dc[:, klo])
                p = -1.0 + h * (b + np.asarray(lo, dtype=np.float64))
                p[:, e // 4] += h * t
                pos[:, vi, :] = p
            out_tri.append(pos)
            out_cell.append(cells[sel])
            out_order.append(np.full(len(sel), ti))
    if not out_tri:
        return np.zeros((0, 3, 3)), np.zeros(0, dtype=np.int64)
    tri = np.concatenate(out_tri)
    tcell = np.concatenate(out_cell)
    order = np.lexsort((np.concatenate(out_order), tcell))
    return tri[order], tcell[order]


# ------------------------------------------------------- mesh properties
def triangle_normals(tri: np.ndarray) -> np.ndarray:
    """(v1 - v0) x (v2 - v0): twice the area times the unit normal."""
    return np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])


def mesh_area(tri: np.ndarray) -> float:
    return float(0.5 * np.linalg.norm(triangle_normals(tri), axis=1).sum())


def enclosed_volume(tri: np.ndarray) -> float:
    """Volume of the region the closed, outward-oriented mesh bounds (divergence
    theorem: the sum of signed tetrahedra against the origin)."""
    return float(np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0)


def weld(tri: np.ndarray):
    """Merge vertices with identical coordinates.  Returns (vertices, faces)."""
    flat = tri.reshape(-1, 3)
    verts, inv = np.unique(flat, axis=0, return_inverse=True)
    return verts, inv.reshape(-1, 3)


def directed_edge_counts(faces: np.ndarray) -> dict:
    """{(a, b): how many faces contain the directed edge a -> b}."""
    counts: dict = {}
    for f in faces:
        for k in range(3):
            key = (int(f[k]), int(f[(k + 1) % 3]))
            counts[key] = counts.get(key, 0) + 1
    return counts


def euler_characteristic(faces: np.ndarray) -> int:
    """V - E + F of the welded mesh (vertices counted from the faces)."""
    v = len(np.unique(faces))
    edges = {tuple(sorted(e)) for e in directed_edge_counts(faces)}
    return v - len(edges) + len(faces)
