"""FP64 CPU oracle for one GridPull optimisation step.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's
CPU-baseline leg; never by the library.  It shares no code with the CUDA path.

Everything here is the plain definition from the paper (Chen, Liu, Han,
"GridPull", ICCV 2023), in float64, vectorised over queries but otherwise in the
order the paper states it:

* grid and cells            - Sec. 3 "Overview", "Discrete Grids"
* trilinear f and grad f     - Eq. 1 and Eq. 3, by solving the 8x8 linear system
* pulled query and L_Pull    - Sec. 3 "Signed Distance Inference", Eq. 4
* M1 / M2 bands              - Sec. 3 (pull band) and "Continuous Distance Fields"
* L_TV                       - Eq. 5
* L_Surface                  - Eq. 6
* L_grad (cosine)            - Eq. 7
* total loss                 - Eq. 8 with alpha, beta, gamma of Sec. 4 "Details"
* query sampling             - Sec. 3 (Gaussian around sampled surface points)
* nearest surface point      - brute force over the whole cloud
* Adam                       - Sec. 4 "Details" (Kingma and Ba's update)

Readings where the paper is silent (the same readings the CUDA path takes):

* the domain is [-1,1]^3 with R cells per axis (R a power of two), h = 2/R and
  vertex (i,j,k) at -1 + h*(i,j,k);
* cell(x) = floor((x + 1) / h) of the exact real value for the float32 input,
  clamped to [0, R-1] for surface points; a query is valid only when that floor
  lies in [0, R-1] on every axis, its cell is in the pull band, and the cell of
  its surface point is in the pull band too;
* the query terms are averaged over the valid queries, L_TV over the TV vertex
  set; the surface term is evaluated at NN(q) of each valid query;
* n = g / max(|g|, 1e-12); the derivative of |r| at r = 0 and sign(0) are 0;
* TV of a vertex uses its six axis neighbours that lie inside [0, R]^3;
* the pull band is the Chebyshev dilation of the occupied cells by M1 cells, the
  TV vertex set the corners of the dilation by M2, the trainable set the corners
  of the dilation by max(M1, M2); a negative M means every cell;
* the sampling sigma of a point is its distance to its k-th nearest other point;
* nearest neighbour: D = ((qx-sx)^2 + (qy-sy)^2) + (qz-sz)^2 in float64 from
  the float32 inputs, ties to the lowest index.
"""
from __future__ import annotations

import math

import numpy as np

# Loss weights of Sec. 4 "Details": alpha (TV), beta (surface), gamma (gradient).
DEFAULT_WEIGHTS = (1.0, 1.0, 0.005)
NORM_FLOOR = 1e-12
# Cap of the residual's conditioning factor kappa = |q - s| / |r| in the
# per-vertex tolerance scale (abs_terms): kappa grows without bound as r -> 0,
# so the scale it multiplies is capped at this factor over the plain terms.
KAPPA_MAX = 64.0


# ------------------------------------------------------------------ grid
def grid_spacing(R: int) -> float:
    return 2.0 / R


def _two_sum(a: np.ndarray, b: float):
    """Error-free sum: a + b == s + e exactly (Knuth's TwoSum)."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def cell_and_local(x: np.ndarray, R: int):
    """Cell index, local coordinate in [0,1] and in-domain flag per point.

    ``x`` is float32 (N,3).  t = (x + 1) * R / 2 is taken exactly: the sum is
    split into s + e without error and R/2 is a power of two, so floor(t) is the
    floor of the real value.  Returns (cell int64 unclamped, local float64,
    inside bool)."""
    x64 = np.asarray(x, dtype=np.float32).astype(np.float64)
    s, e = _two_sum(x64, 1.0)
    half_r = R / 2.0
    t_hi = s * half_r
    t_lo = e * half_r
    c = np.floor(t_hi)
    c = c - ((t_hi == c) & (t_lo < 0))
    local = (t_hi - c) + t_lo
    cell = c.astype(np.int64)
    inside = np.all((cell >= 0) & (cell <= R - 1), axis=1)
    return cell, local, inside


def clamp_cell(cell: np.ndarray, local: np.ndarray, R: int):
    """Clamp a cell to [0, R-1]; the local coordinate follows the clamped cell."""
    cc = np.clip(cell, 0, R - 1)
    return cc, local + (cell - cc)


def vertex_key(ijk: np.ndarray, R: int) -> np.ndarray:
    n = R + 1
    return ijk[..., 0] + n * (ijk[..., 1] + n * ijk[..., 2])


def cell_key(ijk: np.ndarray, R: int) -> np.ndarray:
    return ijk[..., 0] + R * (ijk[..., 1] + R * ijk[..., 2])


def key_to_vertex(key: np.ndarray, R: int) -> np.ndarray:
    n = R + 1
    return np.stack([key % n, (key // n) % n, key // (n * n)], axis=-1)


def key_to_cell(key: np.ndarray, R: int) -> np.ndarray:
    return np.stack([key % R, (key // R) % R, key // (R * R)], axis=-1)


# Corner order: k = dx + 2*dy + 4*dz.
CORNERS = np.array([[k & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], dtype=np.int64)


# ------------------------------------------------------ Eq. 3: trilinear
def _basis(xi: np.ndarray) -> np.ndarray:
    """[1, x, y, z, xy, xz, yz, xyz] of Eq. 3 at local offsets xi (N,3)."""
    x, y, z = xi[:, 0], xi[:, 1], xi[:, 2]
    one = np.ones_like(x)
    return np.stack([one, x, y, z, x * y, x * z, y * z, x * y * z], axis=1)


def _basis_grad(xi: np.ndarray) -> np.ndarray:
    """d basis / d(x,y,z): (N, 3, 8)."""
    x, y, z = xi[:, 0], xi[:, 1], xi[:, 2]
    zero, one = np.zeros_like(x), np.ones_like(x)
    dx = np.stack([zero, one, zero, zero, y, z, zero, y * z], axis=1)
    dy = np.stack([zero, zero, one, zero, x, zero, z, x * z], axis=1)
    dz = np.stack([zero, zero, zero, one, zero, x, y, x * y], axis=1)
    return np.stack([dx, dy, dz], axis=1)


def trilinear_system(h: float) -> np.ndarray:
    """The 8x8 matrix of Eq. 3: row k is the basis at corner k of a cell whose
    lowest vertex is the origin (the polynomial space is translation invariant,
    so each cell is solved in its own frame)."""
    return _basis(CORNERS.astype(np.float64) * h)


def trilinear_eval(d8: np.ndarray, xi: np.ndarray, h: float):
    """f and grad f at local world offsets ``xi`` (N,3) from corner values
    ``d8`` (N,8), by solving Eq. 3 for the coefficients a.

    Also returns the sensitivities df/dd (N,8) and d(grad f)/dd (N,3,8), i.e.
    A^-T basis(xi) and A^-T dbasis(xi), for the explicit backward."""
    A = trilinear_system(h)
    coef = np.linalg.solve(A, d8.T).T                      # (N, 8): a_0..a_7
    b = _basis(xi)
    db = _basis_grad(xi)
    f = np.einsum("nk,nk->n", b, coef)
    g = np.einsum("nak,nk->na", db, coef)
    sens_f = np.linalg.solve(A.T, b.T).T                    # (N, 8)
    sens_g = np.linalg.solve(A.T, db.reshape(-1, 8).T).T.reshape(-1, 3, 8)
    return f, g, sens_f, sens_g


# --------------------------------------------------------------- bands
def occupied_cells(points: np.ndarray, R: int) -> np.ndarray:
    cell, local, _ = cell_and_local(points, R)
    cell, _ = clamp_cell(cell, local, R)
    return np.unique(cell_key(cell, R))


def dilate_cells(cell_keys: np.ndarray, M: int, R: int) -> np.ndarray:
    """Cells within Chebyshev distance M of the given cells (M < 0: every cell)."""
    if M < 0 or (M >= R - 1 and len(cell_keys)):
        return np.arange(R ** 3, dtype=np.int64)
    if len(cell_keys) == 0:
        return np.zeros(0, dtype=np.int64)
    base = key_to_cell(cell_keys, R)
    rng = np.arange(-M, M + 1)
    offs = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), axis=-1).reshape(-1, 3)
    out = []
    for o in offs:
        c = base + o
        ok = np.all((c >= 0) & (c < R), axis=1)
        out.append(cell_key(c[ok], R))
    return np.unique(np.concatenate(out))


def cell_corners(cell_keys: np.ndarray, R: int) -> np.ndarray:
    base = key_to_cell(cell_keys, R)
    return np.unique(np.concatenate([vertex_key(base + c, R) for c in CORNERS]))


def axis_neighbours(vkeys: np.ndarray, R: int):
    """The six axis neighbours of each vertex: keys (N,6) and an in-grid mask."""
    v = key_to_vertex(vkeys, R)
    offs = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]])
    nb = v[:, None, :] + offs[None, :, :]
    ok = np.all((nb >= 0) & (nb <= R), axis=2)
    return vertex_key(np.clip(nb, 0, R), R), ok


def band_sets(points: np.ndarray, R: int, M1: int, M2: int) -> dict:
    """Pull cells (M1 band), TV vertices (corners of the M2 band), trainable
    vertices (corners of the max(M1,M2) band) and the vertices a step reads.
    Sec. 3: the M1-bandwidth of the pull loss and the M2-bandwidth of L_TV; only
    variables in the bands are optimised."""
    occ = occupied_cells(points, R)
    big = -1 if (M1 < 0 or M2 < 0) else max(M1, M2)
    pull = dilate_cells(occ, M1, R)
    tv = cell_corners(dilate_cells(occ, M2, R), R)
    trainable = cell_corners(dilate_cells(occ, big, R), R)
    nb, ok = axis_neighbours(tv, R)
    required = np.unique(np.concatenate([trainable, tv, nb[ok]]))
    return {"occupied": occ, "pull_cells": pull, "tv": tv, "trainable": trainable,
            "required": required}


def _dilate_cells_bitmap(b: np.ndarray, M: int) -> np.ndarray:
    """Chebyshev dilation by M of a boolean cell array (per axis: separable)."""
    out = b
    for ax in range(3):
        src, res = out, out.copy()
        n = src.shape[ax]
        for d in range(1, min(M, n - 1) + 1):
            hi, lo = [slice(None)] * 3, [slice(None)] * 3
            hi[ax], lo[ax] = slice(d, None), slice(None, n - d)
            res[tuple(hi)] |= src[tuple(lo)]
            res[tuple(lo)] |= src[tuple(hi)]
        out = res
    return out


def band_vertex_sets_bitmap(points: np.ndarray, R: int, M1: int, M2: int) -> dict:
    """The TV and trainable vertex sets of band_sets (corners of the M2 and
    max(M1, M2) dilations of the occupied cells) as sorted keys, built on dense
    boolean arrays indexed [k, j, i] instead of sets of keys: the same
    definition, for grids where 125 shifted copies of the occupied set would not
    fit in memory.  Also returns the occupied cell keys."""
    occ_keys = occupied_cells(points, R)
    occ = np.zeros((R, R, R), bool)
    c = key_to_cell(occ_keys, R)
    occ[c[:, 2], c[:, 1], c[:, 0]] = True
    out = {"occupied": occ_keys}
    big = -1 if (M1 < 0 or M2 < 0) else max(M1, M2)
    for name, M in (("tv", M2), ("trainable", big)):
        cells = np.ones_like(occ) if M < 0 else _dilate_cells_bitmap(occ, M)
        v = np.zeros((R + 1,) * 3, bool)
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    v[dz:dz + R, dy:dy + R, dx:dx + R] |= cells
        out[name] = np.flatnonzero(v.reshape(-1)).astype(np.int64)  # i fastest: the vertex key order
        del v, cells
    return out


# ----------------------------------------------------- nearest neighbour
def sq_dist64(q: np.ndarray, s: np.ndarray) -> np.ndarray:
    """((qx-sx)^2 + (qy-sy)^2) + (qz-sz)^2 in float64 for all pairs (Nq, Ns)."""
    q64 = np.asarray(q, np.float32).astype(np.float64)
    s64 = np.asarray(s, np.float32).astype(np.float64)
    dx = q64[:, None, 0] - s64[None, :, 0]
    dy = q64[:, None, 1] - s64[None, :, 1]
    dz = q64[:, None, 2] - s64[None, :, 2]
    d = dx * dx
    d = d + dy * dy
    d = d + dz * dz
    return d


def nearest_point(q: np.ndarray, points: np.ndarray, chunk: int = 512) -> np.ndarray:
    """NN(q): index of the nearest surface point by brute force over the whole
    cloud; equal distances go to the lowest index (np.argmin's first hit)."""
    out = np.empty(len(q), dtype=np.int64)
    for a in range(0, len(q), chunk):
        out[a:a + chunk] = np.argmin(sq_dist64(q[a:a + chunk], points), axis=1)
    return out


def knn_sigma(points: np.ndarray, k: int = 50, idx=None, chunk: int = 256) -> np.ndarray:
    """Distance from each point (or from points[idx]) to its k-th nearest other
    point; the point itself is excluded by index, duplicates count.  A cloud
    with fewer than k + 1 points uses k = J - 1 (sigma = 0 for a single point)."""
    idx = np.arange(len(points)) if idx is None else np.asarray(idx)
    k = min(k, len(points) - 1)
    out = np.zeros(len(idx), dtype=np.float64)
    if k <= 0:
        return out
    for a in range(0, len(idx), chunk):
        sel = idx[a:a + chunk]
        d = sq_dist64(points[sel], points)
        d[np.arange(len(sel)), sel] = np.inf
        out[a:a + chunk] = np.sqrt(np.partition(d, k - 1, axis=1)[:, k - 1])
    return out


# ------------------------------------------------ counter-based sampling
_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def philox4x32(ctr, key):
    """Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) on one counter.

    ctr: four uint32 words, key: two uint32 words.  Each of the ten rounds
    multiplies words 0 and 2 by the round multipliers (32x32 -> 64 bits), mixes
    the high halves with the other words and the key, and the key is bumped by
    the Weyl constants between rounds."""
    c = [int(x) & _MASK32 for x in ctr]
    k = [int(x) & _MASK32 for x in key]
    for _ in range(10):
        p0 = _PHILOX_M0 * c[0]
        p1 = _PHILOX_M1 * c[2]
        c = [(p1 >> 32) ^ c[1] ^ k[0], p1 & _MASK32, (p0 >> 32) ^ c[3] ^ k[1], p0 & _MASK32]
        k = [(k[0] + _PHILOX_W0) & _MASK32, (k[1] + _PHILOX_W1) & _MASK32]
    return c


def philox4x32_vec(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox4x32-10: each counter word may be an array or a scalar."""
    c0 = np.asarray(c0, dtype=np.uint64) & np.uint64(_MASK32)
    n = c0.shape
    c = [c0] + [np.broadcast_to(np.asarray(x, dtype=np.uint64) & np.uint64(_MASK32), n).copy()
                for x in (c1, c2, c3)]
    k = [k0 & _MASK32, k1 & _MASK32]
    m32 = np.uint64(_MASK32)
    sh = np.uint64(32)
    for _ in range(10):
        p0 = np.uint64(_PHILOX_M0) * c[0]          # < 2^64: no wrap
        p1 = np.uint64(_PHILOX_M1) * c[2]
        c = [(p1 >> sh) ^ c[1] ^ np.uint64(k[0]), p1 & m32, (p0 >> sh) ^ c[3] ^ np.uint64(k[1]), p0 & m32]
        k = [(k[0] + _PHILOX_W0) & _MASK32, (k[1] + _PHILOX_W1) & _MASK32]
    return c


def _seed_key(seed: int):
    return int(seed) & _MASK32, (int(seed) >> 32) & _MASK32


def _u24(x: np.ndarray, plus_one: bool) -> np.ndarray:
    """Top 24 bits of a 32-bit word as a float in (0,1] (plus_one) or [0,1)."""
    top = (np.asarray(x, np.uint64) >> np.uint64(8)).astype(np.float64)
    return (top + (1.0 if plus_one else 0.0)) * 2.0 ** -24


def box_muller3(words) -> np.ndarray:
    """Three standard normals from one Philox block (Box-Muller on two pairs)."""
    u1 = _u24(words[0], True)
    u2 = _u24(words[1], False)
    u3 = _u24(words[2], True)
    u4 = _u24(words[3], False)
    r1 = np.sqrt(-2.0 * np.log(u1))
    r2 = np.sqrt(-2.0 * np.log(u3))
    return np.stack([r1 * np.cos(2 * math.pi * u2), r1 * np.sin(2 * math.pi * u2),
                     r2 * np.cos(2 * math.pi * u4)], axis=1)


def feistel_bits(J: int) -> int:
    """Even bit width m >= 2 with 2^m >= J."""
    m = max(2, (int(J) - 1).bit_length())
    return m + (m & 1)


def point_permutation(J: int, seed: int, epoch: int, positions=None) -> np.ndarray:
    """Pi_e(p): the random order in which epoch ``epoch`` visits the points.

    A 4-round balanced Feistel network on m bits (m even, 2^m >= J) whose round
    function is word 0 of Philox4x32-10 at counter (value, round, epoch, 1) and
    key (seed low, seed high), made a bijection of [0, J) by cycle walking."""
    m = feistel_bits(J)
    half = m // 2
    mask = (1 << half) - 1
    pos = np.arange(J, dtype=np.uint64) if positions is None else np.asarray(positions, np.uint64)

    def enc(x):
        left = x >> np.uint64(half)
        right = x & np.uint64(mask)
        for rnd in range(4):
            f = philox4x32_vec(right, rnd, epoch, 1, *_seed_key(seed))[0] & np.uint64(mask)
            left, right = right, left ^ f
        return (left << np.uint64(half)) | right

    y = enc(pos)
    for _ in range(1000):
        bad = y >= np.uint64(J)
        if not bad.any():
            return y.astype(np.int64)
        y[bad] = enc(y[bad])
    raise RuntimeError("cycle walk did not terminate")


def sample_queries(points: np.ndarray, sigma: np.ndarray, seed: int, epoch: int,
                   positions: np.ndarray):
    """Queries at pool positions ``positions`` of epoch ``epoch`` (Sec. 3:
    Gaussian queries around randomly visited surface points, drawn anew each
    epoch).  Position k visits point j = Pi_e(k mod J) and draws
    z ~ N(0, I) from Philox4x32-10 at counter (k, epoch, 0, 0), key (seed low,
    seed high);
    q = s_j + sigma_j * z.  Returns (q float64 (n,3), j int64 (n,))."""
    J = len(points)
    positions = np.asarray(positions, dtype=np.int64)
    j = point_permutation(J, seed, epoch, positions % J)
    z = box_muller3(philox4x32_vec(positions.astype(np.uint64), epoch, 0, 0, *_seed_key(seed)))
    s = np.asarray(points, np.float32).astype(np.float64)[j]
    return s + np.asarray(sigma, np.float64)[j][:, None] * z, j


def sphere_init(vkeys: np.ndarray, R: int, center, radius: float, noise_std: float, seed: int):
    """Geometric initialisation (Sec. 3): |v - c| - radius at each vertex, plus
    noise_std * N(0,1) (the first Box-Muller normal) from Philox4x32-10 at
    counter (vertex key low, vertex key high, 0, 2), key (seed low, seed high)."""
    h = grid_spacing(R)
    v = -1.0 + h * key_to_vertex(np.asarray(vkeys, np.int64), R).astype(np.float64)
    d = np.sqrt(np.sum((v - np.asarray(center, np.float64)) ** 2, axis=1)) - radius
    if noise_std != 0:
        kk = np.asarray(vkeys, np.uint64)
        w = philox4x32_vec(kk & np.uint64(_MASK32), kk >> np.uint64(32), 0, 2, *_seed_key(seed))
        d = d + noise_std * box_muller3(w)[:, 0]
    return d


# ------------------------------------------------- value stores and bands
class SparseValues:
    """Grid values held only at a set of vertices: ``keys`` (sorted, unique
    vertex keys i + (R+1)(j + (R+1)k)) and ``vals`` (float64, one per key).
    The loss functions accept it wherever they accept a dense ((R+1)^3,)
    array; gradients are then returned over the same compact index (entry n
    belongs to keys[n]).  Reading a vertex that is not held is an error."""

    def __init__(self, keys, vals):
        keys = np.asarray(keys, np.int64)
        order = np.argsort(keys, kind="stable")
        self.keys = keys[order]
        self.vals = np.asarray(vals, np.float64)[order]
        if len(self.keys) > 1 and np.any(self.keys[1:] == self.keys[:-1]):
            raise ValueError("duplicate vertex keys")

    def index(self, vkeys):
        vkeys = np.asarray(vkeys, np.int64)
        pos = np.searchsorted(self.keys, vkeys)
        pos_c = np.minimum(pos, max(len(self.keys) - 1, 0))
        if len(self.keys) == 0 or np.any(self.keys[pos_c] != vkeys):
            raise KeyError("vertex not held by the sparse value store")
        return pos_c


def _store(D):
    """(values array, key -> position map) of a dense array or SparseValues."""
    if isinstance(D, SparseValues):
        return D.vals, D.index
    flat = np.asarray(D).reshape(-1)
    return flat, (lambda k: k)


def in_dilated_band(cell_keys, occupied_keys, M: int, R: int, keys_sorted: bool = False) -> np.ndarray:
    """Membership of cells in the Chebyshev dilation by M of the occupied
    cells (Sec. 3 bandwidth), tested per cell against the occupied keys
    instead of building the dilated set: a cell is in the band iff some cell
    within Chebyshev distance M of it is occupied.  M < 0: every cell.
    keys_sorted: the occupied keys are already sorted (np.unique output)."""
    cell_keys = np.asarray(cell_keys, np.int64)
    if M < 0:
        return np.ones(len(cell_keys), bool)
    occ = np.asarray(occupied_keys, np.int64)
    if not keys_sorted:
        occ = np.sort(occ)
    base = key_to_cell(cell_keys, R)
    hit = np.zeros(len(cell_keys), bool)
    rng = np.arange(-M, M + 1)
    for dz in rng:
        for dy in rng:
            for dx in rng:
                c = base + np.array([dx, dy, dz])
                ok = np.all((c >= 0) & (c < R), axis=1) & ~hit
                if not ok.any():
                    continue
                k = cell_key(c[ok], R)
                pos = np.minimum(np.searchsorted(occ, k), max(len(occ) - 1, 0))
                found = (occ[pos] == k) if len(occ) else np.zeros(len(k), bool)
                hit[np.nonzero(ok)[0][found]] = True
    return hit


def _pull_member(pull_cells, cell_keys, R: int) -> np.ndarray:
    """Pull-band membership: ``pull_cells`` is the band's cell keys, or a
    function of an array of cell keys returning booleans."""
    if callable(pull_cells):
        return np.asarray(pull_cells(cell_keys), bool)
    if R <= 256:
        pull = np.zeros(R ** 3, dtype=bool)
        pull[pull_cells] = True
        return pull[cell_keys]
    return np.isin(cell_keys, pull_cells)


# ------------------------------------------------------- loss and gradient
def _norm(v: np.ndarray) -> np.ndarray:
    return np.sqrt(np.sum(v * v, axis=1))


def _eval_at(D: np.ndarray, cell: np.ndarray, local: np.ndarray, R: int):
    """Corner keys, f, grad f and sensitivities at points with given cells."""
    h = grid_spacing(R)
    keys = np.stack([vertex_key(cell + c, R) for c in CORNERS], axis=1)   # (N, 8)
    vals, index = _store(D)
    d8 = vals[index(keys)]
    f, g, sf, sg = trilinear_eval(d8, local * h, h)
    return keys, f, g, sf, sg


def _unit(g: np.ndarray):
    """n = g / max(|g|, 1e-12) and the Jacobian map v -> dn/dg^T v."""
    gl = _norm(g)
    den = np.maximum(gl, NORM_FLOOR)
    n = g / den[:, None]
    big = gl > NORM_FLOOR

    def vjp(v):
        proj = v - n * np.sum(n * v, axis=1, keepdims=True)
        return np.where(big[:, None], proj, v) / den[:, None]
    return n, vjp


def query_terms(D: np.ndarray, R: int, pull_cells: np.ndarray, q: np.ndarray, s: np.ndarray,
                beta: float, gamma: float, with_grad: bool = True):
    """Per-query terms of Eq. 4, 6 and 7 and, optionally, their gradient.

    D: float64 dense grid values of shape ((R+1)^3,) indexed by vertex key,
    or a SparseValues holding at least the corners of the valid queries' cells
    (gradients are then over its compact index).  pull_cells: the pull band's
    cell keys, or a membership function of cell keys (in_dilated_band).
    q, s: float32 (B,3) query and its nearest surface point NN(q).
    Returns dict with per-query l_pull, l_grad, l_surf, valid, the sums, B_v and
    (if with_grad) the gradient of (1/B_v) * sum(l_pull + beta*l_surf + gamma*l_grad)
    with respect to D, accumulated in query order."""
    q = np.asarray(q, np.float32)
    s = np.asarray(s, np.float32)
    cq, lq, inside = cell_and_local(q, R)
    cs, ls, _ = cell_and_local(s, R)
    cs, ls = clamp_cell(cs, ls, R)
    cq_c = np.clip(cq, 0, R - 1)
    valid = inside & _pull_member(pull_cells, cell_key(cq_c, R), R) & _pull_member(pull_cells, cell_key(cs, R), R)
    idx = np.nonzero(valid)[0]
    Bv = len(idx)
    out = {"valid": valid, "Bv": Bv}
    zeros = np.zeros(len(q))
    out["l_pull"], out["l_grad"], out["l_surf"] = zeros.copy(), zeros.copy(), zeros.copy()
    vals_D, index = _store(D)
    grad = np.zeros_like(vals_D) if with_grad else None
    if Bv == 0:
        out.update(sum_pull=0.0, sum_grad=0.0, sum_surf=0.0, grad=grad)
        return out
    kq, f, g, sfq, sgq = _eval_at(D, cq_c[idx], lq[idx], R)
    ks, fs, gs, sfs, sgs = _eval_at(D, cs[idx], ls[idx], R)
    q64 = q[idx].astype(np.float64)
    s64 = s[idx].astype(np.float64)
    n, n_vjp = _unit(g)
    ns, ns_vjp = _unit(gs)
    # Pulled query p = q - f * n (Sec. 3) and L_Pull = |p - NN(q)| (Eq. 4).
    r = (q64 - s64) - f[:, None] * n
    l_pull = _norm(r)
    l_grad = 1.0 - np.sum(n * ns, axis=1)        # Eq. 7
    l_surf = np.abs(fs)                          # Eq. 6
    out["l_pull"][idx], out["l_grad"][idx], out["l_surf"][idx] = l_pull, l_grad, l_surf
    out["sum_pull"], out["sum_grad"], out["sum_surf"] = l_pull.sum(), l_grad.sum(), l_surf.sum()
    out["pulled"] = q64 - f[:, None] * n
    out["f"], out["g"], out["fs"], out["gs"] = f, g, fs, gs
    if with_grad:
        w = 1.0 / Bv
        u = np.where(l_pull[:, None] > 0, r / np.where(l_pull > 0, l_pull, 1.0)[:, None], 0.0)
        dL_df = -w * np.sum(u * n, axis=1)
        dL_dn = -w * f[:, None] * u - w * gamma * ns
        dL_dg = n_vjp(dL_dn)
        dL_dns = -w * gamma * n
        dL_dgs = ns_vjp(dL_dns)
        dL_dfs = w * beta * np.sign(fs)
        cq_grad = dL_df[:, None] * sfq + np.einsum("na,nak->nk", dL_dg, sgq)
        cs_grad = dL_dfs[:, None] * sfs + np.einsum("na,nak->nk", dL_dgs, sgs)
        keys = index(np.concatenate([kq, ks], axis=1).reshape(-1))  # query order
        vals = np.concatenate([cq_grad, cs_grad], axis=1).reshape(-1)
        np.add.at(grad, keys, vals)
        # Conditioning of each vertex's sum: the magnitudes of the elementary
        # products it is made of, before any cancellation.  A component of
        # dL/dg is only known to within u times the size of the vector it is
        # projected from (dL/dn / |g|), and dL/df to within u times w (|u.n|
        # <= 1); the unit residual u = r/|r| itself carries a relative error
        # kappa = |q - s| / |r| times u (r is a difference of vectors of size
        # |q - s|).  Those sizes, times |w_c| and |dw_c/dx_a|, are the scale
        # against which a float32 evaluation is compared.
        kappa_raw = np.maximum(1.0, np.linalg.norm(q64 - s64, axis=1) / np.maximum(l_pull, 1e-300))
        kappa = np.minimum(kappa_raw, KAPPA_MAX)
        out["kappa_max"] = float(kappa_raw.max())
        sq_g = kappa * np.linalg.norm(dL_dn, axis=1) / np.maximum(_norm(g), NORM_FLOOR)
        ss_g = np.linalg.norm(dL_dns, axis=1) / np.maximum(_norm(gs), NORM_FLOOR)
        tq = (w * kappa)[:, None] * np.abs(sfq) + sq_g[:, None] * np.abs(sgq).sum(axis=1)
        ts = np.abs(dL_dfs)[:, None] * np.abs(sfs) + ss_g[:, None] * np.abs(sgs).sum(axis=1)
        out["abs_terms"] = np.zeros_like(vals_D)
        np.add.at(out["abs_terms"], keys, np.concatenate([tq, ts], axis=1).reshape(-1))
        # The plain absolute sum of the contributions added at each vertex,
        # sum_k |c_k|: the condition of the sum itself (abs_terms >= this).
        out["abs_contrib"] = np.zeros_like(vals_D)
        np.add.at(out["abs_contrib"], keys, np.abs(vals))
    out["grad"] = grad
    return out


def _tv_diffs(D, R: int, tv_keys: np.ndarray):
    """d_i - d_n for the six axis neighbours of each TV vertex (0 where the
    neighbour is outside [0, R]^3), the neighbour keys, the in-grid mask and the
    store's value array and key map."""
    vals, index = _store(D)
    nb, ok = axis_neighbours(tv_keys, R)
    dn = np.zeros(nb.shape)
    dn[ok] = vals[index(nb[ok])]
    di = vals[index(tv_keys)][:, None]
    return np.where(ok, di - dn, 0.0), nb, ok, vals, index


def tv_term(D: np.ndarray, R: int, tv_keys: np.ndarray, with_grad: bool = True, n_tv=None):
    """Eq. 5 per TV vertex, averaged over the TV set, and its gradient.

    ``n_tv`` (default len(tv_keys)) is the divisor |T| of the mean: pass the
    whole set's size to evaluate a subset of the TV vertices' terms."""
    T = len(tv_keys) if n_tv is None else int(n_tv)
    vals, _ = _store(D)
    grad = np.zeros_like(vals) if with_grad else None
    if len(tv_keys) == 0 or T == 0:
        return 0.0, grad, np.zeros(0)
    diff, nb, ok, vals, index = _tv_diffs(D, R, tv_keys)
    tv = np.sqrt(np.sum(diff * diff, axis=1))
    loss = tv.sum() / T
    if with_grad:
        pos = tv > 0
        coef = np.where(pos[:, None], diff / np.where(pos, tv, 1.0)[:, None], 0.0) / T
        np.add.at(grad, index(tv_keys), coef.sum(axis=1))
        np.add.at(grad, index(nb[ok]), -coef[ok])
    return loss, grad, tv


def tv_term_abs(D: np.ndarray, R: int, tv_keys: np.ndarray, n_tv=None) -> np.ndarray:
    """Per vertex, the sum of |(d_i - d_n) / TV| over the terms of the L_TV
    gradient that land on it (conditioning of that sum)."""
    T = len(tv_keys) if n_tv is None else int(n_tv)
    vals, _ = _store(D)
    out = np.zeros_like(vals)
    if len(tv_keys) == 0 or T == 0:
        return out
    diff, nb, ok, vals, index = _tv_diffs(D, R, tv_keys)
    tv = np.sqrt(np.sum(diff * diff, axis=1))
    pos = tv > 0
    coef = np.abs(np.where(pos[:, None], diff / np.where(pos, tv, 1.0)[:, None], 0.0)) / T
    np.add.at(out, index(tv_keys), coef.sum(axis=1))
    np.add.at(out, index(nb[ok]), coef[ok])
    return out


def step_loss_grad(D: np.ndarray, R: int, sets: dict, q: np.ndarray, s: np.ndarray,
                   weights=DEFAULT_WEIGHTS, with_grad: bool = True) -> dict:
    """L = L_Pull + alpha L_TV + beta L_Surface + gamma L_grad (Eq. 8) and dL/dD.

    sets: "pull_cells" (keys or a membership function), "tv" (the TV vertex
    keys whose terms are evaluated) and optionally "n_tv" (|T| when "tv" is a
    subset).  D: dense array or SparseValues (see query_terms)."""
    alpha, beta, gamma = weights
    n_tv = sets.get("n_tv")
    qt = query_terms(D, R, sets["pull_cells"], q, s, beta, gamma, with_grad)
    tv_loss, tv_grad, tv_vals = tv_term(D, R, sets["tv"], with_grad, n_tv)
    tv_abs = tv_term_abs(D, R, sets["tv"], n_tv) if with_grad else None
    Bv = qt["Bv"]
    mean = (lambda x: x / Bv) if Bv else (lambda x: 0.0)
    res = {
        "Bv": Bv, "valid": qt["valid"],
        "l_pull": mean(qt["sum_pull"]), "l_grad": mean(qt["sum_grad"]),
        "l_surf": mean(qt["sum_surf"]), "l_tv": tv_loss,
        "per_query": qt, "tv_vals": tv_vals,
    }
    res["loss"] = res["l_pull"] + alpha * res["l_tv"] + beta * res["l_surf"] + gamma * res["l_grad"]
    if with_grad:
        res["grad"] = qt["grad"] + alpha * tv_grad
        zero = np.zeros_like(_store(D)[0])
        res["abs_terms"] = qt.get("abs_terms", zero) + alpha * tv_abs
        res["abs_contrib"] = qt.get("abs_contrib", zero) + alpha * tv_abs
        res["kappa_max"] = qt.get("kappa_max", 1.0)
    return res


# ------------------------------------------------------------------- Adam
def adam(d, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, Algorithm 1) at step t >= 1, float64."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return d - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
