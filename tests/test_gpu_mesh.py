"""Parity of gp_mesh_extract (through the C ABI) with the FP64 mesh oracle.

Contract: the meshed cells, each cell's triangle count and the triangles' order
are bit-exact (every decision is the float32 comparison d < iso on the same
values on both sides); vertex positions agree within POS_TOL.  The GPU forms
t = (iso - d_lo) / (d_hi - d_lo) with three correctly rounded float32
operations on exact inputs and adds h t to the exact corner -1 + h i, so its
error is at most (3 h t + h t + 1) 2^-24 <= 1.2e-7 for h <= 1/4 and |x| <= 1;
POS_TOL is twice that.  Inputs come from the seeded generators; expected values
from the oracle only.
"""
import ctypes

import numpy as np
import pytest

from oracle import gridpull as o
from oracle import mesh as om
from paper_2308_13175_gb300 import synth

from gpu_common import build_lib, dense_from_band, export_band, have_gpu

pytestmark = pytest.mark.gpu

POS_TOL = 2.5e-7


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


def _band(gb, ctx, pts, R, M1, M2):
    import torch
    return gb.gp_build_band(ctx, torch.from_numpy(np.ascontiguousarray(pts)).cuda(), R, M1, M2, 0)


def _set_values(gb, band, fn):
    """Write fn(world xyz of each stored slot) into the band (float32)."""
    import torch
    ijk, _, _, exists = export_band(band)
    R = band.info["R"]
    x = -1.0 + (2.0 / R) * ijk.astype(np.float64)
    vals = np.where(exists, fn(x), 0.0).astype(np.float32)
    gb.gp_band_set_values(band, torch.from_numpy(vals).cuda())
    return vals


def _compare(gb, band, pts, R, M1, M2, iso=0.0):
    """GPU soup against the oracle over the oracle's own meshed-cell set."""
    tri, cells = gb.gp_mesh_extract(band, iso)
    tri = tri.cpu().numpy().astype(np.float64)
    cells = cells.cpu().numpy()
    ijk, d, _, exists = export_band(band)
    D = dense_from_band(d, ijk, exists, R)
    sets = o.band_sets(pts, R, M1, M2)
    want_cells = om.meshed_cells(sets["trainable"], R)
    want_tri, want_cell = om.marching_cubes(D, R, want_cells, float(np.float32(iso)))
    # the GPU writes bricks in storage order; a stable sort by cell keeps each
    # cell's triangles in fan order
    order = np.argsort(cells, kind="stable")
    np.testing.assert_array_equal(cells[order], want_cell)
    err = np.abs(tri[order] - want_tri).max() if len(tri) else 0.0
    assert err <= POS_TOL, f"max vertex error {err:.3e}"
    return tri, cells, want_cells, D


def test_mesh_dense_random_field_covers_every_case(gb, ctx):
    """A dense band (every cell meshed) holding i.i.d. normal values: all 256
    sign patterns of a cell occur."""
    R = 32
    pts = synth.sphere_cloud(2000, 0.5, seed=0)
    band = _band(gb, ctx, pts, R, -1, -1)
    rng = np.random.default_rng(7)
    _set_values(gb, band, lambda x: rng.standard_normal(len(x)))
    tri, cells, want_cells, D = _compare(gb, band, pts, R, -1, -1)
    assert len(want_cells) == R ** 3
    base = o.key_to_cell(want_cells, R)
    case = np.zeros(len(want_cells), dtype=np.int64)
    for k, c in enumerate(o.CORNERS):
        case |= (D[o.vertex_key(base + c, R)] < 0).astype(np.int64) << k
    assert len(np.unique(case)) == 256
    band.close()


def test_mesh_large_band_takes_the_warp_form(gb, ctx):
    """A dense R = 128 band has 17^3 = 4,913 active bricks, enough for the
    warp-per-brick kernels (32 bricks per SM on 152 SMs); random values put
    many triangles on every lane."""
    R = 128
    pts = synth.sphere_cloud(2000, 0.5, seed=0)
    band = _band(gb, ctx, pts, R, -1, -1)
    rng = np.random.default_rng(5)
    _set_values(gb, band, lambda x: rng.standard_normal(len(x)))
    gb.gp_profile(ctx, True)
    _compare(gb, band, pts, R, -1, -1)
    gb.gp_profile(ctx, False)
    names = set(gb.gp_profile_read(ctx))
    assert {"k_mesh_count_w", "k_mesh_emit_w"} <= names, names
    band.close()


@pytest.mark.parametrize("R,M", [(64, 2), (128, 1), (256, 2)])
def test_mesh_band_skips_cells_not_optimised(gb, ctx, R, M):
    """The single-object cloud's band with a noisy sphere field: only cells whose
    8 corners are trainable are meshed (256^3 with M = 2 is the benchmark's
    band)."""
    pts = synth.object_cloud(100_000, seed=1)
    band = _band(gb, ctx, pts, R, M, M)
    h = 2.0 / R
    c = 0.5 * (pts.min(0) + pts.max(0))
    gb.gp_band_init_sphere(band, c, 0.3, 0.7 * h, 11)
    tri, cells, want_cells, _ = _compare(gb, band, pts, R, M, M)
    assert len(tri) > 1000
    assert set(np.unique(cells).tolist()) <= set(want_cells.tolist())
    band.close()


def test_mesh_iso_levels_and_ties(gb, ctx):
    """Values on a coarse lattice so that many equal the level exactly (they
    count as positive), at levels 0 and 0.25, and a level below every value."""
    R = 16
    pts = synth.sphere_cloud(2000, 0.5, seed=0)
    band = _band(gb, ctx, pts, R, -1, -1)
    rng = np.random.default_rng(3)
    _set_values(gb, band, lambda x: 0.25 * rng.integers(-2, 3, len(x)))
    for iso in (0.0, 0.25, -0.125):
        _compare(gb, band, pts, R, -1, -1, iso)
    tri, _ = gb.gp_mesh_extract(band, -1.0)
    assert tri.shape[0] == 0
    band.close()


def test_mesh_of_a_sphere_is_a_closed_genus_zero_surface(gb, ctx):
    R = 64
    pts = synth.sphere_cloud(5000, 0.5, seed=0)
    band = _band(gb, ctx, pts, R, -1, -1)
    centre = np.array([0.03, -0.02, 0.01])
    _set_values(gb, band, lambda x: np.linalg.norm(x - centre, axis=1) - 0.5)
    tri, _ = gb.gp_mesh_extract(band, 0.0, with_cells=False)
    tri = tri.cpu().numpy().astype(np.float64)
    _, faces = om.weld(tri)
    counts = om.directed_edge_counts(faces)
    assert max(counts.values()) == 1 and all((b, a) in counts for (a, b) in counts)
    assert om.euler_characteristic(faces) == 2
    band.close()


def test_mesh_sizing_capacity_and_errors(gb, ctx):
    import torch
    R = 16
    pts = synth.sphere_cloud(2000, 0.5, seed=0)
    band = _band(gb, ctx, pts, R, -1, -1)
    _set_values(gb, band, lambda x: np.linalg.norm(x, axis=1) - 0.5)
    lib = gb.load()
    n = ctypes.c_int64(-5)
    ctx.check(lib.gp_mesh_extract(band.handle, 0.0, None, None, 0, ctypes.byref(n)))
    T = int(n.value)
    assert T > 0
    # too small a buffer: the total comes back and nothing is written
    small = torch.full((T - 1, 9), 7.0, device="cuda")
    st = lib.gp_mesh_extract(band.handle, 0.0, ctypes.c_void_p(small.data_ptr()), None, T - 1, ctypes.byref(n))
    assert st == gb.GP_OK and n.value == T
    assert bool((small == 7.0).all())
    # exact capacity: written, and equal to the binding's result
    full = torch.empty((T, 9), device="cuda")
    st = lib.gp_mesh_extract(band.handle, 0.0, ctypes.c_void_p(full.data_ptr()), None, T, ctypes.byref(n))
    assert st == gb.GP_OK and n.value == T
    ref, _ = gb.gp_mesh_extract(band, 0.0)
    assert torch.equal(full.view(-1, 3, 3), ref)
    # argument errors
    assert lib.gp_mesh_extract(band.handle, float("nan"), None, None, 0, ctypes.byref(n)) == 1
    assert lib.gp_mesh_extract(band.handle, 0.0, None, None, -1, ctypes.byref(n)) == 1
    assert lib.gp_mesh_extract(band.handle, 0.0, None, None, 4, ctypes.byref(n)) == 1
    assert lib.gp_mesh_extract(band.handle, 0.0, None, None, 0, None) == 1
    # a field with no crossing
    _set_values(gb, band, lambda x: np.ones(len(x)))
    tri, cells = gb.gp_mesh_extract(band, 0.0)
    assert tri.shape == (0, 3, 3) and cells.shape == (0,)
    band.close()
