"""Helpers shared by the GPU parity tests: build the library, move band
exports to numpy, compare against the oracle with the stated tolerances."""
import numpy as np
import pytest

# Tolerance of the parity contract: float32 GPU vs float64 oracle.
REL_TOL = 1e-5


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def build_lib():
    from paper_2308_13175_gb300 import build
    return build.build()


def export_band(band):
    """(ijk, values, flags, exists) of every stored slot, as numpy."""
    from paper_2308_13175_gb300 import binding as gb
    ijk, d, fl = gb.gp_band_export(band)
    ijk = ijk.cpu().numpy().astype(np.int64)
    d = d.cpu().numpy()
    fl = fl.cpu().numpy()
    return ijk, d, fl, (fl & 4) != 0


def vertex_keys(ijk, R):
    n = R + 1
    return ijk[:, 0] + n * (ijk[:, 1] + n * ijk[:, 2])


def dense_from_band(values, ijk, exists, R):
    """Float64 dense grid ((R+1)^3,) holding the band's stored values."""
    D = np.zeros((R + 1) ** 3, dtype=np.float64)
    D[vertex_keys(ijk[exists], R)] = values[exists].astype(np.float64)
    return D


def assert_rel(got, want, tol=REL_TOL, what="value"):
    got, want = float(got), float(want)
    assert abs(got - want) <= tol * abs(want) + 1e-30, f"{what}: got {got!r}, want {want!r}"


def strict_bound_failures(g, ref, tol=REL_TOL):
    """Vertices outside the stricter per-vertex bound
    |g_i - ref_i| <= tol * max(|ref_i|, 1e-3 max|ref|), reported beside the
    contract (it ignores cancellation inside a vertex's sum)."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0, 0.0
    floor = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
    rel = np.abs(g - ref) / np.maximum(floor, 1e-300)
    return int(np.count_nonzero(rel > tol)), float(rel.max())


def assert_grad_close(g, ref, scale=None, tol=REL_TOL, what="grad", kappa_max=None):
    """Norm-wise relative error <= tol, and per vertex
    |g_i - ref_i| <= tol * scale_i, where scale_i is the oracle's conditioning
    of that vertex's sum (the sizes of the products it adds up; >= |ref_i| and
    pinned to at most 64 times the absolute sum of its contributions).
    Without a scale the per-vertex check uses max(|ref_i|, 1e-3 max|ref|).
    Prints how many vertices miss that stricter bound and, when given, the
    largest residual conditioning factor kappa of the records."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    nrm = np.linalg.norm(ref)
    err = np.linalg.norm(g - ref)
    nfail, worst_rel = strict_bound_failures(g, ref, tol)
    print(f"[{what}] norm err {err / max(nrm, 1e-300):.3e}; vertices over tol*max(|g*|, 1e-3 |g*|_inf): "
          f"{nfail} of {ref.size} (worst {worst_rel:.3e})"
          + (f"; kappa max {kappa_max:.3g}" if kappa_max is not None else ""))
    assert err <= tol * nrm, f"{what}: |g - ref| / |ref| = {err / max(nrm, 1e-300):.3e}"
    if scale is None:
        scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
    scale = np.maximum(np.asarray(scale, np.float64), np.abs(ref))
    per = np.abs(g - ref) / np.maximum(scale, 1e-300)
    worst = int(np.argmax(per))
    assert per[worst] <= tol, (f"{what}: vertex {worst} err {abs(g[worst] - ref[worst]):.3e} = {per[worst]:.3e} of "
                               f"its scale {scale[worst]:.3e} (got {g[worst]}, want {ref[worst]})")
