"""ctypes binding of libgridpull.so: the C ABI of ``include/gridpull.h`` under
the same names, with torch tensors for device memory and torch's current CUDA
stream.  Argument marshalling only: every step runs in the library's kernels.

The library is loaded on first use; a missing library raises ``RuntimeError``
(there is no fallback path)."""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB as _LIB_PATH

_lib = None
_lock = threading.Lock()

GP_OK, GP_ERR_ARG, GP_ERR_OOM, GP_ERR_CUDA, GP_ERR_TIMEOUT, GP_ERR_STATE, GP_ERR_NUMERIC = range(7)
GP_BAND_DETERMINISTIC = 1
GP_STEP_DETERMINISTIC = 1
GP_STEP_NO_TV = 2
GP_STEP_LOSS_ONLY = 4
GP_SAMPLE_SPATIAL = 1
GP_QUERY_DIRECT = 0
GP_QUERY_WINDOW = 1
GP_QUERY_WINDOW_STAGED = 2
GP_MULTI_DETERMINISTIC = 2
GP_LOSS_TOTAL, GP_LOSS_PULL, GP_LOSS_GRAD, GP_LOSS_SURF, GP_LOSS_TV, GP_LOSS_BV, GP_LOSS_T = range(7)

STATUS_NAMES = {0: "GP_OK", 1: "GP_ERR_ARG", 2: "GP_ERR_OOM", 3: "GP_ERR_CUDA", 4: "GP_ERR_TIMEOUT",
                5: "GP_ERR_STATE", 6: "GP_ERR_NUMERIC"}

# Every function the header declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_i32 = ctypes.c_int32
_f = ctypes.c_float


class GridDesc(ctypes.Structure):
    _fields_ = [("R", _i32), ("M1", _i32), ("M2", _i32), ("knn_k", _i32), ("nn_grid", _i32), ("flags", _u32)]


class BandInfo(ctypes.Structure):
    _fields_ = [("R", _i32), ("nb", _i32), ("n_bricks", _i64), ("n_active_bricks", _i64), ("V_stored", _i64),
                ("V_trainable", _i64), ("V_tv", _i64), ("n_pull_cells", _i64), ("n_occupied_cells", _i64),
                ("J", _i64), ("nn_grid", _i32), ("knn_k", _i32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class LossW(ctypes.Structure):
    _fields_ = [("alpha", _f), ("beta", _f), ("gamma", _f)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", _f), ("beta1", _f), ("beta2", _f), ("eps", _f)]


class MultiInfo(ctypes.Structure):
    _fields_ = [("n", _i32), ("flags", _u32), ("records_per_tile", _i32), ("blocks_per_sm_nn", _i32),
                ("blocks_per_sm_tv", _i32), ("blocks_per_sm_query", _i32), ("error_bits", _i32),
                ("reserved", _i32), ("total_B", _i64), ("V_total", _i64), ("step", _i64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


SIGNATURES = {
    "gp_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "gp_set_stream": (ctypes.c_int, [_vp, _vp]),
    "gp_destroy": (None, [_vp]),
    "gp_last_error": (ctypes.c_char_p, [_vp]),
    "gp_version": (ctypes.c_char_p, []),
    "gp_profile": (ctypes.c_int, [_vp, ctypes.c_int]),
    "gp_profile_read": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(_i64), _i32, ctypes.POINTER(_i32)]),
    "gp_launch_count": (_i64, [_vp]),
    "gp_build_band": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(GridDesc), ctypes.POINTER(_vp)]),
    "gp_band_destroy": (None, [_vp]),
    "gp_band_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(BandInfo)]),
    "gp_band_init_sphere": (ctypes.c_int, [_vp, _f, _f, _f, _f, _f, _u64]),
    "gp_band_set_values": (ctypes.c_int, [_vp, _vp]),
    "gp_band_export": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "gp_band_values": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "gp_band_sigma": (ctypes.c_int, [_vp, _vp]),
    "gp_band_reset_adam": (ctypes.c_int, [_vp]),
    "gp_band_check": (ctypes.c_int, [_vp]),
    "gp_sample": (ctypes.c_int, [_vp, _u64, _u32, _i64, _i64, _i64, _u32, _vp, _vp, _vp]),
    "gp_nn": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "gp_nn_work": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, ctypes.POINTER(_i64)]),
    "gp_step": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, ctypes.POINTER(LossW), _vp, _vp, _u32]),
    "gp_update": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(Adam), _i64]),
    "gp_step_update": (ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.POINTER(LossW), ctypes.POINTER(Adam), _i64, _vp,
                                      _u32]),
    "gp_band_set_query_tiles": (ctypes.c_int, [_vp, _i32, _i32]),
    "gp_band_set_query_form": (ctypes.c_int, [_vp, _i32]),
    "gp_band_query_shape": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "gp_band_autotune": (ctypes.c_int, [_vp, _vp, _i64, _vp, ctypes.POINTER(LossW), ctypes.POINTER(_i32),
                                        ctypes.POINTER(_i32)]),
    "gp_multi_create": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                       _u64, _u32, ctypes.POINTER(_vp)]),
    "gp_multi_step": (ctypes.c_int, [_vp, ctypes.POINTER(LossW), ctypes.POINTER(Adam), _f, _i64, _vp]),
    "gp_multi_autotune": (ctypes.c_int, [_vp, ctypes.POINTER(LossW)]),
    "gp_multi_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(MultiInfo)]),
    "gp_multi_set_step": (ctypes.c_int, [_vp, _i64]),
    "gp_multi_buffers": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "gp_multi_destroy": (None, [_vp]),
    "gp_step_dense_noalloc": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i64, ctypes.POINTER(LossW), _vp, _vp]),
    "gp_mesh_extract": (ctypes.c_int, [_vp, _f, _vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "gp_mesh_case_table": (ctypes.c_int, [_vp, _vp]),
    "gp_mesh_quadrature": (ctypes.c_int, [_vp, _vp, _i64, _i32, _vp, _vp, _vp]),
    "gp_eval_nearest": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_double), _i32,
                                       ctypes.POINTER(ctypes.c_double)]),
}


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libgridpull.so (built by ``build.build()``) and declare its ABI."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libgridpull.so not built ({_LIB_PATH}); run paper_2308_13175_gb300.build.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class GridPullError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, numel=None, name="tensor"):
    import torch
    if t is None:
        return
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements, has {t.numel()}")


class Context:
    """gp_ctx on one device, following torch's current stream at each call."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = load()
        self.device = device
        h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream(device).cuda_stream
        st = self.lib.gp_create(ctypes.byref(h), device, ctypes.c_void_p(s))
        if st != GP_OK:
            raise GridPullError(st, "gp_create failed")
        self.handle = h

    def sync_stream(self):
        import torch
        self.lib.gp_set_stream(self.handle, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def check(self, st: int):
        if st != GP_OK:
            raise GridPullError(st, self.lib.gp_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Band:
    """A gp_band: grid, brick table, values, Adam moments and point cell list."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle
        info = BandInfo()
        ctx.check(ctx.lib.gp_band_get_info(handle, ctypes.byref(info)))
        self.info = info.as_dict()

    @property
    def V_stored(self) -> int:
        return self.info["V_stored"]

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.gp_band_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ the C ABI
def gp_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def gp_profile(ctx: Context, enable: bool):
    ctx.check(ctx.lib.gp_profile(ctx.handle, 1 if enable else 0))


def gp_profile_read(ctx: Context, max_kernels: int = 64):
    """{kernel name: (launches, total_ms)} of the launches recorded since the
    last read (synchronises the stream)."""
    names = ctypes.create_string_buffer(32 * max_kernels)
    ms = (ctypes.c_double * max_kernels)()
    cnt = (_i64 * max_kernels)()
    n = _i32()
    ctx.sync_stream()
    ctx.check(ctx.lib.gp_profile_read(ctx.handle, names, ms, cnt, max_kernels, ctypes.byref(n)))
    out = {}
    for k in range(min(n.value, max_kernels)):
        name = names.raw[32 * k:32 * (k + 1)].split(b"\0", 1)[0].decode()
        out[name] = (int(cnt[k]), float(ms[k]))
    return out


def gp_launch_count(ctx: Context) -> int:
    return int(ctx.lib.gp_launch_count(ctx.handle))


def gp_build_band(ctx: Context, points, R: int, M1: int, M2: int, knn_k: int = 50, nn_grid: int = 0,
                  deterministic: bool = False) -> Band:
    import torch
    _need(points, torch.float32, name="points")
    if points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must be (J, 3)")
    ctx.sync_stream()
    desc = GridDesc(R, M1, M2, knn_k, nn_grid, GP_BAND_DETERMINISTIC if deterministic else 0)
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.gp_build_band(ctx.handle, _ptr(points), points.shape[0], ctypes.byref(desc), ctypes.byref(h)))
    return Band(ctx, h)


def gp_band_init_sphere(band: Band, center, radius: float, noise_std: float = 0.0, seed: int = 0):
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_band_init_sphere(band.handle, float(center[0]), float(center[1]),
                                                    float(center[2]), float(radius), float(noise_std), int(seed)))


def gp_band_set_values(band: Band, d):
    import torch
    _need(d, torch.float32, band.V_stored, "values")
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_band_set_values(band.handle, _ptr(d)))


def gp_band_export(band: Band):
    """Returns (ijk int32 (V,3), values float32 (V,), flags uint8 (V,)) on the device."""
    import torch
    V = band.V_stored
    dev = torch.device("cuda", band.ctx.device)
    ijk = torch.empty((V, 3), dtype=torch.int32, device=dev)
    d = torch.empty(V, dtype=torch.float32, device=dev)
    fl = torch.empty(V, dtype=torch.uint8, device=dev)
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_band_export(band.handle, _ptr(ijk), _ptr(d), _ptr(fl)))
    return ijk, d, fl


def gp_band_values(band: Band):
    """Zero-copy (D, m, v) views of the band's own buffers as torch tensors."""
    import torch
    pd, pm, pv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    band.ctx.check(band.ctx.lib.gp_band_values(band.handle, ctypes.byref(pd), ctypes.byref(pm), ctypes.byref(pv)))
    return tuple(_wrap_device(p.value, band.V_stored, band) for p in (pd, pm, pv))


def _wrap_device(addr: int, n: int, owner, typestr: str = "<f4"):
    import torch

    class _CAI:
        def __init__(self):
            self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (addr, False), "version": 3,
                                             "strides": None}
    t = torch.as_tensor(_CAI(), device=torch.device("cuda", owner.ctx.device))
    return t


def gp_band_sigma(band: Band):
    import torch
    out = torch.empty(band.info["J"], dtype=torch.float32, device=torch.device("cuda", band.ctx.device))
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_band_sigma(band.handle, _ptr(out)))
    return out


def gp_band_reset_adam(band: Band):
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_band_reset_adam(band.handle))


def gp_band_check(band: Band):
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_band_check(band.handle))


def gp_sample(band: Band, seed: int, epoch: int, Q: int, first: int, count: int, out=None, src_out=None,
              pos_out=None, spatial: bool = False):
    import torch
    if out is None:
        out = torch.empty((count, 3), dtype=torch.float32, device=torch.device("cuda", band.ctx.device))
    _need(out, torch.float32, 3 * count, "q")
    _need(src_out, torch.int32, count, "src")
    _need(pos_out, torch.int32, count, "pos")
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_sample(band.handle, int(seed), int(epoch), int(Q), int(first), int(count),
                                          GP_SAMPLE_SPATIAL if spatial else 0, _ptr(out), _ptr(src_out),
                                          _ptr(pos_out)))
    return out


def gp_mesh_case_table():
    """The library's marching-cubes case table (host only): (ntri uint8 (256,),
    edges uint8 (256, 15), 255 past each case's last triangle)."""
    import numpy as np
    lib = load()
    ntri = np.zeros(256, dtype=np.uint8)
    edges = np.zeros((256, 15), dtype=np.uint8)
    st = lib.gp_mesh_case_table(ntri.ctypes.data_as(ctypes.c_void_p), edges.ctypes.data_as(ctypes.c_void_p))
    if st != GP_OK:
        raise GridPullError(st, "gp_mesh_case_table")
    return ntri, edges


def gp_mesh_extract(band: Band, iso: float = 0.0, with_cells: bool = True):
    """Marching-cubes triangle soup of the band's optimised cells at level iso.

    Returns (tri float32 (T, 3, 3), cells int64 (T,) or None) on the device: one
    sizing call (cap = 0), then the extracting call."""
    import torch
    n = ctypes.c_int64(0)
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_mesh_extract(band.handle, float(iso), None, None, 0, ctypes.byref(n)))
    dev = torch.device("cuda", band.ctx.device)
    T = int(n.value)
    tri = torch.empty((T, 3, 3), dtype=torch.float32, device=dev)
    cells = torch.empty(T, dtype=torch.int64, device=dev) if with_cells else None
    if T:
        band.ctx.check(band.ctx.lib.gp_mesh_extract(band.handle, float(iso), _ptr(tri), _ptr(cells), T,
                                                    ctypes.byref(n)))
        if int(n.value) != T:
            raise GridPullError(5, f"gp_mesh_extract: {n.value} triangles on the second pass, {T} on the first")
    return tri, cells


def gp_mesh_quadrature(ctx: Context, tri, m: int = 4):
    """(points (T m^2, 3), unit normals (T m^2, 3), weights (T m^2,)) float32 on
    the device: the centroids of the m^2 sub-triangles of every triangle."""
    import torch
    _need(tri, torch.float32, name="triangles")
    T = tri.numel() // 9
    n = T * int(m) * int(m)
    dev = torch.device("cuda", ctx.device)
    pts = torch.empty((n, 3), dtype=torch.float32, device=dev)
    nrm = torch.empty((n, 3), dtype=torch.float32, device=dev)
    w = torch.empty(n, dtype=torch.float32, device=dev)
    ctx.sync_stream()
    ctx.check(ctx.lib.gp_mesh_quadrature(ctx.handle, _ptr(tri), T, int(m), _ptr(pts), _ptr(nrm), _ptr(w)))
    return pts, nrm, w


def gp_eval_nearest(band: Band, q, q_nrm=None, q_w=None, target_nrm=None, taus=()):
    """One direction of the metrics (see the header): a dict with W, mean_d,
    mean_d2, max_d, mean_cos and below (one fraction per tau)."""
    import torch
    _need(q, torch.float32, name="q")
    n = q.numel() // 3
    _need(q_nrm, torch.float32, 3 * n, "q normals")
    _need(q_w, torch.float32, n, "q weights")
    _need(target_nrm, torch.float32, 3 * band.info["J"], "target normals")
    k = len(taus)
    tau = (ctypes.c_double * max(k, 1))(*[float(t) for t in taus])
    out = (ctypes.c_double * (5 + k))()
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_eval_nearest(band.handle, _ptr(q), _ptr(q_nrm), _ptr(q_w), n, _ptr(target_nrm),
                                                tau, k, out))
    v = list(out)
    return {"W": v[0], "mean_d": v[1], "mean_d2": v[2], "max_d": v[3], "mean_cos": v[4], "below": v[5:5 + k]}


def gp_nn(band: Band, q, nn_out=None, rec_out=None, hint=None, nvalid_out=None):
    import torch
    _need(q, torch.float32, name="q")
    n = q.numel() // 3
    _need(nn_out, torch.int32, n, "nn")
    _need(rec_out, torch.float32, 6 * n, "records")
    _need(hint, torch.int32, n, "hint")
    _need(nvalid_out, torch.int32, 1, "nvalid")
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_nn(band.handle, _ptr(q), n, _ptr(hint), _ptr(nn_out), _ptr(rec_out),
                                      _ptr(nvalid_out)))
    return nn_out, rec_out


def gp_nn_work(band: Band, q, nn_out, hint=None) -> int:
    """gp_nn's search with a count of the point distances it evaluates."""
    import torch
    _need(q, torch.float32, name="q")
    n = q.numel() // 3
    _need(nn_out, torch.int32, n, "nn")
    _need(hint, torch.int32, n, "hint")
    band.ctx.sync_stream()
    work = _i64(0)
    band.ctx.check(band.ctx.lib.gp_nn_work(band.handle, _ptr(q), n, _ptr(hint), _ptr(nn_out), ctypes.byref(work)))
    return int(work.value)


def gp_step(band: Band, rec, B: int, grad, loss, weights=(1.0, 1.0, 0.005), nvalid=None, d=None, flags: int = 0):
    import torch
    _need(rec, torch.float32, 6 * B, "records")
    _need(grad, torch.float32, band.V_stored, "grad")
    _need(loss, torch.float32, 8, "loss")
    _need(nvalid, torch.int32, 1, "nvalid")
    _need(d, torch.float32, band.V_stored, "values")
    w = LossW(*[float(x) for x in weights])
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_step(band.handle, _ptr(rec), int(B), _ptr(nvalid), _ptr(d), ctypes.byref(w),
                                        _ptr(grad), _ptr(loss), int(flags)))


def gp_band_autotune(band: Band, rec, B: int, weights=(1.0, 1.0, 0.005), nvalid=None) -> dict:
    """Times the fused step kernel's launch shapes and forms on these records
    and keeps the fastest in the band; returns {"records_per_thread",
    "blocks_per_sm", "form"} (form: GP_QUERY_*)."""
    import torch
    _need(rec, torch.float32, 6 * B, "records")
    _need(nvalid, torch.int32, 1, "nvalid")
    w = LossW(*[float(x) for x in weights])
    rpt, bps = _i32(0), _i32(0)
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_band_autotune(band.handle, _ptr(rec), int(B), _ptr(nvalid), ctypes.byref(w),
                                                 ctypes.byref(rpt), ctypes.byref(bps)))
    return gp_band_query_shape(band)


def gp_step_update(band: Band, rec, B: int, loss, lr: float, step: int, weights=(1.0, 1.0, 0.005), nvalid=None,
                   flags: int = 0, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """gp_step then gp_update in one call without a gradient array; the band's
    value buffer alternates (gp_band_values gives the current one)."""
    import torch
    _need(rec, torch.float32, 6 * B, "records")
    _need(loss, torch.float32, 8, "loss")
    _need(nvalid, torch.int32, 1, "nvalid")
    w = LossW(*[float(x) for x in weights])
    hp = Adam(float(lr), float(beta1), float(beta2), float(eps))
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_step_update(band.handle, _ptr(rec), int(B), _ptr(nvalid), ctypes.byref(w),
                                               ctypes.byref(hp), int(step), _ptr(loss), int(flags)))


def gp_band_set_query_tiles(band: Band, records_per_thread: int, blocks_per_sm: int):
    band.ctx.check(band.ctx.lib.gp_band_set_query_tiles(band.handle, int(records_per_thread), int(blocks_per_sm)))


def gp_band_set_query_form(band: Band, form: int):
    band.ctx.check(band.ctx.lib.gp_band_set_query_form(band.handle, int(form)))


def gp_band_query_shape(band: Band) -> dict:
    rpt, bps, form = _i32(0), _i32(0), _i32(0)
    band.ctx.check(band.ctx.lib.gp_band_query_shape(band.handle, ctypes.byref(rpt), ctypes.byref(bps),
                                                    ctypes.byref(form)))
    return {"records_per_thread": rpt.value, "blocks_per_sm": bps.value, "form": form.value}


def gp_update(band: Band, grad, lr: float, step: int, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    import torch
    _need(grad, torch.float32, band.V_stored, "grad")
    hp = Adam(float(lr), float(beta1), float(beta2), float(eps))
    band.ctx.sync_stream()
    band.ctx.check(band.ctx.lib.gp_update(band.handle, _ptr(grad), ctypes.byref(hp), int(step)))


def gp_step_dense_noalloc(ctx: Context, R: int, d, rec, B: int, grad, loss, weights=(1.0, 1.0, 0.005)):
    """Query terms and gradient on a caller-owned dense grid; allocates nothing
    (for callers that may not allocate device memory themselves)."""
    import torch
    n1 = R + 1
    _need(d, torch.float32, n1 ** 3, "values")
    _need(rec, torch.float32, 6 * B, "records")
    _need(grad, torch.float32, n1 ** 3, "grad")
    _need(loss, torch.float32, 8, "loss")
    w = LossW(*[float(x) for x in weights])
    ctx.sync_stream()
    ctx.check(ctx.lib.gp_step_dense_noalloc(ctx.handle, int(R), _ptr(d), _ptr(rec), int(B), ctypes.byref(w),
                                            _ptr(grad), _ptr(loss)))


# ----------------------------------------------------------- many clouds
class Multi:
    """A gp_multi: several bands stepped together, one launch per stage.  Holds
    references to its bands, which the C side needs alive."""

    def __init__(self, ctx: Context, handle, bands, Q, B):
        self.ctx = ctx
        self.handle = handle
        self.bands = list(bands)
        self.Q = [int(x) for x in Q]
        self.B = [int(x) for x in B]

    @property
    def n(self) -> int:
        return len(self.bands)

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.gp_multi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gp_multi_create(ctx: Context, bands, Q, B, seed: int = 0, spatial: bool = True,
                    deterministic: bool = False) -> Multi:
    n = len(bands)
    arr = (_vp * n)(*[b.handle for b in bands])
    qa = (_i64 * n)(*[int(x) for x in Q])
    ba = (_i64 * n)(*[int(x) for x in B])
    out = _vp()
    ctx.sync_stream()
    flags = (GP_SAMPLE_SPATIAL if spatial else 0) | (GP_MULTI_DETERMINISTIC if deterministic else 0)
    ctx.check(ctx.lib.gp_multi_create(ctx.handle, arr, n, qa, ba, int(seed), flags, ctypes.byref(out)))
    return Multi(ctx, out, bands, Q, B)


def gp_multi_step(m: Multi, loss, weights=(1.0, 1.0, 0.005), lr: float = 1e-3, beta1: float = 0.9,
                  beta2: float = 0.999, eps: float = 1e-8, lr_decay: float = 1.0, lr_every: int = 0):
    import torch
    _need(loss, torch.float32, 8 * m.n, "loss")
    w = LossW(*[float(x) for x in weights])
    hp = Adam(float(lr), float(beta1), float(beta2), float(eps))
    m.ctx.sync_stream()
    m.ctx.check(m.ctx.lib.gp_multi_step(m.handle, ctypes.byref(w), ctypes.byref(hp), float(lr_decay), int(lr_every),
                                        _ptr(loss)))


def gp_multi_autotune(m: Multi, weights=(1.0, 1.0, 0.005)):
    w = LossW(*[float(x) for x in weights])
    m.ctx.sync_stream()
    m.ctx.check(m.ctx.lib.gp_multi_autotune(m.handle, ctypes.byref(w)))
    return gp_multi_get_info(m)


def gp_multi_get_info(m: Multi) -> dict:
    info = MultiInfo()
    m.ctx.sync_stream()
    m.ctx.check(m.ctx.lib.gp_multi_get_info(m.handle, ctypes.byref(info)))
    return info.as_dict()


def gp_multi_set_step(m: Multi, step: int):
    m.ctx.sync_stream()
    m.ctx.check(m.ctx.lib.gp_multi_set_step(m.handle, int(step)))


def gp_multi_buffers(m: Multi, k: int):
    """Zero-copy views of cloud k's records (B_k, 6), sources (B_k,) and
    gradient (V_stored,) as the last step left them."""
    pr, ps, pg = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    m.ctx.check(m.ctx.lib.gp_multi_buffers(m.handle, int(k), ctypes.byref(pr), ctypes.byref(ps), ctypes.byref(pg)))
    Bk = m.B[k]
    rec = _wrap_device(pr.value, 6 * Bk, m).view(Bk, 6)
    src = _wrap_device(ps.value, Bk, m, "<i4")
    grad = _wrap_device(pg.value, m.bands[k].V_stored, m)
    return rec, src, grad
