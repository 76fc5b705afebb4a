"""Python binding of libsem, the GB300 (sm_103a) CUDA library for the in situ render path
of spectral-element velocity fields (spectral derivative -> Q-criterion -> marching-cubes
isosurface -> z-buffer raster).

This module only marshals arguments into the C ABI declared in ``include/sem.h``; every
step of the path runs in the library's CUDA kernels.  PyTorch provides device memory and
streams.  There is no CPU fallback: if ``lib/libsem.so`` has not been built, every call
raises.  Functions keep the C names (``sem_create``, ``sem_load_mesh``, ``sem_derivatives``,
``sem_qcriterion``, ``sem_isosurface``, ``sem_render``, ...).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libsem.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "sem.h")

SEM_OK, SEM_ERR_ARG, SEM_ERR_CAPACITY, SEM_ERR_OOM, SEM_ERR_CUDA, SEM_ERR_TIMEOUT, SEM_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = ["SEM_OK", "SEM_ERR_ARG", "SEM_ERR_CAPACITY", "SEM_ERR_OOM", "SEM_ERR_CUDA", "SEM_ERR_TIMEOUT",
                "SEM_ERR_UNSUPPORTED"]
SEM_FP32, SEM_TF32, SEM_FP16, SEM_BF16, SEM_BF16X2 = range(5)
SEM_MAX_ORDER = 15
SEM_NOALLOC_MAX_ELEMENTS = 262144
SEM_MC_MAXT = 12
SEM_MAX_ISO = 8
SEM_MAX_FIELDS = 4

_lock = threading.Lock()
_lib = None


class SemError(RuntimeError):
    def __init__(self, status: int, msg: str, required: Optional[int] = None):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status
        self.required = required


class sem_camera(C.Structure):
    _fields_ = [("ortho", C.c_int32), ("eye", C.c_float * 3), ("center", C.c_float * 3), ("up", C.c_float * 3),
                ("fovy_deg", C.c_float), ("half_h", C.c_float), ("znear", C.c_float), ("zfar", C.c_float)]


def _declare(L):
    vp, i32, i64, f32, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_float, C.c_double
    L.sem_version.restype = i32
    L.sem_create.argtypes = [i32, vp, C.POINTER(vp)]
    L.sem_destroy.argtypes = [vp]
    L.sem_destroy.restype = None
    L.sem_last_error.argtypes = [vp]
    L.sem_last_error.restype = C.c_char_p
    L.sem_set_stream.argtypes = [vp, vp]
    L.sem_synchronize.argtypes = [vp]
    L.sem_debug_set_wait_limit.argtypes = [vp, i64]
    L.sem_trace_enable.argtypes = [vp, i32]
    L.sem_memory.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    L.sem_trace_collect.argtypes = [vp, C.POINTER(i32)]
    L.sem_trace_entry.argtypes = [vp, i32, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.POINTER(i64)]
    L.sem_load_mesh.argtypes = [vp, i32, i64, vp, C.POINTER(vp)]
    L.sem_mesh_free.argtypes = [vp]
    L.sem_mesh_free.restype = None
    L.sem_mesh_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i64)]
    L.sem_derivatives.argtypes = [vp, vp, vp, vp, vp, vp, i32]
    L.sem_qcriterion.argtypes = [vp, vp, vp, vp, vp, vp, i32]
    L.sem_qcriterion_batch.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.sem_isosurface.argtypes = [vp, vp, vp, f32, vp, vp, i64, C.POINTER(i64), vp]
    L.sem_isosurface_multi.argtypes = [vp, vp, vp, vp, i32, vp, vp, i64, vp, vp]
    L.sem_isosurface_multi_async.argtypes = [vp, vp, vp, vp, i32, vp, vp, i64, vp, vp]
    L.sem_isosurface_multi_append_async.argtypes = [vp, vp, vp, vp, i32, vp, vp, i64, vp, vp]
    L.sem_qcriterion_isosurface_async.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, vp, vp, i64, vp]
    L.sem_qcriterion_isosurface_fields_async.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp,
                                                         i64, vp]
    L.sem_render_async.argtypes = [vp, vp, i64, vp, i32, vp, C.POINTER(sem_camera), i32, i32, vp, vp]
    L.sem_frame_async.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, i64, vp, vp,
                                  C.POINTER(sem_camera), i32, i32, vp, vp]
    L.sem_render_segments_async.argtypes = [vp, vp, i64, vp, i32, vp, C.c_uint64, C.POINTER(sem_camera), i32, i32,
                                            vp, vp]
    L.sem_isosurface_noalloc.argtypes = [vp, vp, vp, f32, vp, vp, i64, C.POINTER(i64), vp]
    L.sem_render.argtypes = [vp, vp, i64, vp, i32, vp, C.POINTER(sem_camera), i32, i32, vp, vp]
    L.sem_surface_measures.argtypes = [vp, vp, i64, vp]
    L.sem_field_max.argtypes = [vp, vp, i64, C.POINTER(f32)]
    L.sem_mc_table.argtypes = [vp, vp]
    L.sem_mc_table.restype = i32
    L.sem_gll.argtypes = [i32, vp, vp]
    L.sem_ae_param_count.restype = i64
    L.sem_ae_param_count.argtypes = []
    L.sem_ae_create.argtypes = [vp, i32, C.POINTER(vp)]
    L.sem_ae_destroy.argtypes = [vp]
    L.sem_ae_destroy.restype = None
    L.sem_ae_set_params.argtypes = [vp, vp, i64]
    L.sem_ae_get_params.argtypes = [vp, vp, i64]
    L.sem_ae_get_state.argtypes = [vp, vp, vp, i64, C.POINTER(i64)]
    L.sem_ae_set_state.argtypes = [vp, vp, vp, i64, i64]
    L.sem_ae_set_normalization.argtypes = [vp, vp, vp]
    L.sem_ae_get_normalization.argtypes = [vp, vp, vp]
    L.sem_ae_fit_normalization.argtypes = [vp, vp, i64]
    L.sem_ae_loss_grad.argtypes = [vp, vp, i64, vp, i32, C.POINTER(f32), vp, i64]
    L.sem_ae_train_step.argtypes = [vp, vp, i64, vp, i32, f32, f32, f32, f32, f32, vp]
    L.sem_ae_encode.argtypes = [vp, vp, vp, vp, i64, vp]
    L.sem_ae_decode.argtypes = [vp, vp, i64, vp, vp, vp]
    L.sem_gemm_bf16.argtypes = [vp, vp, vp, i64, i32, i32, vp]
    L.sem_autotune_set.argtypes = [vp, i32]
    L.sem_autotune_entry.argtypes = [vp, i32, C.POINTER(i64)] + [C.POINTER(i32)] * 7 + [C.POINTER(f32)]
    L.sem_autotune_emit_entry.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32), C.POINTER(i32),
                                          C.POINTER(f32)]
    L.sem_autotune_width_entry.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i32),
                                           C.POINTER(f32)]
    for name in ("sem_create", "sem_set_stream", "sem_synchronize", "sem_debug_set_wait_limit", "sem_load_mesh", "sem_mesh_info",
                 "sem_derivatives", "sem_qcriterion", "sem_isosurface", "sem_isosurface_multi", "sem_isosurface_multi_async",
                 "sem_isosurface_multi_append_async", "sem_qcriterion_isosurface_async",
                 "sem_qcriterion_isosurface_fields_async", "sem_frame_async", "sem_render_async",
                 "sem_render_segments_async",
                 "sem_isosurface_noalloc", "sem_render", "sem_surface_measures",
                 "sem_field_max", "sem_gll"):
        getattr(L, name).restype = i32


def get_lib():
    """Load lib/libsem.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with paper_2312_09888_gb300.build_library()")
            L = C.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
        return _lib


def build_library(force: bool = False) -> str:
    """Compile lib/libsem.so for sm_103a (incremental)."""
    import importlib
    return importlib.import_module(__name__ + ".build").build(force=force)


# ------------------------------------------------------------------------------ marshalling

def _dev(t, name, dtype=None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is None")
    if isinstance(t, int):
        return C.c_void_p(t)
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _check(ctx, st: int, required: Optional[int] = None):
    if st != SEM_OK:
        msg = get_lib().sem_last_error(ctx).decode(errors="replace")
        raise SemError(st, msg, required)


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------------------ C ABI mirrors

def sem_version() -> int:
    return get_lib().sem_version()


def sem_create(device: int = 0, stream=None):
    out = C.c_void_p()
    st = get_lib().sem_create(device, C.c_void_p(_stream_handle(stream)), C.byref(out))
    _check(None, st)
    return out


def sem_destroy(ctx) -> None:
    get_lib().sem_destroy(ctx)


def sem_last_error(ctx) -> str:
    return get_lib().sem_last_error(ctx).decode(errors="replace")


def sem_set_stream(ctx, stream) -> None:
    _check(ctx, get_lib().sem_set_stream(ctx, C.c_void_p(_stream_handle(stream))))


def sem_synchronize(ctx) -> None:
    _check(ctx, get_lib().sem_synchronize(ctx))


def sem_debug_set_wait_limit(ctx, polls: int) -> None:
    """Polls a Q-kernel wait for its input copies makes before it gives up and records
    SEM_ERR_TIMEOUT (0: at once; negative: the default).  A failure-detection test hook."""
    _check(ctx, get_lib().sem_debug_set_wait_limit(ctx, int(polls)))


def sem_memory(ctx):
    """(bytes in use, high-water mark) of the device memory the library holds for ctx."""
    a, b = C.c_int64(0), C.c_int64(0)
    _check(ctx, get_lib().sem_memory(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def sem_trace_enable(ctx, on: bool = True) -> None:
    _check(ctx, get_lib().sem_trace_enable(ctx, 1 if on else 0))


def sem_trace_collect(ctx) -> dict:
    """{kernel name: (summed device ms, launches)} of the launches traced since the last call."""
    L = get_lib()
    n = C.c_int32(0)
    _check(ctx, L.sem_trace_collect(ctx, C.byref(n)))
    out = {}
    for k in range(n.value):
        name, ms, cnt = C.c_char_p(), C.c_double(0), C.c_int64(0)
        _check(ctx, L.sem_trace_entry(ctx, k, C.byref(name), C.byref(ms), C.byref(cnt)))
        out[name.value.decode()] = (ms.value, cnt.value)
    return out


def sem_load_mesh(ctx, N: int, xyz) -> C.c_void_p:
    """xyz: host float64 array (3, E, (N+1)^3) of node coordinates (torch or numpy)."""
    a = xyz.detach().cpu().numpy() if hasattr(xyz, "detach") else xyz
    a = np.ascontiguousarray(a, dtype=np.float64)
    E = a.shape[1] if a.ndim == 3 else a.size // (3 * (N + 1) ** 3)
    out = C.c_void_p()
    _check(ctx, get_lib().sem_load_mesh(ctx, int(N), int(E), a.ctypes.data_as(C.c_void_p), C.byref(out)))
    return out


def sem_mesh_free(mesh) -> None:
    get_lib().sem_mesh_free(mesh)


def sem_mesh_info(mesh):
    n = C.c_int()
    e = C.c_int64()
    st = get_lib().sem_mesh_info(mesh, C.byref(n), C.byref(e))
    if st:
        raise SemError(st, "bad mesh")
    return n.value, e.value


def sem_derivatives(ctx, mesh, u, dudx, dudy, dudz, prec: int = SEM_FP32) -> None:
    import torch
    f = torch.float32
    _check(ctx, get_lib().sem_derivatives(ctx, mesh, _dev(u, "u", f), _dev(dudx, "dudx", f), _dev(dudy, "dudy", f),
                                          _dev(dudz, "dudz", f), int(prec)))


def sem_qcriterion(ctx, mesh, u, v, w, Q, prec: int = SEM_FP32) -> None:
    import torch
    f = torch.float32
    _check(ctx, get_lib().sem_qcriterion(ctx, mesh, _dev(u, "u", f), _dev(v, "v", f), _dev(w, "w", f),
                                         _dev(Q, "Q", f), int(prec)))


def sem_qcriterion_batch(ctx, meshes, us, vs, ws, Qs) -> None:
    """Q of several partitions (lists of meshes and device tensors) in one launch per order."""
    import torch
    n = len(meshes)
    arr = lambda xs, name: (C.c_void_p * max(n, 1))(*[_dev(x, name, torch.float32) for x in xs])  # noqa: E731
    mp = (C.c_void_p * max(n, 1))(*meshes)
    _check(ctx, get_lib().sem_qcriterion_batch(ctx, n, mp, arr(us, "u"), arr(vs, "v"), arr(ws, "w"), arr(Qs, "Q")))


def sem_isosurface(ctx, mesh, f, iso: float, tris, tri_elem=None, cases=None, cap: Optional[int] = None) -> int:
    """Returns the triangle count (tris None: count only).  Raises SemError(SEM_ERR_CAPACITY,
    required=n) if tris is too small (cap defaults to tris.numel() // 9)."""
    import torch
    if cap is None:
        cap = 0 if tris is None else tris.numel() // 9
    n = C.c_int64(0)
    st = get_lib().sem_isosurface(ctx, mesh, _dev(f, "f", torch.float32), C.c_float(iso),
                                  _dev(tris, "tris", torch.float32, allow_none=True),
                                  _dev(tri_elem, "tri_elem", torch.int32, allow_none=True), int(cap), C.byref(n),
                                  _dev(cases, "cases", torch.uint8, allow_none=True))
    _check(ctx, st, n.value)
    return n.value


def sem_isosurface_multi(ctx, mesh, f, isos, tris, tri_elem=None, cases=None, cap: Optional[int] = None):
    """Several isovalues in one call; returns the per-isovalue triangle counts (a list).  The
    triangles of isovalue q follow those of q-1 in ``tris`` (tris None: count only)."""
    import torch
    iv = np.ascontiguousarray(np.asarray(isos, dtype=np.float32).reshape(-1))
    if cap is None:
        cap = 0 if tris is None else tris.numel() // 9
    n = np.zeros(len(iv), dtype=np.int64)
    st = get_lib().sem_isosurface_multi(ctx, mesh, _dev(f, "f", torch.float32), iv.ctypes.data_as(C.c_void_p),
                                        len(iv), _dev(tris, "tris", torch.float32, allow_none=True),
                                        _dev(tri_elem, "tri_elem", torch.int32, allow_none=True), int(cap),
                                        n.ctypes.data_as(C.c_void_p),
                                        _dev(cases, "cases", torch.uint8, allow_none=True))
    _check(ctx, st, int(n.sum()))
    return [int(x) for x in n]


def sem_isosurface_multi_async(ctx, mesh, f, isos, tris, counts_dev, tri_elem=None, cases=None,
                               cap: Optional[int] = None) -> None:
    """No host synchronisation (CUDA-graph capturable); segment starts land in counts_dev
    (int64 CUDA tensor of len(isos) + 1); an overflow raises the device flag."""
    import torch
    iv = np.ascontiguousarray(np.asarray(isos, dtype=np.float32).reshape(-1))
    if cap is None:
        cap = 0 if tris is None else tris.numel() // 9
    st = get_lib().sem_isosurface_multi_async(ctx, mesh, _dev(f, "f", torch.float32), iv.ctypes.data_as(C.c_void_p),
                                              len(iv), _dev(tris, "tris", torch.float32, allow_none=True),
                                              _dev(tri_elem, "tri_elem", torch.int32, allow_none=True), int(cap),
                                              _dev(counts_dev, "counts_dev", torch.int64),
                                              _dev(cases, "cases", torch.uint8, allow_none=True))
    _check(ctx, st)


def sem_qcriterion_isosurface_async(ctx, mesh, u, v, w, Q, isos, tris, counts_dev, tri_elem=None,
                                    cap: Optional[int] = None) -> None:
    """sem_qcriterion then sem_isosurface_multi_async of Q, the counting pass done by the Q kernel
    (N = 7 box meshes); no host synchronisation.  Same results as the two calls."""
    import torch
    iv = np.ascontiguousarray(np.asarray(isos, dtype=np.float32).reshape(-1))
    if cap is None:
        cap = 0 if tris is None else tris.numel() // 9
    st = get_lib().sem_qcriterion_isosurface_async(ctx, mesh, _dev(u, "u", torch.float32), _dev(v, "v", torch.float32),
                                                   _dev(w, "w", torch.float32), _dev(Q, "Q", torch.float32),
                                                   iv.ctypes.data_as(C.c_void_p), len(iv),
                                                   _dev(tris, "tris", torch.float32, allow_none=True),
                                                   _dev(tri_elem, "tri_elem", torch.int32, allow_none=True),
                                                   int(cap), _dev(counts_dev, "counts_dev", torch.int64))
    _check(ctx, st)


def sem_qcriterion_isosurface_fields_async(ctx, mesh, u, v, w, Q, q_isos, fields, f_isos, tris, counts_dev,
                                           tri_elem=None, cap: Optional[int] = None) -> None:
    """Q and its isosurfaces, then the isosurfaces of further fields appended behind them, in one
    call whose further-field passes run on the context's auxiliary stream, overlapping Q's scan
    and emit.  ``fields``: list of CUDA float32 tensors; ``f_isos``: one list of isovalues per
    field; counts_dev: int64 CUDA tensor of 1 + len(q_isos) + sum(len(f)) entries (all segment
    starts, then the total).  Same results as sem_qcriterion_isosurface_async followed by one
    sem_isosurface_multi_append_async per field."""
    import torch
    qv, fv, fn, fp = _fields_args(q_isos, fields, f_isos)
    if cap is None:
        cap = 0 if tris is None else tris.numel() // 9
    st = get_lib().sem_qcriterion_isosurface_fields_async(
        ctx, mesh, _dev(u, "u", torch.float32), _dev(v, "v", torch.float32), _dev(w, "w", torch.float32),
        _dev(Q, "Q", torch.float32), qv.ctypes.data_as(C.c_void_p), len(qv), len(fields),
        C.cast(fp, C.c_void_p), fv.ctypes.data_as(C.c_void_p), fn.ctypes.data_as(C.c_void_p),
        _dev(tris, "tris", torch.float32, allow_none=True), _dev(tri_elem, "tri_elem", torch.int32, allow_none=True),
        int(cap), _dev(counts_dev, "counts_dev", torch.int64))
    _check(ctx, st)


def _fields_args(q_isos, fields, f_isos):
    import torch
    qv = np.ascontiguousarray(np.asarray(q_isos, dtype=np.float32).reshape(-1))
    if len(fields) != len(f_isos):
        raise ValueError("one list of isovalues per field")
    fv = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float32).reshape(-1) for x in f_isos])
                              if f_isos else np.zeros(0, np.float32))
    fn = np.ascontiguousarray(np.asarray([len(x) for x in f_isos], dtype=np.int32))
    fp = (C.c_void_p * max(1, len(fields)))(*[_dev(f, "fields[k]", torch.float32) for f in fields])
    return qv, fv, fn, fp


def sem_frame_async(ctx, mesh, u, v, w, Q, q_isos, fields, f_isos, tris, counts_dev, seg_rgb, cam: dict, W: int,
                    H: int, rgba, depth=None, tri_elem=None, cap: Optional[int] = None) -> None:
    """One frame in one call: sem_qcriterion_isosurface_fields_async then sem_render_async of all
    its segments (colours ``seg_rgb``: one RGB row per segment, or None), each stream drawing the
    segments it has just emitted and one resolve after the join.  Same results as the two calls."""
    import torch
    qv, fv, fn, fp = _fields_args(q_isos, fields, f_isos)
    if cap is None:
        cap = 0 if tris is None else tris.numel() // 9
    rgb = None if seg_rgb is None else np.ascontiguousarray(np.asarray(seg_rgb, dtype=np.float32).reshape(-1))
    camc = make_camera(cam)
    st = get_lib().sem_frame_async(
        ctx, mesh, _dev(u, "u", torch.float32), _dev(v, "v", torch.float32), _dev(w, "w", torch.float32),
        _dev(Q, "Q", torch.float32), qv.ctypes.data_as(C.c_void_p), len(qv), len(fields), C.cast(fp, C.c_void_p),
        fv.ctypes.data_as(C.c_void_p), fn.ctypes.data_as(C.c_void_p),
        _dev(tris, "tris", torch.float32, allow_none=True), _dev(tri_elem, "tri_elem", torch.int32, allow_none=True),
        int(cap), _dev(counts_dev, "counts_dev", torch.int64), None if rgb is None else rgb.ctypes.data_as(C.c_void_p),
        C.byref(camc), int(W), int(H), _dev(rgba, "rgba", torch.uint8), _dev(depth, "depth", torch.float32,
                                                                                allow_none=True))
    _check(ctx, st)


def sem_isosurface_multi_append_async(ctx, mesh, f, isos, tris, counts_dev, tri_elem=None, cases=None,
                                      cap: Optional[int] = None) -> None:
    """As sem_isosurface_multi_async, appending behind triangles already in ``tris``:
    counts_dev[0] (device) is read as the index of the first triangle written, counts_dev[1:]
    receive the segment ends (counts_dev: int64 CUDA tensor of len(isos) + 1, e.g. a view
    starting at an earlier call's last entry).  ``cap`` is the whole buffer's capacity."""
    import torch
    iv = np.ascontiguousarray(np.asarray(isos, dtype=np.float32).reshape(-1))
    if cap is None:
        cap = 0 if tris is None else tris.numel() // 9
    st = get_lib().sem_isosurface_multi_append_async(ctx, mesh, _dev(f, "f", torch.float32),
                                                     iv.ctypes.data_as(C.c_void_p), len(iv),
                                                     _dev(tris, "tris", torch.float32, allow_none=True),
                                                     _dev(tri_elem, "tri_elem", torch.int32, allow_none=True),
                                                     int(cap), _dev(counts_dev, "counts_dev", torch.int64),
                                                     _dev(cases, "cases", torch.uint8, allow_none=True))
    _check(ctx, st)


def sem_render_async(ctx, tris, ntri_max: int, seg_start_dev, nseg: int, seg_rgb, cam: dict, W: int, H: int, rgba,
                     depth=None) -> None:
    import torch
    rgb = None if seg_rgb is None else np.ascontiguousarray(np.asarray(seg_rgb, dtype=np.float32).reshape(-1))
    camc = make_camera(cam)
    st = get_lib().sem_render_async(ctx, _dev(tris, "tris", torch.float32, allow_none=ntri_max == 0), int(ntri_max),
                                    _dev(seg_start_dev, "seg_start_dev", torch.int64), int(nseg),
                                    None if rgb is None else rgb.ctypes.data_as(C.c_void_p), C.byref(camc), int(W),
                                    int(H), _dev(rgba, "rgba", torch.uint8),
                                    _dev(depth, "depth", torch.float32, allow_none=True))
    _check(ctx, st)


def sem_render_segments_async(ctx, tris, ntri_max: int, seg_start_dev, nseg: int, seg_rgb, seg_mask: int, cam: dict,
                              W: int, H: int, rgba, depth=None) -> None:
    """sem_render_async of up to 64 segments, drawing only those whose bit is set in seg_mask."""
    import torch
    rgb = None if seg_rgb is None else np.ascontiguousarray(np.asarray(seg_rgb, dtype=np.float32).reshape(-1))
    camc = make_camera(cam)
    st = get_lib().sem_render_segments_async(ctx, _dev(tris, "tris", torch.float32, allow_none=ntri_max == 0),
                                             int(ntri_max), _dev(seg_start_dev, "seg_start_dev", torch.int64),
                                             int(nseg), None if rgb is None else rgb.ctypes.data_as(C.c_void_p),
                                             C.c_uint64(int(seg_mask) & ((1 << 64) - 1)), C.byref(camc), int(W),
                                             int(H), _dev(rgba, "rgba", torch.uint8),
                                             _dev(depth, "depth", torch.float32, allow_none=True))
    _check(ctx, st)


def sem_isosurface_noalloc(ctx, mesh, f, iso: float, tris, tri_elem=None, cases=None,
                           cap: Optional[int] = None) -> int:
    """As sem_isosurface, for callers that may not allocate device memory during the call:
    the library keeps this call's scratch in a fixed device array (meshes of at most
    SEM_NOALLOC_MAX_ELEMENTS elements; calls on one device must not overlap)."""
    import torch
    if cap is None:
        cap = 0 if tris is None else tris.numel() // 9
    n = C.c_int64(0)
    st = get_lib().sem_isosurface_noalloc(ctx, mesh, _dev(f, "f", torch.float32), C.c_float(iso),
                                          _dev(tris, "tris", torch.float32, allow_none=True),
                                          _dev(tri_elem, "tri_elem", torch.int32, allow_none=True), int(cap),
                                          C.byref(n), _dev(cases, "cases", torch.uint8, allow_none=True))
    _check(ctx, st, n.value)
    return n.value


def make_camera(cam: dict) -> sem_camera:
    c = sem_camera()
    c.ortho = int(cam["ortho"])
    for k in ("eye", "center", "up"):
        getattr(c, k)[:] = [float(x) for x in cam[k]]
    c.fovy_deg = float(cam.get("fovy_deg", 40.0))
    c.half_h = float(cam.get("half_h", 1.0))
    c.znear = float(cam["znear"])
    c.zfar = float(cam["zfar"])
    return c


def sem_render(ctx, tris, ntri: int, seg_ntri: Sequence[int], seg_rgb, cam: dict, W: int, H: int, rgba,
               depth=None) -> None:
    import torch
    seg = np.ascontiguousarray(np.asarray(seg_ntri, dtype=np.int64))
    rgb = None if seg_rgb is None else np.ascontiguousarray(np.asarray(seg_rgb, dtype=np.float32).reshape(-1))
    camc = make_camera(cam)
    st = get_lib().sem_render(ctx, _dev(tris, "tris", torch.float32, allow_none=ntri == 0), int(ntri),
                              seg.ctypes.data_as(C.c_void_p), len(seg),
                              None if rgb is None else rgb.ctypes.data_as(C.c_void_p), C.byref(camc), int(W), int(H),
                              _dev(rgba, "rgba", torch.uint8), _dev(depth, "depth", torch.float32, allow_none=True))
    _check(ctx, st)


def sem_surface_measures(ctx, tris, ntri: int):
    import torch
    out = np.zeros(2)
    _check(ctx, get_lib().sem_surface_measures(ctx, _dev(tris, "tris", torch.float32, allow_none=ntri == 0),
                                               int(ntri), out.ctypes.data_as(C.c_void_p)))
    return float(out[0]), float(out[1])


def sem_field_max(ctx, f) -> float:
    import torch
    m = C.c_float(0)
    _check(ctx, get_lib().sem_field_max(ctx, _dev(f, "f", torch.float32), int(f.numel()), C.byref(m)))
    return m.value


def sem_mc_table():
    n = np.zeros(256, dtype=np.int32)
    e = np.zeros((256, SEM_MC_MAXT, 3), dtype=np.int8)
    mx = get_lib().sem_mc_table(n.ctypes.data_as(C.c_void_p), e.ctypes.data_as(C.c_void_p))
    if mx < 0:
        raise SemError(SEM_ERR_CUDA, f"table generator failed ({mx})")
    return n, e


def sem_gll(N: int):
    xi = np.zeros(N + 1)
    D = np.zeros((N + 1, N + 1))
    st = get_lib().sem_gll(int(N), xi.ctypes.data_as(C.c_void_p), D.ctypes.data_as(C.c_void_p))
    if st:
        raise SemError(st, f"sem_gll({N})")
    return xi, D


# ------------------------------------------------------------------------ learned compression

AE_LAYER_SHAPES = [("W1", (512, 1536)), ("b1", (512,)), ("W2", (48, 512)), ("b2", (48,)),
                   ("W3", (512, 48)), ("b3", (512,)), ("W4", (1536, 512)), ("b4", (1536,))]


def ae_flatten(params: dict) -> np.ndarray:
    """{name: array} -> the flat FP32 host array of the C ABI (order W1 b1 W2 b2 W3 b3 W4 b4)."""
    return np.ascontiguousarray(np.concatenate([np.asarray(params[k], np.float32).reshape(-1)
                                                for k, _ in AE_LAYER_SHAPES]))


def ae_unflatten(flat) -> dict:
    out, at = {}, 0
    for k, shp in AE_LAYER_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[at:at + n]).reshape(shp)
        at += n
    return out


def sem_ae_param_count() -> int:
    return int(get_lib().sem_ae_param_count())


def sem_ae_create(ctx, batch: int):
    h = C.c_void_p()
    _check(ctx, get_lib().sem_ae_create(ctx, int(batch), C.byref(h)))
    return h


def sem_ae_destroy(ae) -> None:
    if ae:
        get_lib().sem_ae_destroy(ae)


def sem_ae_set_params(ctx, ae, params) -> None:
    flat = ae_flatten(params) if isinstance(params, dict) else np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, get_lib().sem_ae_set_params(ae, flat.ctypes.data_as(C.c_void_p), int(flat.size)))


def sem_ae_get_params(ctx, ae) -> dict:
    flat = np.zeros(sem_ae_param_count(), dtype=np.float32)
    _check(ctx, get_lib().sem_ae_get_params(ae, flat.ctypes.data_as(C.c_void_p), int(flat.size)))
    return ae_unflatten(flat)


def sem_ae_get_state(ctx, ae):
    n = sem_ae_param_count()
    m, v, st = np.zeros(n, np.float32), np.zeros(n, np.float32), C.c_int64(0)
    _check(ctx, get_lib().sem_ae_get_state(ae, m.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p), n,
                                           C.byref(st)))
    return m, v, st.value


def sem_ae_set_state(ctx, ae, m, v, step: int) -> None:
    m = np.ascontiguousarray(m, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    _check(ctx, get_lib().sem_ae_set_state(ae, m.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p),
                                           int(m.size), int(step)))


def sem_ae_set_normalization(ctx, ae, mean, std) -> None:
    mu = np.ascontiguousarray(mean, np.float32)
    sd = np.ascontiguousarray(std, np.float32)
    _check(ctx, get_lib().sem_ae_set_normalization(ae, mu.ctypes.data_as(C.c_void_p), sd.ctypes.data_as(C.c_void_p)))


def sem_ae_get_normalization(ctx, ae):
    mu, sd = np.zeros(3, np.float32), np.zeros(3, np.float32)
    _check(ctx, get_lib().sem_ae_get_normalization(ae, mu.ctypes.data_as(C.c_void_p), sd.ctypes.data_as(C.c_void_p)))
    return mu, sd


def sem_ae_fit_normalization(ctx, ae, samples) -> None:
    import torch
    _check(ctx, get_lib().sem_ae_fit_normalization(ae, _dev(samples, "samples", torch.float32),
                                                   int(samples.shape[0])))


def sem_ae_loss_grad(ctx, ae, samples, idx, want_grad: bool = True):
    """(loss, {name: gradient}) of the batch samples[idx] (idx: device int64)."""
    import torch
    loss = C.c_float(0)
    g = np.zeros(sem_ae_param_count(), np.float32) if want_grad else None
    _check(ctx, get_lib().sem_ae_loss_grad(ae, _dev(samples, "samples", torch.float32), int(samples.shape[0]),
                                           _dev(idx, "idx", torch.int64),
                                           int(idx.numel()), C.byref(loss),
                                           g.ctypes.data_as(C.c_void_p) if g is not None else None,
                                           sem_ae_param_count()))
    return loss.value, (ae_unflatten(g) if g is not None else None)


def sem_ae_train_step(ctx, ae, samples, idx, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                      eps: float = 1e-8, weight_decay: float = 0.0, loss_dev=None) -> None:
    import torch
    _check(ctx, get_lib().sem_ae_train_step(ae, _dev(samples, "samples", torch.float32), int(samples.shape[0]),
                                            _dev(idx, "idx", torch.int64), int(idx.numel()), float(lr), float(beta1),
                                            float(beta2), float(eps), float(weight_decay),
                                            _dev(loss_dev, "loss_dev", torch.float32, allow_none=True)))


def sem_ae_encode(ctx, ae, u, v, w, latent) -> None:
    """latent: device int16/uint16-sized tensor of E*48 BF16 values (torch.bfloat16 works)."""
    import torch
    E = u.numel() // 512
    _check(ctx, get_lib().sem_ae_encode(ae, _dev(u, "u", torch.float32), _dev(v, "v", torch.float32),
                                        _dev(w, "w", torch.float32), int(E), _dev(latent, "latent")))


def sem_ae_decode(ctx, ae, latent, E: int, u, v, w) -> None:
    import torch
    _check(ctx, get_lib().sem_ae_decode(ae, _dev(latent, "latent"), int(E), _dev(u, "u", torch.float32),
                                        _dev(v, "v", torch.float32), _dev(w, "w", torch.float32)))


def sem_autotune_set(ctx, on: bool) -> None:
    _check(ctx, get_lib().sem_autotune_set(ctx, 1 if on else 0))


def sem_autotune_emit_choices(ctx) -> list:
    """[(N, E, isovalues, units per atomic, ms)] of the tuned isosurface emit launches."""
    out, k = [], 0
    L = get_lib()
    while True:
        N, E, nq, units, ms = C.c_int32(0), C.c_int64(0), C.c_int32(0), C.c_int32(0), C.c_float(0)
        st = L.sem_autotune_emit_entry(ctx, k, C.byref(N), C.byref(E), C.byref(nq), C.byref(units), C.byref(ms))
        if st != SEM_OK:
            return out
        out.append((N.value, E.value, nq.value, units.value, ms.value))
        k += 1


def sem_autotune_width_choices(ctx) -> list:
    """Launch widths the autotuner chose: (kind, N, size, width, ms) per entry (see sem.h)."""
    out = []
    k = 0
    while True:
        kind, N, size, width, ms = C.c_int(), C.c_int(), C.c_int64(), C.c_int(), C.c_float()
        if get_lib().sem_autotune_width_entry(ctx, k, C.byref(kind), C.byref(N), C.byref(size), C.byref(width),
                                              C.byref(ms)) != SEM_OK:
            return out
        out.append((kind.value, N.value, size.value, width.value, ms.value))
        k += 1


def sem_autotune_choices(ctx) -> list:
    """[(M, N, K, epilogue, BN, stages, split, persistent, ms)] of the tuned GEMM shapes."""
    out, k = [], 0
    L = get_lib()
    while True:
        M = C.c_int64(0)
        v = [C.c_int32(0) for _ in range(7)]
        ms = C.c_float(0)
        st = L.sem_autotune_entry(ctx, k, C.byref(M), *[C.byref(x) for x in v], C.byref(ms))
        if st != SEM_OK:
            return out
        out.append((M.value, *[x.value for x in v], ms.value))
        k += 1


def sem_gemm_bf16(ctx, A, B, C_out) -> None:
    """C_out[M][N] = A[M][K] B[N][K]^T (torch.bfloat16 A, B; float32 C) on the tensor cores."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    _check(ctx, get_lib().sem_gemm_bf16(ctx, _dev(A, "A", torch.bfloat16), _dev(B, "B", torch.bfloat16), int(M),
                                        int(N), int(K), _dev(C_out, "C", torch.float32)))


def exported_symbols():
    """Function names declared in include/sem.h (for the ABI test)."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"SEM_API[^;(]*?\b(sem_\w+)\s*\(", txt)))


# ------------------------------------------------------------------------------ convenience

class Session:
    """A context plus its meshes, freed together (``with Session() as s: ...``)."""

    def __init__(self, device: int = 0, stream=None):
        self.ctx = sem_create(device, stream)
        self._meshes = []

    def mesh(self, N: int, xyz):
        m = sem_load_mesh(self.ctx, N, xyz)
        self._meshes.append(m)
        return m

    def close(self):
        for m in self._meshes:
            sem_mesh_free(m)
        self._meshes = []
        if self.ctx:
            sem_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
