"""FP64 CPU oracle for the SEM Q-isosurface render path (ctypes wrapper of sem_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers.  The CUDA library never imports this module, and
the two share no code.  Functions whose result no closed form, invariant or brute-force
check pins are marked "parity unpinned" in their docstring; every function here has at
least one pin in ``tests/test_oracle_*.py``.

All arrays are numpy float64 (inputs are promoted exactly from the FP32 the GPU uses).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sem_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsem_oracle.so")
_lock = threading.Lock()
_lib = None

MAXT = 12


def build(force: bool = False) -> str:
    """Compile sem_oracle.c with gcc (no FMA contraction) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            d, i64, i32, vp = C.c_double, C.c_int64, C.c_int, C.c_void_p
            L = _lib
            L.orc_gll.argtypes = [i32, vp, vp]
            L.orc_dmat.argtypes = [i32, vp, vp]
            L.orc_gradient.argtypes = [i32, i64, vp, i32, vp, vp]
            L.orc_q_from_gradient.argtypes = [i64, vp, vp]
            L.orc_qcriterion.argtypes = [i32, i64, vp, vp, vp]
            L.orc_mc_table.argtypes = [vp, vp]
            L.orc_isosurface.argtypes = [i32, i64, vp, vp, d, vp, vp, i64, vp, vp, vp]
            L.orc_render.argtypes = [vp, i64, vp, i32, vp, i32, vp, vp, vp, d, d, d, d, i32, i32, vp, vp, vp]
            L.orc_surface_measures.argtypes = [vp, i64, vp, vp]
        return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def gll(N: int):
    """GLL nodes and weights (Canuto et al. Sec. 2.3)."""
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    rc = lib().orc_gll(N, _p(xi), _p(w))
    if rc:
        raise ValueError(f"orc_gll rc={rc}")
    return xi, w


def dmat(N: int) -> np.ndarray:
    """(N+1)x(N+1) collocation derivative matrix on the GLL nodes, D[i,j] = l_j'(xi_i)."""
    xi, _ = gll(N)
    D = np.zeros((N + 1, N + 1))
    lib().orc_dmat(N, _p(xi), _p(D))
    return D


def gradient(N: int, xyz, fields) -> np.ndarray:
    """Physical gradient (isoparametric chain rule).  xyz (3,E,NP^3); fields (nf,E,NP^3)
    -> (nf, 3, E, NP^3): d field_q / d x_a."""
    xyz = _f64(xyz)
    fields = _f64(fields)
    if fields.ndim == 2:
        fields = fields[None]
    nf, E = fields.shape[0], fields.shape[1]
    out = np.zeros((nf, 3) + fields.shape[1:])
    rc = lib().orc_gradient(N, E, _p(xyz), nf, _p(fields), _p(out))
    if rc:
        raise ValueError(f"orc_gradient rc={rc}")
    return out


def q_from_gradient(grad) -> np.ndarray:
    """Q = -1/2 sum_ij J_ij J_ji from grad (3, 3, ...) with grad[i, j] = du_i/dx_j."""
    g = _f64(grad)
    shp = g.shape[2:]
    Q = np.zeros(shp)
    lib().orc_q_from_gradient(int(np.prod(shp)), _p(g), _p(Q))
    return Q


def qcriterion(N: int, xyz, uvw) -> np.ndarray:
    """Q-criterion of the velocity (3,E,NP^3) on the mesh xyz (3,E,NP^3) -> (E,NP^3)."""
    xyz = _f64(xyz)
    uvw = _f64(uvw)
    E = uvw.shape[1]
    Q = np.zeros(uvw.shape[1:])
    rc = lib().orc_qcriterion(N, E, _p(xyz), _p(uvw), _p(Q))
    if rc:
        raise ValueError(f"orc_qcriterion rc={rc}")
    return Q


def mc_table():
    """(ntri[256], tri[256, MAXT, 3]) generated from the face-consistent rule."""
    n = np.zeros(256, dtype=np.int32)
    t = np.zeros((256, MAXT, 3), dtype=np.int32)
    mx = lib().orc_mc_table(_p(n), _p(t))
    if mx < 0:
        raise RuntimeError(f"table rule failed ({mx})")
    return n, t


def isosurface(N: int, xyz, f, iso: float, cap: int = None, want_tris: bool = True):
    """Marching cubes over each element's N^3 GLL sub-hexes.

    Returns dict(cases (E,N^3) u8, elem_ntri (E,) i64, ntri, tris (ntri,3,3) f64,
    tri_elem (ntri,) i32)."""
    xyz = _f64(xyz)
    f = _f64(f)
    E = f.shape[0]
    cases = np.zeros((E, N ** 3), dtype=np.uint8)
    en = np.zeros(E, dtype=np.int64)
    nt = C.c_int64(0)
    L = lib()
    if cap is None:
        L.orc_isosurface(N, E, _p(xyz), _p(f), float(iso), _p(cases), _p(en), 0, None, None, C.byref(nt))
        cap = nt.value
    if not want_tris:
        return dict(cases=cases, elem_ntri=en, ntri=int(en.sum()))
    tris = np.zeros((max(cap, 1), 3, 3))
    te = np.zeros(max(cap, 1), dtype=np.int32)
    rc = L.orc_isosurface(N, E, _p(xyz), _p(f), float(iso), _p(cases), _p(en), cap, _p(tris), _p(te),
                          C.byref(nt))
    if rc:
        raise ValueError(f"orc_isosurface rc={rc}")
    n = nt.value
    return dict(cases=cases, elem_ntri=en, ntri=n, tris=tris[:n], tri_elem=te[:n])


def render(tris, seg_ntri, seg_rgb, cam: dict, W: int = None, H: int = None):
    """Z-buffer raster of a triangle soup (ntri,3,3), coloured per contiguous segment.

    Returns (rgba (H,W,4) u8, depth (H,W) f64, winner (H,W) i64 triangle index or -1)."""
    tris = _f64(tris).reshape(-1, 9)
    W = cam["W"] if W is None else W
    H = cam["H"] if H is None else H
    seg_end = np.cumsum(np.asarray(seg_ntri, dtype=np.int64))
    rgb = _f64(seg_rgb).reshape(-1, 3)
    rgba = np.zeros((H, W, 4), dtype=np.uint8)
    depth = np.zeros((H, W))
    win = np.zeros((H, W), dtype=np.int64)
    rc = lib().orc_render(_p(tris), tris.shape[0], _p(seg_end), len(seg_end), _p(rgb), int(cam["ortho"]),
                          _p(_f64(cam["eye"])), _p(_f64(cam["center"])), _p(_f64(cam["up"])),
                          float(cam["fovy_deg"]), float(cam["half_h"]), float(cam["znear"]),
                          float(cam["zfar"]), W, H, _p(rgba), _p(depth), _p(win))
    if rc:
        raise ValueError(f"orc_render rc={rc}")
    return rgba, depth, win


def surface_measures(tris):
    """(area, enclosed volume) of a triangle soup, FP64."""
    tris = _f64(tris).reshape(-1, 9)
    a = C.c_double(0)
    v = C.c_double(0)
    lib().orc_surface_measures(_p(tris), tris.shape[0], C.byref(a), C.byref(v))
    return a.value, v.value
