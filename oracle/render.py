"""Oracle: ctypes binding of ``render.c`` (test infrastructure only).

``build()`` compiles the FP64 compositing oracle with gcc (OpenMP, strict
floating point: no contraction into fused multiply-adds) into
``oracle/_build/liborc_render.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "render.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc_render.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Splats(C.Structure):
    _fields_ = [("n", C.c_int), ("mean2d", C.c_void_p), ("conic", C.c_void_p),
                ("opacity", C.c_void_p), ("rgb", C.c_void_p), ("mask", C.c_void_p)]


class _Frame(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("tile_w", C.c_int),
                ("tile_h", C.c_int), ("bg", C.c_double * 3), ("eps", C.c_double),
                ("eps_T", C.c_double)]


class _Grads(C.Structure):
    _fields_ = [("dmean2d", C.c_void_p), ("dconic", C.c_void_p), ("dopacity", C.c_void_p),
                ("drgb", C.c_void_p), ("dmask", C.c_void_p), ("dalpha", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_render_tiled.restype = C.c_int64
        _lib.orc_render_tiled.argtypes = [C.POINTER(_Splats), C.POINTER(_Frame), C.c_void_p,
                                          C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]
        _lib.orc_render_bruteforce.restype = None
        _lib.orc_render_bruteforce.argtypes = [C.POINTER(_Splats), C.POINTER(_Frame),
                                               C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                               C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.orc_render_backward.restype = None
        _lib.orc_render_backward.argtypes = [C.POINTER(_Splats), C.POINTER(_Frame), C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.POINTER(_Grads)]
    return _lib


def _c64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class SplatsF64:
    """FP64 per-Gaussian render inputs kept alive for the C calls."""

    def __init__(self, mean2d, conic, opacity, rgb, mask):
        n = int(np.asarray(opacity).shape[0])
        self.mean2d = _c64(mean2d, (n, 2))
        self.conic = _c64(conic, (n, 3))
        self.opacity = _c64(opacity, (n,))
        self.rgb = _c64(rgb, (n, 3))
        self.mask = _c64(mask, (n,))
        self.n = n
        self.c = _Splats(n, self.mean2d.ctypes.data, self.conic.ctypes.data,
                         self.opacity.ctypes.data, self.rgb.ctypes.data, self.mask.ctypes.data)


def _frame(width, height, tile_w, tile_h, bg, eps, eps_T=None):
    return _Frame(int(width), int(height), int(tile_w), int(tile_h),
                  (C.c_double * 3)(*[float(x) for x in bg]), float(eps),
                  float(10 * eps if eps_T is None else eps_T))


def render_tiled(splats: SplatsF64, width, height, tile_w, tile_h, vals, ranges,
                 bg=(0.0, 0.0, 0.0), masked=True, eps=1e-3, eps_T=None):
    f = _frame(width, height, tile_w, tile_h, bg, eps, eps_T)
    vals = np.ascontiguousarray(vals, dtype=np.uint32)
    ranges = np.ascontiguousarray(ranges, dtype=np.uint32)
    img = np.zeros((3, height, width), np.float64)
    T = np.zeros((height, width), np.float64)
    nc = np.zeros((height, width), np.int32)
    fl = np.zeros((height, width), np.uint8)
    frags = lib().orc_render_tiled(C.byref(splats.c), C.byref(f), vals.ctypes.data,
                                   ranges.ctypes.data, int(masked), img.ctypes.data,
                                   T.ctypes.data, nc.ctypes.data, fl.ctypes.data)
    return dict(image=img, final_T=T, n_contrib=nc, flags=fl, frags=int(frags))


def render_bruteforce(splats: SplatsF64, width, height, tile_w, tile_h, rect, depth_bits,
                      bg=(0.0, 0.0, 0.0), masked=True, eps=1e-3, eps_T=None):
    f = _frame(width, height, tile_w, tile_h, bg, eps, eps_T)
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    depth_bits = np.ascontiguousarray(depth_bits, dtype=np.uint32)
    img = np.zeros((3, height, width), np.float64)
    T = np.zeros((height, width), np.float64)
    nc = np.zeros((height, width), np.int32)
    fl = np.zeros((height, width), np.uint8)
    lib().orc_render_bruteforce(C.byref(splats.c), C.byref(f), rect.ctypes.data,
                                depth_bits.ctypes.data, int(masked), img.ctypes.data,
                                T.ctypes.data, nc.ctypes.data, fl.ctypes.data)
    return dict(image=img, final_T=T, n_contrib=nc, flags=fl)


def render_backward(splats: SplatsF64, width, height, tile_w, tile_h, vals, ranges,
                    dL_dimage, bg=(0.0, 0.0, 0.0)):
    f = _frame(width, height, tile_w, tile_h, bg, 0.0)
    vals = np.ascontiguousarray(vals, dtype=np.uint32)
    ranges = np.ascontiguousarray(ranges, dtype=np.uint32)
    g = _c64(dL_dimage, (3, height, width))
    n = splats.n
    out = dict(dmean2d=np.zeros((n, 2)), dconic=np.zeros((n, 3)), dopacity=np.zeros(n),
               drgb=np.zeros((n, 3)), dmask=np.zeros(n), dalpha=np.zeros(n))
    gr = _Grads(*[out[k].ctypes.data for k in
                  ("dmean2d", "dconic", "dopacity", "drgb", "dmask", "dalpha")])
    lib().orc_render_backward(C.byref(splats.c), C.byref(f), vals.ctypes.data,
                              ranges.ctypes.data, g.ctypes.data, C.byref(gr))
    return out
