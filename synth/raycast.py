"""ctypes wrapper of synth/raycast.c: the noise-free depth of a scene, in the operation
order of Scene.render_clean_numpy's casts (the same float64 depths, about nine times
faster).  Input generation only; none of the method's arithmetic."""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "raycast.c")
LIB = os.path.join(HERE, "libraycast.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.raycast_depth.restype = None
        L.raycast_depth.argtypes = [i32, i32, dbl, dbl, dbl, dbl, vp, i32, vp, i32, vp, vp, i32, vp, vp, dbl, vp, vp]
        _lib = L
    return _lib


def depth(scene, T, box_windows) -> np.ndarray:
    """Noise-free depth [H, W] float64 of ``scene`` from pose T; box_windows: per box the
    pixel rectangle (y0, y1, x0, x1) holding its projection, or None for the whole image."""
    c = scene.camera
    rects = np.array([[r.axis, r.value, r.lo[0], r.lo[1], r.hi[0], r.hi[1]] for r in scene.rects],
                     dtype=np.float64).reshape(-1, 6)
    boxes = np.array([list(b.lo) + list(b.hi) for b in scene.boxes], dtype=np.float64).reshape(-1, 6)
    win = np.array([[-1, 0, 0, 0] if w is None else list(w) for w in box_windows], dtype=np.int32).reshape(-1, 4)
    fac = np.array([[f.x, f.side, f.y_top, f.y_bot, f.z0, f.z1, f.cell[0], f.cell[1], f.win[0], f.win[1],
                     f.recess, f.windows.shape[0], f.windows.shape[1]] for f in scene.facades],
                   dtype=np.float64).reshape(-1, 13)
    wins = np.concatenate([f.windows.astype(np.uint8).reshape(-1) for f in scene.facades]) if scene.facades \
        else np.zeros(1, np.uint8)
    T = np.ascontiguousarray(T, dtype=np.float64)
    out = np.empty((c.height, c.width), np.float64)
    buf = np.empty(3 * c.width * c.height, np.float64)
    lib().raycast_depth(c.width, c.height, c.fx, c.fy, c.cx, c.cy, T.ctypes.data, len(rects), rects.ctypes.data,
                        len(boxes), boxes.ctypes.data, win.ctypes.data, len(fac), fac.ctypes.data,
                        wins.ctypes.data, float(scene.d_max), buf.ctypes.data, out.ctypes.data)
    return out
