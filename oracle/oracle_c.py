"""ctypes wrapper of oracle/denser_oracle_c.c -- TEST INFRASTRUCTURE ONLY.

The C oracle restates the same method as oracle/denser_oracle.py (Section III-A
allocation and Eq. 1 fusion; Section III-B/C primal-dual iteration and energies) in
the same operation order, so that it reaches the numpy oracle's allocation, fusion
and iterates bit for bit, on maps and iteration counts that numpy cannot run in a
test's time.  It runs its loops over blocks with OpenMP (Jacobi updates: the result
does not depend on the thread count).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may use this module.  It shares no code with the CUDA path.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "denser_oracle_c.c")
LIB = os.path.join(HERE, "liboracle_c.so")
BV = 512

_lib = None


def build(force: bool = False) -> str:
    """Compiles the C oracle (gcc, -O2, OpenMP, no floating-point contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        sig = {
            "ocl_new": (vp, [dbl, dbl, dbl, dbl, dbl, dbl, i64]),
            "ocl_free": (None, [vp]),
            "ocl_num_blocks": (i64, [vp]),
            "ocl_load_blocks": (i64, [vp, vp, vp, vp, i64]),
            "ocl_alloc": (i64, [vp, vp, i32, i32, dbl, dbl, dbl, dbl, vp, i64]),
            "ocl_fuse": (None, [vp, vp, i32, i32, dbl, dbl, dbl, dbl, vp, i64]),
            "ocl_iterate": (i32, [vp, i32, i32]),
            "ocl_energies": (i32, [vp, vp, vp]),
            "ocl_get": (None, [vp, vp, vp, vp, vp, vp, vp]),
            "ocl_set_state": (None, [vp, vp, vp, vp]),
            "ocl_set_threads": (None, [i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def set_threads(n: int = 0):
    """Threads of the C oracle's loops from now on (0: one per processor)."""
    lib().ocl_set_threads(int(n))


def _p(a):
    return None if a is None else a.ctypes.data


class CMap:
    """A sparse grid of the C oracle: the same state as denser_oracle.SparseGrid
    (keys in block-index order, f, w, u, u_bar [nb][512], p [3][nb][512], all float64)."""

    def __init__(self, params, capacity: int):
        self.params = params
        self.capacity = int(capacity)
        self.h = lib().ocl_new(params.voxel_size, params.mu, params.lam, params.sigma, params.tau,
                               params.theta, self.capacity)
        if not self.h:
            raise MemoryError("C oracle: out of host memory")

    def close(self):
        if self.h:
            lib().ocl_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def n_blocks(self) -> int:
        return int(lib().ocl_num_blocks(self.h))

    def alloc_blocks(self, depth, K, T_gc, segment: int = 0) -> int:
        d = np.ascontiguousarray(depth, dtype=np.float32)
        T = np.ascontiguousarray(T_gc, dtype=np.float64).reshape(16)
        n = lib().ocl_alloc(self.h, _p(d), K.width, K.height, K.fx, K.fy, K.cx, K.cy, _p(T), int(segment))
        if n < 0:
            raise MemoryError("C oracle: block capacity exceeded")
        return int(n)

    def fuse_depth(self, depth, K, T_gc, segment: int = 0):
        d = np.ascontiguousarray(depth, dtype=np.float32)
        T = np.ascontiguousarray(T_gc, dtype=np.float64).reshape(16)
        lib().ocl_fuse(self.h, _p(d), K.width, K.height, K.fx, K.fy, K.cx, K.cy, _p(T), int(segment))

    def load_blocks(self, coords, f=None, w=None):
        c = np.ascontiguousarray(coords, dtype=np.int64).reshape(-1, 4)
        fa = None if f is None else np.ascontiguousarray(f, dtype=np.float64).reshape(-1, BV)
        wa = None if w is None else np.ascontiguousarray(w, dtype=np.float64).reshape(-1, BV)
        if lib().ocl_load_blocks(self.h, _p(c), _p(fa), _p(wa), len(c)) < 0:
            raise ValueError("C oracle: duplicate key or capacity exceeded")

    def iterate(self, iters: int, threads: int = 0):
        """``iters`` Chambolle-Pock iterations from the current state."""
        if lib().ocl_iterate(self.h, int(iters), int(threads)) != 0:
            raise MemoryError("C oracle: out of host memory")

    def regularize(self, iters: int, threads: int = 0, warm: bool = False):
        """From p = u = u^ = 0 (step 1 of Section III-C), or from the stored state."""
        if not warm:
            lib().ocl_set_state(self.h, None, None, None)
        self.iterate(iters, threads)

    def energies(self):
        P, D = ctypes.c_double(), ctypes.c_double()
        if lib().ocl_energies(self.h, ctypes.byref(P), ctypes.byref(D)) != 0:
            raise MemoryError("C oracle: out of host memory")
        return P.value, D.value

    def set_state(self, u=None, u_bar=None, p=None):
        n = self.n_blocks
        ua = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(n, BV)
        ba = None if u_bar is None else np.ascontiguousarray(u_bar, dtype=np.float64).reshape(n, BV)
        pa = None if p is None else np.ascontiguousarray(p, dtype=np.float64).reshape(3, n, BV)
        lib().ocl_set_state(self.h, _p(ua), _p(ba), _p(pa))

    def snapshot(self) -> dict:
        n = self.n_blocks
        out = {"coords": np.empty((n, 4), np.int64), "f": np.empty((n, BV)), "w": np.empty((n, BV)),
               "u": np.empty((n, BV)), "u_bar": np.empty((n, BV)), "p": np.empty((3, n, BV))}
        lib().ocl_get(self.h, _p(out["coords"]), _p(out["f"]), _p(out["w"]), _p(out["u"]), _p(out["u_bar"]),
                      _p(out["p"]))
        out["omega"] = out["w"] > 0
        return out


def run_pipeline(depths, K, poses, params, iters: int, segment: int = 0, capacity: int = None,
                 threads: int = 0) -> CMap:
    """alloc(k) then fuse(k) for every depth map, then ``iters`` iterations from zero."""
    cap = capacity or 1 << 16
    m = CMap(params, cap)
    for dm, T in zip(depths, poses):
        m.alloc_blocks(dm, K, T, segment)
        m.fuse_depth(dm, K, T, segment)
    if iters > 0:
        m.regularize(iters, threads)
    return m
