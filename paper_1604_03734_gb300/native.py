"""ctypes binding of libdenser.so: the C ABI of include/denser.h, same names.

Argument marshalling only.  Every computation runs in the library's CUDA
kernels; if the library is missing this module raises instead of falling back
to anything else.  Buffers may be torch tensors (CPU or CUDA) or numpy arrays;
they must be contiguous and of the dtype the C function documents.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

DENSER_OK = 0
DENSER_ERR_INVALID_ARG = -1
DENSER_ERR_HASH_FULL = -2
DENSER_ERR_POOL_FULL = -3
DENSER_ERR_CUDA = -4
DENSER_ERR_TIMEOUT = -5
DENSER_ERR_RANGE = -6
DENSER_ERR_TOO_LARGE = -7
DENSER_NOALLOC_MAX_BLOCKS = 16384
DENSER_MAX_BATCH = 16
DENSER_FP32, DENSER_FP16, DENSER_BF16 = 0, 1, 2

# every symbol include/denser.h declares
EXPORTS = ("denser_default_params", "denser_create", "denser_destroy", "denser_reset",
           "denser_last_error", "denser_sync", "denser_alloc_blocks", "denser_fuse_depth", "denser_integrate",
           "denser_integrate_batch",
           "denser_alloc_points", "denser_fuse_points", "denser_integrate_points",
           "denser_regularize", "denser_energy", "denser_extract", "denser_extract_dual", "denser_extract_surface",
           "denser_load_blocks", "denser_load_state", "denser_num_blocks", "denser_launch_count",
           "denser_set_schedule", "denser_get_schedule", "denser_energy_noalloc",
           "denser_set_fusion_profiling", "denser_get_fusion_profile", "denser_net_check",
           "denser_net_targets_div", "denser_net_loss_div",
           "denser_net_gather", "denser_net_targets", "denser_net_apply", "denser_conv3", "denser_conv3_wgrad",
           "denser_relu_backward", "denser_net_loss", "denser_adam", "denser_pack_weights",
           "denser_stereo_default_params", "denser_census", "denser_diffusion_tensor", "denser_disparity_assign",
           "denser_tgv_iterate", "denser_stereo_workspace_size", "denser_stereo_estimate",
           "denser_disparity_to_depth")


class denser_params(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_double), ("mu", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("sigma", ctypes.c_double), ("tau", ctypes.c_double), ("theta", ctypes.c_double),
                ("hash_slots", ctypes.c_uint32), ("max_blocks", ctypes.c_uint32),
                ("max_new_blocks", ctypes.c_uint32), ("precision", ctypes.c_int32),
                ("gap_every", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class denser_fusion_profile(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int64), ("maps", ctypes.c_int64), ("listed_blocks", ctypes.c_int64),
                ("new_blocks", ctypes.c_int64), ("key_pass_ms", ctypes.c_double), ("alloc_rest_ms", ctypes.c_double),
                ("cull_ms", ctypes.c_double), ("fuse_ms", ctypes.c_double)]


class denser_intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class denser_reg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("primal", ctypes.c_double),
                ("dual", ctypes.c_double), ("gap", ctypes.c_double), ("rel_gap", ctypes.c_double),
                ("sweep_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("sweep_launches", ctypes.c_int32), ("gap_evals", ctypes.c_int32),
                ("n_blocks", ctypes.c_int64), ("n_omega", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class denser_schedule(ctypes.Structure):
    _fields_ = [("sweep_kernel", ctypes.c_int32), ("order", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


class denser_stereo_params(ctypes.Structure):
    _fields_ = [("max_disp", ctypes.c_int32), ("lambda_", ctypes.c_float), ("alpha1", ctypes.c_float),
                ("alpha2", ctypes.c_float), ("beta", ctypes.c_float), ("gamma", ctypes.c_float),
                ("theta0", ctypes.c_float), ("theta_decay", ctypes.c_float), ("outer", ctypes.c_int32),
                ("inner", ctypes.c_int32)]


class DenserError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"denser error {code}: {msg}")
        self.code = code


_lib = None
_vp, _i32, _i64, _u64, _dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_1604_03734_gb300.build.build()")
        L = ctypes.CDLL(LIB)
        P = ctypes.POINTER
        sig = {
            "denser_default_params": (None, [P(denser_params)]),
            "denser_create": (_i32, [P(denser_params), _i32, P(_vp)]),
            "denser_destroy": (None, [_vp]),
            "denser_reset": (_i32, [_vp, _vp]),
            "denser_last_error": (ctypes.c_char_p, [_vp]),
            "denser_sync": (_i32, [_vp, _vp]),
            "denser_alloc_blocks": (_i32, [_vp, _vp, P(denser_intrinsics), P(_dbl), _i32, _vp, P(_i32)]),
            "denser_fuse_depth": (_i32, [_vp, _vp, P(denser_intrinsics), P(_dbl), _i32, _vp]),
            "denser_integrate": (_i32, [_vp, _vp, P(denser_intrinsics), P(_dbl), _i32, _vp, P(_i32)]),
            "denser_integrate_batch": (_i32, [_vp, _vp, _i32, P(denser_intrinsics), P(_dbl), _i32, _vp, P(_i32)]),
            "denser_alloc_points": (_i32, [_vp, _vp, _i64, P(_dbl), _i32, _vp, P(_i32)]),
            "denser_fuse_points": (_i32, [_vp, _vp, _i64, P(_dbl), _i32, _vp]),
            "denser_integrate_points": (_i32, [_vp, _vp, _i64, P(_dbl), _i32, _vp, P(_i32)]),
            "denser_regularize": (_i32, [_vp, _i32, _dbl, _i32, _vp, P(denser_reg_stats)]),
            "denser_energy": (_i32, [_vp, P(_dbl), P(_dbl), _vp]),
            "denser_extract": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i64, P(_i64), _vp]),
            "denser_extract_dual": (_i32, [_vp, _vp, _vp, _i64, _vp]),
            "denser_extract_surface": (_i32, [_vp, _vp, _vp, _i64, P(_i64), _vp, _vp]),
            "denser_load_blocks": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp]),
            "denser_load_state": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp]),
            "denser_num_blocks": (_i64, [_vp, _vp]),
            "denser_launch_count": (_u64, [_vp]),
            "denser_set_fusion_profiling": (_i32, [_vp, _i32]),
            "denser_net_check": (_i32, [_vp]),
            "denser_net_targets_div": (_i32, [_vp, _vp, _i64, _vp, _vp]),
            "denser_net_loss_div": (_i32, [_vp, _vp, ctypes.c_float, ctypes.c_float, _vp, _vp, _i64, _vp]),
            "denser_get_fusion_profile": (_i32, [_vp, _vp]),
            "denser_set_schedule": (_i32, [_vp, P(denser_schedule)]),
            "denser_get_schedule": (_i32, [_vp, P(denser_schedule)]),
            "denser_energy_noalloc": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _dbl, _vp, _vp]),
            "denser_net_gather": (_i32, [_vp, _vp, _i64, _vp, _vp]),
            "denser_net_targets": (_i32, [_vp, _vp, _i64, _vp, _vp, ctypes.c_float, ctypes.c_float, _vp]),
            "denser_net_apply": (_i32, [_vp, _vp, _i64, _vp, _i32, _vp]),
            "denser_conv3": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _i64, _vp]),
            "denser_conv3_wgrad": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp]),
            "denser_relu_backward": (_i32, [_vp, _vp, _vp, _i64, _vp]),
            "denser_net_loss": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _vp]),
            "denser_adam": (_i32, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, _i32, _vp]),
            "denser_pack_weights": (_i32, [_vp, _vp, _vp, _vp]),
            "denser_stereo_default_params": (None, [P(denser_stereo_params)]),
            "denser_census": (_i32, [_vp, _i32, _i32, _vp, _vp]),
            "denser_diffusion_tensor": (_i32, [_vp, _i32, _i32, ctypes.c_float, ctypes.c_float, _vp, _vp]),
            "denser_disparity_assign": (_i32, [_vp, _vp, _i32, _i32, _i32, ctypes.c_float, _dbl, _vp, _vp, _vp]),
            "denser_tgv_iterate": (_i32, [_vp, _vp, _i32, _i32, ctypes.c_float, ctypes.c_float, _dbl, _i32, _vp,
                                          _vp]),
            "denser_stereo_workspace_size": (ctypes.c_size_t, [_i32, _i32]),
            "denser_stereo_estimate": (_i32, [_vp, _vp, _i32, _i32, P(denser_stereo_params), _vp, ctypes.c_size_t,
                                              _vp, _vp]),
            "denser_disparity_to_depth": (_i32, [_vp, _i32, _i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                                 _vp, _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ------------------------------------------------------------- marshalling
def _ptr(buf, dtype=None):
    """Raw address of a contiguous torch tensor or numpy array (None -> NULL)."""
    if buf is None:
        return None
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffer must be C-contiguous")
        if dtype is not None and buf.dtype != np.dtype(dtype):
            raise TypeError(f"expected {np.dtype(dtype)}, got {buf.dtype}")
        return buf.ctypes.data
    import torch
    if isinstance(buf, torch.Tensor):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None:
            want = {np.float32: torch.float32, np.int32: torch.int32, np.uint8: torch.uint8,
                    np.float64: torch.float64, np.int64: torch.int64}[dtype]
            if buf.dtype != want:
                raise TypeError(f"expected {want}, got {buf.dtype}")
        return buf.data_ptr()
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, rc):
    if rc != DENSER_OK:
        msg = lib().denser_last_error(ctx)
        raise DenserError(rc, msg.decode() if msg else "")
    return rc


def _pose(T):
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    return a, a.ctypes.data_as(ctypes.POINTER(_dbl))


def intrinsics(fx, fy, cx, cy, width, height) -> denser_intrinsics:
    return denser_intrinsics(float(fx), float(fy), float(cx), float(cy), int(width), int(height))


# ------------------------------------------------------------ the C calls
def denser_default_params(**overrides) -> denser_params:
    p = denser_params()
    lib().denser_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, "lambda_" if k == "lambda" else k, v)
    return p


def denser_create(params: denser_params, device: int = 0):
    ctx = _vp()
    rc = lib().denser_create(ctypes.byref(params), device, ctypes.byref(ctx))
    if rc != DENSER_OK:
        raise DenserError(rc, "denser_create failed")
    return ctx


def denser_destroy(ctx):
    lib().denser_destroy(ctx)


def denser_reset(ctx, stream=None):
    return _check(ctx, lib().denser_reset(ctx, _stream(stream)))


def denser_last_error(ctx) -> str:
    m = lib().denser_last_error(ctx)
    return m.decode() if m else ""


def denser_sync(ctx, stream=None):
    return _check(ctx, lib().denser_sync(ctx, _stream(stream)))


def denser_alloc_blocks(ctx, depth, K: denser_intrinsics, T_gc, segment=0, stream=None, count=False):
    """Returns the number of new blocks when ``count`` (waits), else None."""
    keep, tp = _pose(T_gc)
    n = _i32(0)
    _check(ctx, lib().denser_alloc_blocks(ctx, _ptr(depth, np.float32), ctypes.byref(K), tp, segment,
                                          _stream(stream), ctypes.byref(n) if count else None))
    return n.value if count else None


def denser_integrate(ctx, depth, K: denser_intrinsics, T_gc, segment=0, stream=None, count=False):
    """Allocation then fusion of one depth map; returns the number of new blocks when
    ``count`` (waits), else None."""
    keep, tp = _pose(T_gc)
    n = _i32(0)
    _check(ctx, lib().denser_integrate(ctx, _ptr(depth, np.float32), ctypes.byref(K), tp, segment,
                                       _stream(stream), ctypes.byref(n) if count else None))
    return n.value if count else None


def denser_integrate_batch(ctx, depths, K: denser_intrinsics, T_gc, segment=0, stream=None, count=False):
    """Allocation and fusion of depth maps [n, H, W] in order (the result of n
    denser_integrate calls) with poses [n, 4, 4]; returns the number of new blocks when
    ``count`` (waits), else None."""
    n_frames = int(depths.shape[0])
    if tuple(depths.shape[1:]) != (K.height, K.width):
        raise ValueError(f"depth maps {tuple(depths.shape)} do not match the camera's {K.height} x {K.width}")
    tp_arr = np.ascontiguousarray(np.asarray(T_gc, dtype=np.float64).reshape(n_frames, 16))
    n = _i32(0)
    _check(ctx, lib().denser_integrate_batch(ctx, _ptr(depths, np.float32), n_frames, ctypes.byref(K),
                                             tp_arr.ctypes.data_as(ctypes.POINTER(_dbl)), segment, _stream(stream),
                                             ctypes.byref(n) if count else None))
    return n.value if count else None


def _npoints(points):
    return 0 if points is None else int(points.shape[0])


def denser_alloc_points(ctx, points, T_gs, segment=0, stream=None, count=False):
    """Allocation along a laser scan's rays; points float32 [n, 3] (sensor frame)."""
    keep, tp = _pose(T_gs)
    n = _i32(0)
    _check(ctx, lib().denser_alloc_points(ctx, _ptr(points, np.float32), _npoints(points), tp, segment,
                                          _stream(stream), ctypes.byref(n) if count else None))
    return n.value if count else None


def denser_fuse_points(ctx, points, T_gs, segment=0, stream=None):
    keep, tp = _pose(T_gs)
    return _check(ctx, lib().denser_fuse_points(ctx, _ptr(points, np.float32), _npoints(points), tp, segment,
                                                _stream(stream)))


def denser_integrate_points(ctx, points, T_gs, segment=0, stream=None, count=False):
    keep, tp = _pose(T_gs)
    n = _i32(0)
    _check(ctx, lib().denser_integrate_points(ctx, _ptr(points, np.float32), _npoints(points), tp, segment,
                                              _stream(stream), ctypes.byref(n) if count else None))
    return n.value if count else None


def denser_fuse_depth(ctx, depth, K: denser_intrinsics, T_gc, segment=0, stream=None):
    keep, tp = _pose(T_gc)
    return _check(ctx, lib().denser_fuse_depth(ctx, _ptr(depth, np.float32), ctypes.byref(K), tp, segment,
                                               _stream(stream)))


def denser_regularize(ctx, max_iters, gap_tol=0.0, start=0, stream=None, stats=True):
    st = denser_reg_stats()
    _check(ctx, lib().denser_regularize(ctx, int(max_iters), float(gap_tol), int(start), _stream(stream),
                                        ctypes.byref(st) if stats else None))
    return st if stats else None


def denser_energy(ctx, stream=None):
    P, D = _dbl(), _dbl()
    _check(ctx, lib().denser_energy(ctx, ctypes.byref(P), ctypes.byref(D), _stream(stream)))
    return P.value, D.value


def denser_extract(ctx, coords=None, f=None, w=None, omega=None, u=None, capacity_blocks=0, stream=None):
    n = _i64(0)
    _check(ctx, lib().denser_extract(ctx, _ptr(coords, np.int32), _ptr(f, np.float32), _ptr(w, np.float32),
                                     _ptr(omega, np.uint8), _ptr(u, np.float32), int(capacity_blocks),
                                     ctypes.byref(n), _stream(stream)))
    return n.value


def denser_extract_dual(ctx, u_bar=None, p=None, capacity_blocks=0, stream=None):
    return _check(ctx, lib().denser_extract_dual(ctx, _ptr(u_bar, np.float32), _ptr(p, np.float32),
                                                 int(capacity_blocks), _stream(stream)))


def denser_extract_surface(ctx, tri_pos=None, tri_ids=None, capacity=0, block_first=None, stream=None) -> int:
    """Triangles of the zero level set of u over Omega (float32 [cap][3][3] positions,
    int64 [cap][3] vertex ids, int64 [n_blocks + 1] first triangle per block); returns
    the total triangle count.  A total above `capacity` with a triangle buffer raises
    DenserError (DENSER_ERR_TOO_LARGE) after the first `capacity` triangles are written;
    count first with the triangle buffers None."""
    n = _i64(0)
    _check(ctx, lib().denser_extract_surface(ctx, _ptr(tri_pos, np.float32), _ptr(tri_ids, np.int64),
                                             int(capacity), ctypes.byref(n), _ptr(block_first, np.int64),
                                             _stream(stream)))
    return n.value


def denser_load_blocks(ctx, coords, f=None, w=None, n=None, stream=None):
    n = len(coords) if n is None else n
    return _check(ctx, lib().denser_load_blocks(ctx, _ptr(coords, np.int32), _ptr(f, np.float32),
                                                _ptr(w, np.float32), int(n), _stream(stream)))


def denser_load_state(ctx, u=None, u_bar=None, p=None, n=0, stream=None):
    return _check(ctx, lib().denser_load_state(ctx, _ptr(u, np.float32), _ptr(u_bar, np.float32),
                                               _ptr(p, np.float32), int(n), _stream(stream)))


def denser_num_blocks(ctx, stream=None) -> int:
    n = lib().denser_num_blocks(ctx, _stream(stream))
    if n < 0:
        _check(ctx, int(n))
    return int(n)


def denser_launch_count(ctx) -> int:
    return int(lib().denser_launch_count(ctx))


def denser_net_targets_div(ctx, blocks, n, target, stream=None):
    return _check(ctx, lib().denser_net_targets_div(ctx, _tptr(blocks), int(n), _tptr(target), _stream(stream)))


def denser_net_loss_div(out, target, u_weight, div_weight, dout, loss, n, stream=None):
    rc = lib().denser_net_loss_div(_tptr(out), _tptr(target), float(u_weight), float(div_weight), _tptr(dout),
                                   _tptr(loss), int(n), _stream(stream))
    if rc != DENSER_OK:
        raise DenserError(rc, "denser_net_loss_div failed")
    return rc


def denser_net_check(stream=None) -> int:
    """Waits for the stream; the C status (DENSER_ERR_TIMEOUT if a tensor-core wait ran out)."""
    return int(lib().denser_net_check(_stream(stream)))


def denser_set_fusion_profiling(ctx, enable: bool = True):
    return _check(ctx, lib().denser_set_fusion_profiling(ctx, 1 if enable else 0))


def denser_get_fusion_profile(ctx) -> dict:
    pr = denser_fusion_profile()
    _check(ctx, lib().denser_get_fusion_profile(ctx, ctypes.byref(pr)))
    return {name: getattr(pr, name) for name, _ in pr._fields_}


def denser_set_schedule(ctx, sweep_kernel=2, order=1, ctas_per_sm=0, use_graph=1):
    sch = denser_schedule(int(sweep_kernel), int(order), int(ctas_per_sm), int(use_graph))
    return _check(ctx, lib().denser_set_schedule(ctx, ctypes.byref(sch)))


def denser_get_schedule(ctx) -> dict:
    sch = denser_schedule()
    _check(ctx, lib().denser_get_schedule(ctx, ctypes.byref(sch)))
    return {"sweep_kernel": sch.sweep_kernel, "order": sch.order, "ctas_per_sm": sch.ctas_per_sm,
            "use_graph": sch.use_graph}


def denser_energy_noalloc(coords, f, w, u, p, n_blocks, lam, out, stream=None) -> int:
    """Energies {P, D} into ``out`` (2 float64, host or device) from caller-owned device
    buffers, with no device allocation; returns the C status code (0 = OK)."""
    return int(lib().denser_energy_noalloc(_ptr(coords, np.int32), _ptr(f, np.float32), _ptr(w, np.float32),
                                           _ptr(u, np.float32), _ptr(p, np.float32), int(n_blocks), float(lam),
                                           _ptr(out, np.float64), _stream(stream)))


def _tptr(t):
    """Address of a contiguous torch tensor of any dtype (None -> NULL)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def denser_net_gather(ctx, blocks, n, x, stream=None):
    return _check(ctx, lib().denser_net_gather(ctx, _tptr(blocks), int(n), _tptr(x), _stream(stream)))


def denser_net_targets(ctx, blocks, n, target, mask, u_weight=1.0, p_weight=1.0, stream=None):
    return _check(ctx, lib().denser_net_targets(ctx, _tptr(blocks), int(n), _tptr(target), _tptr(mask),
                                                float(u_weight), float(p_weight), _stream(stream)))


def denser_net_apply(ctx, blocks, n, out, with_dual=1, stream=None):
    return _check(ctx, lib().denser_net_apply(ctx, _tptr(blocks), int(n), _tptr(out), int(with_dual),
                                              _stream(stream)))


def _ok(rc, what):
    if rc != DENSER_OK:
        raise DenserError(rc, what)


def denser_conv3(x, w, bias, relu, y_bf16, y_f32, n, stream=None):
    _ok(lib().denser_conv3(_tptr(x), _tptr(w), _tptr(bias), int(relu), _tptr(y_bf16), _tptr(y_f32), int(n),
                           _stream(stream)), "denser_conv3")


def denser_conv3_wgrad(h, dz, dw, db, n, stream=None):
    _ok(lib().denser_conv3_wgrad(_tptr(h), _tptr(dz), _tptr(dw), _tptr(db), int(n), _stream(stream)),
        "denser_conv3_wgrad")


def denser_relu_backward(dh, h, dz, count, stream=None):
    _ok(lib().denser_relu_backward(_tptr(dh), _tptr(h), _tptr(dz), int(count), _stream(stream)),
        "denser_relu_backward")


def denser_net_loss(out, target, mask, dout, loss, n, stream=None):
    _ok(lib().denser_net_loss(_tptr(out), _tptr(target), _tptr(mask), _tptr(dout), _tptr(loss), int(n),
                              _stream(stream)), "denser_net_loss")


def denser_adam(w, grad, m, v, count, lr, beta1, beta2, eps, step, stream=None):
    _ok(lib().denser_adam(_tptr(w), _tptr(grad), _tptr(m), _tptr(v), int(count), float(lr), float(beta1),
                          float(beta2), float(eps), int(step), _stream(stream)), "denser_adam")


def denser_pack_weights(w32, wf, wb, stream=None):
    _ok(lib().denser_pack_weights(_tptr(w32), _tptr(wf), _tptr(wb), _stream(stream)), "denser_pack_weights")


# ------------------------------------------------------------ stereo
def denser_stereo_default_params(**overrides) -> denser_stereo_params:
    p = denser_stereo_params()
    lib().denser_stereo_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, "lambda_" if k == "lambda" else k, v)
    return p


def _hw(img):
    return int(img.shape[1]), int(img.shape[0])


def denser_census(img, sig, stream=None):
    W, H = _hw(img)
    _ok(lib().denser_census(_tptr(img), W, H, _tptr(sig), _stream(stream)), "denser_census")


def denser_diffusion_tensor(img, tensor, gamma=4.0, beta=1.0, stream=None):
    W, H = _hw(img)
    _ok(lib().denser_diffusion_tensor(_tptr(img), W, H, float(gamma), float(beta), _tptr(tensor), _stream(stream)),
        "denser_diffusion_tensor")


def denser_disparity_assign(sig_left, sig_right, max_disp, lam, theta, d, a, stream=None):
    W, H = _hw(sig_right)
    _ok(lib().denser_disparity_assign(_tptr(sig_left), _tptr(sig_right), W, H, int(max_disp), float(lam),
                                      float(theta), _tptr(d), _tptr(a), _stream(stream)), "denser_disparity_assign")


def denser_tgv_iterate(a, tensor, alpha1, alpha2, theta, iters, state, stream=None):
    W, H = _hw(a)
    _ok(lib().denser_tgv_iterate(_tptr(a), _tptr(tensor), W, H, float(alpha1), float(alpha2), float(theta),
                                 int(iters), _tptr(state), _stream(stream)), "denser_tgv_iterate")


def denser_stereo_workspace_size(width, height) -> int:
    return int(lib().denser_stereo_workspace_size(int(width), int(height)))


def denser_stereo_estimate(img_left, img_right, params, workspace, disparity, stream=None):
    W, H = _hw(img_right)
    nbytes = workspace.numel() * workspace.element_size()
    _ok(lib().denser_stereo_estimate(_tptr(img_left), _tptr(img_right), W, H, ctypes.byref(params), _tptr(workspace),
                                     nbytes, _tptr(disparity), _stream(stream)), "denser_stereo_estimate")


def denser_disparity_to_depth(disparity, fx, baseline, min_disp, depth, stream=None):
    W, H = _hw(disparity)
    _ok(lib().denser_disparity_to_depth(_tptr(disparity), W, H, float(fx), float(baseline), float(min_disp),
                                        _tptr(depth), _stream(stream)), "denser_disparity_to_depth")


# ------------------------------------------------------------ convenience
class DenserMap:
    """Owns one context; numpy-returning helpers built on the calls above."""

    def __init__(self, device=0, **params):
        self.params = denser_default_params(**params)
        self.ctx = denser_create(self.params, device)

    def close(self):
        if self.ctx is not None:
            denser_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def snapshot(self, dual=False):
        """Host copies: coords [n,4], f, w, u [n,512], omega bool [n,512] (+ u_bar, p)."""
        n = denser_num_blocks(self.ctx)
        out = {"coords": np.zeros((n, 4), np.int32), "f": np.zeros((n, 512), np.float32),
               "w": np.zeros((n, 512), np.float32), "omega": np.zeros((n, 512), np.uint8),
               "u": np.zeros((n, 512), np.float32)}
        denser_extract(self.ctx, out["coords"], out["f"], out["w"], out["omega"], out["u"], n)
        if dual:
            out["u_bar"] = np.zeros((n, 512), np.float32)
            out["p"] = np.zeros((3, n, 512), np.float32)
            denser_extract_dual(self.ctx, out["u_bar"], out["p"], n)
        return out

    def surface(self, with_ids=True, stream=None):
        """Host copies of the surface triangles: positions float32 [n, 3, 3] (metres) and,
        with_ids, vertex ids int64 [n, 3]."""
        n = denser_extract_surface(self.ctx, stream=stream)
        pos = np.zeros((n, 3, 3), np.float32)
        ids = np.zeros((n, 3), np.int64) if with_ids else None
        if n:
            denser_extract_surface(self.ctx, pos, ids, n, stream=stream)
        return (pos, ids) if with_ids else pos
