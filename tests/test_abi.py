"""The C-ABI library builds, loads and exports every symbol include/denser.h declares.
No compute call: these run without a GPU."""

import ctypes
import os
import re

import pytest

from paper_1604_03734_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "denser.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(denser_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def library():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declarations_are_bound():
    assert sorted(native.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(library):
    for name in _declared():
        assert hasattr(library, name), name


def test_binding_loads_and_default_params(library):
    p = native.denser_default_params()
    assert p.voxel_size == 0.1 and p.mu == 0.3 and p.lambda_ == 0.8
    assert p.sigma == 0.5 and p.theta == 1.0 and abs(p.tau - 1 / 6) < 1e-15
    assert p.hash_slots == 1 << 20 and p.precision == native.DENSER_FP32


def test_null_context_is_rejected(library):
    L = native.lib()
    assert L.denser_sync(None, None) == native.DENSER_ERR_INVALID_ARG
    assert L.denser_integrate_batch(None, None, 1, None, None, 0, None, None) == native.DENSER_ERR_INVALID_ARG
    assert L.denser_launch_count(None) == 0
    assert L.denser_set_fusion_profiling(None, 1) == native.DENSER_ERR_INVALID_ARG
    assert L.denser_get_fusion_profile(None, None) == native.DENSER_ERR_INVALID_ARG
    assert L.denser_last_error(None) == b"null context"


def test_struct_sizes_match_header():
    assert ctypes.sizeof(native.denser_params) == 6 * 8 + 6 * 4
    assert ctypes.sizeof(native.denser_intrinsics) == 4 * 8 + 2 * 4
    assert ctypes.sizeof(native.denser_reg_stats) == 2 * 4 + 6 * 8 + 2 * 4 + 2 * 8
    assert ctypes.sizeof(native.denser_fusion_profile) == 4 * 8 + 4 * 8


def test_batch_binding_checks_shapes_without_a_gpu(library):
    """The binding of denser_integrate_batch checks the maps' shape against the camera
    before any call, and the library rejects a null context."""
    import numpy as np
    K = native.intrinsics(100.0, 100.0, 2.5, 2.0, 5, 4)
    poses = np.stack([np.eye(4)] * 2)
    with pytest.raises(ValueError):
        native.denser_integrate_batch(None, np.zeros((2, 4, 4), np.float32), K, poses)
    with pytest.raises(native.DenserError):
        native.denser_integrate_batch(None, np.zeros((2, 4, 5), np.float32), K, poses)
    with pytest.raises(ValueError):  # one pose per map
        native.denser_integrate_batch(None, np.zeros((2, 4, 5), np.float32), K, poses[:1])
