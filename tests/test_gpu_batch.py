"""Batched allocation + fusion (denser_integrate_batch) through the C ABI.

A batch of depth maps must leave exactly the map that one denser_integrate call per
map leaves: the same blocks and block indices (new blocks ordered by the first map that
reached them, then by key), the same w and the same f, bit for bit, since every voxel
takes its maps in order with the same operations.  The oracle (one alloc + fuse per
map, Section III-A) is the reference for both: keys, indices and w bit-exact, f within
1e-4.
"""

import numpy as np
import pytest

from synth.scenes import street_scene, tiny_scene
from tests.pipelines import oracle_coords, run_oracle

pytestmark = pytest.mark.gpu
TOL = 1e-4

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import native as N  # noqa: E402

N.lib()


def _K(sc):
    c = sc.camera
    return N.intrinsics(c.fx, c.fy, c.cx, c.cy, c.width, c.height)


def sequential(sc, depths, segment=0, **params):
    m = N.DenserMap(**params)
    K = _K(sc)
    total = 0
    for k in range(len(depths)):
        d = torch.from_numpy(np.ascontiguousarray(depths[k])).cuda()
        total += N.denser_integrate(m.ctx, d, K, sc.poses[k], segment, count=True)
    snap = m.snapshot()
    m.close()
    return snap, total


def batched(sc, depths, poses=None, segment=0, group=None, kind="device", **params):
    """denser_integrate_batch over all maps (group=None) or over consecutive groups."""
    m = N.DenserMap(**params)
    K = _K(sc)
    poses = np.asarray(sc.poses if poses is None else poses, dtype=np.float64)
    n = len(depths)
    group = group or n
    total = 0
    for first in range(0, n, group):
        d = torch.from_numpy(np.ascontiguousarray(depths[first:first + group]))
        d = d.cuda() if kind == "device" else (d.pin_memory() if kind == "pinned" else d)
        total += N.denser_integrate_batch(m.ctx, d, K, poses[first:first + group], segment, count=True)
    snap = m.snapshot()
    m.close()
    return snap, total


def assert_same(got, want, what=""):
    for key in ("coords", "f", "w"):
        np.testing.assert_array_equal(got[key], want[key], err_msg=f"{what} {key}")


@pytest.fixture(scope="module")
def tiny():
    s = tiny_scene(seed=0)
    return s, s.depth_maps()


def test_tiny_batch_equals_sequential_and_oracle(tiny):
    sc, d = tiny
    want, n_seq = sequential(sc, d)
    got, n_bat = batched(sc, d)
    assert n_bat == n_seq
    assert_same(got, want)
    g, news, _ = run_oracle(sc, d, 0)
    assert n_bat == sum(news)
    np.testing.assert_array_equal(got["coords"], oracle_coords(g))
    np.testing.assert_array_equal(got["w"], g.w.astype(np.float32))
    assert np.max(np.abs(got["f"] - g.f)) <= TOL


@pytest.mark.parametrize("kind", ["pinned", "pageable"])
def test_host_depths(tiny, kind):
    sc, d = tiny
    want, _ = sequential(sc, d)
    got, _ = batched(sc, d, kind=kind)
    assert_same(got, want, kind)


def test_rotated_ragged_camera_and_segment():
    """Yawed poses, a 131 x 47 image (not a multiple of a warp or a tile), segment 5."""
    sc = tiny_scene(seed=3, n_frames=5, yaw_jitter=0.15, width=131, height=47, focal=90.0)
    d = sc.depth_maps()
    want, n_seq = sequential(sc, d, segment=5)
    got, n_bat = batched(sc, d, segment=5)
    assert n_bat == n_seq and n_seq > 0
    assert_same(got, want)
    assert np.all(got["coords"][:, 0] == 5)


def test_more_maps_than_one_launch_and_invalid_maps():
    """20 street maps (one launch of 16, one of 4), two of them without a valid pixel,
    in groups of 7 (ragged) and all at once."""
    sc = street_scene(seed=2, length=12.0)
    d = sc.depth_maps(range(20))
    d[3] = np.nan
    d[11] = 0.0
    want, n_seq = sequential(sc, d)
    assert n_seq > 1000
    for group in (None, 7, 1):
        got, n_bat = batched(sc, d, poses=np.asarray(sc.poses[:20]), group=group)
        assert n_bat == n_seq
        assert_same(got, want, f"group {group}")


def test_street_segment_against_oracle():
    """Ten maps of the driving street (1241 x 376, 15% invalid pixels) against the
    oracle: keys, indices and w bit-exact, f within 1e-4."""
    sc = street_scene(seed=0, length=20.0)
    d = sc.depth_maps(range(10))
    got, n_bat = batched(sc, d, poses=np.asarray(sc.poses[:10]))
    g, news, _ = run_oracle(sc, d, 0)
    assert n_bat == sum(news) == g.n_blocks
    np.testing.assert_array_equal(got["coords"], oracle_coords(g))
    np.testing.assert_array_equal(got["w"], g.w.astype(np.float32))
    assert np.max(np.abs(got["f"] - g.f)) <= TOL


def test_batch_then_regularize_matches_sequential(tiny):
    """The regularised state after a batch equals the one after per-map calls."""
    sc, d = tiny
    outs = []
    for mode in ("seq", "batch"):
        m = N.DenserMap()
        K = _K(sc)
        if mode == "seq":
            for k in range(len(d)):
                N.denser_integrate(m.ctx, torch.from_numpy(np.ascontiguousarray(d[k])).cuda(), K, sc.poses[k], 0)
        else:
            N.denser_integrate_batch(m.ctx, torch.from_numpy(np.ascontiguousarray(d)).cuda(), K,
                                     np.asarray(sc.poses), 0)
        N.denser_regularize(m.ctx, 30, 0.0, 0)
        outs.append(m.snapshot(dual=True))
        m.close()
    for key in outs[0]:
        np.testing.assert_array_equal(outs[1][key], outs[0][key], err_msg=key)


def test_invalid_arguments(tiny):
    sc, d = tiny
    K = _K(sc)
    dd = torch.from_numpy(np.ascontiguousarray(d)).cuda()
    poses = np.asarray(sc.poses, dtype=np.float64).copy()
    with N.DenserMap() as m:
        with pytest.raises(N.DenserError):
            N.denser_integrate_batch(m.ctx, dd[:0], K, poses[:0], 0)
        bad = poses.copy()
        bad[2, 0, 3] = np.nan
        with pytest.raises(N.DenserError):
            N.denser_integrate_batch(m.ctx, dd, K, bad, 0)
        with pytest.raises(N.DenserError):
            N.denser_integrate_batch(m.ctx, dd, K, poses, 200)
        with pytest.raises(ValueError):
            N.denser_integrate_batch(m.ctx, dd[:, :, 1:].contiguous(), K, poses, 0)
        # nothing was allocated by the rejected calls
        assert N.denser_num_blocks(m.ctx) == 0
