"""Pins of the oracle's allocation and fusion against geometry the paper fixes.

Allocation (Section III-A, reading R1) is pinned by a hand-counted one-pixel
case and by a world-frame ray march; fusion (Eq. 1) by plane closed forms, a
one-pixel viewing cone under a rotated camera, and repeated identical frames.
"""

import math

import numpy as np
import pytest

from oracle.denser_oracle import (BLOCK, Intrinsics, Params, SparseGrid, alloc_blocks,
                                  frame_block_keys, fuse_depth, local_offsets, run_pipeline)

P = Params()


def _rot(a, b, c):
    ca, sa, cb, sb, cc, sc = math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(c), math.sin(c)
    Rz = np.array([[cc, -sc, 0], [sc, cc, 0], [0, 0, 1]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    return Rz @ Ry @ Rx


def _pose(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def _voxel_centres(grid):
    """World centres [nb*512, 3] of every allocated voxel: ((i+0.5)s, (j+0.5)s, (k+0.5)s)."""
    lx, ly, lz = local_offsets()
    C = grid.coords()
    i = (C[:, 1:2] * BLOCK + lx[None, :]).reshape(-1)
    j = (C[:, 2:3] * BLOCK + ly[None, :]).reshape(-1)
    k = (C[:, 3:4] * BLOCK + lz[None, :]).reshape(-1)
    s = grid.params.voxel_size
    return np.stack([(i + 0.5) * s, (j + 0.5) * s, (k + 0.5) * s], axis=1)


# ------------------------------------------------------------ allocation
def test_alloc_one_pixel_hand_count():
    # Pixel (0,0) of a camera with cx = cy = 0.5 looks down the optical axis.
    K = Intrinsics(100.0, 100.0, 0.5, 0.5, 1, 1)
    depth = np.array([[4.0]], np.float32)
    # samples z = 4 + n*0.05, n = -6..6, global z = z + 0.0037 in [3.7037, 4.3037];
    # divided by the 0.8 m block size: [4.63, 5.38] -> bz in {4, 5}; x = 0.0123 -> bx 0.
    keys = frame_block_keys(depth, K, _pose(np.eye(3), (0.0123, 0.0071, 0.0037)), P)
    assert keys == {(0, 0, 0, 4), (0, 0, 0, 5)}
    # A negative x offset must floor to block -1, not truncate to 0.
    keys = frame_block_keys(depth, K, _pose(np.eye(3), (-0.0123, 0.0071, 0.0037)), P, segment=3)
    assert keys == {(3, -1, 0, 4), (3, -1, 0, 5)}
    # mu = 1.0: N = 20 samples each side, z + 0.0037 in [3.0037, 5.0037] -> bz 3..6.
    keys = frame_block_keys(depth, K, _pose(np.eye(3), (0.0123, 0.0071, 0.0037)), Params(mu=1.0))
    assert keys == {(0, 0, 0, b) for b in (3, 4, 5, 6)}


def test_alloc_invalid_pixels_allocate_nothing():
    K = Intrinsics(100.0, 100.0, 2.0, 1.0, 4, 2)
    depth = np.array([[0.0, -1.0, np.nan, np.inf], [-np.inf, 0.0, -0.0, 0.0]], np.float32)
    assert frame_block_keys(depth, K, np.eye(4), P) == set()


def test_alloc_matches_world_ray_march():
    """Blocks touched by samples of each pixel's world ray o + z*R*dir (a different
    evaluation order of the same geometry) equal the oracle's set."""
    rng = np.random.default_rng(5)
    K = Intrinsics(140.0, 95.0, 9.137, 6.291, 17, 11)   # fx != fy on purpose
    R = _rot(0.3, -0.2, 0.7)
    t = np.array([-3.21, 1.7, 0.4])
    T = _pose(R, t)
    depth = rng.uniform(0.2, 9.0, (K.height, K.width)).astype(np.float32)
    depth[rng.random(depth.shape) < 0.2] = 0.0
    ref = frame_block_keys(depth, K, T, P)
    s, mu = P.voxel_size, P.mu
    h = s / 2
    n_side = int(round(mu / h))
    brute = set()
    for y in range(K.height):
        for x in range(K.width):
            d = float(depth[y, x])
            if not d > 0:
                continue
            ray = R @ np.array([(x + 0.5 - K.cx) / K.fx, (y + 0.5 - K.cy) / K.fy, 1.0])
            for n in range(-n_side, n_side + 1):
                z = d + n * h
                if z <= 0:
                    continue
                g = t + z * ray
                brute.add((0,) + tuple(int(math.floor(c / (8 * s))) for c in g))
    assert brute == ref
    assert len(ref) > 30


# ----------------------------------------------------------------- fusion
def _fuse_one(depth, K, T, params=P, frames=1):
    g = SparseGrid(params)
    alloc_blocks(g, depth, K, T)
    for _ in range(frames):
        fuse_depth(g, depth, K, T)
    return g


def test_fuse_fronto_parallel_wall_closed_form():
    K = Intrinsics(60.0, 60.0, 20.137, 15.291, 40, 30)
    t = np.array([0.0123, 0.0071, 0.0037])
    Z0 = 6.0
    g = _fuse_one(np.full((K.height, K.width), Z0, np.float32), K, _pose(np.eye(3), t))
    pc = _voxel_centres(g) - t          # R = I
    zc = pc[:, 2]
    f, w = g.f.reshape(-1), g.w.reshape(-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        ax, ay = pc[:, 0] / zc, pc[:, 1] / zc
    # inside the viewing frustum by a clear margin, in front, within the band
    lo_x, hi_x = -K.cx / K.fx, (K.width - K.cx) / K.fx
    lo_y, hi_y = -K.cy / K.fy, (K.height - K.cy) / K.fy
    m = 1e-6
    inside = (zc > 0.05) & (ax > lo_x + m) & (ax < hi_x - m) & (ay > lo_y + m) & (ay < hi_y - m)
    outside = (zc <= 0) | (ax < lo_x - m) | (ax > hi_x + m) | (ay < lo_y - m) | (ay > hi_y + m)
    band = Z0 - zc >= -P.mu
    upd = inside & band
    assert upd.sum() > 1000
    np.testing.assert_array_equal(w[upd], 1.0)
    np.testing.assert_allclose(f[upd], np.minimum(1.0, (Z0 - zc[upd]) / P.mu), rtol=0, atol=1e-12)
    assert np.all(w[outside | (inside & (Z0 - zc < -P.mu - 1e-9))] == 0)


def test_fuse_ground_plane_closed_form():
    K = Intrinsics(80.0, 80.0, 30.137, 20.291, 60, 40)
    t = np.array([0.0123, 0.0071, 0.0037])
    h = 1.65 - t[1]
    rows = np.arange(K.height) + 0.5 - K.cy
    d_row = np.where(rows > 0, h * K.fy / np.where(rows > 0, rows, 1), 0.0)
    d_row[d_row > 25] = 0
    depth32 = np.repeat(d_row[:, None], K.width, axis=1).astype(np.float32)
    g = _fuse_one(depth32, K, _pose(np.eye(3), t))
    pc = _voxel_centres(g) - t
    f, w = g.f.reshape(-1), g.w.reshape(-1)
    sel = (w == 1) & (f < 1.0 - 1e-9)
    assert sel.sum() > 100
    d_read = pc[sel, 2] + P.mu * f[sel]
    # the depth read must be the stored depth of the row whose cell holds the voxel's ray
    ang = pc[sel, 1] / pc[sel, 2]
    r = np.round(h * K.fy / d_read + K.cy - 0.5).astype(int)
    assert np.all(ang >= (r - K.cy) / K.fy - 1e-12) and np.all(ang < (r + 1 - K.cy) / K.fy + 1e-12)
    np.testing.assert_allclose(d_read, depth32[r, 0].astype(np.float64), rtol=0, atol=1e-9)


def test_fuse_side_wall_columns_closed_form():
    K = Intrinsics(70.0, 70.0, 25.137, 10.291, 50, 20)
    t = np.array([0.0123, 0.0071, 0.0037])
    X0 = 3.0
    hx = X0 - t[0]
    cols = np.arange(K.width) + 0.5 - K.cx
    d_col = np.where(cols > 0, hx * K.fx / np.where(cols > 0, cols, 1), 0.0)
    d_col[d_col > 25] = 0
    depth32 = np.repeat(d_col[None, :], K.height, axis=0).astype(np.float32)
    g = _fuse_one(depth32, K, _pose(np.eye(3), t))
    pc = _voxel_centres(g) - t
    f, w = g.f.reshape(-1), g.w.reshape(-1)
    sel = (w == 1) & (f < 1.0 - 1e-9)
    assert sel.sum() > 100
    d_read = pc[sel, 2] + P.mu * f[sel]
    ang = pc[sel, 0] / pc[sel, 2]
    c = np.round(hx * K.fx / d_read + K.cx - 0.5).astype(int)
    assert np.all(ang >= (c - K.cx) / K.fx - 1e-12) and np.all(ang < (c + 1 - K.cx) / K.fx + 1e-12)
    np.testing.assert_allclose(d_read, depth32[0, c].astype(np.float64), rtol=0, atol=1e-9)


def test_fuse_single_pixel_cone_rotated_camera():
    """Only voxels inside the one valid pixel's viewing cone and within the band are
    updated; the camera frame comes from a library matrix inverse of the pose."""
    K = Intrinsics(50.0, 45.0, 10.137, 8.291, 20, 16)
    R = _rot(0.25, -0.4, 0.9)
    t = np.array([1.3, -0.7, 2.2])
    T = _pose(R, t)
    px0, py0, d0 = 13, 5, 3.3
    depth = np.zeros((K.height, K.width), np.float32)
    depth[py0, px0] = d0
    g = _fuse_one(depth, K, T)
    pg = _voxel_centres(g)
    Tinv = np.linalg.inv(T)
    pc = pg @ Tinv[:3, :3].T + Tinv[:3, 3]
    zc = pc[:, 2]
    ax, ay = pc[:, 0] / zc, pc[:, 1] / zc
    m = 1e-9
    in_cone = (zc > 0) & (ax > (px0 - K.cx) / K.fx + m) & (ax < (px0 + 1 - K.cx) / K.fx - m) \
        & (ay > (py0 - K.cy) / K.fy + m) & (ay < (py0 + 1 - K.cy) / K.fy - m)
    out_cone = (zc <= 0) | (ax < (px0 - K.cx) / K.fx - m) | (ax > (px0 + 1 - K.cx) / K.fx + m) \
        | (ay < (py0 - K.cy) / K.fy - m) | (ay > (py0 + 1 - K.cy) / K.fy + m)
    band = float(np.float32(d0)) - zc >= -P.mu
    f, w = g.f.reshape(-1), g.w.reshape(-1)
    upd = in_cone & band
    assert upd.sum() >= 1
    np.testing.assert_array_equal(w[upd], 1.0)
    np.testing.assert_allclose(f[upd], np.minimum(1.0, (float(np.float32(d0)) - zc[upd]) / P.mu), atol=1e-9)
    assert np.all(w[out_cone] == 0)


def test_fuse_repeated_identical_frames():
    K = Intrinsics(60.0, 60.0, 20.137, 15.291, 40, 30)
    T = _pose(np.eye(3), (0.0123, 0.0071, 0.0037))
    depth = np.full((K.height, K.width), 5.0, np.float32)
    g1 = _fuse_one(depth, K, T, frames=1)
    g5 = _fuse_one(depth, K, T, frames=5)
    np.testing.assert_array_equal(g5.w, 5 * g1.w)
    np.testing.assert_allclose(g5.f, g1.f, atol=1e-14)


def test_alloc_block_order_is_sorted_per_call():
    K = Intrinsics(60.0, 60.0, 20.137, 15.291, 40, 30)
    T = _pose(_rot(0.1, 0.2, -0.3), (0.3, -0.2, 0.1))
    depth = np.random.default_rng(1).uniform(1, 6, (30, 40)).astype(np.float32)
    g = SparseGrid(P)
    n = alloc_blocks(g, depth, K, T, segment=2)
    keys = [(k[0], k[3], k[2], k[1]) for k in g.keys]
    assert n == len(keys) and keys == sorted(keys)
    assert len(set(g.keys)) == n


def test_fuse_invalid_depths_update_nothing():
    """Pixels whose depth is not a finite positive number carry no observation: voxels
    just in front of the camera (z_c below mu, where a depth of 0 would pass Eq. 1's
    truncation test) stay unobserved under a map of zeros, negatives, NaN and infinities."""
    K = Intrinsics(60.0, 60.0, 20.137, 15.291, 40, 30)
    T = _pose(np.eye(3), (0.0123, 0.0071, 0.0037))
    g = SparseGrid(P)
    g.add_blocks([(0, bx, by, 0) for by in (-1, 0) for bx in (-1, 0)])
    depth = np.zeros((K.height, K.width), np.float32)
    depth[::3] = -1.0
    depth[1::5] = np.nan
    depth[:, ::7] = np.inf
    depth[2::6, 1::4] = -0.0
    mask = fuse_depth(g, depth, K, T)
    assert not mask.any() and np.all(g.w == 0) and np.all(g.f == 0)
    # the same blocks do see a valid map: the voxels in front of the camera are reachable
    fuse_depth(g, np.full((K.height, K.width), 0.5, np.float32), K, T)
    assert np.count_nonzero(g.w) > 40


def test_fuse_touches_its_own_segment_only():
    """Segments are separate maps that share the hash: a depth map fused into segment 1
    leaves segment 0's blocks at the same coordinates untouched, and gives segment 1
    what a map holding only those blocks gets."""
    K = Intrinsics(60.0, 60.0, 20.137, 15.291, 40, 30)
    T = _pose(_rot(0.05, -0.1, 0.02), (0.0123, 0.0071, 0.0037))
    depth = np.random.default_rng(7).uniform(2.0, 4.0, (K.height, K.width)).astype(np.float32)
    alone = SparseGrid(P)
    alloc_blocks(alone, depth, K, T, segment=1)
    both = SparseGrid(P)
    both.add_blocks([(0,) + tuple(k[1:]) for k in alone.keys] + list(alone.keys))
    fuse_depth(alone, depth, K, T, segment=1)
    fuse_depth(both, depth, K, T, segment=1)
    n = alone.n_blocks
    assert np.all(both.w[:n] == 0) and np.all(both.f[:n] == 0)
    assert np.array_equal(both.w[n:], alone.w) and np.array_equal(both.f[n:], alone.f)
    assert np.count_nonzero(alone.w) > 1000


def test_pipeline_allocates_before_it_fuses():
    """Section III-A takes each depth map through allocation and then fusion, so a single
    map already observes the blocks it allocates: the pipeline of one wall map gives the
    wall's closed-form field."""
    K = Intrinsics(60.0, 60.0, 20.137, 15.291, 40, 30)
    T = _pose(np.eye(3), (0.0123, 0.0071, 0.0037))
    depth = np.full((K.height, K.width), 6.0, np.float32)
    g = run_pipeline([depth], K, [T], P, 0)
    ref = _fuse_one(depth, K, T)
    assert g.keys == ref.keys and np.array_equal(g.w, ref.w) and np.array_equal(g.f, ref.f)
    assert np.count_nonzero(g.w) > 1000
