"""Pins of the laser oracle (oracle/laser_oracle.py) to facts that do not come from it:

* an axis-aligned ray: every voxel from the sensor's to mu behind the hit, each once,
  with the closed-form u_SDF = r - (c_z - t_z) and f = min(1, u_SDF/mu);
* oblique rays: the voxels found lie in cells the ray segment crosses (slab test, an
  independent geometric routine) and include every cell the segment crosses for
  longer than h (such a chord must hold a sample);
* ray order does not change f or w (bit for bit), repeated rays give the same f;
* over scans, a voxel seen by one ray per scan follows Eq. 1 applied in turn;
* allocation along an axis-aligned ray is the closed-form block range; with only the
  band allocated, fusion reaches every voxel within mu of the hit, none more than mu
  behind it, and gives free-space voxels u_TSDF = 1;
* invalid points (NaN, infinite, zero range) are skipped.
"""

import numpy as np
import pytest

from oracle import denser_oracle as O
from oracle import laser_oracle as L

S_VOX = 0.1
T0 = np.eye(4)
T0[:3, 3] = (0.0123, 0.0071, 0.0037)


def box_grid(lo, hi, params=None):
    g = O.SparseGrid(params or O.Params())
    keys = [(0, x, y, z) for z in range(lo[2], hi[2]) for y in range(lo[1], hi[1]) for x in range(lo[0], hi[0])]
    g.add_blocks(keys)
    return g


def voxel_centre(flat, grid, s=S_VOX):
    b, l = flat // 512, flat % 512
    k = np.array(grid.keys)[b]
    ijk = k[:, 1:4] * 8 + np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    return (ijk + 0.5) * s, ijk


def test_ray_along_negative_x_closed_form():
    """Voxels with negative indices (floor, not truncation, to their blocks)."""
    g = box_grid((-6, -1, -1), (1, 1, 1))
    r = 2.3456
    cnt = L.fuse_scan(g, np.array([[-r, 0.0, 0.0]], np.float32), T0)
    flat = np.nonzero(cnt.reshape(-1))[0]
    c, ijk = voxel_centre(flat, g)
    t = T0[:3, 3]
    rr = float(np.float32(r))
    assert np.all(ijk[:, 1] == 0) and np.all(ijk[:, 2] == 0)
    k_far = int(np.floor((t[0] - np.floor((rr + 0.3) / 0.05) * 0.05) / S_VOX))
    expect = [k for k in range(k_far, int(np.floor(t[0] / S_VOX)) + 1) if rr - (t[0] - (k + 0.5) * S_VOX) >= -0.3]
    assert sorted(ijk[:, 0].tolist()) == expect and min(expect) < -8
    usdf = rr - (t[0] - c[:, 0])
    np.testing.assert_allclose(g.f.reshape(-1)[flat], np.minimum(1.0, usdf / 0.3), atol=2.0 ** -30)


@pytest.mark.parametrize("r", [3.4567, 3.448])
def test_axis_aligned_ray_closed_form(r):
    """With r = 3.448 the last sample (n = M = 74, at z = t_z + 3.7) is the first one in
    its voxel, whose centre is still within mu of the hit: the walk must reach it."""
    g = box_grid((-1, -1, -1), (1, 1, 8))
    cnt = L.fuse_scan(g, np.array([[0.0, 0.0, r]], np.float32), T0)
    flat = np.nonzero(cnt.reshape(-1))[0]
    c, ijk = voxel_centre(flat, g)
    t = T0[:3, 3]
    # the ray is the line x = t_x, y = t_y: one column of voxels
    assert np.all(ijk[:, 0] == int(np.floor(t[0] / S_VOX))) and np.all(ijk[:, 1] == int(np.floor(t[1] / S_VOX)))
    rr = float(np.float32(r))
    k0 = int(np.floor(t[2] / S_VOX))
    k_end = int(np.floor((t[2] + np.floor((rr + 0.3) / 0.05) * 0.05) / S_VOX))
    usdf = rr - (c[:, 2] - t[2])
    expect = [k for k in range(k0, k_end + 1) if rr - ((k + 0.5) * S_VOX - t[2]) >= -0.3]
    assert sorted(ijk[:, 2].tolist()) == expect
    assert np.all(cnt.reshape(-1)[flat] == 1)
    np.testing.assert_allclose(g.f.reshape(-1)[flat], np.minimum(1.0, usdf / 0.3), atol=2.0 ** -30)


def slab_chord(p0, p1, lo, hi):
    """Length of the segment p0-p1 inside the box [lo, hi] (slab method)."""
    d = p1 - p0
    t0, t1 = 0.0, 1.0
    for a in range(3):
        if abs(d[a]) < 1e-300:
            if p0[a] < lo[a] or p0[a] >= hi[a]:
                return 0.0
            continue
        ta, tb = (lo[a] - p0[a]) / d[a], (hi[a] - p0[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0) * np.linalg.norm(d)


def test_oblique_rays_against_slab_geometry():
    rng = np.random.default_rng(0)
    p = O.Params()
    h = 0.5 * S_VOX
    T = T0.copy()
    a = 0.3
    T[:3, :3] = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        pt = (d * rng.uniform(0.5, 2.0)).astype(np.float32)
        valid, r, dg, t = L.ray_setup(pt[None], T)
        # the global direction is R p / |p|, by a library matrix product
        np.testing.assert_allclose(dg[0], T[:3, :3] @ (pt.astype(np.float64) / np.linalg.norm(pt.astype(np.float64))),
                                   atol=1e-15)
        v = L.ray_voxels(r[0], dg[0], t, p)
        assert len(np.unique(v, axis=0)) == len(v)  # each voxel once
        p0 = t
        p1 = t + dg[0] * (np.floor((r[0] + p.mu) / h) * h)
        found = {tuple(x) for x in v.tolist()}
        lo = np.floor(np.minimum(p0, p1) / S_VOX).astype(int) - 1
        hi = np.floor(np.maximum(p0, p1) / S_VOX).astype(int) + 2
        for i in range(lo[0], hi[0]):
            for j in range(lo[1], hi[1]):
                for k in range(lo[2], hi[2]):
                    cell_lo = np.array([i, j, k]) * S_VOX
                    chord = slab_chord(p0, p1, cell_lo, cell_lo + S_VOX)
                    if (i, j, k) in found:
                        assert chord > 0 or np.allclose(p0, p1)
                    elif chord > h + 1e-9:
                        pytest.fail(f"cell {(i, j, k)} crossed for {chord} m but not found")


def test_ray_order_and_repeats():
    sc_pts = np.array([[0.3, -0.2, 2.5], [0.1, 0.05, 2.7], [-0.2, 0.1, 2.6], [0.0, 0.0, 2.65]], np.float32)
    g1 = box_grid((-2, -2, -1), (2, 2, 6))
    g2 = box_grid((-2, -2, -1), (2, 2, 6))
    L.fuse_scan(g1, sc_pts, T0)
    L.fuse_scan(g2, sc_pts[::-1].copy(), T0)
    assert np.array_equal(g1.w, g2.w) and np.array_equal(g1.f, g2.f)
    g3 = box_grid((-2, -2, -1), (2, 2, 6))
    L.fuse_scan(g3, np.repeat(sc_pts[:1], 3, axis=0), T0)
    g4 = box_grid((-2, -2, -1), (2, 2, 6))
    L.fuse_scan(g4, sc_pts[:1], T0)
    hit = g4.w > 0
    assert np.array_equal(g3.w[hit], 3 * g4.w[hit]) and np.array_equal(g3.w > 0, hit)
    np.testing.assert_allclose(g3.f[hit], g4.f[hit], atol=2.0 ** -29)


def test_scans_follow_eq1_in_turn():
    g = box_grid((-1, -1, -1), (1, 1, 8))
    ranges = [3.40, 3.47, 3.52, 3.44]
    f_ref = {}
    w_ref = {}
    t = T0[:3, 3]
    for r in ranges:
        rr = float(np.float32(r))
        cnt = L.fuse_scan(g, np.array([[0.0, 0.0, r]], np.float32), T0)
        for fl in np.nonzero(cnt.reshape(-1))[0]:
            c, _ = voxel_centre(np.array([fl]), g)
            u = min(1.0, (rr - (c[0, 2] - t[2])) / 0.3)
            w0 = w_ref.get(fl, 0.0)
            f_ref[fl] = (u + w0 * f_ref.get(fl, 0.0)) / (w0 + 1)  # Eq. 1
            w_ref[fl] = w0 + 1
    for fl, f in f_ref.items():
        assert g.w.reshape(-1)[fl] == w_ref[fl]
        assert abs(g.f.reshape(-1)[fl] - f) <= 1e-8


def test_allocation_band_axis_aligned():
    p = O.Params()
    t = T0[:3, 3]
    bs = 0.8
    # the last band samples (n = -6 and n = +6) are the only ones in their blocks
    for r in (5.4321, 6.4 - 0.0037 - 0.29, 4.8 - 0.0037 + 0.29):
        rr = float(np.float32(r))
        keys = L.scan_block_keys(np.array([[0.0, 0.0, r]], np.float32), T0, p)
        z_lo, z_hi = t[2] + rr - 6 * 0.05, t[2] + rr + 6 * 0.05
        expect = {(0, int(np.floor(t[0] / bs)), int(np.floor(t[1] / bs)), bz)
                  for bz in range(int(np.floor(z_lo / bs)), int(np.floor(z_hi / bs)) + 1)}
        assert keys == expect, r
    # a point closer than mu: band samples at or behind the sensor (rho <= 0) allocate
    # nothing, so the block just behind the sensor (z < 0, the sensor at z = 0.0037) is
    # not taken
    keys = L.scan_block_keys(np.array([[0.0, 0.0, 0.1]], np.float32), T0, p)
    assert keys == {(0, 0, 0, 0)}
    r = 5.4321
    rr = float(np.float32(r))
    keys = L.scan_block_keys(np.array([[0.0, 0.0, r]], np.float32), T0, p)
    expect = keys
    # with only the band allocated, fusion updates every voxel of the ray within mu of
    # the hit (they lie in band blocks), nothing more than mu behind it, and in front
    # only voxels of the same blocks (free space, u_TSDF = 1)
    g = O.SparseGrid(p)
    assert L.alloc_scan(g, np.array([[0.0, 0.0, r]], np.float32), T0) == len(expect)
    cnt = L.fuse_scan(g, np.array([[0.0, 0.0, r]], np.float32), T0)
    c, ijk = voxel_centre(np.nonzero(cnt.reshape(-1))[0], g)
    usdf = rr - (c[:, 2] - t[2])
    assert np.all(usdf >= -0.3)
    k_hit = [k for k in range(int(np.floor((t[2] + rr - 0.3) / S_VOX)), int(np.floor((t[2] + rr + 0.3) / S_VOX)) + 1)
             if abs(rr - ((k + 0.5) * S_VOX - t[2])) <= 0.3 - 1e-9]
    assert set(k_hit) <= set(ijk[:, 2].tolist())
    assert np.all(np.floor(ijk[:, 2] / 8) >= min(k[3] for k in expect))
    np.testing.assert_allclose(g.f.reshape(-1)[np.nonzero(cnt.reshape(-1))[0]][usdf >= 0.3], 1.0)


def test_invalid_points_are_skipped():
    g = box_grid((-2, -2, -1), (2, 2, 6))
    # NaN, zero range, infinite, and beyond the 2^22-sample range limit (about 210 km)
    pts = np.array([[np.nan, 0, 1], [0, 0, 0], [np.inf, 1, 1], [0, 0, 3.0e5]], np.float32)
    assert L.alloc_scan(O.SparseGrid(O.Params()), pts, T0) == 0
    cnt = L.fuse_scan(g, pts, T0)
    assert cnt.sum() == 0 and np.all(g.w == 0)


def test_scan_touches_its_own_segment_and_orders_new_blocks():
    """A scan fused into segment 2 leaves the same blocks of segment 0 untouched and gives
    segment 2 what a map holding only those blocks gets; the blocks a scan allocates are
    appended in ascending (segment, bz, by, bx) order."""
    rng = np.random.default_rng(12)
    pts = (rng.standard_normal((60, 3)) * np.array([1.5, 0.6, 0.4]) + np.array([0.0, 0.5, 4.0])).astype(np.float32)
    T = T0.copy()
    alone = O.SparseGrid(O.Params())
    n = L.alloc_scan(alone, pts, T, segment=2)
    keys = [(k[0], k[3], k[2], k[1]) for k in alone.keys]
    assert n == len(keys) > 4 and keys == sorted(keys)
    both = O.SparseGrid(O.Params())
    both.add_blocks([(0,) + tuple(k[1:]) for k in alone.keys] + list(alone.keys))
    L.fuse_scan(alone, pts, T, segment=2)
    L.fuse_scan(both, pts, T, segment=2)
    assert np.all(both.w[:n] == 0) and np.array_equal(both.w[n:], alone.w) and np.array_equal(both.f[n:], alone.f)
    assert np.count_nonzero(alone.w) > 100
