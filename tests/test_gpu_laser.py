"""Laser scans through the C ABI against the oracle (oracle/laser_oracle.py).

Allocation (block keys, indices) and the per-voxel observation counts w are bit-exact;
f within 1e-5 (float32 signed distances and float32 storage against float64).  Ray
order does not change anything (fixed-point sums).  At full size (64 x 2000-ray scans of
the 100 m street) the allocation is compared whole, and fusion on sampled blocks with
the oracle fed exactly the rays whose sample segment crosses each block.
"""

import numpy as np
import pytest

from oracle import denser_oracle as O
from oracle import laser_oracle as L
from synth.scenes import Lidar, street_scene, tiny_scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import native as N  # noqa: E402

N.lib()
F_TOL = 1e-5
SMALL = Lidar(beams=16, azimuths=256)


def scans(scene, lidar, frames):
    return [np.ascontiguousarray(scene.lidar_scan(k, lidar)) for k in frames]


def run_both(scene, pts_list, frames, params=None, kind="device", **gpu_params):
    prm = params or O.Params()
    g = O.SparseGrid(prm)
    m = N.DenserMap(**gpu_params)
    news_o, news_g = [], []
    for pts, k in zip(pts_list, frames):
        T = scene.poses[k]
        news_o.append(L.alloc_scan(g, pts, T))
        L.fuse_scan(g, pts, T)
        p = torch.from_numpy(pts)
        p = p.cuda() if kind == "device" else (p.pin_memory() if kind == "pinned" else p)
        news_g.append(N.denser_integrate_points(m.ctx, p, T, 0, count=True))
    return g, m, news_o, news_g


@pytest.mark.parametrize("jitter", [0.0, 0.05])
def test_tiny_scans_parity(jitter):
    sc = tiny_scene(seed=1, yaw_jitter=jitter)
    frames = range(4)
    pts = scans(sc, SMALL, frames)
    g, m, news_o, news_g = run_both(sc, pts, frames)
    snap = m.snapshot()
    m.close()
    assert news_o == news_g and sum(news_o) > 50
    np.testing.assert_array_equal(snap["coords"], g.coords().astype(np.int32))
    np.testing.assert_array_equal(snap["w"], g.w.astype(np.float32))
    assert np.max(np.abs(snap["f"] - g.f)) <= F_TOL
    assert (g.w > 0).sum() > 5000


def test_host_inputs_and_separate_calls_agree():
    sc = tiny_scene(seed=2)
    frames = range(3)
    pts = scans(sc, SMALL, frames)
    ref = None
    for kind in ("device", "pinned", "pageable"):
        _, m, _, _ = run_both(sc, pts, frames, kind=kind)
        snap = m.snapshot()
        m.close()
        if ref is None:
            ref = snap
        for key in ("coords", "f", "w"):
            np.testing.assert_array_equal(snap[key], ref[key], err_msg=kind)
    with N.DenserMap() as m:
        for pts_k, k in zip(pts, frames):
            N.denser_alloc_points(m.ctx, torch.from_numpy(pts_k).cuda(), sc.poses[k])
            N.denser_fuse_points(m.ctx, torch.from_numpy(pts_k).cuda(), sc.poses[k])
        snap = m.snapshot()
    for key in ("coords", "f", "w"):
        np.testing.assert_array_equal(snap[key], ref[key])


def test_ray_order_does_not_matter():
    sc = tiny_scene(seed=3)
    pts = scans(sc, SMALL, [0])[0]
    perm = np.random.default_rng(0).permutation(len(pts))
    outs = []
    for p in (pts, np.ascontiguousarray(pts[perm])):
        with N.DenserMap() as m:
            N.denser_integrate_points(m.ctx, torch.from_numpy(p).cuda(), sc.poses[0])
            outs.append(m.snapshot())
    for key in ("coords", "f", "w"):
        np.testing.assert_array_equal(outs[0][key], outs[1][key])


def test_depth_and_laser_in_one_map_then_regularize():
    sc = tiny_scene(seed=4)
    d = sc.depth_maps()
    pts = scans(sc, SMALL, [2, 3])
    cam = sc.camera
    Ko = O.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    g = O.SparseGrid(O.Params())
    with N.DenserMap() as m:
        K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        for k in range(2):
            O.alloc_blocks(g, d[k], Ko, sc.poses[k])
            O.fuse_depth(g, d[k], Ko, sc.poses[k])
            N.denser_integrate(m.ctx, torch.from_numpy(d[k]).cuda(), K, sc.poses[k])
        for p, k in zip(pts, [2, 3]):
            L.alloc_scan(g, p, sc.poses[k])
            L.fuse_scan(g, p, sc.poses[k])
            N.denser_integrate_points(m.ctx, torch.from_numpy(p).cuda(), sc.poses[k])
        O.regularize(g, 30)
        N.denser_regularize(m.ctx, 30)
        snap = m.snapshot()
    np.testing.assert_array_equal(snap["coords"], g.coords().astype(np.int32))
    np.testing.assert_array_equal(snap["w"], g.w.astype(np.float32))
    assert np.max(np.abs(snap["u"] - g.u)) <= 1e-4


def test_edge_cases():
    sc = tiny_scene(seed=0)
    T = sc.poses[0]
    with N.DenserMap() as m:
        assert N.denser_integrate_points(m.ctx, np.zeros((0, 3), np.float32), T, count=True) == 0
        bad = np.array([[np.nan, 0, 1], [0, 0, 0], [np.inf, 1, 1], [0, 0, 3.0e5], [0, 0, -np.inf]], np.float32)
        assert N.denser_integrate_points(m.ctx, bad, T, count=True) == 0
        assert N.denser_num_blocks(m.ctx) == 0
        with pytest.raises(N.DenserError):
            N.denser_integrate_points(m.ctx, bad, T, segment=200)
        T_bad = T.copy()
        T_bad[0, 0] = np.nan
        with pytest.raises(N.DenserError):
            N.denser_integrate_points(m.ctx, bad, T_bad)
        # one ray straight ahead, then the same ray again: w counts both scans
        ray = np.array([[0.0, 0.0, 3.4567]], np.float32)
        N.denser_integrate_points(m.ctx, ray, T)
        N.denser_integrate_points(m.ctx, ray, T)
        snap = m.snapshot()
    g = O.SparseGrid(O.Params())
    for _ in range(2):
        L.alloc_scan(g, ray, T)
        L.fuse_scan(g, ray, T)
    np.testing.assert_array_equal(snap["w"], g.w.astype(np.float32))
    assert set(np.unique(snap["w"]).tolist()) == {0.0, 2.0}
    assert np.max(np.abs(snap["f"] - g.f)) <= F_TOL


def crossing_rays(pts, T, lo, hi, mu, h):
    """Indices of the rays whose sample segment [t, t + dg (M h)] crosses the box
    [lo, hi] (slab test, vectorised); a superset of the rays with a sample inside."""
    valid, r, dg, t = L.ray_setup(pts, T, O.Params())
    idx = np.nonzero(valid)[0]
    M = np.floor((r[idx] + mu) / h)
    p0 = np.broadcast_to(t, (len(idx), 3))
    d = dg[idx] * (M * h)[:, None]
    t0 = np.zeros(len(idx))
    t1 = np.ones(len(idx))
    with np.errstate(divide="ignore", invalid="ignore"):
        for a in range(3):
            ta = (lo[a] - p0[:, a]) / d[:, a]
            tb = (hi[a] - p0[:, a]) / d[:, a]
            par = d[:, a] == 0
            inside = (p0[:, a] >= lo[a]) & (p0[:, a] <= hi[a])
            tmin = np.where(par, np.where(inside, -np.inf, np.inf), np.minimum(ta, tb))
            tmax = np.where(par, np.where(inside, np.inf, -np.inf), np.maximum(ta, tb))
            t0 = np.maximum(t0, tmin)
            t1 = np.minimum(t1, tmax)
    return idx[t0 <= t1]


def test_fullsize_street_scans():
    sc = street_scene(seed=0)
    lid = Lidar()
    frames = [0, 20, 40]
    pts = scans(sc, lid, frames)
    prm = O.Params()
    g = O.SparseGrid(prm)
    nb_after = []
    with N.DenserMap(max_blocks=1 << 16) as m:
        for p, k in zip(pts, frames):
            n_o = L.alloc_scan(g, p, sc.poses[k])
            nb_after.append(g.n_blocks)
            assert N.denser_integrate_points(m.ctx, torch.from_numpy(p).cuda(), sc.poses[k], count=True) == n_o
        snap = m.snapshot()
    np.testing.assert_array_equal(snap["coords"], g.coords().astype(np.int32))
    nb = len(snap["coords"])
    assert nb > 2000 and len(pts[0]) == 128000
    # fusion on sampled blocks: the oracle sees exactly the rays that can reach them
    rng = np.random.default_rng(1)
    s, h = prm.voxel_size, 0.5 * prm.voxel_size
    checked = 0
    for b in rng.choice(nb, 12, replace=False):
        key = tuple(int(v) for v in snap["coords"][b])
        lo = np.array(key[1:4]) * 8 * s - s
        hi = lo + 10 * s
        g.w[b] = 0.0
        g.f[b] = 0.0
        for j, (p, k) in enumerate(zip(pts, frames)):
            if b >= nb_after[j]:
                continue  # not allocated yet when scan j was fused
            sel = crossing_rays(p, sc.poses[k], lo, hi, prm.mu, h)
            flat, u = L.scan_observations(g, p[sel], sc.poses[k])
            inb = flat // 512 == b
            loc = flat[inb] % 512
            cnt = np.bincount(loc, minlength=512).astype(np.float64)
            S = np.zeros(512, np.int64)
            np.add.at(S, loc, np.rint(u[inb] * L.FIX).astype(np.int64))
            upd = cnt > 0
            wn = g.w[b] + cnt
            g.f[b] = np.where(upd, (g.w[b] * g.f[b] + S / L.FIX) / np.where(upd, wn, 1.0), g.f[b])
            g.w[b] = wn
        np.testing.assert_array_equal(snap["w"][b], g.w[b].astype(np.float32))
        assert np.max(np.abs(snap["f"][b] - g.f[b])) <= F_TOL
        checked += int((g.w[b] > 0).sum())
    assert checked > 500
