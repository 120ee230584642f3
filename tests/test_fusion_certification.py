"""Soundness of the fusion kernel's float32 certification, on the CPU.

The fusion kernel (Section III-A, Eq. 1) takes each voxel's integer decisions (in front
of the camera, inside the image, which pixel, u_SDF >= -mu) in float32 together with a
forward error bound (one projection bound shared by a block's voxels where the block
lies clear of the camera plane, else per voxel), and recomputes the voxel in float64
only when the bound cannot decide.  This test restates that float32 path in numpy (float32 operations round to
nearest like the GPU's; fused multiply-adds are rounded once, exactly) and checks, on
random poses far from the origin and on depth maps whose neighbouring pixels disagree
(so that a wrong pixel shows), that every decision it certifies is the oracle's
float64 decision, and that it leaves few voxels undecided.  No GPU.
"""

import numpy as np
import pytest

from oracle import denser_oracle as O
from tests.oracle_helpers import grid_from_blocks

F32 = np.float32
EPS22 = F32(2.0 ** -22)
EPS23 = F32(2.0 ** -23)


def fma32(a, b, c):
    """float32 fma(a, b, c) rounded once: the product of two float32 values is exact in
    float64; the sum's float64 rounding error is recovered exactly (two-sum), and only a
    float64 sum that sits exactly halfway between two float32 values needs it."""
    p = np.asarray(a, np.float64) * np.asarray(b, np.float64)
    c = np.asarray(c, np.float64)
    s = p + c
    bp = s - c
    err = (p - bp) + (c - (s - bp))
    r = s.astype(F32)
    lo = np.where(r.astype(np.float64) <= s, r, np.nextafter(r, F32(-np.inf)))
    hi = np.nextafter(lo, F32(np.inf))
    mid = (lo.astype(np.float64) + hi.astype(np.float64)) * 0.5
    at_mid = (s == mid) & (err != 0)
    return np.where(at_mid, np.where(err > 0, hi, lo), r).astype(F32)


def rcp32(z, ulps=0):
    """float32 reciprocal: the correctly rounded value (float64 quotient rounded to float32;
    a tie would need 1/z within 2^-53 of a float32 midpoint, which a float32 z cannot
    give) moved by `ulps` units in the last place.  The kernel uses the hardware's
    approximate reciprocal, within 1 ulp of 1/z: one of the values at -1, 0, +1."""
    r = (1.0 / np.asarray(z, np.float64)).astype(F32)
    for _ in range(abs(ulps)):
        r = np.nextafter(r, F32(np.inf) if ulps > 0 else F32(-np.inf))
    return r.astype(F32)


# the approximate reciprocal's possible values: 1/z at -1, 0 or +1 ulp, and 1/(z - dz)
# one ulp low (the smaller bound; a larger one only defers more voxels)
RCP_CASES = [(-1, -1), (0, -1), (1, -1)]


def floor32(v):
    return np.floor(np.asarray(v, F32)).astype(np.int64)


def shared_bound(hi, lo, dl, M, sf, fxf, fyf, cxf, cyf, rcp_ulps):
    """The projection-error bounds (x, y) shared by a block's voxels, per block ([nb] each;
    -1 where the block reaches too close to the camera plane), in the origin kernel's
    float32 operations."""
    up, eps22 = F32(1.00000095), EPS22
    s25 = F32(F32(25.0) * sf)
    X = []
    for r in range(3):
        ext = F32(F32(7.0) * F32(F32(abs(M[3 * r]) + abs(M[3 * r + 1])) + abs(M[3 * r + 2])))
        X.append(F32(F32(F32(np.abs(hi[r]) + np.abs(lo[r])) + ext) * up))
    dxb, dyb, dzb = [fma32(eps22, F32(Xr + s25), dl) for Xr in X]
    mneg = F32(F32(7.0) * F32(F32(min(M[6], F32(0)) + min(M[7], F32(0))) + min(M[8], F32(0))))
    zlo = F32(F32(F32(hi[2] + lo[2]) + mneg) - F32(F32(4.76837158e-7) * X[2]))
    gap = F32(zlo - dzb)
    ok = gap > F32(1e-30)
    izb = F32(rcp32(np.where(ok, gap, F32(1)), rcp_ulps) * up)
    izl = F32(rcp32(np.where(ok, zlo, F32(1)), rcp_ulps) * up)
    rxb, ryb = F32(F32(X[0] * izl) * up), F32(F32(X[1] * izl) * up)
    cx, cy = abs(cxf), abs(cyf)
    pxb, pyb = F32(fma32(fxf, rxb, cx) * up), F32(fma32(fyf, ryb, cy) * up)
    ex = F32(F32(F32(F32(F32(fxf * fma32(rxb, dzb, dxb)) * izb) * F32(1.01))
                 + F32(F32(eps22 * F32(fxf * rxb)) + F32(EPS23 * F32(pxb + cx)))) + F32(1e-6))
    ey = F32(F32(F32(F32(F32(fyf * fma32(ryb, dzb, dyb)) * izb) * F32(1.01))
                 + F32(F32(eps22 * F32(fyf * ryb)) + F32(EPS23 * F32(pyb + cy)))) + F32(1e-6))
    return (np.where(ok, F32(ex * up), F32(-1)).astype(F32), np.where(ok, F32(ey * up), F32(-1)).astype(F32))


def kernel_decisions(keys, depth, K, T, prm, rcp=(0, 0), with_shared=False, bound_scale=1.0):
    """The float32 path of the fusion kernel for every voxel of `keys`: (decided, update,
    u_tsdf) per voxel, each [nb, 512] (with_shared: also which blocks take the bound
    shared by their voxels).  rcp: the ulp offsets of the two reciprocals (1/z,
    1/(z - dz)) from their correctly rounded values.  bound_scale multiplies the pixel and
    truncation bounds (1: the kernel's; 0 only to show that the checks below catch an
    unsound bound)."""
    s = prm.voxel_size
    Ri, ti = O.pose_inverse(T)
    keys = np.asarray(keys, np.int64)
    nb = len(keys)
    # the block's float64 origin as a float32 hi/lo pair with its bound
    g = [(keys[:, a].astype(np.float64) * 8.0 + 0.5) * s for a in (1, 2, 3)]
    c0 = [((Ri[r, 0] * g[0] + Ri[r, 1] * g[1]) + Ri[r, 2] * g[2]) + ti[r] for r in range(3)]
    hi = [c.astype(F32) for c in c0]
    lo = [(c0[r] - hi[r].astype(np.float64)).astype(F32) for r in range(3)]
    amax = np.max(np.abs(np.stack(c0)), axis=0)
    gmax = (8.0 * np.abs(keys[:, 1:]).sum(axis=1) + 24.0) * s
    dl = np.ldexp(amax + gmax + np.abs(ti).sum() + 1.0, -44).astype(F32)[:, None]
    M = (Ri * s).astype(F32).reshape(-1)
    l = np.arange(512)
    lxf, lyf, lzf = (l % 8).astype(F32), ((l // 8) % 8).astype(F32), (l // 64).astype(F32)
    myz = [fma32(M[3 * r + 1], lyf, M[3 * r + 2] * lzf) for r in range(3)]
    m = [fma32(M[3 * r], lxf, myz[r]) for r in range(3)]
    x, y, z = [((hi[r][:, None] + m[r][None, :]) + lo[r][:, None]).astype(F32) for r in range(3)]
    sf = F32(s)
    s25 = F32(25.0) * sf
    dx, dy, dz = [fma32(EPS22, (np.abs(v) + s25).astype(F32), dl) for v in (x, y, z)]
    fxf, fyf, cxf, cyf = F32(K.fx), F32(K.fy), F32(K.cx), F32(K.cy)
    muf, imuf = F32(prm.mu), F32(1.0 / prm.mu)
    Wf, Hf = F32(K.width), F32(K.height)

    decided = np.zeros((nb, 512), bool)
    upd = np.zeros((nb, 512), bool)
    ut = np.zeros((nb, 512), F32)
    with np.errstate(all="ignore"):
        # the bound the origin kernel shares among a block's voxels (shared_projection_bound),
        # every operation rounded as written there; its reciprocals one ulp low like 1/(z - dz)
        ex_sh, ey_sh = shared_bound(hi, lo, dl[:, 0], M, sf, fxf, fyf, cxf, cyf, rcp[1])
        ex_sh, ey_sh = ex_sh[:, None], ey_sh[:, None]
    shared = np.broadcast_to(ex_sh >= 0, (nb, 512))
    behind = ~shared & ((z + dz) <= 0)
    decided |= behind
    front = shared | ((z - dz) > 0)
    with np.errstate(all="ignore"):
        inv = rcp32(z, rcp[0])
        rx, ry = (x * inv).astype(F32), (y * inv).astype(F32)
        px, py = fma32(fxf, rx, cxf), fma32(fyf, ry, cyf)
        iz = rcp32((z - dz).astype(F32), rcp[1])
        ex = (fxf * (dx + np.abs(rx) * dz) * iz * F32(1.01) + EPS22 * (fxf * np.abs(rx))
              + EPS23 * (np.abs(px) + np.abs(cxf)) + F32(1e-6)).astype(F32)
        ey = (fyf * (dy + np.abs(ry) * dz) * iz * F32(1.01) + EPS22 * (fyf * np.abs(ry))
              + EPS23 * (np.abs(py) + np.abs(cyf)) + F32(1e-6)).astype(F32)
        ex = np.where(shared, ex_sh, ex).astype(F32)
        ey = np.where(shared, ey_sh, ey).astype(F32)
        ex, ey = (ex * F32(bound_scale)).astype(F32), (ey * F32(bound_scale)).astype(F32)
        outside = front & (((px + ex) < 0) | ((px - ex) >= Wf) | ((py + ey) < 0) | ((py - ey) >= Hf))
        decided |= outside
        small = (ex < F32(2.0 ** 20)) & (ey < F32(2.0 ** 20))
        pxi, pyi = floor32(px - ex), floor32(py - ey)
        pix_ok = front & ~outside & small & (pxi == floor32(px + ex)) & (pyi == floor32(py + ey))
        d = depth[np.clip(pyi, 0, K.height - 1), np.clip(pxi, 0, K.width - 1)].astype(F32)
        invalid = pix_ok & ~(np.isfinite(d) & (d > 0))
        decided |= invalid
        dh = (d - hi[2][:, None]).astype(F32)
        us = ((dh - m[2][None, :]) - lo[2][:, None]).astype(F32)
        eu = (EPS22 * (np.abs(dh) + np.abs(m[2][None, :]) + np.abs(us) + muf + s25) + dl + F32(1e-7)).astype(F32)
        eu = (eu * F32(bound_scale)).astype(F32)
        cert = pix_ok & ~invalid & (np.abs(us + muf) > eu)
        decided |= cert
        upd |= cert & (us >= -muf)
        ut = np.where(cert, np.minimum(F32(1.0), us * imuf), ut).astype(F32)
    if with_shared:
        return decided, upd, ut, ex_sh[:, 0] >= 0
    return decided, upd, ut


def random_pose(rng, far):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = rng.uniform(-far, far, 3)
    return T


@pytest.mark.parametrize("rcp", RCP_CASES)
@pytest.mark.parametrize("seed,far", [(0, 5.0), (1, 300.0), (2, 2000.0)])
def test_certified_decisions_are_the_oracles(seed, far, rcp):
    rng = np.random.default_rng(seed)
    prm = O.Params()
    W, H = 173, 61
    K = O.Intrinsics(float(rng.uniform(80, 400)), float(rng.uniform(80, 400)), float(rng.uniform(70, 100)),
                     float(rng.uniform(25, 35)), W, H)
    T = random_pose(rng, far)
    # depth maps whose neighbouring pixels disagree, with invalid pixels of both kinds
    depth = rng.uniform(0.5, 12.0, (H, W)).astype(F32)
    depth[rng.random((H, W)) < 0.1] = 0.0
    depth[rng.random((H, W)) < 0.05] = np.nan
    # blocks around points in the viewing frustum (and some behind the camera)
    n = 160
    u, v = rng.uniform(-5, W + 5, n), rng.uniform(-5, H + 5, n)
    zc = rng.uniform(-2.0, 13.0, n)
    pc = np.stack([(u - K.cx) * zc / K.fx, (v - K.cy) * zc / K.fy, zc])
    pg = T[:3, :3] @ pc + T[:3, 3:4]
    keys = sorted({(0,) + tuple(int(b) for b in np.floor(pg[:, i] / (8 * prm.voxel_size))) for i in range(n)})
    g = grid_from_blocks(keys)
    want = O.fuse_depth(g, depth, K, T)
    decided, upd, ut, shared = kernel_decisions(keys, depth, K, T, prm, rcp, with_shared=True)
    assert decided.mean() > 0.97, decided.mean()
    assert shared.mean() > 0.8, shared.mean()  # most blocks take the bound shared by their voxels
    np.testing.assert_array_equal(upd[decided], want[decided])
    both = decided & upd
    assert both.sum() > 1000
    assert np.max(np.abs(ut[both].astype(np.float64) - g.f[both])) <= 2e-6


def _lattice_case():
    """A camera on the voxel lattice: identity rotation, fx = fy = 100 px, principal point
    on a pixel edge.  Voxel centres ((i + 0.5) s, ...) then project to rational pixel
    coordinates, many of them exactly on a pixel edge in float64."""
    prm = O.Params()
    K = O.Intrinsics(100.0, 100.0, 80.0, 48.0, 160, 96)
    keys = [(0, bx, by, bz) for bz in range(0, 3) for by in range(-2, 2) for bx in range(-3, 3)]
    g = grid_from_blocks(keys)
    C = g.coords()
    l = np.arange(512)
    s = prm.voxel_size
    xc = ((C[:, 1:2] * 8 + l % 8) + 0.5) * s
    yc = ((C[:, 2:3] * 8 + (l // 8) % 8) + 0.5) * s
    zc = ((C[:, 3:4] * 8 + l // 64) + 0.5) * s
    px = np.floor(K.fx * xc / zc + K.cx).astype(np.int64)
    py = np.floor(K.fy * yc / zc + K.cy).astype(np.int64)
    return prm, K, keys, g, zc, px, py


@pytest.mark.parametrize("rcp", RCP_CASES)
def test_pixel_edges_are_deferred_or_right(rcp):
    """Projections on pixel edges, against a checkerboard of valid and invalid pixels:
    a pixel off by one in either direction flips the update."""
    prm, K, keys, g, zc, px, py = _lattice_case()
    yy, xx = np.mgrid[0:K.height, 0:K.width]
    depth = np.where((xx + yy) % 2 == 0, F32(20.0), F32(0.0)).astype(F32)
    want = O.fuse_depth(g, depth, K, np.eye(4))
    decided, upd, ut = kernel_decisions(keys, depth, K, np.eye(4), prm, rcp)
    assert 0.5 < decided.mean() < 1.0  # the edge cases are deferred to float64
    assert want.sum() > 2000
    np.testing.assert_array_equal(upd[decided], want[decided])


@pytest.mark.parametrize("rcp", RCP_CASES)
def test_truncation_edges_are_deferred_or_right(rcp):
    """Depths set to z - mu within a few float32 ulps put u_SDF on the truncation edge of
    Eq. 1 (one voxel per pixel)."""
    rng = np.random.default_rng(7)
    prm, K, keys, g, zc, px, py = _lattice_case()
    ok = (px >= 0) & (px < K.width) & (py >= 0) & (py < K.height)
    depth = rng.uniform(0.3, 3.0, (K.height, K.width)).astype(F32)
    sel = np.flatnonzero(ok.reshape(-1))
    rng.shuffle(sel)
    for f in sel:
        b, v = divmod(int(f), 512)
        depth[py[b, v], px[b, v]] = F32(zc[b, v] - prm.mu) + F32(rng.integers(-3, 4)) * F32(2.0 ** -22)
    want = O.fuse_depth(g, depth, K, np.eye(4))
    decided, upd, ut = kernel_decisions(keys, depth, K, np.eye(4), prm, rcp)
    assert 0.5 < decided.mean() < 1.0
    np.testing.assert_array_equal(upd[decided], want[decided])
    both = decided & upd
    assert np.max(np.abs(ut[both].astype(np.float64) - g.f[both])) <= 2e-6


def test_the_edge_cases_catch_an_unsound_bound():
    """The checks above have teeth: with no error bound (float32 decisions taken as
    final) the pixel-edge and truncation-edge cases certify decisions that differ from
    the oracle's."""
    prm, K, keys, g, zc, px, py = _lattice_case()
    yy, xx = np.mgrid[0:K.height, 0:K.width]
    depth = np.where((xx + yy) % 2 == 0, F32(20.0), F32(0.0)).astype(F32)
    want = O.fuse_depth(g, depth, K, np.eye(4))
    decided, upd, _ = kernel_decisions(keys, depth, K, np.eye(4), prm, bound_scale=0.0)
    assert np.any(upd[decided] != want[decided])
    rng = np.random.default_rng(7)
    ok = (px >= 0) & (px < K.width) & (py >= 0) & (py < K.height)
    depth = rng.uniform(0.3, 3.0, (K.height, K.width)).astype(F32)
    for f in np.flatnonzero(ok.reshape(-1)):
        b, v = divmod(int(f), 512)
        depth[py[b, v], px[b, v]] = F32(zc[b, v] - prm.mu) + F32(rng.integers(-3, 4)) * F32(2.0 ** -22)
    g2 = grid_from_blocks(keys)
    want = O.fuse_depth(g2, depth, K, np.eye(4))
    decided, upd, _ = kernel_decisions(keys, depth, K, np.eye(4), prm, bound_scale=0.0)
    assert np.any(upd[decided] != want[decided])
