"""Soundness of the allocation kernel's float32 key certification, on the CPU.

The allocation kernel (Section III-A, reading R1) finds the block keys of a ray's band
samples in float32: the certified floors at the band's two ends and, for each axis
whose floor changes, the first sample of each new floor (estimated from the line, then
confirmed by certified comparisons of q with the new floor's boundary on both sides).  Floors that the error bound cannot
certify send the ray to a per-sample walk, and samples that stay uncertified there to
float64.  This test restates the float32 path ray by ray in numpy (float32 operations
rounded to nearest, fused multiply-adds rounded once) and checks that every ray it
decides without float64 gets exactly the oracle's key set, on random poses far from
the origin and on a camera whose band samples fall exactly on block faces.  No GPU.
"""

import math

import numpy as np
import pytest

from oracle import denser_oracle as O
from tests.test_fusion_certification import fma32, random_pose

F32 = np.float32
MAGIC = F32(12582912.0)  # 1.5 2^23
COORD_BIAS = 1 << 18


def f32(v):
    return F32(v)


def fma(a, b, c):
    return F32(fma32(F32(a), F32(b), F32(c)))


def band_floor(dv, nf, hf, D, tf, e):
    """(floor of q = fma(fma(nf, hf, dv), D, tf), certified)."""
    q = fma(fma(nf, hf, dv), D, tf)
    tq = F32(q + MAGIC)
    nq = F32(tq - MAGIC)
    down = nq > q
    fr = F32(q - (F32(nq - F32(1)) if down else nq))
    return int(nq) - (1 if down else 0), bool(fr >= e and F32(F32(1) - fr) > e)


class Setup:
    def __init__(self, K, T, prm):
        self.h = 0.5 * prm.voxel_size
        self.bs = 8.0 * prm.voxel_size
        self.N = int(math.ceil(prm.mu / self.h - 1e-9))
        self.hf, self.nhf = f32(self.h), f32(self.N * self.h)
        self.ifx, self.ify, self.ibs = f32(1.0 / K.fx), f32(1.0 / K.fy), f32(1.0 / self.bs)
        self.cx_hi = f32(K.cx)
        self.cx_lo = f32(K.cx - float(self.cx_hi))
        self.cy_hi = f32(K.cy)
        self.cy_lo = f32(K.cy - float(self.cy_hi))
        T = np.asarray(T, np.float64)
        self.Rf = T[:3, :3].astype(F32).reshape(-1)
        tb = T[:3, 3] / self.bs
        self.Ti = [int(max(-2.0 * COORD_BIAS, min(2.0 * COORD_BIAS, math.floor(v)))) for v in tb]
        self.tf = [f32(tb[r] - self.Ti[r]) for r in range(3)]
        self.e_scale = F32(1)  # the kernel's bounds; 0 only to show the checks catch an unsound bound


def ray_keys(S, x, y, dv):
    """The float32 path for pixel (x, y) of depth dv: its key set, or None when some
    decision needs float64."""
    eps = F32(2.0 ** -20)
    ua = F32(F32(F32(F32(x) + F32(0.5)) - S.cx_hi) - S.cx_lo)
    va = F32(F32(F32(F32(y) + F32(0.5)) - S.cy_hi) - S.cy_lo)
    ax, ay = F32(ua * S.ifx), F32(va * S.ify)
    zmax, zmin = F32(dv + S.nhf), F32(dv - S.nhf)
    ez = F32(F32(eps * zmax + F32(1e-30)) * S.e_scale)
    D, e = [], []
    for r in range(3):
        R0, R1, R2 = S.Rf[3 * r], S.Rf[3 * r + 1], S.Rf[3 * r + 2]
        D.append(F32(fma(R0, ax, fma(R1, ay, R2)) * S.ibs))
        DA = F32(F32(F32(abs(F32(R0 * ax)) + abs(F32(R1 * ay))) + abs(R2)) * S.ibs)
        qm = max(abs(fma(zmin, D[r], S.tf[r])), abs(fma(zmax, D[r], S.tf[r])))
        if not qm < F32(2.0 ** 21):
            return None
        e.append(F32(fma(F32(1.25) * eps, F32(DA * F32(zmax + S.nhf)), F32(0.25) * eps * F32(qm + F32(1))) * S.e_scale))
    keys = events_path(S, dv, D, e, ez)
    return keys if keys is not None else per_sample_path(S, dv, D, e, ez)


def events_path(S, dv, D, e, ez):
    N = S.N
    if not fma(F32(-N), S.hf, dv) > ez:
        return None
    klo, khi = [], []
    for r in range(3):
        a, ok_a = band_floor(dv, F32(-N), S.hf, D[r], S.tf[r], e[r])
        b, ok_b = band_floor(dv, F32(N), S.hf, D[r], S.tf[r], e[r])
        if not (ok_a and ok_b):
            return None
        klo.append(a)
        khi.append(b)
    events = []
    for r in range(3):
        span = khi[r] - klo[r]
        if span == 0:
            continue
        slope = F32(S.hf * D[r])
        if abs(span) > 2 or not abs(slope) < F32(0.5):
            return None
        step = 1 if span > 0 else -1
        q0 = fma(dv, D[r], S.tf[r])
        for v in range(klo[r] + step, khi[r] + step, step):
            T = F32(v if step > 0 else v + 1)
            est = F32(F32(T - q0) / slope)
            # the kernel divides approximately (within 2 ulps): est moved by S.est_ulps
            for _ in range(abs(S.est_ulps)):
                est = np.nextafter(est, F32(np.inf) if S.est_ulps > 0 else F32(-np.inf))
            est = min(max(est, F32(-1e6)), F32(1e6))
            nc = int(math.ceil(est)) if step > 0 else int(math.floor(est)) + 1
            nc = min(max(nc, -N + 1), N)
            tries = 0
            while True:
                da = F32(fma(fma(F32(nc - 1), S.hf, dv), D[r], S.tf[r]) - T)
                db = F32(fma(fma(F32(nc), S.hf, dv), D[r], S.tf[r]) - T)
                ok2 = (da >= e[r] or da < -e[r]) and (db >= e[r] or db < -e[r])
                if not ok2 or tries > 2:
                    return None
                at_b = db >= 0 if step > 0 else db < 0
                at_a = da >= 0 if step > 0 else da < 0
                if at_b and not at_a:
                    break
                if not at_b:
                    if nc >= N:
                        return None
                    nc += 1
                else:
                    if nc <= -N + 1:
                        return None
                    nc -= 1
                tries += 1
            events.append((nc, r, v))
    events.sort(key=lambda ev: ev[0])  # stable, as the kernel's insertion sort
    k = list(klo)
    keys = {tuple(S.Ti[r] + k[r] for r in range(3))}
    i = 0
    while i < len(events):
        n = events[i][0]
        while i < len(events) and events[i][0] == n:
            k[events[i][1]] = events[i][2]
            i += 1
        keys.add(tuple(S.Ti[r] + k[r] for r in range(3)))
    return keys


def per_sample_path(S, dv, D, e, ez):
    keys = set()
    for n in range(-S.N, S.N + 1):
        z = fma(F32(n), S.hf, dv)
        if z < -ez:
            continue
        if not z > ez:
            return None
        k = []
        for r in range(3):
            f, ok = band_floor(dv, F32(n), S.hf, D[r], S.tf[r], e[r])
            if not ok:
                return None
            k.append(S.Ti[r] + f)
        keys.add(tuple(k))
    return keys


def oracle_ray_keys(K, T, prm, x, y, dv):
    depth = np.zeros((K.height, K.width), np.float32)
    depth[y, x] = dv
    return {k[1:] for k in O.frame_block_keys(depth, K, T, prm)}


def check_rays(K, T, prm, pixels, depths, min_decided, est_ulps=0):
    S = Setup(K, T, prm)
    S.est_ulps = est_ulps
    decided = 0
    for (x, y), dv in zip(pixels, depths):
        got = ray_keys(S, x, y, F32(dv))
        if got is None:
            continue
        decided += 1
        assert got == oracle_ray_keys(K, T, prm, x, y, F32(dv)), (x, y, dv)
    assert decided >= min_decided * len(pixels), decided


@pytest.mark.parametrize("est_ulps", [-2, 0, 2])
@pytest.mark.parametrize("seed,far", [(0, 3.0), (1, 400.0), (2, 3000.0)])
def test_certified_rays_match_the_oracle(seed, far, est_ulps):
    rng = np.random.default_rng(seed)
    prm = O.Params()
    K = O.Intrinsics(float(rng.uniform(150, 800)), float(rng.uniform(150, 800)), float(rng.uniform(100, 140)),
                     float(rng.uniform(40, 60)), 240, 100)
    T = random_pose(rng, far)
    n = 1500
    pixels = list(zip(rng.integers(0, K.width, n).tolist(), rng.integers(0, K.height, n).tolist()))
    depths = rng.uniform(0.2, 45.0, n).astype(F32)
    check_rays(K, T, prm, pixels, depths, 0.99, est_ulps)


@pytest.mark.parametrize("est_ulps", [-2, 0, 2])
def test_samples_on_block_faces(est_ulps):
    """Identity pose, principal point on a pixel centre: the central pixel's ray runs
    along +z and, for depths on a multiple of the sample spacing, its samples land on
    block faces; neighbouring pixels graze them."""
    prm = O.Params()
    K = O.Intrinsics(500.0, 500.0, 60.5, 30.5, 121, 61)
    T = np.eye(4)
    pixels, depths = [], []
    for k in range(1, 60):
        for dx, dy in ((0, 0), (1, 0), (0, 1), (-1, -1), (2, -3)):
            pixels.append((60 + dx, 30 + dy))
            depths.append(F32(k * 0.05))
    check_rays(K, T, prm, pixels, np.array(depths, F32), 0.05, est_ulps)


def test_the_block_faces_catch_an_unsound_bound():
    """The face case has teeth: with no error bound (float32 floors taken as final) some
    ray it decides gets a key set other than the oracle's."""
    prm = O.Params()
    K = O.Intrinsics(500.0, 500.0, 60.5, 30.5, 121, 61)
    T = np.eye(4)
    S = Setup(K, T, prm)
    S.est_ulps = 0
    S.e_scale = F32(0)
    wrong = 0
    for k in range(1, 60):
        for dx, dy in ((0, 0), (1, 0), (0, 1), (-1, -1), (2, -3)):
            x, y, dv = 60 + dx, 30 + dy, F32(k * 0.05)
            got = ray_keys(S, x, y, dv)
            wrong += got is not None and got != oracle_ray_keys(K, T, prm, x, y, dv)
    assert wrong > 0
