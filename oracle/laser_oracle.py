"""CPU FP64 oracle of laser-scan allocation and ray fusion -- TEST INFRASTRUCTURE ONLY.

The paper fuses depth maps by projecting voxels into them (Eq. 1) and notes that the
method extends to laser sensors by updating only the voxels along each ray, from the
sensor to mu behind the observed surface (Section III-A, after Eq. 1).  It gives no
more detail; the readings taken here:

  L1  a scan is a set of points p in the sensor frame (float32) with a sensor->global
      pose T (float64, rotation R, origin t); a point is valid when finite with range
      r = |p| > 0 and M = floor((r + mu)/h) < 2^22 (a range limit of about 200 km at
      10 cm voxels that keeps every ray's walk bounded).  Its ray has the unit
      direction d = p / r, dg = R d in the global frame, and starts at t;
  L2  allocation follows reading R1 along the ray: a block is allocated when it holds
      a band sample at range rho = r + n h, n = -N..N, rho > 0 (h = s/2,
      N = ceil(mu/h)), at g = dg rho + t;
  L3  the voxels "along the ray" are those holding a ray sample at range rho = n h,
      n = 0..M, M = floor((r + mu)/h) (from the sensor to mu behind the hit), in an
      allocated block of the scan's segment; a voxel counts once per ray (a ray never
      re-enters a voxel, so repeats are consecutive);
  L4  the signed distance of such a voxel (centre c) is the range difference along
      the ray, u_SDF = r - (c - t) . dg; it is observed when u_SDF >= -mu, with
      u_TSDF = min(1, u_SDF/mu) (readings R2 and Eq. 1's truncation test);
  L5  one scan updates a voxel once with all its observations: w <- w + n and
      f <- (w_old f_old + sum u_TSDF) / w, what n applications of Eq. 1 give in exact
      arithmetic, but independent of the order of the rays.  The sum is taken in fixed
      point, each u_TSDF rounded to a multiple of 2^-30 (ties to even), so that it is
      exact and order-free.

Expression order where a float64 value decides an integer (written out so that an
implementation following the same order reaches the same integers):
    r   = sqrt((x*x + y*y) + z*z);   d = (x/r, y/r, z/r)
    dg_i = (R_i0*d0 + R_i1*d1) + R_i2*d2
    g_i = dg_i*rho + t_i;   block_i = floor(g_i / (8 s));   voxel_i = floor(g_i / s)
    rho = r + n*h (allocation), rho = n*h (fusion);  M = floor((r + mu) / h)
    e_i = (v_i + 0.5)*s - t_i;   u_SDF = r - ((e_0*dg_0 + e_1*dg_1) + e_2*dg_2)

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It shares no code with the CUDA path.
"""

from __future__ import annotations

import numpy as np

from .denser_oracle import BLOCK, BLOCK_VOXELS, SparseGrid, band_samples

FIX = 2.0 ** 30  # fixed-point scale of the per-scan sums (L5)


def ray_setup(points, T, params=None):
    """(valid [n], r [n], dg [n, 3], t [3]) of a scan (L1), float64 in the stated order."""
    P = np.asarray(points, dtype=np.float32).astype(np.float64).reshape(-1, 3)
    T = np.asarray(T, dtype=np.float64)
    R, t = T[:3, :3], T[:3, 3]
    x, y, z = P[:, 0], P[:, 1], P[:, 2]
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.sqrt((x * x + y * y) + z * z)
        valid = np.isfinite(r) & (r > 0)
        if params is not None:
            valid &= np.floor((r + params.mu) / (0.5 * params.voxel_size)) < 2.0 ** 22
        d = np.stack([x / r, y / r, z / r], axis=1)
    dg = np.stack([(R[i, 0] * d[:, 0] + R[i, 1] * d[:, 1]) + R[i, 2] * d[:, 2] for i in range(3)], axis=1)
    return valid, r, dg, t


def scan_block_keys(points, T, params, segment: int = 0) -> set:
    """Block keys a scan allocates (L2)."""
    s = params.voxel_size
    h = 0.5 * s
    bs = 8.0 * s
    N = band_samples(params)
    valid, r, dg, t = ray_setup(points, T, params)
    r, dg = r[valid], dg[valid]
    keys = set()
    for n in range(-N, N + 1):
        rho = r + float(n) * h
        ok = rho > 0
        kb = np.stack([np.floor((dg[:, i] * rho + t[i]) / bs) for i in range(3)], axis=1)
        trip = kb[ok].astype(np.int64)
        keys.update((segment, int(a), int(b), int(c)) for a, b, c in np.unique(trip, axis=0))
    return keys


def alloc_scan(grid: SparseGrid, points, T, segment: int = 0) -> int:
    """Allocates the scan's blocks not yet in the map, new keys appended in ascending
    (segment, bz, by, bx) order; returns how many were new."""
    keys = scan_block_keys(points, T, grid.params, segment)
    new = sorted((k for k in keys if k not in grid.index), key=lambda k: (k[0], k[3], k[2], k[1]))
    return grid.add_blocks(new)


def ray_voxels(r, dg, t, params):
    """Per ray (L3): the distinct voxels [m, 3] (int64) of its samples rho = n h,
    n = 0..M, in sample order."""
    s = params.voxel_size
    h = 0.5 * s
    M = int(np.floor((r + params.mu) / h))
    rho = np.arange(M + 1, dtype=np.float64) * h
    v = np.stack([np.floor((dg[i] * rho + t[i]) / s) for i in range(3)], axis=1).astype(np.int64)
    keep = np.ones(len(v), dtype=bool)
    keep[1:] = np.any(v[1:] != v[:-1], axis=1)
    return v[keep]


def scan_observations(grid: SparseGrid, points, T, segment: int = 0):
    """All (flat voxel index, u_TSDF) observations of a scan (L3, L4), ray by ray."""
    p = grid.params
    s = p.voxel_size
    valid, r, dg, t = ray_setup(points, T, p)
    flat_all, u_all = [], []
    for i in np.nonzero(valid)[0]:
        v = ray_voxels(r[i], dg[i], t, p)
        blk = v // BLOCK  # floor division: block of each voxel
        loc = v - blk * BLOCK
        idx = np.array([grid.index.get((segment, int(a), int(b), int(c)), -1) for a, b, c in blk], dtype=np.int64)
        inb = idx >= 0
        if not np.any(inb):
            continue
        v, loc, idx = v[inb], loc[inb], idx[inb]
        e = [(v[:, k].astype(np.float64) + 0.5) * s - t[k] for k in range(3)]
        usdf = r[i] - ((e[0] * dg[i, 0] + e[1] * dg[i, 1]) + e[2] * dg[i, 2])
        obs = usdf >= -p.mu
        if not np.any(obs):
            continue
        flat = idx * BLOCK_VOXELS + loc[:, 0] + BLOCK * loc[:, 1] + BLOCK * BLOCK * loc[:, 2]
        flat_all.append(flat[obs])
        u_all.append(np.minimum(1.0, usdf[obs] / p.mu))
    if not flat_all:
        return np.zeros(0, np.int64), np.zeros(0)
    return np.concatenate(flat_all), np.concatenate(u_all)


def fuse_scan(grid: SparseGrid, points, T, segment: int = 0) -> np.ndarray:
    """Ray fusion of one scan (L3-L5); returns the per-voxel observation counts."""
    flat, u = scan_observations(grid, points, T, segment)
    nv = grid.n_blocks * BLOCK_VOXELS
    cnt = np.bincount(flat, minlength=nv).astype(np.float64)
    q = np.rint(u * FIX).astype(np.int64)  # L5: fixed point, exact sum
    S = np.zeros(nv, dtype=np.int64)
    np.add.at(S, flat, q)
    w = grid.w.reshape(-1)
    f = grid.f.reshape(-1)
    upd = cnt > 0
    w_new = w + cnt
    f_new = np.where(upd, (w * f + S.astype(np.float64) / FIX) / np.where(upd, w_new, 1.0), f)
    grid.w[:] = w_new.reshape(grid.w.shape)
    grid.f[:] = f_new.reshape(grid.f.shape)
    return cnt.reshape(grid.w.shape)
