"""CPU FP64 oracle for the DENSER hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct restatement of the paper's method:
  * block allocation of the hashing voxel grid (Section III-A, "Fusing Data");
  * projective TSDF fusion (Section III-A, Eq. 1);
  * the observed-voxel indicator Omega and the Omega-aware gradient and
    divergence (Section III-B, Eq. 3 and Eq. 4);
  * the Chambolle-Pock primal-dual iteration (Section III-C, steps 1-4,
    constants from Table I);
  * the primal and dual energies and their gap (Section III-B Eq. 2, the
    saddle-point form of Section III-C).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module.  It shares no code with the CUDA path.

Every floating-point quantity is float64.  Where a float decides an integer
(a block key, a pixel index, the truncation test) the expression order is
written out below, operation by operation, with no fused multiply-add
(numpy's elementwise operators round each step), so that an implementation
that follows the same order reaches the same integers.

Readings of the paper taken here (the paper is silent or garbled):
  R1  allocation band: a block is allocated when a sample of a valid pixel's
      ray at depth z = d + n*s/2, n = -N..N, N = ceil(mu/(s/2)), z > 0, lies in it;
  R2  u_TSDF = min(1, u_SDF/mu) (normalised), no weight cap;
  R3  "nearest pixel" = floor of the continuous projection, pixel x covers [x, x+1);
  R4  Omega = allocated and w > 0;
  R5  gradient differences are not divided by the voxel size; neighbours in
      unallocated blocks are in Omega-bar (play the role of i = V_x);
  R6  divergence = exact negative adjoint of the gradient (reproduces every
      non-conflicting case of Eq. 4; gives 0 where two cases conflict);
  R7  primal step u~ = u + tau*div p (Chambolle-Pock sign; the printed minus
      ascends the TV term);
  R8  relaxation u^ = u_k + theta*(u_k - u_{k-1});
  R9  Table I step sizes read as sigma = 0.5, theta = 1.0, tau = 1/6;
  R10 energy = sum ||grad u||_2 + (lambda/2) sum w (u - f)^2 (the weighted
      data term whose proximal map is the printed primal update); isotropic TV.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BLOCK = 8
BLOCK_VOXELS = BLOCK ** 3


@dataclass(frozen=True)
class Params:
    """Method constants; defaults are Table I's 10 cm column with the 0.3 m truncation
    band of the synthetic workloads."""
    voxel_size: float = 0.1
    mu: float = 0.3
    lam: float = 0.8
    sigma: float = 0.5
    tau: float = 1.0 / 6.0
    theta: float = 1.0


@dataclass(frozen=True)
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


def band_samples(params: Params) -> int:
    """N of reading R1: samples every s/2 along the ray cover [d - mu, d + mu]."""
    h = 0.5 * params.voxel_size
    return int(math.ceil(params.mu / h - 1e-9))


# --------------------------------------------------------------- the map
class SparseGrid:
    """Hashing voxel grid (Section III-A): 8^3 blocks keyed by (segment, bx, by, bz).

    A dict plays the hash table; block b owns voxels b*512 + lx + 8*ly + 64*lz.
    Block indices are assigned in allocation order; the new keys of one
    allocation call are appended in ascending (segment, bz, by, bx) order.
    """

    def __init__(self, params: Params = Params()):
        self.params = params
        self.keys: list = []
        self.index: dict = {}
        self.f = np.zeros((0, BLOCK_VOXELS))
        self.w = np.zeros((0, BLOCK_VOXELS))
        self.u = np.zeros((0, BLOCK_VOXELS))
        self.u_bar = np.zeros((0, BLOCK_VOXELS))
        self.p = np.zeros((3, 0, BLOCK_VOXELS))

    @property
    def n_blocks(self) -> int:
        return len(self.keys)

    def add_blocks(self, keys) -> int:
        """Append blocks (already ordered) with zero state; returns how many were new."""
        new = [k for k in keys if k not in self.index]
        for k in new:
            self.index[k] = len(self.keys)
            self.keys.append(k)
        n = len(new)
        if n:
            z = np.zeros((n, BLOCK_VOXELS))
            self.f = np.concatenate([self.f, z])
            self.w = np.concatenate([self.w, z])
            self.u = np.concatenate([self.u, z])
            self.u_bar = np.concatenate([self.u_bar, z])
            self.p = np.concatenate([self.p, np.zeros((3, n, BLOCK_VOXELS))], axis=1)
        return n

    def coords(self) -> np.ndarray:
        """[nb, 4] int64 rows (segment, bx, by, bz) in block-index order."""
        return np.array(self.keys, dtype=np.int64).reshape(-1, 4)


def local_offsets():
    l = np.arange(BLOCK_VOXELS)
    return l % BLOCK, (l // BLOCK) % BLOCK, l // (BLOCK * BLOCK)


# ---------------------------------------------------------- allocation
def frame_block_keys(depth: np.ndarray, K: Intrinsics, T_gc: np.ndarray, params: Params,
                     segment: int = 0) -> set:
    """Set of block keys a depth map observes (Section III-A allocation rule, reading R1).

    For every valid pixel (x, y) (finite d > 0) and n = -N..N:
        z  = d + n*h,                     h = s/2          (skip z <= 0)
        X  = ((x + 0.5) - cx) * z / fx,   Y likewise,  Z = z
        g  = R [X Y Z]^T + t,   each row summed left to right
        b  = floor(g / (8 s))
    """
    s = params.voxel_size
    h = 0.5 * s
    bs = 8.0 * s
    N = band_samples(params)
    d32 = np.asarray(depth, dtype=np.float32)
    valid = np.isfinite(d32) & (d32 > 0)
    ys, xs = np.nonzero(valid)
    d = d32[ys, xs].astype(np.float64)
    uu = (xs.astype(np.float64) + 0.5) - K.cx
    vv = (ys.astype(np.float64) + 0.5) - K.cy
    R = np.asarray(T_gc, dtype=np.float64)[:3, :3]
    t = np.asarray(T_gc, dtype=np.float64)[:3, 3]
    keys = set()
    for n in range(-N, N + 1):
        z = d + float(n) * h
        ok = z > 0
        X = (uu * z) / K.fx
        Y = (vv * z) / K.fy
        Z = z
        g = []
        for r in range(3):
            g.append(((R[r, 0] * X + R[r, 1] * Y) + R[r, 2] * Z) + t[r])
        kb = [np.floor(gi / bs) for gi in g]
        trip = np.stack(kb, axis=1)[ok].astype(np.int64)
        keys.update((segment, int(a), int(b), int(c)) for a, b, c in np.unique(trip, axis=0))
    return keys


def alloc_blocks(grid: SparseGrid, depth, K: Intrinsics, T_gc, segment: int = 0) -> int:
    """Allocate every observed block not yet in the map; new keys appended in ascending
    (segment, bz, by, bx) order.  Returns the number of new blocks."""
    keys = frame_block_keys(depth, K, T_gc, grid.params, segment)
    new = sorted((k for k in keys if k not in grid.index), key=lambda k: (k[0], k[3], k[2], k[1]))
    return grid.add_blocks(new)


# ------------------------------------------------------------- fusion
def pose_inverse(T_gc: np.ndarray):
    """(R^T, -R^T t) of a rigid camera->global pose; -R^T t summed left to right."""
    T = np.asarray(T_gc, dtype=np.float64)
    R, t = T[:3, :3], T[:3, 3]
    Ri = R.T.copy()
    ti = np.array([-((R[0, r] * t[0] + R[1, r] * t[1]) + R[2, r] * t[2]) for r in range(3)])
    return Ri, ti


def fuse_depth(grid: SparseGrid, depth, K: Intrinsics, T_gc, segment: int = 0,
               blocks=None) -> np.ndarray:
    """Projective TSDF fusion of one depth map into every allocated voxel of ``segment``
    (Section III-A, steps 1-4 and Eq. 1).  Returns the per-voxel update mask.

    Per voxel (i, j, k) with centre p_g = ((i+0.5)s, (j+0.5)s, (k+0.5)s):
        p_c = R^T p_g + (-R^T t)            rows summed left to right
        skip if z_c <= 0
        px = floor((fx*x_c)/z_c + cx),  py = floor((fy*y_c)/z_c + cy)     (reading R3)
        skip if the pixel is outside the map or its depth is invalid
        u_SDF = d - z_c;  skip if u_SDF < -mu                               (Eq. 1)
        u_TSDF = min(1, u_SDF/mu)                                           (reading R2)
        w <- w + 1;  f <- (u_TSDF + w_old f_old) / w                        (Eq. 1)
    """
    p = grid.params
    s = p.voxel_size
    H, W = K.height, K.width
    d32 = np.asarray(depth, dtype=np.float32).reshape(H, W)
    Ri, ti = pose_inverse(T_gc)
    lx, ly, lz = local_offsets()
    sel = [b for b, k in enumerate(grid.keys) if k[0] == segment] if blocks is None else list(blocks)
    mask_all = np.zeros((grid.n_blocks, BLOCK_VOXELS), dtype=bool)
    if not sel:
        return mask_all
    sel = np.array(sel)
    C = grid.coords()[sel]
    i = C[:, 1:2] * BLOCK + lx[None, :]
    j = C[:, 2:3] * BLOCK + ly[None, :]
    k = C[:, 3:4] * BLOCK + lz[None, :]
    gx = (i.astype(np.float64) + 0.5) * s
    gy = (j.astype(np.float64) + 0.5) * s
    gz = (k.astype(np.float64) + 0.5) * s
    xc = ((Ri[0, 0] * gx + Ri[0, 1] * gy) + Ri[0, 2] * gz) + ti[0]
    yc = ((Ri[1, 0] * gx + Ri[1, 1] * gy) + Ri[1, 2] * gz) + ti[1]
    zc = ((Ri[2, 0] * gx + Ri[2, 1] * gy) + Ri[2, 2] * gz) + ti[2]
    front = zc > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        pxf = np.floor((K.fx * xc) / zc + K.cx)
        pyf = np.floor((K.fy * yc) / zc + K.cy)
    inside = front & (pxf >= 0) & (pxf < W) & (pyf >= 0) & (pyf < H)
    px = np.where(inside, pxf, 0).astype(np.int64)
    py = np.where(inside, pyf, 0).astype(np.int64)
    d = d32[py, px].astype(np.float64)
    valid = inside & np.isfinite(d) & (d > 0)
    usdf = d - zc
    upd = valid & (usdf >= -p.mu)
    utsdf = np.minimum(1.0, usdf / p.mu)
    w_old = grid.w[sel]
    f_old = grid.f[sel]
    w_new = np.where(upd, w_old + 1.0, w_old)
    f_new = np.where(upd, (utsdf + w_old * f_old) / np.where(upd, w_new, 1.0), f_old)
    grid.w[sel] = w_new
    grid.f[sel] = f_new
    mask_all[sel] = upd
    return mask_all


# ------------------------------------------------- Omega, grad and div
def omega(grid: SparseGrid) -> np.ndarray:
    """Observed-voxel indicator (Section III-B, reading R4): allocated and w > 0."""
    return (grid.w > 0).reshape(-1)


def voxel_neighbours(grid: SparseGrid):
    """Flat indices of each voxel's +axis and -axis neighbours, -1 where the
    neighbour's block is not allocated.  Returns (fwd[3, N], bwd[3, N])."""
    nb = grid.n_blocks
    lx, ly, lz = local_offsets()
    loc = (lx, ly, lz)
    stride = (1, BLOCK, BLOCK * BLOCK)
    fwd = np.full((3, nb * BLOCK_VOXELS), -1, dtype=np.int64)
    bwd = np.full((3, nb * BLOCK_VOXELS), -1, dtype=np.int64)
    base = np.arange(nb)[:, None] * BLOCK_VOXELS + np.arange(BLOCK_VOXELS)[None, :]
    for a in range(3):
        for sign, out in ((+1, fwd), (-1, bwd)):
            nbr_block = np.full(nb, -1, dtype=np.int64)
            for b, key in enumerate(grid.keys):
                q = list(key)
                q[1 + a] += sign
                nbr_block[b] = grid.index.get(tuple(q), -1)
            edge = (loc[a] == (BLOCK - 1)) if sign > 0 else (loc[a] == 0)
            same = base + sign * stride[a]
            wrap = nbr_block[:, None] * BLOCK_VOXELS + np.arange(BLOCK_VOXELS)[None, :] \
                - sign * (BLOCK - 1) * stride[a]
            wrap = np.where(nbr_block[:, None] >= 0, wrap, -1)
            out[a] = np.where(edge[None, :], wrap, same).reshape(-1)
    return fwd, bwd


def edge_mask(om: np.ndarray, fwd: np.ndarray) -> np.ndarray:
    """e[a, v] = v in Omega and v + a in Omega (a forward difference exists), Eq. 3."""
    has = fwd >= 0
    nb_om = np.where(has, om[np.where(has, fwd, 0)], False)
    return om[None, :] & nb_om


def gradient(u: np.ndarray, om: np.ndarray, fwd: np.ndarray) -> np.ndarray:
    """Omega-aware forward difference, Eq. 3: u_{v+a} - u_v where both voxels are in
    Omega, else 0.  u is flat [N]; returns [3, N]."""
    e = edge_mask(om, fwd)
    g = np.zeros((3, u.size))
    for a in range(3):
        g[a] = np.where(e[a], u[np.where(e[a], fwd[a], 0)] - u, 0.0)
    return g


def divergence(p: np.ndarray, om: np.ndarray, fwd: np.ndarray, bwd: np.ndarray) -> np.ndarray:
    """Omega-aware divergence, Eq. 4, as the negative adjoint of ``gradient`` (reading R6):
    (div p)_v = sum_a [ e_a(v) p^a_v - e_a(v-a) p^a_{v-a} ]."""
    e = edge_mask(om, fwd)
    d = np.zeros(p.shape[1])
    for a in range(3):
        own = np.where(e[a], p[a], 0.0)
        hb = bwd[a] >= 0
        bi = np.where(hb, bwd[a], 0)
        back = np.where(hb & e[a][bi], p[a][bi], 0.0)
        d = d + (own - back)
    return d


# -------------------------------------------------------- primal-dual
class PDProblem:
    """Flat views of one map's regularisation problem (Section III-B/C)."""

    def __init__(self, grid: SparseGrid):
        self.grid = grid
        self.om = omega(grid)
        self.fwd, self.bwd = voxel_neighbours(grid)
        self.f = grid.f.reshape(-1).copy()
        self.w = grid.w.reshape(-1).copy()

    def grad(self, u):
        return gradient(u, self.om, self.fwd)

    def div(self, p):
        return divergence(p, self.om, self.fwd, self.bwd)


def pd_iterate(prob: PDProblem, u, u_bar, p, iters: int, params: Params, literal_sign: bool = False):
    """Chambolle-Pock iterations of Section III-C (steps 2-4), Jacobi over all voxels.

        p~ = p + sigma grad(u^);          p = p~ / max(1, ||p~||_2)
        u~ = u + tau div(p)               (reading R7; literal_sign=True uses u - tau div p)
        u  = (u~ + tau lam w f)/(1 + tau lam w)   on Omega; u unchanged on Omega-bar
        u^ = u + theta (u - u_old)        (reading R8)
    """
    sg, tau, lam, th = params.sigma, params.tau, params.lam, params.theta
    om, f, w = prob.om, prob.f, prob.w
    for _ in range(iters):
        pt = p + sg * prob.grad(u_bar)
        nrm = np.sqrt(pt[0] * pt[0] + pt[1] * pt[1] + pt[2] * pt[2])
        p = pt / np.maximum(1.0, nrm)[None, :]
        u_old = u
        dv = prob.div(p)
        ut = (u - tau * dv) if literal_sign else (u + tau * dv)
        u = np.where(om, (ut + tau * lam * w * f) / (1.0 + tau * lam * w), u)
        u_bar = u + th * (u - u_old)
    return u, u_bar, p


def energies(prob: PDProblem, u, p, params: Params):
    """Primal P(u), dual D(p) of the saddle problem (reading R10):
        P(u) = sum_Omega ||grad u||_2 + (lam/2) sum_Omega w (u - f)^2
        D(p) = sum_Omega [ -f div p - (div p)^2 / (2 lam w) ]      (min over u of the Lagrangian)
    """
    om, f, w, lam = prob.om, prob.f, prob.w, params.lam
    g = prob.grad(u)
    tv = np.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2])
    P = np.sum(np.where(om, tv + 0.5 * lam * w * (u - f) ** 2, 0.0))
    dv = prob.div(p)
    wd = np.where(om, w, 1.0)
    D = np.sum(np.where(om, -f * dv - dv * dv / (2.0 * lam * wd), 0.0))
    return float(P), float(D)


def regularize(grid: SparseGrid, iters: int, params: Params = None, warm: bool = False,
               literal_sign: bool = False):
    """Run ``iters`` iterations from p = u = u^ = 0 (step 1), or from the grid's stored
    state when ``warm``; stores the result in the grid and returns the PDProblem."""
    params = params or grid.params
    prob = PDProblem(grid)
    N = grid.n_blocks * BLOCK_VOXELS
    if warm:
        u, ub, p = grid.u.reshape(-1).copy(), grid.u_bar.reshape(-1).copy(), grid.p.reshape(3, -1).copy()
    else:
        u, ub, p = np.zeros(N), np.zeros(N), np.zeros((3, N))
    u, ub, p = pd_iterate(prob, u, ub, p, iters, params, literal_sign)
    grid.u = u.reshape(-1, BLOCK_VOXELS)
    grid.u_bar = ub.reshape(-1, BLOCK_VOXELS)
    grid.p = p.reshape(3, -1, BLOCK_VOXELS)
    return prob


# ----------------------------------------------------------- pipeline
def run_pipeline(depths, K: Intrinsics, poses, params: Params, iters: int, segment: int = 0):
    """alloc(k) then fuse(k) for every frame, then ``iters`` primal-dual iterations."""
    grid = SparseGrid(params)
    for dm, T in zip(depths, poses):
        alloc_blocks(grid, dm, K, T, segment)
        fuse_depth(grid, dm, K, T, segment)
    if iters > 0:
        regularize(grid, iters)
    return grid
