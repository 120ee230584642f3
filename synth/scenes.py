"""Seeded synthetic street scenes and their depth maps.

This module only makes inputs: pinhole depth maps of a scene made of planes
and axis-aligned boxes, the camera intrinsics and the camera-to-global poses.
It holds none of the fusion or regularisation arithmetic; both the CPU oracle
and the CUDA path consume what it returns.

The scenes stand in for the paper's KITTI-VO driving sequences (Section V),
which are not available here: a road plane, facades with window recesses,
parked cars as boxes, and a forward-moving camera.

Conventions (shared by every consumer):
  * camera frame: x right, y down, z forward; the road is the plane y = +1.65;
  * a pose ``T_gc`` is a 4x4 float64 row-major matrix mapping camera -> global;
  * pixel (x, y) covers [x, x+1) x [y, y+1); its ray passes through its centre;
  * a depth value is the camera-frame z of the first hit (a z-buffer), 0 where
    the ray hits nothing within ``d_max`` or the pixel is dropped as invalid.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Generic offsets keep lattice-aligned geometry away from exact rounding ties.
CAM_OFFSET = (0.0123, 0.0071, 0.0037)
PP_OFFSET = (0.137, 0.291)
ROAD_Y = 1.65


@dataclass(frozen=True)
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @staticmethod
    def pinhole(width: int, height: int, focal: float) -> "Camera":
        return Camera(float(focal), float(focal), width / 2.0 + PP_OFFSET[0],
                      height / 2.0 + PP_OFFSET[1], int(width), int(height))


@dataclass(frozen=True)
class Lidar:
    """A spinning multi-beam laser: ``beams`` elevations evenly spaced in
    [el_lo, el_hi] degrees (up positive), ``azimuths`` rays per turn.  The default is
    shaped like the 64-beam scanner of the paper's driving sequences."""
    beams: int = 64
    azimuths: int = 2000
    el_lo: float = -24.9
    el_hi: float = 2.0
    r_max: float = 40.0
    noise: float = 0.02
    invalid_prob: float = 0.05


@dataclass
class Box:
    lo: np.ndarray
    hi: np.ndarray


@dataclass
class Rect:
    """Axis-aligned rectangle in the plane ``coord[axis] == value``."""
    axis: int
    value: float
    lo: np.ndarray  # lower bounds of the two in-plane coordinates (ascending axis order)
    hi: np.ndarray


@dataclass
class Facade:
    """Vertical facade plane x = ``x`` (sign ``side``) with rectangular recesses.

    Cells of ``cell`` (z, y) metres tile the facade; a cell with a window has a
    ``win`` (z, y) opening centred in it, ``recess`` metres deep, away from the street.
    """
    x: float
    side: int
    y_top: float
    y_bot: float
    z0: float
    z1: float
    windows: np.ndarray  # bool [n_cells_z, n_cells_y]
    cell: tuple = (2.0, 3.0)
    win: tuple = (1.2, 1.5)
    recess: float = 0.3


@dataclass
class Scene:
    camera: Camera
    poses: list
    rects: list = field(default_factory=list)
    boxes: list = field(default_factory=list)
    facades: list = field(default_factory=list)
    d_max: float = 30.0
    noise_sigma: float = 0.0      # constant part of the depth noise (m)
    noise_quad: float = 0.0       # sigma += noise_quad * z^2
    invalid_prob: float = 0.0
    seed: int = 0
    name: str = ""

    # ------------------------------------------------------------------ rays
    def _rays(self):
        c = self.camera
        xs = (np.arange(c.width, dtype=np.float64) + 0.5 - c.cx) / c.fx
        ys = (np.arange(c.height, dtype=np.float64) + 0.5 - c.cy) / c.fy
        dx, dy = np.meshgrid(xs, ys)
        return np.stack([dx, dy, np.ones_like(dx)], axis=0)  # [3, H, W]

    def render_clean(self, frame: int) -> np.ndarray:
        """Noise-free depth (float64, 0 = no hit within d_max) for one pose: the casts of
        render_clean_numpy, evaluated by synth/raycast.c in the same operation order."""
        from . import raycast
        T = self.poses[frame]
        wins = [_box_pixel_window(b, self.camera, T) for b in self.boxes]
        return raycast.depth(self, T, wins)

    def render_clean_numpy(self, frame: int) -> np.ndarray:
        """The same depth cast with numpy array operations."""
        T = self.poses[frame]
        R, o = T[:3, :3], T[:3, 3]
        dcam = self._rays()
        D = np.einsum("ij,jhw->ihw", R, dcam)  # world ray directions, camera z = 1
        best = np.full(D.shape[1:], np.inf)
        for r in self.rects:
            _hit_rect(best, o, D, r)
        for b in self.boxes:
            _hit_box(best, o, D, b, self.camera, T)
        for f in self.facades:
            _hit_facade(best, o, D, f)
        best[~(best <= self.d_max)] = 0.0
        return best

    def render(self, frame: int, rng: np.random.Generator) -> np.ndarray:
        d = self.render_clean(frame)
        valid = d > 0
        if self.noise_sigma > 0 or self.noise_quad > 0:
            sig = self.noise_sigma + self.noise_quad * d * d
            d = d + rng.standard_normal(d.shape) * sig
        if self.invalid_prob > 0:
            valid &= rng.random(d.shape) >= self.invalid_prob
        valid &= d > 0
        out = np.where(valid, d, 0.0).astype(np.float32)
        return out

    # ---------------------------------------------------------------- laser
    def lidar_scan(self, frame: int, lidar: "Lidar") -> np.ndarray:
        """Points [n, 3] float32 in the sensor frame (the camera frame of pose ``frame``:
        x right, y down, z forward) of one spinning-lidar sweep: ``lidar.beams``
        elevations x ``lidar.azimuths`` azimuths, every ray cast from the pose's origin.
        A ray with no hit within ``lidar.r_max``, or dropped (``lidar.invalid_prob``),
        gives a NaN point.  Range noise N(0, lidar.noise) from PCG64([seed, 2, frame])."""
        T = self.poses[frame]
        R, o = T[:3, :3], T[:3, 3]
        el = np.linspace(lidar.el_lo, lidar.el_hi, lidar.beams) * (np.pi / 180.0)
        az = (np.arange(lidar.azimuths) + 0.5) * (2.0 * np.pi / lidar.azimuths)
        E, A = np.meshgrid(el, az, indexing="ij")
        # unit directions in the sensor frame: elevation up is -y
        ds = np.stack([np.cos(E) * np.sin(A), -np.sin(E), np.cos(E) * np.cos(A)], axis=0)
        D = np.einsum("ij,jhw->ihw", R, ds)
        best = np.full(D.shape[1:], np.inf)
        for r in self.rects:
            _hit_rect(best, o, D, r)
        for b in self.boxes:
            _hit_box(best, o, D, b, None, T)
        for f in self.facades:
            _hit_facade(best, o, D, f)
        rng = np.random.Generator(np.random.PCG64([self.seed, 2, frame]))
        rng_noise = rng.standard_normal(best.shape) * lidar.noise
        drop = rng.random(best.shape) < lidar.invalid_prob
        valid = (best <= lidar.r_max) & ~drop
        rho = np.where(valid, best + rng_noise, np.nan)
        pts = (ds * rho[None]).reshape(3, -1).T
        return np.ascontiguousarray(pts, dtype=np.float32)

    # ---------------------------------------------------------------- stereo
    def _cast(self, T, D):
        best = np.full(D.shape[1:], np.inf)
        for r in self.rects:
            _hit_rect(best, T[:3, 3], D, r)
        for b in self.boxes:
            _hit_box(best, T[:3, 3], D, b, None, T)
        for f in self.facades:
            _hit_facade(best, T[:3, 3], D, f)
        return best

    def intensity(self, T: np.ndarray, rng=None, noise: float = 0.01) -> np.ndarray:
        """Grey image [H, W] float32 in [0, 1] seen from pose T: surfaces carry a fixed,
        band-limited value-noise texture of their world position (octaves 0.0125 - 0.4 m,
        those finer than 4 pixels faded out), so that nearby views of a point see the same
        value; rays with no hit within d_max see a smooth sky gradient.  Additive
        N(0, noise) pixel noise from ``rng``."""
        c = self.camera
        R, o = T[:3, :3], T[:3, 3]
        D = np.einsum("ij,jhw->ihw", R, self._rays())
        lam = self._cast(T, D)
        hit = lam <= self.d_max
        P = o[:, None, None] + D * np.where(hit, lam, 0.0)[None]
        # metres per pixel at the hit (lam is the camera-frame depth: D has z = 1)
        fp = np.where(hit, lam, 1.0) / c.fx
        img = texture_value(P.reshape(3, -1).T, fp.reshape(-1)).reshape(c.height, c.width)
        sky = 0.85 + 0.1 * (np.arange(c.height)[:, None] / c.height) * np.ones((1, c.width))
        img = np.where(hit, img, sky)
        if rng is not None and noise > 0:
            img = img + rng.standard_normal(img.shape) * noise
        return np.clip(img, 0.0, 1.0).astype(np.float32)

    def stereo_pair(self, frame: int, baseline: float = 0.54, noise: float = 0.01):
        """(I_left, I_right, d_right, T_right): a rectified pair whose right camera sits at
        the pose of ``frame`` and whose left camera is ``baseline`` metres along its -x
        axis; the true disparity on the right image is f * baseline / z (0 where the
        right view sees nothing), so that I_left(x + d) = I_right(x).  Noise from
        PCG64([seed, 3, frame])."""
        TR = self.poses[frame]
        TL = TR.copy()
        TL[:3, 3] = TR[:3, 3] - baseline * TR[:3, 0]
        rng = np.random.Generator(np.random.PCG64([self.seed, 3, frame]))
        IL = self.intensity(TL, rng, noise)
        IR = self.intensity(TR, rng, noise)
        z = self.render_clean(frame)
        d = np.where(z > 0, self.camera.fx * baseline / np.where(z > 0, z, 1.0), 0.0).astype(np.float32)
        return IL, IR, d, TR

    def depth_map(self, k: int) -> np.ndarray:
        """Depth map of frame k; its noise comes from PCG64([seed, 1, k])."""
        return self.render(k, np.random.Generator(np.random.PCG64([self.seed, 1, k])))

    def depth_maps(self, frames=None, workers: int = 1) -> np.ndarray:
        """Depth maps [n, H, W] float32; frame k draws its noise from PCG64([seed, 1, k]), so
        the result does not depend on ``workers`` (> 1: that many processes, started with
        'spawn' so that a parent which already uses a GPU is safe)."""
        n = len(self.poses)
        frames = list(range(n)) if frames is None else list(frames)
        c = self.camera
        out = np.zeros((len(frames), c.height, c.width), np.float32)
        if workers > 1 and len(frames) > 1:
            import multiprocessing as mp
            with mp.get_context("spawn").Pool(workers) as pool:
                for i, img in enumerate(pool.imap(self.depth_map, frames, chunksize=8)):
                    out[i] = img
            return out
        for i, k in enumerate(frames):
            out[i] = self.depth_map(k)
        return out


# ---------------------------------------------------------------- texture
def _lattice_hash(i, j, k):
    """Deterministic values in [0, 1) on an integer lattice (a 64-bit integer mix)."""
    h = (i.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)) ^ (j.astype(np.uint64) * np.uint64(0xC2B2AE3D27D4EB4F)) \
        ^ (k.astype(np.uint64) * np.uint64(0x165667B19E3779F9))
    h ^= h >> np.uint64(29)
    h *= np.uint64(0xBF58476D1CE4E5B9)
    h ^= h >> np.uint64(32)
    return (h >> np.uint64(11)).astype(np.float64) / float(1 << 53)


def texture_value(P: np.ndarray, footprint=None, cell: float = 0.1) -> np.ndarray:
    """Band-limited value noise of world points P [n, 3]: trilinear interpolation of
    lattice values over octaves of 0.0125 .. 0.4 m, in [0, 1].  ``footprint`` [n] (metres
    per pixel at each point) fades out the octaves finer than 4 pixels, so that nearby
    views of a point sample the same, alias-free texture and close surfaces keep detail."""
    out = np.zeros(len(P))
    total = np.zeros(len(P))
    fp = np.zeros(len(P)) if footprint is None else np.asarray(footprint, dtype=np.float64)
    for scale in (cell / 8, cell / 4, cell / 2, cell, 2 * cell, 4 * cell):
        wgt = np.clip((scale / np.maximum(fp, 1e-12) - 2.0) / 2.0, 0.0, 1.0) if footprint is not None else \
            np.ones(len(P))
        q = P / scale
        b = np.floor(q)
        f = q - b
        b = b.astype(np.int64)
        acc = np.zeros(len(P))
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    wv = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * \
                         (f[:, 2] if dz else 1 - f[:, 2])
                    with np.errstate(over="ignore"):
                        acc += wv * _lattice_hash(b[:, 0] + dx, b[:, 1] + dy, b[:, 2] + dz)
        out += wgt * acc
        total += wgt
    return np.where(total > 0, out / np.maximum(total, 1e-12), 0.5)


# ---------------------------------------------------------------- primitives
def _in_range(a, lo, hi):
    return (a >= lo) & (a <= hi)


def _hit_rect(best, o, D, r: Rect):
    a = r.axis
    with np.errstate(divide="ignore", invalid="ignore"):
        lam = (r.value - o[a]) / D[a]
    ok = lam > 0
    others = [i for i in range(3) if i != a]
    for k, ax in enumerate(others):
        c = o[ax] + lam * D[ax]
        ok &= _in_range(c, r.lo[k], r.hi[k])
    upd = ok & (lam < best)
    best[upd] = lam[upd]


def _box_pixel_window(b: Box, cam: Camera, T: np.ndarray):
    """Pixel rectangle that contains the box's projection, or None for the whole image."""
    corners = np.array([[x, y, z] for x in (b.lo[0], b.hi[0]) for y in (b.lo[1], b.hi[1])
                        for z in (b.lo[2], b.hi[2])])
    R, t = T[:3, :3], T[:3, 3]
    pc = (corners - t) @ R  # R^T (p - t)
    if np.any(pc[:, 2] <= 0.05):
        return None
    px = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    py = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    x0 = max(int(np.floor(px.min())) - 1, 0)
    x1 = min(int(np.ceil(px.max())) + 1, cam.width)
    y0 = max(int(np.floor(py.min())) - 1, 0)
    y1 = min(int(np.ceil(py.max())) + 1, cam.height)
    if x0 >= x1 or y0 >= y1:
        return (0, 0, 0, 0)
    return (y0, y1, x0, x1)


def _hit_box(best, o, D, b: Box, cam, T: np.ndarray):
    win = _box_pixel_window(b, cam, T) if cam is not None else None
    if win is None:
        sl = (slice(None), slice(None))
    else:
        y0, y1, x0, x1 = win
        if y0 == y1:
            return
        sl = (slice(y0, y1), slice(x0, x1))
    Ds = D[:, sl[0], sl[1]]
    with np.errstate(divide="ignore", invalid="ignore"):
        t_near = np.full(Ds.shape[1:], -np.inf)
        t_far = np.full(Ds.shape[1:], np.inf)
        for a in range(3):
            inv = 1.0 / Ds[a]
            t1 = (b.lo[a] - o[a]) * inv
            t2 = (b.hi[a] - o[a]) * inv
            lo = np.minimum(t1, t2)
            hi = np.maximum(t1, t2)
            par = Ds[a] == 0
            inside = (o[a] >= b.lo[a]) & (o[a] <= b.hi[a])
            lo = np.where(par, np.where(inside, -np.inf, np.inf), lo)
            hi = np.where(par, np.where(inside, np.inf, -np.inf), hi)
            t_near = np.maximum(t_near, lo)
            t_far = np.minimum(t_far, hi)
    hit = (t_near <= t_far) & (t_near > 0)
    sub = best[sl[0], sl[1]]
    upd = hit & (t_near < sub)
    sub[upd] = t_near[upd]


def _hit_facade(best, o, D, f: Facade):
    toward = (f.x - o[0]) * D[0] > 0
    sel = np.nonzero(toward.ravel())[0]
    if sel.size == 0:
        return
    Dx, Dy, Dz = (D[a].ravel()[sel] for a in range(3))
    lam = (f.x - o[0]) / Dx
    y = o[1] + lam * Dy
    z = o[2] + lam * Dz
    ok = _in_range(y, f.y_top, f.y_bot) & _in_range(z, f.z0, f.z1)
    depth = np.where(ok, lam, np.inf)
    # window recesses: cells indexed from (z0, y_top)
    cz, cy = f.cell
    wz, wy = f.win
    iz = np.floor((z - f.z0) / cz)
    iy = np.floor((y - f.y_top) / cy)
    nz, ny = f.windows.shape
    inside_grid = ok & (iz >= 0) & (iz < nz) & (iy >= 0) & (iy < ny)
    izc = np.clip(np.where(inside_grid, iz, 0), 0, nz - 1).astype(np.int64)
    iyc = np.clip(np.where(inside_grid, iy, 0), 0, ny - 1).astype(np.int64)
    has_win = inside_grid & f.windows[izc, iyc]
    wz0 = f.z0 + izc * cz + 0.5 * (cz - wz)
    wy0 = f.y_top + iyc * cy + 0.5 * (cy - wy)
    wz1, wy1 = wz0 + wz, wy0 + wy
    in_win = has_win & (z > wz0) & (z < wz1) & (y > wy0) & (y < wy1)
    if np.any(in_win):
        w = np.nonzero(in_win)[0]
        xb = f.x + f.side * f.recess
        lam_b = (xb - o[0]) / Dx[w]
        # the ray may leave the opening's (y, z) rectangle through a side wall first
        lam_exit = np.full(w.size, np.inf)
        with np.errstate(divide="ignore", invalid="ignore"):
            for ob, Db, lo, hi in ((o[1], Dy[w], wy0[w], wy1[w]), (o[2], Dz[w], wz0[w], wz1[w])):
                t_hi = np.where(Db > 0, (hi - ob) / Db, np.inf)
                t_lo = np.where(Db < 0, (lo - ob) / Db, np.inf)
                lam_exit = np.minimum(lam_exit, np.minimum(t_hi, t_lo))
        depth[w] = np.minimum(lam_b, lam_exit)
    flat = best.reshape(-1)
    cur = flat[sel]
    upd = depth < cur
    flat[sel[upd]] = depth[upd]


# ------------------------------------------------------------------ scenes
def _poses_along_z(n: int, step: float, yaw_jitter: float = 0.0, rng=None) -> list:
    poses = []
    for k in range(n):
        T = np.eye(4)
        if yaw_jitter > 0:
            a = rng.uniform(-yaw_jitter, yaw_jitter)
            b = rng.uniform(-yaw_jitter, yaw_jitter)
            ca, sa, cb, sb = np.cos(a), np.sin(a), np.cos(b), np.sin(b)
            Ry = np.array([[ca, 0, sa], [0, 1, 0], [-sa, 0, ca]])
            Rx = np.array([[1, 0, 0], [0, cb, -sb], [0, sb, cb]])
            T[:3, :3] = Ry @ Rx
        T[:3, 3] = (CAM_OFFSET[0], CAM_OFFSET[1], CAM_OFFSET[2] + step * k)
        poses.append(T)
    return poses


def tiny_scene(seed: int = 0, n_frames: int = 4, yaw_jitter: float = 0.0,
               wall_z: float = 12.0, cube_at=(-1.5, 7.0), noise: float = 0.02,
               width: int = 320, height: int = 96, focal: float = 200.0) -> Scene:
    """Plain-method tiny workload: 4 depth maps 320x96, f = 200 px, poses 0.5 m apart
    along +z; ground plane, one fronto-parallel wall (z = 12 m, x in [-6, 6], 4 m high)
    and one 1 m cube on the ground; N(0, 0.02 m) depth noise; d_max = 30 m."""
    rng = np.random.Generator(np.random.PCG64([seed, 0]))
    cam = Camera.pinhole(width, height, focal)
    poses = _poses_along_z(n_frames, 0.5, yaw_jitter, rng)
    ground = Rect(1, ROAD_Y, np.array([-6.0, -5.0]), np.array([6.0, wall_z]))
    wall = Rect(2, wall_z, np.array([-6.0, ROAD_Y - 4.0]), np.array([6.0, ROAD_Y]))
    cx, cz = cube_at
    cube = Box(np.array([cx - 0.5, ROAD_Y - 1.0, cz - 0.5]), np.array([cx + 0.5, ROAD_Y, cz + 0.5]))
    return Scene(cam, poses, rects=[ground, wall], boxes=[cube], d_max=30.0,
                 noise_sigma=noise, seed=seed, name="tiny")


def street_scene(seed: int = 0, length: float = 100.0, frame_step: float = 0.5,
                 width: int = 1241, height: int = 376, focal: float = 718.0,
                 n_cars: int = 20, invalid_prob: float = 0.15, noise_quad: float = 0.001,
                 d_max: float = 40.0) -> Scene:
    """Driving-shaped street: road plane, facades at x = +-8 m (12 m high) with random
    window recesses (1.2 x 1.5 m, 0.3 m deep, ~30% of a 2 x 3 m lattice), ``n_cars``
    car boxes (about 4.2 x 1.5 x 1.8 m +-10%, |x| in [2.5, 6], z in [5, length]);
    depth noise sigma = noise_quad * z^2 m; ``invalid_prob`` of pixels dropped;
    ``length / frame_step`` poses along +z."""
    rng = np.random.Generator(np.random.PCG64([seed, 0]))
    cam = Camera.pinhole(width, height, focal)
    n_frames = int(round(length / frame_step))
    z1 = length + d_max
    poses = _poses_along_z(n_frames, frame_step)
    road = Rect(1, ROAD_Y, np.array([-8.0, -1.0]), np.array([8.0, z1]))
    facades = []
    for side, x in ((+1, 8.0), (-1, -8.0)):
        nz = int(np.ceil((z1 + 1.0) / 2.0))
        ny = 4
        win = rng.random((nz, ny)) < 0.3
        facades.append(Facade(x=x, side=side, y_top=ROAD_Y - 12.0, y_bot=ROAD_Y,
                              z0=-1.0, z1=z1, windows=win))
    boxes = []
    for _ in range(n_cars):
        L = 4.2 * rng.uniform(0.9, 1.1)
        Hh = 1.5 * rng.uniform(0.9, 1.1)
        Wd = 1.8 * rng.uniform(0.9, 1.1)
        xc = rng.uniform(2.5, 6.0) * (1 if rng.random() < 0.5 else -1)
        zc = rng.uniform(5.0, length)
        boxes.append(Box(np.array([xc - Wd / 2, ROAD_Y - Hh, zc - L / 2]),
                         np.array([xc + Wd / 2, ROAD_Y, zc + L / 2])))
    return Scene(cam, poses, rects=[road], boxes=boxes, facades=facades, d_max=d_max,
                 noise_quad=noise_quad, invalid_prob=invalid_prob, seed=seed, name="street")


def segment_scenes(n_segments: int = 64, lo: float = 50.0, hi: float = 500.0, base_seed: int = 1,
                   **kw) -> list:
    """Independent street segments with lengths uniform in [lo, hi] m, seeds base_seed.."""
    rng = np.random.Generator(np.random.PCG64([base_seed, 7]))
    lengths = rng.uniform(lo, hi, n_segments)
    return [street_scene(seed=base_seed + i, length=float(np.round(Lm / 0.5) * 0.5), **kw)
            for i, Lm in enumerate(lengths)]


# ------------------------------------------------------- many maps in parallel
_WORKER_SCENES: dict = {}


def _street_frame(task):
    """Depth map k of street_scene(seed, length), built once per worker process."""
    seed, length, k = task
    sc = _WORKER_SCENES.get((seed, length))
    if sc is None:
        sc = _WORKER_SCENES[(seed, length)] = street_scene(seed=seed, length=length)
    return sc.depth_map(k)


def street_depth_maps(specs, workers: int = 1, chunksize: int = 8):
    """Depth maps of several streets, in order: for each (seed, length) of ``specs`` its
    frames 0, 1, ...; yields (spec index, frame, depth map).  With workers > 1 they are
    made by a 'spawn' process pool (safe in a parent that already uses a GPU) and handed
    over one by one, so the caller holds only what it has not consumed yet."""
    tasks = []
    for i, (seed, length) in enumerate(specs):
        n = int(round(length / 0.5))
        tasks += [(i, seed, length, k) for k in range(n)]
    if workers <= 1:
        for i, seed, length, k in tasks:
            yield i, k, _street_frame((seed, length, k))
        return
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        for (i, seed, length, k), d in zip(tasks, pool.imap(_street_frame, [t[1:] for t in tasks],
                                                             chunksize=chunksize)):
            yield i, k, d
