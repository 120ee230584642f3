"""Small builders for oracle tests: maps made directly from block lists."""

import numpy as np

from oracle.denser_oracle import BLOCK_VOXELS, Intrinsics, Params, SparseGrid


def grid_from_blocks(keys, f=None, w=None, params=Params()):
    """SparseGrid holding ``keys`` (in the given order) with per-voxel f, w [nb, 512]."""
    g = SparseGrid(params)
    g.add_blocks([tuple(int(v) for v in k) for k in keys])
    if f is not None:
        g.f[:] = f
    if w is not None:
        g.w[:] = w
    return g


def box_keys(nx, ny, nz, seg=0, origin=(0, 0, 0)):
    """Keys of a fully allocated nx*ny*nz box of blocks in (bz, by, bx) order."""
    ox, oy, oz = origin
    return [(seg, ox + x, oy + y, oz + z) for z in range(nz) for y in range(ny) for x in range(nx)]


def random_fw(rng, nb, p_omega=0.8, wmax=5):
    f = rng.uniform(-1, 1, (nb, BLOCK_VOXELS))
    w = rng.integers(1, wmax + 1, (nb, BLOCK_VOXELS)).astype(np.float64)
    w[rng.random((nb, BLOCK_VOXELS)) >= p_omega] = 0.0
    return f, w


def intrinsics_of(cam):
    return Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
