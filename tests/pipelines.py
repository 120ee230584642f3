"""Runs one scene through the oracle and through the C ABI on the same inputs."""

import numpy as np

from oracle import denser_oracle as O


def oracle_params(**kw):
    return O.Params(**kw)


def oracle_K(cam):
    return O.Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)


def run_oracle(scene, depths, iters, params=None, frames=None, segment=0):
    params = params or O.Params()
    K = oracle_K(scene.camera)
    g = O.SparseGrid(params)
    news = []
    frames = range(len(depths)) if frames is None else frames
    for k in frames:
        news.append(O.alloc_blocks(g, depths[k], K, scene.poses[k], segment))
        O.fuse_depth(g, depths[k], K, scene.poses[k], segment)
    prob = O.regularize(g, iters) if iters > 0 else None
    return g, news, prob


def run_gpu(scene, depths, iters, segment=0, frames=None, stream=None, device_depth=True, **params):
    """Returns (DenserMap, per-frame new counts, reg stats or None)."""
    import torch
    from paper_1604_03734_gb300 import native as N
    m = N.DenserMap(**params)
    cam = scene.camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    frames = range(len(depths)) if frames is None else frames
    news = []
    for k in frames:
        d = torch.from_numpy(np.ascontiguousarray(depths[k]))
        if device_depth:
            d = d.cuda()
        news.append(N.denser_alloc_blocks(m.ctx, d, K, scene.poses[k], segment, stream, count=True))
        N.denser_fuse_depth(m.ctx, d, K, scene.poses[k], segment, stream)
    st = N.denser_regularize(m.ctx, iters, 0.0, 0, stream) if iters > 0 else None
    return m, news, st


def oracle_coords(g):
    return g.coords().astype(np.int32)
