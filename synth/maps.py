"""Seeded synthetic map states: block coordinates and per-voxel f, w, u.

This module only makes inputs for tests and measurements that start from a map
rather than from depth maps (surface extraction): the blocks around the surface of a
street-like scene and a regularised-looking u on them.  It holds none of the
method's arithmetic; both the CPU oracle and the CUDA path consume what it returns.

Layout (the library's): coords int32 [n, 4] = (segment, bx, by, bz), voxel l of a
block at local (l % 8, l // 8 % 8, l // 64), centre ((8 b + local) + 1/2) s.
"""

from __future__ import annotations

import numpy as np

ROAD_Y = 1.65


def _centres(coords: np.ndarray, s: float) -> np.ndarray:
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], axis=1)
    ijk = coords[:, None, 1:4].astype(np.int64) * 8 + loc[None]
    return (ijk + 0.5) * s  # [n, 512, 3]


def street_sdf(p: np.ndarray, boxes, margin: float = 2.0) -> np.ndarray:
    """Signed distance-like field of a street (positive in free space): the road
    y = ROAD_Y (y down), facades at |x| = 8 m, and solid boxes.  p: [n, k, 3] points
    in n groups (blocks).  A box only changes the groups whose first point lies within
    `margin` of its extent (farther ones are left to the road and facades, which are
    closer there); `margin` must exceed the group's size."""
    x, y = p[..., 0], p[..., 1]
    d = np.minimum(ROAD_Y - y, 8.0 - np.abs(x))
    for c, h in boxes:
        near = np.nonzero(np.all(np.abs(p[:, 0] - c) <= h + margin, axis=1))[0]
        q = np.abs(p[near] - c) - h
        outside = np.sqrt(np.sum(np.maximum(q, 0.0) ** 2, axis=-1))
        inside = np.minimum(np.max(q, axis=-1), 0.0)
        d[near] = np.minimum(d[near], outside + inside)
    return d


def street_map(seed: int = 0, length: float = 100.0, s: float = 0.1, mu: float = 0.3, n_boxes: int = 20,
               noise: float = 0.05, unobserved: float = 0.05, segment: int = 0):
    """Blocks within reach of the street surface and a noisy normalised field on them.

    Returns coords int32 [n, 4], f, w, u float32 [n, 512].  u = clip(sdf/mu, -1, 1) plus
    N(0, noise); w is an observation count in 1..20, 0 (unobserved) for voxels more than
    mu behind the surface and for a random `unobserved` share of the rest; f = u plus
    N(0, noise).  Streams of one PCG64 generator: boxes, w, u noise, f noise."""
    rng = np.random.default_rng([seed, 7])
    boxes = []
    for _ in range(n_boxes):
        side = rng.choice([-1.0, 1.0])
        c = np.array([side * rng.uniform(2.5, 6.0), ROAD_Y - 0.75, rng.uniform(5.0, length - 5.0)])
        h = np.array([0.75, 0.75, 2.1]) * rng.uniform(0.9, 1.1, 3)
        boxes.append((c, h))
    bs = 8 * s
    reach = mu + bs * np.sqrt(3.0)
    bx = np.arange(int(np.floor(-9.0 / bs)), int(np.ceil(9.0 / bs)) + 1)
    by = np.arange(int(np.floor(-11.0 / bs)), int(np.ceil((ROAD_Y + 1.0) / bs)) + 1)
    bz = np.arange(int(np.floor(-1.0 / bs)), int(np.ceil((length + 1.0) / bs)) + 1)
    Z, Y, X = np.meshgrid(bz, by, bx, indexing="ij")  # ascending (bz, by, bx)
    cand = np.stack([np.full(X.size, segment), X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    centre = (cand[:, 1:4] + 0.5) * bs
    keep = np.abs(street_sdf(centre[:, None, :], boxes)[:, 0]) <= reach
    # facades end 12 m up: drop blocks above the top
    keep &= centre[:, 1] >= ROAD_Y - 12.0 - bs
    coords = cand[keep].astype(np.int32)
    p = _centres(coords, s)
    d = street_sdf(p, boxes, margin=2.0 + bs)
    del p
    n = len(coords)
    w = rng.integers(1, 21, size=(n, 512)).astype(np.float32)
    w[d < -mu] = 0.0
    w[rng.random((n, 512)) < unobserved] = 0.0
    u = (np.clip(d / mu, -1.0, 1.0) + rng.normal(0.0, noise, (n, 512))).astype(np.float32)
    f = (u + rng.normal(0.0, noise, (n, 512))).astype(np.float32)
    return coords, f, w, u


def random_map(seed: int = 0, box=(3, 3, 2), extra: int = 6, s: float = 0.1, unobserved: float = 0.05):
    """A small map: a box of blocks plus scattered single blocks (some in segment 1),
    u a smooth field with noise and exact zeros, w with unobserved voxels."""
    rng = np.random.default_rng([seed, 11])
    keys = [(0, x, y, z) for z in range(box[2]) for y in range(box[1]) for x in range(box[0])]
    while len(keys) < box[0] * box[1] * box[2] + extra:
        k = (int(rng.integers(0, 2)), int(rng.integers(-4, 6)), int(rng.integers(-3, 5)), int(rng.integers(-2, 4)))
        if k not in keys:
            keys.append(k)
    coords = np.array(keys, dtype=np.int32)
    p = _centres(coords, s)
    u = np.sin(2.1 * p[..., 0] + 0.3) * np.cos(1.7 * p[..., 1]) + 0.4 * np.sin(2.9 * p[..., 2]) - 0.1
    u = u + rng.normal(0.0, 0.05, u.shape)
    u[rng.random(u.shape) < 0.01] = 0.0
    w = rng.integers(1, 9, size=u.shape).astype(np.float32)
    w[rng.random(u.shape) < unobserved] = 0.0
    f = np.clip(u, -1, 1).astype(np.float32)
    return coords, f, w, u.astype(np.float32)
