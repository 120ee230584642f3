"""Pins of the surface-extraction oracle (oracle/surface_oracle.py) to facts that do not
come from the oracle itself:

* the Kuhn split: six tetrahedra of volume 1/6 filling the cube, orientation signs
  equal to the determinant;
* a plane level set: every vertex on the plane, area = the closed-form cross-section,
  normals along +grad u;
* a sphere: area and enclosed volume converge to 4 pi r^2 and 4/3 pi r^3;
* random fields with a non-negative border: the mesh is a closed, consistently
  oriented 2-manifold, and its enclosed volume equals the brute-force volume of
  {u < 0} under linear interpolation, tetrahedron by tetrahedron, from scipy's
  convex hull;
* Omega restriction: values on Omega-bar never change the output, and a cube with
  an unobserved corner is never meshed;
* translation by one block moves every vertex by 8 s and keeps the topology.
"""

import itertools
from collections import Counter

import numpy as np
import pytest

from oracle import surface_oracle as S

spatial = pytest.importorskip("scipy.spatial")


def box_keys(nx, ny, nz, origin=(0, 0, 0), seg=0):
    return [(seg, origin[0] + bx, origin[1] + by, origin[2] + bz)
            for bz in range(nz) for by in range(ny) for bx in range(nx)]


def centres(keys, s):
    """[nb*512, 3] voxel-centre world positions ((i, j, k) + 1/2) s, written out here
    independently of the oracle: voxel l of block (bx, by, bz) has
    (i, j, k) = 8 (bx, by, bz) + (l % 8, l // 8 % 8, l // 64)."""
    out = []
    for _, bx, by, bz in keys:
        for l in range(512):
            i, j, k = 8 * bx + l % 8, 8 * by + (l // 8) % 8, 8 * bz + l // 64
            out.append(((i + 0.5) * s, (j + 0.5) * s, (k + 0.5) * s))
    return np.array(out)


def field(keys, s, fn):
    """u [nb, 512] from a function of the voxel-centre world positions."""
    w = centres(keys, s)
    return fn(w[:, 0], w[:, 1], w[:, 2]).reshape(len(keys), 512)


def test_kuhn_split_fills_the_cube():
    tets = S.kuhn_tets()
    assert len(tets) == 6
    total = 0.0
    for codes, orient in tets:
        P = np.array([S.corner_offset(c) for c in codes], dtype=float)
        det = np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))
        assert np.sign(det) == orient and abs(abs(det) - 1.0) < 1e-12
        total += abs(det) / 6.0
        # monotone edges: a lower tetrahedron index is a bitwise subset
        for i, j in itertools.combinations(range(4), 2):
            assert codes[i] & codes[j] == codes[i]
    assert abs(total - 1.0) < 1e-12
    # random points of the cube fall in exactly one tetrahedron (x_pi0 >= x_pi1 >= x_pi2)
    rng = np.random.default_rng(0)
    for x in rng.random((200, 3)):
        inside = 0
        for codes, _ in tets:
            P = np.array([S.corner_offset(c) for c in codes], dtype=float)
            bc = np.linalg.solve(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]).T, x - P[0])
            inside += bool(np.all(bc >= -1e-12) and bc.sum() <= 1 + 1e-12)
        assert inside == 1


def test_plane_closed_form():
    s = 0.1
    keys = box_keys(3, 3, 3)
    z0 = 1.2345
    u = field(keys, s, lambda x, y, z: (z - z0) / 0.3)
    om = np.ones_like(u, dtype=bool)
    pos, ids = S.extract_surface(keys, u, om, s)
    assert len(pos) > 0
    assert np.max(np.abs(pos[:, :, 2] - z0)) < 1e-12
    # 24 x 24 voxel centres in x, y: 23 x 23 cells of s^2
    assert abs(S.mesh_area(pos) - (23 * s) ** 2) < 1e-10
    n = np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0])
    assert np.all(n[:, 2] > 0)  # from the negative side (z < z0) to the positive
    assert np.allclose(n[:, :2], 0.0, atol=1e-14)


def test_sphere_area_and_volume_converge():
    errs = []
    for s in (0.2, 0.1, 0.05):
        nblk = int(np.ceil(2.4 / (8 * s)))
        keys = box_keys(nblk, nblk, nblk)
        c = np.array([1.2, 1.2, 1.2]) + 0.0123
        r = 0.8
        u = field(keys, s, lambda x, y, z: np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - r)
        pos, _ = S.extract_surface(keys, u, np.ones_like(u, dtype=bool), s)
        ea = abs(S.mesh_area(pos) / (4 * np.pi * r * r) - 1)
        ev = abs(S.mesh_volume(pos) / (4 / 3 * np.pi * r ** 3) - 1)
        errs.append((ea, ev))
    assert errs[-1][0] < 0.02 and errs[-1][1] < 0.01, errs
    # second-order convergence of the volume: halving s cuts the error at least 2.5 x
    assert errs[2][1] < errs[1][1] / 2.5 < errs[0][1] / 6.0, errs


def negative_volume_brute_force(keys, u, om, s):
    """Volume of {u < 0} under linear interpolation on each Kuhn tetrahedron of each
    meshed cube: the convex hull of the negative corners and the edge zeros."""
    nb = len(keys)
    uf = u.reshape(-1)
    corners = S.corner_indices(keys, nb)
    world = S.voxel_world(keys, s)
    total = 0.0
    for cube in range(nb * 512):
        cs = corners[cube]
        if np.any(cs < 0) or not np.all(om.reshape(-1)[cs]):
            continue
        for codes, _ in S.kuhn_tets():
            P = world[[cs[c] for c in codes]]
            U = uf[[cs[c] for c in codes]]
            if np.all(U >= 0):
                continue
            if np.all(U < 0):
                total += abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))) / 6
                continue
            pts = [P[i] for i in range(4) if U[i] < 0]
            for i, j in itertools.combinations(range(4), 2):
                if (U[i] < 0) != (U[j] < 0):
                    t = U[i] / (U[i] - U[j])
                    pts.append(P[i] + t * (P[j] - P[i]))
            pts = np.array(pts)
            if len(pts) >= 4 and np.linalg.matrix_rank(pts[1:] - pts[0], tol=1e-12) == 3:
                total += spatial.ConvexHull(pts).volume
    return total


@pytest.mark.parametrize("seed", [0, 1])
def test_random_field_closed_oriented_and_volume(seed):
    rng = np.random.default_rng(seed)
    s = 0.1
    keys = box_keys(2, 2, 1)
    w = centres(keys, s)
    u = rng.normal(0.2, 1.0, size=len(keys) * 512)
    ijk = np.floor(w / s).astype(int)
    border = (ijk[:, 0] == 0) | (ijk[:, 0] == 15) | (ijk[:, 1] == 0) | (ijk[:, 1] == 15) | \
             (ijk[:, 2] == 0) | (ijk[:, 2] == 7)
    u[border] = np.abs(u[border]) + 0.1
    u = u.reshape(len(keys), 512)
    om = np.ones_like(u, dtype=bool)
    pos, ids = S.extract_surface(keys, u, om, s)
    assert len(pos) > 50
    # vertices with the same edge id coincide
    flat_ids, flat_pos = ids.reshape(-1), pos.reshape(-1, 3)
    first = {}
    for i, p in zip(flat_ids.tolist(), flat_pos):
        if i in first:
            assert np.array_equal(first[i], p)
        else:
            first[i] = p
    # closed and consistently oriented: each directed edge once, its reverse once
    directed = Counter()
    for a, b, c in ids.tolist():
        for e in ((a, b), (b, c), (c, a)):
            directed[e] += 1
    assert all(n == 1 for n in directed.values())
    assert all(directed[(b, a)] == 1 for (a, b) in directed)
    vol = S.mesh_volume(pos)
    ref = negative_volume_brute_force(keys, u, om, s)
    assert ref > 0 and abs(vol - ref) <= 1e-9 * ref, (vol, ref)


def test_omega_restriction():
    rng = np.random.default_rng(5)
    s = 0.1
    keys = box_keys(2, 1, 1)
    u = field(keys, s, lambda x, y, z: (x - 0.77) + 0.3 * (y - 0.41))
    om = rng.random(u.shape) > 0.05
    pos, ids = S.extract_surface(keys, u, om, s)
    u2 = u.copy()
    u2[~om] = rng.normal(size=int((~om).sum()))
    pos2, ids2 = S.extract_surface(keys, u2, om, s)
    assert np.array_equal(pos, pos2) and np.array_equal(ids, ids2)
    # a triangle's cube (the lower end of its first vertex's edge lies in it) has all
    # eight corners observed: check through the cube set that produced the ids
    corners = S.corner_indices(keys, len(keys))
    omf = om.reshape(-1)
    meshed = {c for c in range(len(keys) * 512) if np.all(corners[c] >= 0) and np.all(omf[corners[c]])}
    full_pos, _ = S.extract_surface(keys, u, np.ones_like(om), s)
    assert len(full_pos) > len(pos)
    # every vertex id's lower end is a corner of some meshed cube
    for v in set((ids // 8).reshape(-1).tolist()):
        assert any(v in corners[c] for c in meshed if abs(c - v) < 600)


def test_translation_by_one_block():
    s = 0.1
    keys = box_keys(2, 2, 2)
    keys_t = box_keys(2, 2, 2, origin=(1, 0, -1))
    fn = lambda x, y, z: np.sin(3 * x) + np.cos(2 * y) * z - 0.4
    u = field(keys, s, fn)
    shift = np.array([8 * s, 0.0, -8 * s])
    u_t = field(keys_t, s, lambda x, y, z: fn(x - shift[0], y - shift[1], z - shift[2]))
    om = np.ones_like(u, dtype=bool)
    pos, ids = S.extract_surface(keys, u, om, s)
    pos_t, ids_t = S.extract_surface(keys_t, u_t, om, s)
    assert len(pos) == len(pos_t) > 0
    assert np.array_equal(ids, ids_t)  # same block order, same local structure
    assert np.max(np.abs(pos_t - (pos + shift))) < 1e-12


def test_segments_do_not_connect():
    s = 0.1
    keys = [(0, 0, 0, 0), (1, 1, 0, 0)]  # +x neighbour key but another segment
    u = field(keys, s, lambda x, y, z: x - 0.751)
    pos, ids = S.extract_surface(keys, u, np.ones_like(u, dtype=bool), s)
    # the level set x = 0.751 lies between voxel centres 0.75 and 0.85, across the
    # blocks: no cube spans both segments, so nothing is meshed
    assert len(pos) == 0
    keys2 = [(0, 0, 0, 0), (0, 1, 0, 0)]
    pos2, _ = S.extract_surface(keys2, field(keys2, s, lambda x, y, z: x - 0.751),
                                np.ones((2, 512), dtype=bool), s)
    assert len(pos2) > 0 and abs(S.mesh_area(pos2) - (7 * s) ** 2) < 1e-10


def test_zero_corner_is_non_negative():
    """S3: u = 0 counts as non-negative.  On the plane through the voxel centres of
    layer k = 4 the zero corners are the upper ends of the crossing edges, so every
    vertex sits at t = 1 of an edge whose lower end is in layer 3."""
    s = 0.1
    keys = box_keys(1, 1, 1)
    u = field(keys, s, lambda x, y, z: np.round(z / s - 0.5) - 4.0)
    pos, ids = S.extract_surface(keys, u, np.ones_like(u, dtype=bool), s)
    assert len(pos) > 0
    assert np.max(np.abs(pos[:, :, 2] - 4.5 * s)) < 1e-12
    lower = ids // 8
    assert np.all(lower // 64 == 3)
    assert abs(S.mesh_area(pos) - (7 * s) ** 2) < 1e-10


def test_blocks_partition_the_mesh():
    """Meshing the blocks one call at a time (each call takes the cubes whose lower
    corner lies in its block) gives the whole mesh's triangles, split by block, in the
    same order."""
    rng = np.random.default_rng(31)
    s = 0.1
    keys = box_keys(2, 2, 1)
    u = rng.normal(0.1, 1.0, size=(len(keys), 512))
    om = rng.random((len(keys), 512)) < 0.95
    pos, ids = S.extract_surface(keys, u, om, s)
    parts = [S.extract_surface(keys, u, om, s, blocks=[b]) for b in range(len(keys))]
    assert sum(len(pp) for pp, _ in parts) == len(pos)
    assert sum(len(pp) > 0 for pp, _ in parts) >= 3
    assert np.array_equal(np.concatenate([pp for pp, _ in parts]), pos)
    assert np.array_equal(np.concatenate([ii for _, ii in parts]), ids)
