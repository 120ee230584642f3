"""CPU FP64 oracle of surface extraction from the regularised map -- TEST INFRASTRUCTURE ONLY.

The paper's pipeline extracts a surface from the regularised model and hands it
to other components (Section II, Fig. 1); it names no extraction method.  The
reading taken here (S1-S5) is the zero level set of u, triangulated cube by cube
over the voxel-centre lattice and restricted to the observed set Omega:

  S1  a cube is the 2x2x2 voxel centres v + {0,1}^3; it is meshed only when all
      eight corners are in Omega (u is meaningless on Omega-bar, Section III-B,
      so no surface is invented at the border of the observed set);
  S2  each cube is split into the six tetrahedra of the Kuhn (Freudenthal)
      triangulation along its main diagonal: for a permutation pi of the axes the
      tetrahedron c0 = 0, c1 = e_pi0, c2 = e_pi0 + e_pi1, c3 = (1,1,1).  The same
      split in every cube triangulates the whole lattice consistently, so the mesh
      is closed wherever the negative region stays inside the meshed cubes;
  S3  a corner is negative when u < 0 (behind the observed surface: u is the
      normalised signed distance d - z, positive in free space); u = 0 is
      non-negative;
  S4  a vertex lies on a tetrahedron edge whose ends differ in sign, at the linear
      zero t = u_a / (u_a - u_b) measured from the edge's componentwise-lower end
      a (Kuhn edges are monotone, so the lower end is the one of lower tetrahedron
      index), world position ((i, j, k) + 1/2) s along the edge;
  S5  triangles are wound so that their normal (v1 - v0) x (v2 - v0) points from
      the negative to the non-negative side (towards the camera).

Output order: blocks by index, cubes by local linear index lx + 8 ly + 64 lz of
their lower corner, tetrahedra in the lexicographic order of pi, triangles within
a tetrahedron as listed in ``_tet_triangles``.  A vertex is identified by its edge:
id = (flat voxel index of the lower end) * 8 + direction bits (1 = +x, 2 = +y,
4 = +z), flat index = block * 512 + local index.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It shares no code with the CUDA path.
"""

from __future__ import annotations

import itertools

import numpy as np

BLOCK = 8
BLOCK_VOXELS = BLOCK ** 3

# S2: the six permutations of the axes, in lexicographic order
KUHN_PERMS = list(itertools.permutations(range(3)))


def perm_sign(seq) -> int:
    """+1 for an even permutation of sorted(seq), -1 for an odd one (inversion count)."""
    inv = sum(1 for i in range(len(seq)) for j in range(i + 1, len(seq)) if seq[i] > seq[j])
    return -1 if inv % 2 else 1


def kuhn_tets():
    """[(corner bit codes c0..c3, orientation sign)] for the six tetrahedra of S2.

    A corner code has bit a set when the corner is offset by +1 along axis a.  The
    orientation sign is that of det[c1 - c0, c2 - c0, c3 - c0], which equals the
    sign of the permutation (column operations reduce it to det[e_pi0, e_pi1, e_pi2])."""
    out = []
    for pi in KUHN_PERMS:
        c1 = 1 << pi[0]
        c2 = c1 | (1 << pi[1])
        out.append(((0, c1, c2, 7), perm_sign(pi)))
    return out


def corner_offset(code: int):
    return (code & 1, (code >> 1) & 1, (code >> 2) & 1)


def _tet_triangles(neg, orient):
    """Triangles of one tetrahedron as lists of three (i, j) tetrahedron-vertex pairs
    with i < j (the edge from vertex i to vertex j), wound per S5.

    neg[i]: vertex i is negative; orient: the tetrahedron's orientation sign.

    One vertex alone on its side: the triangle cuts the three edges at that vertex,
    taken in the order of an even permutation that brings it first, (i; j, k, l) in
    {(0; 1,2,3), (1; 0,3,2), (2; 3,0,1), (3; 2,1,0)}; for a positively oriented
    tetrahedron that triangle's normal points away from the lone vertex.  Two and
    two: with A < B the negatives and C < D the non-negatives, the quadrilateral
    AC, AD, BD, BC is split along AC-BD; for (A, B, C, D) an even permutation of a
    positively oriented tetrahedron its normal points from {A, B} to {C, D}."""
    k = int(sum(neg))
    if k == 0 or k == 4:
        return []
    e = lambda i, j: (min(i, j), max(i, j))
    if k in (1, 3):
        lone = [i for i in range(4) if neg[i] == (k == 1)][0]
        others = {0: (1, 2, 3), 1: (0, 3, 2), 2: (3, 0, 1), 3: (2, 1, 0)}[lone]
        tri = [e(lone, others[0]), e(lone, others[1]), e(lone, others[2])]
        # normal away from the lone vertex when orient > 0; it must point to the
        # non-negative side, i.e. away from a lone negative, towards a lone non-negative
        away_ok = k == 1
        if (orient > 0) != away_ok:
            tri = [tri[0], tri[2], tri[1]]
        return [tri]
    A, B = [i for i in range(4) if neg[i]]
    C, D = [i for i in range(4) if not neg[i]]
    s = orient * perm_sign((A, B, C, D))
    tris = [[e(A, C), e(A, D), e(B, D)], [e(A, C), e(B, D), e(B, C)]]
    if s < 0:
        tris = [[t[0], t[2], t[1]] for t in tris]
    return tris


def corner_indices(keys, n_blocks: int):
    """[nb*512, 8] flat voxel index of each cube corner (corner code order), -1 where
    the corner's block is not allocated.  keys: (segment, bx, by, bz) per block."""
    index = {tuple(int(c) for c in k): b for b, k in enumerate(keys)}
    l = np.arange(BLOCK_VOXELS)
    lx, ly, lz = l % BLOCK, (l // BLOCK) % BLOCK, l // (BLOCK * BLOCK)
    out = np.full((n_blocks * BLOCK_VOXELS, 8), -1, dtype=np.int64)
    for code in range(8):
        ox, oy, oz = corner_offset(code)
        nx, ny, nz = lx + ox, ly + oy, lz + oz
        cx, cy, cz = nx // BLOCK, ny // BLOCK, nz // BLOCK  # block carry (0 or 1)
        nl = (nx % BLOCK) + BLOCK * (ny % BLOCK) + BLOCK * BLOCK * (nz % BLOCK)
        for b, k in enumerate(keys):
            seg, bx, by, bz = (int(c) for c in k)
            col = np.full(BLOCK_VOXELS, -1, dtype=np.int64)
            for carry in set(zip(cx.tolist(), cy.tolist(), cz.tolist())):
                nbk = index.get((seg, bx + carry[0], by + carry[1], bz + carry[2]), -1)
                if nbk < 0:
                    continue
                sel = (cx == carry[0]) & (cy == carry[1]) & (cz == carry[2])
                col[sel] = nbk * BLOCK_VOXELS + nl[sel]
            out[b * BLOCK_VOXELS:(b + 1) * BLOCK_VOXELS, code] = col
    return out


def voxel_world(keys, voxel_size: float):
    """[nb*512, 3] world position ((i, j, k) + 1/2) s of every voxel centre."""
    c = np.asarray(keys, dtype=np.int64).reshape(-1, 4)
    l = np.arange(BLOCK_VOXELS)
    loc = np.stack([l % BLOCK, (l // BLOCK) % BLOCK, l // (BLOCK * BLOCK)], axis=1)
    ijk = c[:, None, 1:4] * BLOCK + loc[None, :, :]
    return ((ijk.astype(np.float64) + 0.5) * voxel_size).reshape(-1, 3)


def extract_surface(keys, u, om, voxel_size: float, blocks=None):
    """Zero level set of u over Omega (S1-S5).

    keys: [nb] (segment, bx, by, bz) in block-index order; u: [nb, 512]; om: [nb, 512]
    bool; blocks: optional block indices whose cubes (by lower corner) alone are meshed.
    Returns (pos [n, 3, 3] float64 world metres, ids [n, 3] int64 edge ids)."""
    nb = len(keys)
    u = np.asarray(u, dtype=np.float64).reshape(-1)
    om = np.asarray(om, dtype=bool).reshape(-1)
    corners = corner_indices(keys, nb)
    world = voxel_world(keys, voxel_size)
    valid = np.all(corners >= 0, axis=1)
    valid[valid] = np.all(om[corners[valid]], axis=1)
    # only cubes with a sign change can hold a triangle
    cu = np.where(valid[:, None], u[np.where(corners >= 0, corners, 0)], 0.0)
    neg = cu < 0
    crossing = valid & np.any(neg, axis=1) & ~np.all(neg, axis=1)
    if blocks is not None:
        chosen = np.zeros(nb, dtype=bool)
        chosen[np.asarray(blocks, dtype=np.int64)] = True
        crossing &= np.repeat(chosen, BLOCK_VOXELS)
    tets = kuhn_tets()
    pos, ids = [], []
    for cube in np.nonzero(crossing)[0]:  # ascending = block, then local index
        for codes, orient in tets:
            vidx = [int(corners[cube, c]) for c in codes]
            vu = [u[v] for v in vidx]
            for tri in _tet_triangles([x < 0 for x in vu], orient):
                tp, ti = [], []
                for i, j in tri:
                    a, b = vidx[i], vidx[j]
                    t = vu[i] / (vu[i] - vu[j])
                    tp.append(world[a] + t * (world[b] - world[a]))
                    ti.append(a * 8 + (codes[j] ^ codes[i]))
                pos.append(tp)
                ids.append(ti)
    if not pos:
        return np.zeros((0, 3, 3)), np.zeros((0, 3), dtype=np.int64)
    return np.asarray(pos, dtype=np.float64), np.asarray(ids, dtype=np.int64)


# ------------------------------------------------------------- mesh measures
def mesh_area(pos) -> float:
    """Total triangle area."""
    if len(pos) == 0:
        return 0.0
    n = np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0])
    return float(0.5 * np.linalg.norm(n, axis=1).sum())


def mesh_volume(pos) -> float:
    """Signed volume enclosed by a closed mesh (divergence theorem); positive when the
    normals point outwards from the enclosed region."""
    if len(pos) == 0:
        return 0.0
    return float(np.einsum("ij,ij->i", pos[:, 0], np.cross(pos[:, 1], pos[:, 2])).sum() / 6.0)
