"""Planted mistakes in the oracles must fail their pins.

Each case below changes one expression of an oracle -- a dropped term or factor, a
wrong sign, a shifted, swapped or transposed index, a missing clamp or mask -- and runs
that oracle's pin tests against the changed copy in a child process.  A case passes
when at least one pin fails there, so every pin set is shown to catch the slips it
exists to catch, not only to agree with the oracle as written.

The oracle files are never modified.  A changed Python oracle lives only in the child
process (compiled from the changed text and installed under the oracle's module name
before the pins are imported); a changed C oracle is written to a temporary directory
and built into a library of its own there.  Every case states, as its reason, which
part of the paper or of a stated reading the change breaks.

Changes that leave the method's result as it is are not cases: taking the other
diagonal of a surface quadrilateral, say, meshes the same plane (u is linear on each
tetrahedron), updating u on Omega-bar changes nothing there (w = 0 and div p = 0), and
the segment's place in the key order never shows (one allocation call adds keys of one
segment).
"""

import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PY_DENSER = ("denser_oracle", ["tests/test_oracle_fusion_pins.py", "tests/test_oracle_regularizer_pins.py"])
PY_LASER = ("laser_oracle", ["tests/test_oracle_laser_pins.py"])
PY_STEREO = ("stereo_oracle", ["tests/test_oracle_stereo_pins.py"])
PY_SURFACE = ("surface_oracle", ["tests/test_oracle_surface_pins.py"])
PY_NET = ("net_oracle", ["tests/test_oracle_net_pins.py"])
C_DENSER = ("denser_oracle_c", ["tests/test_oracle_c_pins.py"])

# (id, oracle, text as it stands, planted text, what the change breaks)
CASES = [
    # ---------------------------------------------- allocation (Section III-A, reading R1)
    ("alloc-band-step", PY_DENSER, "z = d + float(n) * h", "z = d + float(n) * s",
     "band samples half a voxel apart"),
    ("alloc-band-end", PY_DENSER, "for n in range(-N, N + 1):\n        z = d",
     "for n in range(-N, N):\n        z = d", "the band reaches mu behind the surface"),
    ("alloc-pixel-centre", PY_DENSER, "uu = (xs.astype(np.float64) + 0.5) - K.cx", "uu = xs.astype(np.float64) - K.cx",
     "rays through pixel centres"),
    ("alloc-focal-swap", PY_DENSER, "Y = (vv * z) / K.fy", "Y = (vv * z) / K.fx", "pinhole back-projection"),
    ("alloc-rotation-transposed", PY_DENSER, "g.append(((R[r, 0] * X + R[r, 1] * Y) + R[r, 2] * Z) + t[r])",
     "g.append(((R[0, r] * X + R[1, r] * Y) + R[2, r] * Z) + t[r])", "camera-to-global pose"),
    ("alloc-truncation", PY_DENSER, "kb = [np.floor(gi / bs) for gi in g]", "kb = [np.trunc(gi / bs) for gi in g]",
     "block of a negative coordinate"),
    ("alloc-key-order", PY_DENSER, "key=lambda k: (k[0], k[3], k[2], k[1]))", "key=lambda k: (k[0], k[1], k[2], k[3]))",
     "new blocks in (segment, bz, by, bx) order"),
    # ----------------------------------------------------- fusion (Section III-A, Eq. 1)
    ("fuse-inverse-rotation", PY_DENSER, "Ri = R.T.copy()", "Ri = R.copy()", "global-to-camera transform"),
    ("fuse-inverse-translation", PY_DENSER, "ti = np.array([-((R[0, r]", "ti = np.array([((R[0, r]",
     "global-to-camera transform"),
    ("fuse-voxel-centre", PY_DENSER, "gx = (i.astype(np.float64) + 0.5) * s", "gx = i.astype(np.float64) * s",
     "voxel centres"),
    ("fuse-pixel-round", PY_DENSER, "pxf = np.floor((K.fx * xc) / zc + K.cx)", "pxf = np.round((K.fx * xc) / zc + K.cx)",
     "pixel (x, y) covers [x, x + 1)"),
    ("fuse-sdf-sign", PY_DENSER, "usdf = d - zc", "usdf = zc - d", "u_SDF = d - z_c, positive in front"),
    ("fuse-no-truncation-test", PY_DENSER, "upd = valid & (usdf >= -p.mu)", "upd = valid",
     "Eq. 1 skips voxels more than mu behind"),
    ("fuse-no-clamp", PY_DENSER, "utsdf = np.minimum(1.0, usdf / p.mu)", "utsdf = usdf / p.mu",
     "u_TSDF = min(1, u_SDF / mu)"),
    ("fuse-unweighted-average", PY_DENSER, "(utsdf + w_old * f_old)", "(utsdf + f_old)",
     "Eq. 1 running weighted average"),
    # ---------------------------------------- Omega, Eq. 3, Eq. 4 (Section III-B)
    ("omega-unobserved", PY_DENSER, "return (grid.w > 0).reshape(-1)", "return (grid.w >= 0).reshape(-1)",
     "Omega = observed voxels"),
    ("neighbour-wrong-side", PY_DENSER, "q[1 + a] += sign", "q[1 + a] -= sign", "neighbour block across a face"),
    ("edge-own-omega", PY_DENSER, "return om[None, :] & nb_om", "return nb_om",
     "Eq. 3 needs both voxels in Omega"),
    ("gradient-sign", PY_DENSER, "u[np.where(e[a], fwd[a], 0)] - u", "u - u[np.where(e[a], fwd[a], 0)]",
     "Eq. 3 forward difference"),
    ("divergence-unmasked-back", PY_DENSER, "back = np.where(hb & e[a][bi], p[a][bi], 0.0)",
     "back = np.where(hb, p[a][bi], 0.0)", "Eq. 4 cases at the Omega boundary"),
    ("divergence-sign", PY_DENSER, "d = d + (own - back)", "d = d + (own + back)", "Eq. 4 backward difference"),
    # ------------------------------------------------- iteration (Section III-C)
    ("dual-projection", PY_DENSER, "p = pt / np.maximum(1.0, nrm)[None, :]",
     "p = pt / np.maximum(1.0, nrm * nrm)[None, :]", "projection onto the unit ball"),
    ("dual-from-u", PY_DENSER, "pt = p + sg * prob.grad(u_bar)", "pt = p + sg * prob.grad(u)",
     "the dual step reads the relaxed primal"),
    ("primal-unweighted-prox", PY_DENSER, "(ut + tau * lam * w * f) / (1.0 + tau * lam * w)",
     "(ut + tau * lam * f) / (1.0 + tau * lam * w)", "the prox of (lam w / 2)(u - f)^2"),
    ("primal-printed-sign", PY_DENSER, "ut = (u - tau * dv) if literal_sign else (u + tau * dv)",
     "ut = (u - tau * dv) if literal_sign else (u - tau * dv)", "reading R7: u + tau div p"),
    ("relaxation-printed", PY_DENSER, "u_bar = u + th * (u - u_old)", "u_bar = u + th * (u - u_bar)",
     "reading R8: extrapolation from the previous iterate"),
    ("energy-half", PY_DENSER, "tv + 0.5 * lam * w * (u - f) ** 2", "tv + lam * w * (u - f) ** 2",
     "reading R10: (lam/2) w (u - f)^2"),
    ("energy-dual-quadratic", PY_DENSER, "dv * dv / (2.0 * lam * wd)", "dv * dv / (lam * wd)",
     "the dual function as min of the Lagrangian"),
    ("energy-dual-sign", PY_DENSER, "-f * dv - dv * dv", "f * dv - dv * dv", "the dual function"),
    ("energy-anisotropic", PY_DENSER, "tv = np.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2])",
     "tv = np.abs(g[0]) + np.abs(g[1]) + np.abs(g[2])", "isotropic TV"),
    # ------------------------------------------------------------ the C restatement
    ("c-band-count", C_DENSER, "const int N = (int)ceil(m->mu / h - 1e-9);", "const int N = (int)floor(m->mu / h - 1e-9);",
     "band samples reach mu"),
    ("c-pixel-centre", C_DENSER, "const double uu = ((double)x + 0.5) - cx;", "const double uu = (double)x - cx;",
     "rays through pixel centres"),
    ("c-truncation", C_DENSER, "k[1 + r] = (int64_t)floor(g / bs);", "k[1 + r] = (int64_t)(g / bs);",
     "block of a negative coordinate"),
    ("c-sdf-sign", C_DENSER, "const double usdf = d - zc;", "const double usdf = zc - d;", "u_SDF = d - z_c"),
    ("c-unweighted-average", C_DENSER, "fb[l] = (utsdf + w_old * fb[l]) / w_new;", "fb[l] = (utsdf + fb[l]) / w_new;",
     "Eq. 1 running weighted average"),
    ("c-neighbour-direction", C_DENSER, "q[1 + (a % 3)] += a < 3 ? 1 : -1;", "q[1 + (a % 3)] += a < 3 ? -1 : 1;",
     "neighbour block across a face"),
    ("c-neighbour-wrap", C_DENSER, "return nb * BV + l - dir * 7 * stride;", "return nb * BV + l;",
     "voxel across a block face"),
    ("c-edge-own-omega", C_DENSER, "return m->w[v] > 0.0 && *fwd >= 0 && m->w[*fwd] > 0.0;",
     "return *fwd >= 0 && m->w[*fwd] > 0.0;", "Eq. 3 needs both voxels in Omega"),
    ("c-divergence-sign", C_DENSER, "d = d + (own - back);", "d = d + (own + back);", "Eq. 4"),
    ("c-projection", C_DENSER, "const double sc = nrm > 1.0 ? nrm : 1.0;", "const double sc = nrm > 1.0 ? nrm * nrm : 1.0;",
     "projection onto the unit ball"),
    ("c-primal-sign", C_DENSER, "const double ut = u_old + tau * dv[v];", "const double ut = u_old - tau * dv[v];",
     "reading R7"),
    ("c-unweighted-prox", C_DENSER, "u = (ut + ((tau * lam) * m->w[v]) * m->f[v])", "u = (ut + (tau * lam) * m->f[v])",
     "the prox of (lam w / 2)(u - f)^2"),
    ("c-relaxation", C_DENSER, "m->ub[v] = u + th * (u - u_old);", "m->ub[v] = u + th * (u - m->ub[v]);", "reading R8"),
    ("c-dual-from-u", C_DENSER, "g[a] = edge(m, nbr, b, l, a, &f) ? m->ub[f] - m->ub[v] : 0.0;",
     "g[a] = edge(m, nbr, b, l, a, &f) ? m->u[f] - m->u[v] : 0.0;", "the dual step reads the relaxed primal"),
    ("c-energy-half", C_DENSER, "sp += tv + ((0.5 * lam) * m->w[v]) * (r * r);", "sp += tv + (lam * m->w[v]) * (r * r);",
     "reading R10"),
    ("c-energy-dual", C_DENSER, "sd += -m->f[v] * d - (d * d) / ((2.0 * lam) * m->w[v]);",
     "sd += -m->f[v] * d - (d * d) / (lam * m->w[v]);", "the dual function"),
    # ------------------------------------------- laser ray fusion (readings L1-L5)
    ("laser-direction-swap", PY_LASER, "d = np.stack([x / r, y / r, z / r], axis=1)",
     "d = np.stack([x / r, z / r, y / r], axis=1)", "L1 ray direction"),
    ("laser-rotation-transposed", PY_LASER, "(R[i, 0] * d[:, 0] + R[i, 1] * d[:, 1]) + R[i, 2] * d[:, 2]",
     "(R[0, i] * d[:, 0] + R[1, i] * d[:, 1]) + R[2, i] * d[:, 2]", "L1 sensor-to-global rotation"),
    ("laser-band-step", PY_LASER, "rho = r + float(n) * h", "rho = r + float(n) * s", "L2 band samples"),
    ("laser-stops-at-hit", PY_LASER, "M = int(np.floor((r + params.mu) / h))", "M = int(np.floor(r / h))",
     "L3 the walk ends mu behind the surface"),
    ("laser-voxel-truncation", PY_LASER, "v = np.stack([np.floor((dg[i] * rho + t[i]) / s)",
     "v = np.stack([np.trunc((dg[i] * rho + t[i]) / s)", "L3 voxel of a negative coordinate"),
    ("laser-repeats", PY_LASER, "keep[1:] = np.any(v[1:] != v[:-1], axis=1)", "keep[1:] = True",
     "L3 a voxel counts once per ray"),
    ("laser-sdf-sign", PY_LASER, "usdf = r[i] - ((e[0] * dg[i, 0] + e[1] * dg[i, 1]) + e[2] * dg[i, 2])",
     "usdf = ((e[0] * dg[i, 0] + e[1] * dg[i, 1]) + e[2] * dg[i, 2]) - r[i]", "L4 range difference"),
    ("laser-voxel-centre", PY_LASER, "e = [(v[:, k].astype(np.float64) + 0.5) * s - t[k] for k in range(3)]",
     "e = [v[:, k].astype(np.float64) * s - t[k] for k in range(3)]", "L4 voxel centres"),
    ("laser-no-truncation-test", PY_LASER, "obs = usdf >= -p.mu", "obs = usdf >= 0", "L4 observed down to -mu"),
    ("laser-no-clamp", PY_LASER, "u_all.append(np.minimum(1.0, usdf[obs] / p.mu))", "u_all.append(usdf[obs] / p.mu)",
     "L4 u_TSDF = min(1, u_SDF / mu)"),
    ("laser-one-count-per-scan", PY_LASER, "w_new = w + cnt", "w_new = w + np.minimum(cnt, 1.0)",
     "L5 w grows by the number of observations"),
    ("laser-unweighted-average", PY_LASER, "(w * f + S.astype(np.float64) / FIX)", "(f + S.astype(np.float64) / FIX)",
     "L5 Eq. 1 weighted average"),
    ("laser-local-index", PY_LASER, "loc[:, 0] + BLOCK * loc[:, 1] + BLOCK * BLOCK * loc[:, 2]",
     "loc[:, 2] + BLOCK * loc[:, 1] + BLOCK * BLOCK * loc[:, 0]", "voxel l = lx + 8 ly + 64 lz"),
    # --------------------------------------------------- stereo (Section IV, D1-D8)
    ("census-ties", PY_STEREO, "sig |= (nb < I).astype(np.uint64)", "sig |= (nb <= I).astype(np.uint64)",
     "D2 Census bit: neighbour darker than the centre"),
    ("census-centre-bit", PY_STEREO, "if dx == 0 and dy == 0:\n                continue",
     "if False:\n                continue", "D2 the centre is not compared with itself"),
    ("hamming-shift-direction", PY_STEREO, "h[d, :, : W - d] = popcount(sigL[:, d:] ^ sigR[:, : W - d])",
     "h[d, :, : W - d] = popcount(sigL[:, : W - d] ^ sigR[:, d:])", "D3 left pixel x + delta"),
    ("hamming-off-image", PY_STEREO, "h = np.full((D, H, W), BITS, dtype=np.int64)\n    for d in range(D):",
     "h = np.full((D, H, W), 0, dtype=np.int64)\n    for d in range(D):", "D3 off-image candidates cost most"),
    ("grad-y-sign", PY_STEREO, "g[1, :-1, :] = u[1:, :] - u[:-1, :]", "g[1, :-1, :] = u[:-1, :] - u[1:, :]",
     "D7 forward differences"),
    ("div-last-column", PY_STEREO, "dx[:, -1] = -px[:, -2]", "dx[:, -1] = px[:, -2]", "D7 div = -grad^T"),
    ("tensor-off-diagonal-sign", PY_STEREO, "T[0, 1] = T[1, 0] = (e - 1.0) * nx * ny",
     "T[0, 1] = T[1, 0] = (1.0 - e) * nx * ny", "D4 eigenvectors along and across the gradient"),
    ("tensor-yy-uses-x", PY_STEREO, "T[1, 1] = 1.0 + (e - 1.0) * ny * ny", "T[1, 1] = 1.0 + (e - 1.0) * nx * nx",
     "D4 tensor"),
    ("assign-coupling-half", PY_STEREO, "e = e + dd * dd / (2.0 * theta)", "e = e + dd * dd / theta",
     "D5 coupling (d - a)^2 / (2 theta)"),
    ("assign-ties-largest", PY_STEREO, "better = e < best", "better = e <= best", "D5 ties to the smallest delta"),
    ("tgv-p-radius", PY_STEREO, "np.sqrt(p[0] ** 2 + p[1] ** 2) / alpha1)[None]",
     "np.sqrt(p[0] ** 2 + p[1] ** 2) / alpha2)[None]", "D6 |p| <= alpha1"),
    ("tgv-prox-theta", PY_STEREO, "d = (d_tmp + (tau / theta) * a) / (1.0 + tau / theta)",
     "d = (d_tmp + tau * a) / (1.0 + tau)", "D6 prox of (d - a)^2 / (2 theta)"),
    ("tgv-w-sign", PY_STEREO, "w = w_old + tau * (p + np.stack([div(q[0]), div(q[1])]))",
     "w = w_old - tau * (p + np.stack([div(q[0]), div(q[1])]))", "D6 primal descent in w"),
    ("tgv-no-relaxation", PY_STEREO, "st.d_bar = 2.0 * d - d_old", "st.d_bar = d", "D6 extrapolation of d"),
    ("tgv-no-relaxation-w", PY_STEREO, "st.w_bar = 2.0 * w - w_old", "st.w_bar = w", "D6 extrapolation of w"),
    # ------------------------------------------------ surface extraction (S1-S5)
    ("surface-orientation", PY_SURFACE, "away_ok = k == 1", "away_ok = k == 3", "S5 normals towards u > 0"),
    ("surface-lone-order", PY_SURFACE, "{0: (1, 2, 3), 1: (0, 3, 2), 2: (3, 0, 1), 3: (2, 1, 0)}",
     "{0: (1, 2, 3), 1: (0, 2, 3), 2: (3, 0, 1), 3: (2, 1, 0)}", "S5 winding of a lone-corner triangle"),
    ("surface-edge-direction", PY_SURFACE, "t = vu[i] / (vu[i] - vu[j])", "t = vu[j] / (vu[j] - vu[i])",
     "S4 vertex where the linear interpolant is zero"),
    ("surface-zero-sign", PY_SURFACE, "_tet_triangles([x < 0 for x in vu], orient)",
     "_tet_triangles([x <= 0 for x in vu], orient)", "S3 u = 0 counts as outside"),
    ("surface-block-carry", PY_SURFACE, "nbk = index.get((seg, bx + carry[0], by + carry[1], bz + carry[2]), -1)",
     "nbk = index.get((seg, bx, by, bz), -1)", "S1 corners in the neighbouring block"),
    ("surface-half-voxel", PY_SURFACE, "return ((ijk.astype(np.float64) + 0.5) * voxel_size).reshape(-1, 3)",
     "return (ijk.astype(np.float64) * voxel_size).reshape(-1, 3)", "voxel centres"),
    ("surface-omega-rule", PY_SURFACE, "valid[valid] = np.all(om[corners[valid]], axis=1)",
     "valid[valid] = np.any(om[corners[valid]], axis=1)", "S1 all eight corners in Omega"),
    ("surface-kuhn-chain", PY_SURFACE, "c2 = c1 | (1 << pi[1])", "c2 = 1 << pi[1]", "S2 Kuhn tetrahedra"),
    # ------------------------------------------------------- warm-start network
    ("conv-taps-transposed", PY_NET, "y += np.einsum(\"oc,nczyx->nozyx\", W[:, :, dz, dy, dx], patch)",
     "y += np.einsum(\"oc,nczyx->nozyx\", W[:, :, dx, dy, dz], patch)", "3^3 correlation taps"),
    ("conv-backward-unflipped", PY_NET, "np.einsum(\"oc,nozyx->nczyx\", W[:, :, dz, dy_, dx], dy)",
     "np.einsum(\"oc,nozyx->nczyx\", W[:, :, 2 - dz, 2 - dy_, 2 - dx], dy)", "input gradient of a correlation"),
    ("conv-bias-mean", PY_NET, "db = dy.sum(axis=(0, 2, 3, 4))", "db = dy.sum(axis=(2, 3, 4)).mean(axis=0)",
     "bias gradient"),
    ("net-relu-on-output", PY_NET, "h = np.maximum(z, 0.0) if li < len(params) - 1 else z\n        acts.append(h)",
     "h = np.maximum(z, 0.0)\n        acts.append(h)", "the last layer is linear"),
    ("net-output-offset", PY_NET, "return h[:, :, 1:-1, 1:-1, 1:-1], acts", "return h[:, :, :-2, :-2, :-2], acts",
     "the output is the centre 8^3"),
    ("net-relu-mask", PY_NET, "dh = dh * (acts[li + 1] > 0)", "dh = dh * (acts[li + 1] >= 0)", "ReLU derivative"),
    ("net-loss-factor", PY_NET, "2.0 * d * mask / out.shape[0]", "d * mask / out.shape[0]",
     "derivative of the squared error"),
    ("bf16-truncation", PY_NET, "np.ldexp(np.rint(m * 256.0) / 256.0, e)", "np.ldexp(np.floor(m * 256.0) / 256.0, e)",
     "nearest BF16"),
    ("gather-halo-offset", PY_NET, "zs = [(1 + l + 8 * oz, l) for l in range(8) if 0 <= 1 + l + 8 * oz < GRID]",
     "zs = [(l + 8 * oz, l) for l in range(8) if 0 <= l + 8 * oz < GRID]", "one-voxel halo along z"),
    ("gather-unobserved-f", PY_NET, "np.where(wv > 0, f3[nb][ix], 0.0)", "f3[nb][ix]", "f only where w > 0"),
    ("warm-no-clamp", PY_NET, "np.clip(o[:, 0], -1.0, 1.0)", "o[:, 0]", "u in [-1, 1]"),
    ("warm-projection", PY_NET, "p = p / np.maximum(1.0, nrm)[None]", "p = p / np.maximum(1.0, nrm * nrm)[None]",
     "projection onto the unit ball"),
    ("inner-edges-axis", PY_NET, "e[1][:, :, :-1, :] = om[:, :, :-1, :] & om[:, :, 1:, :]",
     "e[1][:, :-1, :, :] = om[:, :-1, :, :] & om[:, 1:, :, :]", "Eq. 3 edges along y"),
    ("inner-divergence-sign", PY_NET, "out = out + (q[a] - back)", "out = out + (q[a] + back)", "Eq. 4"),
    ("loss-div-gradient", PY_NET, "(rd - nxt.reshape(-1, 512))", "(rd + nxt.reshape(-1, 512))",
     "adjoint of the inner divergence"),
    # ------------------------------------------------------------------ a second pass
    ("alloc-band-count", PY_DENSER, "return int(math.ceil(params.mu / h - 1e-9))",
     "return int(math.floor(params.mu / h - 1e-9))", "reading R1: the band covers [d - mu, d + mu]"),
    ("alloc-zero-depth", PY_DENSER, "valid = np.isfinite(d32) & (d32 > 0)", "valid = np.isfinite(d32)",
     "invalid pixels allocate nothing"),
    ("fuse-zero-depth", PY_DENSER, "valid = inside & np.isfinite(d) & (d > 0)", "valid = inside & np.isfinite(d)",
     "invalid pixels fuse nothing"),
    ("fuse-image-edge", PY_DENSER, "inside = front & (pxf >= 0) & (pxf < W)", "inside = front & (pxf >= 1) & (pxf < W)",
     "the first pixel column is in the image"),
    ("fuse-other-segments", PY_DENSER, "sel = [b for b, k in enumerate(grid.keys) if k[0] == segment]",
     "sel = [b for b, k in enumerate(grid.keys) if True]", "a depth map fuses into its own segment"),
    ("voxel-layout-transposed", PY_DENSER, "return l % BLOCK, (l // BLOCK) % BLOCK, l // (BLOCK * BLOCK)",
     "return l // (BLOCK * BLOCK), (l // BLOCK) % BLOCK, l % BLOCK", "voxel l = lx + 8 ly + 64 lz"),
    ("neighbour-face-swapped", PY_DENSER, "edge = (loc[a] == (BLOCK - 1)) if sign > 0 else (loc[a] == 0)",
     "edge = (loc[a] == 0) if sign > 0 else (loc[a] == (BLOCK - 1))", "which face a step leaves by"),
    ("dual-norm-xy", PY_DENSER, "nrm = np.sqrt(pt[0] * pt[0] + pt[1] * pt[1] + pt[2] * pt[2])",
     "nrm = np.sqrt(pt[0] * pt[0] + pt[1] * pt[1])", "the 3-vector norm of p"),
    ("warm-relaxed-state", PY_DENSER, "grid.u.reshape(-1).copy(), grid.u_bar.reshape(-1).copy()",
     "grid.u.reshape(-1).copy(), grid.u.reshape(-1).copy()", "a warm start resumes the relaxed primal"),
    ("c-inverse-rotation", C_DENSER, "Ri[3 * r + c] = T[4 * c + r];", "Ri[3 * r + c] = T[4 * r + c];",
     "global-to-camera rotation R^T"),
    ("c-inverse-translation", C_DENSER, "ti[r] = -((T[0 * 4 + r]", "ti[r] = ((T[0 * 4 + r]", "-R^T t"),
    ("c-no-clamp", C_DENSER, "const double utsdf = q < 1.0 ? q : 1.0;", "const double utsdf = q;",
     "u_TSDF = min(1, u_SDF / mu)"),
    ("c-other-segments", C_DENSER, "if (k[0] != segment) continue;\n        double *fb",
     "if (0) continue;\n        double *fb", "a depth map fuses into its own segment"),
    ("c-pixel-round", C_DENSER, "const double pxf = floor((fx * xc) / zc + cx)", "const double pxf = round((fx * xc) / zc + cx)",
     "pixel (x, y) covers [x, x + 1)"),
    ("c-no-truncation-test", C_DENSER, "if (!(usdf >= -mu)) continue;", "if (!(usdf >= 0.0)) continue;",
     "Eq. 1 observes down to -mu"),
    ("c-dual-norm-xy", C_DENSER, "const double nrm = sqrt((q0 * q0 + q1 * q1) + q2 * q2);",
     "const double nrm = sqrt(q0 * q0 + q1 * q1);", "the 3-vector norm of p"),
    ("c-energy-tv-xy", C_DENSER, "const double tv = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);",
     "const double tv = sqrt(g[0] * g[0] + g[1] * g[1]);", "isotropic TV over three axes"),
    ("laser-range-limit", PY_LASER, "valid &= np.floor((r + params.mu) / (0.5 * params.voxel_size)) < 2.0 ** 22",
     "valid &= np.isfinite(r)", "L1 range limit"),
    ("laser-block-truncation", PY_LASER, "blk = v // BLOCK", "blk = (v / BLOCK).astype(np.int64)",
     "block of a negative voxel index"),
    ("laser-behind-sensor", PY_LASER, "ok = rho > 0", "ok = rho > -np.inf", "L2 samples behind the sensor"),
    ("tensor-anisotropic-norm", PY_STEREO, "mag = np.sqrt(g[0] ** 2 + g[1] ** 2)", "mag = np.abs(g[0]) + np.abs(g[1])",
     "D4 |grad I|"),
    ("tensor-normal-swapped", PY_STEREO, "nx = np.where(mag > 0, g[0] / mag, 0.0)",
     "nx = np.where(mag > 0, g[1] / mag, 0.0)", "D4 n = grad I / |grad I|"),
    ("tgv-q-from-w", PY_STEREO, "gw = np.stack([grad(st.w_bar[0]), grad(st.w_bar[1])])",
     "gw = np.stack([grad(st.w[0]), grad(st.w[1])])", "D6 the dual step reads the relaxed primal"),
    ("tgv-p-w-sign", PY_STEREO, "p = st.p + sigma * (apply_T(T, grad(st.d_bar)) - st.w_bar)",
     "p = st.p + sigma * (apply_T(T, grad(st.d_bar)) + st.w_bar)", "D6 K (d, w) = (T grad d - w, grad w)"),
    ("estimate-theta-grows", PY_STEREO, "theta *= prm.theta_decay", "theta /= prm.theta_decay",
     "D5 theta shrinks"),
    ("estimate-no-wta-start", PY_STEREO, "d0 = assign(hvol, np.zeros(IR.shape), prm.lam, np.inf)",
     "d0 = np.zeros(IR.shape)", "D5 start from the winner-takes-all disparity"),
    ("census-mirrored", PY_STEREO, "nb = I[np.clip(ys + dy, 0, H - 1), np.clip(xs + dx, 0, W - 1)]",
     "nb = I[np.clip(ys - dy, 0, H - 1), np.clip(xs - dx, 0, W - 1)]", "D2 bit order over the window"),
    ("surface-perm-sign", PY_SURFACE, "return -1 if inv % 2 else 1", "return 1", "S2 orientation of odd tetrahedra"),
    ("surface-edge-id", PY_SURFACE, "ti.append(a * 8 + (codes[j] ^ codes[i]))", "ti.append(a * 8 + codes[j])",
     "S4 a vertex is named by its lattice edge"),
    ("surface-corner-layout", PY_SURFACE,
     "nl = (nx % BLOCK) + BLOCK * (ny % BLOCK) + BLOCK * BLOCK * (nz % BLOCK)",
     "nl = (nz % BLOCK) + BLOCK * (ny % BLOCK) + BLOCK * BLOCK * (nx % BLOCK)", "voxel l = lx + 8 ly + 64 lz"),
    ("net-unrounded-activations", PY_NET, "h = bf16(np.maximum(z, 0.0)) if li < len(params) - 1 else z",
     "h = np.maximum(z, 0.0) if li < len(params) - 1 else z", "hidden activations stored as BF16"),
    ("net-unrounded-weights", PY_NET, "z = conv3d_same(h, bf16(W), np.asarray(b, dtype=np.float64))",
     "z = conv3d_same(h, W, np.asarray(b, dtype=np.float64))", "weights stored as BF16"),
    ("gather-axes-swapped", PY_NET, "nb = index.get((seg, bx + ox, by + oy, bz + oz))",
     "nb = index.get((seg, bx + oz, by + oy, bz + ox))", "the halo's neighbouring blocks"),
    ("gather-weight-scale", PY_NET, "wv / (wv + 8.0)", "wv / (wv + 1.0)", "input channel w / (w + 8)"),
    ("warm-components-reversed", PY_NET, "p = np.where(edges, o[:, 1:].transpose(1, 0, 2), 0.0)",
     "p = np.where(edges, o[:, :0:-1].transpose(1, 0, 2), 0.0)", "outputs (u, p_x, p_y, p_z)"),
    ("loss-unmasked", PY_NET, "d = (out - target) * mask", "d = out - target", "the loss counts Omega only"),
    ("loss-div-unmasked-u", PY_NET, "ru = np.where(om, out[:, 0] - target[:, 0], 0.0)", "ru = out[:, 0] - target[:, 0]",
     "the divergence loss counts Omega only"),
    # ------------------------------------------------------------------- a third pass
    ("laser-other-segment", PY_LASER, "idx = np.array([grid.index.get((segment, int(a), int(b), int(c)), -1)",
     "idx = np.array([grid.index.get((0, int(a), int(b), int(c)), -1)", "a scan fuses into its own segment"),
    ("laser-key-order", PY_LASER, "key=lambda k: (k[0], k[3], k[2], k[1]))", "key=lambda k: (k[0], k[1], k[2], k[3]))",
     "new blocks in (segment, bz, by, bx) order"),
    ("estimate-alphas-swapped", PY_STEREO, "tgv_iterate(st, a, T, theta, prm.alpha1, prm.alpha2, prm.inner)",
     "tgv_iterate(st, a, T, theta, prm.alpha2, prm.alpha1, prm.inner)", "Table I's alpha1 and alpha2"),
    ("estimate-tensor-of-left", PY_STEREO, "T = diffusion_tensor(IR, prm.gamma, prm.beta)",
     "T = diffusion_tensor(IL, prm.gamma, prm.beta)", "D4 the tensor of the reference image I_R"),
    ("estimate-images-swapped", PY_STEREO, "sL, sR = census(IL), census(IR)", "sL, sR = census(IR), census(IL)",
     "D1 I_L(x + d) against I_R(x)"),
    ("assign-flags-everything", PY_STEREO, "flag |= close & (arg != k)", "flag |= close",
     "D8 a near tie needs another candidate"),
    ("surface-blocks-ignored", PY_SURFACE, "crossing &= np.repeat(chosen, BLOCK_VOXELS)", "crossing &= True",
     "only the chosen blocks' cubes are meshed"),
    ("targets-edges-reversed", PY_NET, "t[:, 3:6] = e.transpose(1, 0, 2)", "t[:, 3:6] = e.transpose(1, 0, 2)[:, ::-1]",
     "target channels (u, Omega, div p, e_x, e_y, e_z)"),
    ("inner-edges-shifted", PY_NET, "e[0][..., :-1] = om[..., :-1] & om[..., 1:]", "e[0][..., 1:] = om[..., :-1] & om[..., 1:]",
     "Eq. 3 edge e_x(v) stored at v"),
    ("c-key-order", C_DENSER, "if (a[3] != b[3]) return a[3] < b[3];", "if (a[3] != b[3]) return a[3] > b[3];",
     "new blocks in (segment, bz, by, bx) order"),
    ("c-band-step", C_DENSER, "const double h = 0.5 * m->s, bs = 8.0 * m->s;", "const double h = m->s, bs = 8.0 * m->s;",
     "band samples half a voxel apart"),
    ("c-row-centre", C_DENSER, "const double vv = ((double)y + 0.5) - cy;", "const double vv = (double)y - cy;",
     "rays through pixel centres"),
    ("c-back-edge", C_DENSER, "if (edge(m, nbr, vb / BV, (int)(vb % BV), a, &f2)) back = pa[vb];", "back = pa[vb];",
     "Eq. 4 cases at the Omega boundary"),
    ("c-face-carry", C_DENSER, "if ((dir > 0 && c < 7) || (dir < 0 && c > 0))", "if ((dir > 0 && c < 7) || (dir < 0 && c >= 0))",
     "a step out of the block's low face"),
    # ------------------------------------------------------------------ a fourth pass
    ("pipeline-fuse-first", PY_DENSER, """        alloc_blocks(grid, dm, K, T, segment)
        fuse_depth(grid, dm, K, T, segment)""", """        fuse_depth(grid, dm, K, T, segment)
        alloc_blocks(grid, dm, K, T, segment)""", "Section III-A: allocate, then fuse, per depth map"),
    ("grid-index-off-by-one", PY_DENSER, "self.index[k] = len(self.keys)\n", "self.index[k] = len(self.keys) + 1\n",
     "block b owns voxels b*512 .. b*512 + 511"),
    ("laser-last-sample", PY_LASER, "rho = np.arange(M + 1, dtype=np.float64) * h", "rho = np.arange(M, dtype=np.float64) * h",
     "L3 samples n = 0..M"),
    ("conv-bias-dropped", PY_NET, "y = np.zeros((n, W.shape[0], D, H, Wd)) + b[None, :, None, None, None]",
     "y = np.zeros((n, W.shape[0], D, H, Wd))", "the bias of each output channel"),
    ("net-backward-offset", PY_NET, "dh[:, :, 1:-1, 1:-1, 1:-1] = dout", "dh[:, :, :-2, :-2, :-2] = dout",
     "the loss reads the centre 8^3"),
    ("tensor-apply-swapped", PY_STEREO, "T[1, 0] * v[0] + T[1, 1] * v[1]", "T[1, 0] * v[1] + T[1, 1] * v[0]",
     "D4 T grad d"),
    ("div-first-column", PY_STEREO, "dx[:, 0] = px[:, 0]", "dx[:, 0] = 0.0", "D7 div = -grad^T"),
    ("c-energy-residual", C_DENSER, "const double r = m->u[v] - m->f[v];", "const double r = m->u[v] + m->f[v];",
     "the data term (u - f)^2"),
    ("c-dual-step-size", C_DENSER, "const double q0 = p0[v] + sg * g[0],", "const double q0 = p0[v] + g[0],",
     "the dual step sigma"),
    # ------------------------------------------------------------------- a fifth pass
    ("surface-corner-axes", PY_SURFACE, "return (code & 1, (code >> 1) & 1, (code >> 2) & 1)",
     "return ((code >> 2) & 1, (code >> 1) & 1, code & 1)", "S2 corner code bit a = axis a"),
    ("div-interior-shift", PY_STEREO, "dx[:, 1:-1] = px[:, 1:-1] - px[:, :-2]", "dx[:, 1:-1] = px[:, 2:] - px[:, 1:-1]",
     "D7 div = -grad^T (backward difference)"),
    ("div-y-rows", PY_STEREO, "dy[1:-1, :] = py[1:-1, :] - py[:-2, :]", "dy[1:-1, :] = py[1:-1, :] - py[2:, :]",
     "D7 div = -grad^T"),
    ("census-bit-stride", PY_STEREO, "            b += 1\n", "            b += 2\n", "D2 62 distinct bits"),
    ("c-sort-descending", C_DENSER, "return key_less(a, b) ? -1 : (key_less(b, a) ? 1 : 0);",
     "return key_less(a, b) ? 1 : (key_less(b, a) ? -1 : 0);", "new blocks in ascending key order"),
]

RUNNER = r"""
import os, sys, types
root, kind, target, changed = sys.argv[1:5]
pins = sys.argv[5:]
sys.path.insert(0, root)
if kind == "py":
    import oracle
    name = "oracle." + target
    mod = types.ModuleType(name)
    mod.__file__ = os.path.join(root, "oracle", target + ".py")
    mod.__package__ = "oracle"
    sys.modules[name] = mod
    setattr(oracle, target, mod)
    exec(compile(open(changed).read(), mod.__file__, "exec"), mod.__dict__)
else:
    from oracle import oracle_c
    oracle_c.SRC = changed
    oracle_c.LIB = changed[:-2] + ".so"
    oracle_c.build(force=True)
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", *pins]))
"""


def _source_path(target):
    return os.path.join(ROOT, "oracle", target + (".c" if target.endswith("_c") else ".py"))


def _run_case(case, workdir):
    cid, (target, pins), old, new, _ = case
    src = open(_source_path(target)).read()
    assert src.count(old) == 1, f"{cid}: the expression to change is not in {target} exactly once"
    kind = "c" if target.endswith("_c") else "py"
    changed = os.path.join(workdir, f"{cid}.{'c' if kind == 'c' else 'py'}")
    with open(changed, "w") as fh:
        fh.write(src.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    try:
        r = subprocess.run([sys.executable, "-c", RUNNER, ROOT, kind, target, changed, *pins], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=600)
    except subprocess.TimeoutExpired:
        return cid, None, "timed out"
    return cid, r.returncode, (r.stdout + r.stderr)[-1500:]


@pytest.fixture(scope="module")
def outcomes():
    with tempfile.TemporaryDirectory() as workdir:
        with ThreadPoolExecutor(max_workers=max(1, min(12, os.cpu_count() or 1))) as ex:
            res = list(ex.map(lambda c: _run_case(c, workdir), CASES))
    return {cid: (rc, tail) for cid, rc, tail in res}


def test_the_unchanged_oracles_pass_their_pins():
    """The harness itself: the oracles as they stand, installed the same way, pass."""
    with tempfile.TemporaryDirectory() as workdir:
        for target, pins in (PY_DENSER, C_DENSER):
            changed = os.path.join(workdir, target + (".c" if target.endswith("_c") else ".py"))
            with open(changed, "w") as fh:
                fh.write(open(_source_path(target)).read())
            kind = "c" if target.endswith("_c") else "py"
            r = subprocess.run([sys.executable, "-c", RUNNER, ROOT, kind, target, changed, pins[0]], cwd=ROOT,
                               env=dict(os.environ, PYTHONDONTWRITEBYTECODE="1"), capture_output=True, text=True,
                               timeout=600)
            assert r.returncode == 0, (r.stdout + r.stderr)[-1500:]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(case, outcomes):
    rc, tail = outcomes[case[0]]
    # 1: a pin failed (not 2, a changed oracle that does not even import, nor 0, all pins passed)
    assert rc == 1, f"{case[0]} ({case[4]}) was not caught: exit {rc}\n{tail}"
