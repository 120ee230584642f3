"""Pins of the oracle's Omega-aware operators and primal-dual solver.

Eq. 3 and Eq. 4 are checked case by case; the divergence against the adjoint
identity; the solver against a closed-form two-voxel TV-L2 problem, an
independent dense-array solve of a fully allocated box, brute-force energies
on a tiny grid, the isolated-region behaviour Section III-B describes, and the
dual function's definition as the minimum of the Lagrangian.
"""

import math

import numpy as np
import pytest

from oracle.denser_oracle import (BLOCK_VOXELS, Params, PDProblem, divergence, energies,
                                  gradient, omega, pd_iterate, regularize, voxel_neighbours)
from tests.oracle_helpers import box_keys, grid_from_blocks, random_fw

P = Params()


def lin(lx, ly, lz, b=0):
    return b * BLOCK_VOXELS + lx + 8 * ly + 64 * lz


# -------------------------------------------------------------- Eq. 3 / 4
def _line_grid(omega_x, two_blocks=False):
    """Voxels (x, 0, 0), x = 0..7 (or 0..15 over two blocks along x); w = 1 where omega_x."""
    keys = [(0, 0, 0, 0), (0, 1, 0, 0)] if two_blocks else [(0, 0, 0, 0)]
    nb = len(keys)
    w = np.zeros((nb, BLOCK_VOXELS))
    for x, o in enumerate(omega_x):
        if o:
            w[x // 8, lin(x % 8, 0, 0)] = 1.0
    return grid_from_blocks(keys, np.zeros((nb, BLOCK_VOXELS)), w)


def test_gradient_cases_eq3():
    om_x = [1, 1, 1, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1]
    g = _line_grid(om_x, two_blocks=True)
    fwd, _ = voxel_neighbours(g)
    om = omega(g)
    u = np.zeros(g.n_blocks * BLOCK_VOXELS)
    vals = np.arange(1, 17, dtype=float) ** 2
    idx = [lin(x % 8, 0, 0, x // 8) for x in range(16)]
    u[idx] = vals
    gx = gradient(u, om, fwd)[0][idx]
    for x in range(16):
        if x == 15:                      # i = V_x: the next block is not allocated
            exp = 0.0
        elif not om_x[x]:                # u_i in Omega-bar
            exp = 0.0
        elif not om_x[x + 1]:            # u_{i+1} in Omega-bar
            exp = 0.0
        else:                            # 1 <= i < V_x, crossing the block face at x = 7
            exp = vals[x + 1] - vals[x]
        assert gx[x] == exp, x
    # y and z by substitution: a voxel pair across the +y and +z block faces
    keys = [(0, 0, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1)]
    w = np.zeros((3, BLOCK_VOXELS))
    w[0, lin(2, 7, 7)] = w[1, lin(2, 0, 7)] = w[2, lin(2, 7, 0)] = 1
    g = grid_from_blocks(keys, np.zeros((3, BLOCK_VOXELS)), w)
    fwd, _ = voxel_neighbours(g)
    u = np.zeros(3 * BLOCK_VOXELS)
    u[lin(2, 7, 7, 0)], u[lin(2, 0, 7, 1)], u[lin(2, 7, 0, 2)] = 0.25, 1.0, -2.0
    gr = gradient(u, omega(g), fwd)
    assert gr[1][lin(2, 7, 7, 0)] == 0.75
    assert gr[2][lin(2, 7, 7, 0)] == -2.25
    assert gr[0][lin(2, 7, 7, 0)] == 0.0


def test_divergence_cases_eq4():
    # Omega pattern along x over two blocks: positions 0..15
    om_x = [1, 1, 1, 1, 0, 1, 1, 0, 1, 1, 0, 1, 1, 1, 1, 1]
    g = _line_grid(om_x, two_blocks=True)
    fwd, bwd = voxel_neighbours(g)
    om = omega(g)
    rng = np.random.default_rng(0)
    idx = [lin(x % 8, 0, 0, x // 8) for x in range(16)]
    # a dual field on the edges that exist (zero elsewhere, as the solver keeps it)
    p = np.zeros((3, g.n_blocks * BLOCK_VOXELS))
    px = rng.uniform(-1, 1, 16)
    for x in range(15):
        if om_x[x] and om_x[x + 1]:
            p[0, idx[x]] = px[x]
    d = divergence(p, om, fwd, bwd)[idx]
    P_ = [p[0, i] for i in idx]
    for x in range(16):
        prev_in = x > 0 and om_x[x - 1]
        next_in = x < 15 and om_x[x + 1]
        if not om_x[x]:
            exp = 0.0                                     # u_i in Omega-bar
        elif x == 0:
            exp = P_[x]                                   # i = 1
        elif x == 15:
            exp = -P_[x - 1]                              # i = V_x
        elif not prev_in and not next_in:
            exp = 0.0                                     # both cases at once: adjoint gives 0
        elif not prev_in:
            exp = P_[x]                                   # u_{i-1} in Omega-bar
        elif not next_in:
            exp = -P_[x - 1]                              # u_{i+1} in Omega-bar
        else:
            exp = P_[x] - P_[x - 1]                       # 1 < i < V_x
        assert d[x] == pytest.approx(exp, abs=1e-15), x


def test_adjoint_identity_random_masks():
    rng = np.random.default_rng(1)
    keys = [(0, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 1, 1, 1), (0, -1, 0, 0), (0, 0, 0, 1),
            (0, 3, 3, 3), (1, 0, 0, 0)]
    f, w = random_fw(rng, len(keys), p_omega=0.6)
    g = grid_from_blocks(keys, f, w)
    fwd, bwd = voxel_neighbours(g)
    om = omega(g)
    N = g.n_blocks * BLOCK_VOXELS
    for _ in range(5):
        u = rng.standard_normal(N)
        p = rng.standard_normal((3, N))
        lhs = np.sum(gradient(u, om, fwd) * p)
        rhs = -np.sum(u * divergence(p, om, fwd, bwd))
        assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


def test_segments_are_not_neighbours():
    keys = [(0, 0, 0, 0), (1, 1, 0, 0)]
    g = grid_from_blocks(keys, np.zeros((2, 512)), np.ones((2, 512)))
    fwd, _ = voxel_neighbours(g)
    assert fwd[0][lin(7, 3, 3, 0)] == -1


# ------------------------------------------------------------ closed form
@pytest.mark.parametrize("f1,f2,w1,w2", [(-0.5, 0.9, 2.0, 3.0), (0.1, 0.6, 2.0, 3.0),
                                         (0.8, -0.7, 1.0, 4.0)])
def test_two_voxel_closed_form(f1, f2, w1, w2):
    """min |u2-u1| + lam/2 (w1 (u1-f1)^2 + w2 (u2-f2)^2): separate by 1/(lam w_i) towards
    each other, or merge at the weighted mean when they would cross."""
    lam = P.lam
    f = np.zeros((1, BLOCK_VOXELS))
    w = np.zeros((1, BLOCK_VOXELS))
    a, b = lin(3, 4, 5), lin(4, 4, 5)
    f[0, a], f[0, b], w[0, a], w[0, b] = f1, f2, w1, w2
    g = grid_from_blocks([(0, 0, 0, 0)], f, w)
    regularize(g, 4000)
    u = g.u.reshape(-1)
    sg = math.copysign(1.0, f2 - f1)
    if abs(f2 - f1) > 1 / (lam * w1) + 1 / (lam * w2):
        e1, e2 = f1 + sg / (lam * w1), f2 - sg / (lam * w2)
    else:
        e1 = e2 = (w1 * f1 + w2 * f2) / (w1 + w2)
    assert abs(u[a] - e1) < 1e-10 and abs(u[b] - e2) < 1e-10
    others = np.ones(BLOCK_VOXELS, bool)
    others[[a, b]] = False
    assert np.all(u[others] == 0)


# --------------------------------------------------------- dense equivalence
def _dense_solve(f, w, iters, prm):
    """Independent dense-array Chambolle-Pock solve on an [X, Y, Z] box whose outer faces
    play i = V_x (Eq. 3 / Eq. 4), written with array slicing."""
    om = w > 0
    u = np.zeros_like(f)
    ub = np.zeros_like(f)
    p = np.zeros((3,) + f.shape)

    def edges():
        e = np.zeros((3,) + f.shape, bool)
        e[0, :-1] = om[:-1] & om[1:]
        e[1, :, :-1] = om[:, :-1] & om[:, 1:]
        e[2, :, :, :-1] = om[:, :, :-1] & om[:, :, 1:]
        return e
    e = edges()

    def grad(x):
        g = np.zeros((3,) + f.shape)
        g[0, :-1] = x[1:] - x[:-1]
        g[1, :, :-1] = x[:, 1:] - x[:, :-1]
        g[2, :, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
        return np.where(e, g, 0.0)

    def div(q):
        q = np.where(e, q, 0.0)
        d = np.zeros(f.shape)
        for a in range(3):
            sh = np.zeros(f.shape)
            if a == 0:
                sh[1:] = q[0, :-1]
            elif a == 1:
                sh[:, 1:] = q[1, :, :-1]
            else:
                sh[:, :, 1:] = q[2, :, :, :-1]
            d = d + (q[a] - sh)
        return d

    for _ in range(iters):
        pt = p + prm.sigma * grad(ub)
        n = np.sqrt(pt[0] ** 2 + pt[1] ** 2 + pt[2] ** 2)
        p = pt / np.maximum(1.0, n)
        uo = u
        ut = u + prm.tau * div(p)
        u = np.where(om, (ut + prm.tau * prm.lam * w * f) / (1 + prm.tau * prm.lam * w), u)
        ub = u + prm.theta * (u - uo)
    return u, p


def _to_dense(g, field, nx, ny, nz):
    out = np.zeros((8 * nx, 8 * ny, 8 * nz))
    for b, (_, bx, by, bz) in enumerate(g.keys):
        blk = field[b].reshape(8, 8, 8)  # [lz, ly, lx]
        out[8 * bx:8 * bx + 8, 8 * by:8 * by + 8, 8 * bz:8 * bz + 8] = blk.transpose(2, 1, 0)
    return out


def test_dense_box_equivalence():
    rng = np.random.default_rng(2)
    nx, ny, nz = 2, 2, 2
    keys = box_keys(nx, ny, nz)
    rng.shuffle(keys)                     # block index order must not matter
    f, w = random_fw(rng, len(keys), p_omega=0.85)
    g = grid_from_blocks(keys, f, w)
    regularize(g, 60)
    fd, wd = _to_dense(g, g.f, nx, ny, nz), _to_dense(g, g.w, nx, ny, nz)
    ud, pd = _dense_solve(fd, wd, 60, P)
    np.testing.assert_allclose(_to_dense(g, g.u, nx, ny, nz), ud, rtol=0, atol=1e-12)
    for a in range(3):
        np.testing.assert_allclose(_to_dense(g, g.p[a], nx, ny, nz), pd[a], rtol=0, atol=1e-12)


# ----------------------------------------------------- energies and the gap
def _tiny_problem(seed=3):
    """One block whose observed voxels form a 4x4x4 cube (64 voxels)."""
    rng = np.random.default_rng(seed)
    f = np.zeros((1, BLOCK_VOXELS))
    w = np.zeros((1, BLOCK_VOXELS))
    for x in range(4):
        for y in range(4):
            for z in range(4):
                i = lin(x + 2, y + 1, z + 3)
                f[0, i] = rng.uniform(-1, 1)
                w[0, i] = rng.integers(1, 4)
    return grid_from_blocks([(0, 5, -2, 7)], f, w)


def _brute_energies(g, u, p, prm):
    """Direct summation over voxels of Eq. 2 (reading R10) and of the dual function."""
    f, w = g.f[0], g.w[0]
    om = w > 0
    lam = prm.lam

    def at(x, y, z):
        if 0 <= x < 8 and 0 <= y < 8 and 0 <= z < 8:
            return lin(x, y, z)
        return None
    Pv = 0.0
    for z in range(8):
        for y in range(8):
            for x in range(8):
                i = lin(x, y, z)
                if not om[i]:
                    continue
                sq = 0.0
                for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    j = at(x + dx, y + dy, z + dz)
                    if j is not None and om[j]:
                        sq += (u[j] - u[i]) ** 2
                Pv += math.sqrt(sq) + 0.5 * lam * w[i] * (u[i] - f[i]) ** 2
    # dual: min over u of <grad u, p> + lam/2 sum w (u - f)^2, voxel by voxel after
    # writing <grad u, p> = sum_v u_v * c_v, c_v collecting the terms that touch u_v.
    c = np.zeros(BLOCK_VOXELS)
    for z in range(8):
        for y in range(8):
            for x in range(8):
                i = lin(x, y, z)
                for a, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
                    j = at(x + dx, y + dy, z + dz)
                    if j is not None and om[i] and om[j]:
                        c[j] += p[a, i]
                        c[i] -= p[a, i]
    Dv = 0.0
    for i in range(BLOCK_VOXELS):
        if om[i]:
            ustar = f[i] - c[i] / (lam * w[i])
            Dv += c[i] * ustar + 0.5 * lam * w[i] * (ustar - f[i]) ** 2
    return Pv, Dv


def test_energies_match_brute_force_and_gap_decreases():
    g = _tiny_problem()
    prob = PDProblem(g)
    N = BLOCK_VOXELS
    u, ub, p = np.zeros(N), np.zeros(N), np.zeros((3, N))
    gaps = []
    for k in range(60):
        u, ub, p = pd_iterate(prob, u, ub, p, 10, P)
        Pv, Dv = energies(prob, u, p, P)
        if k in (0, 5, 30):
            Pb, Db = _brute_energies(g, u, p, P)
            assert abs(Pv - Pb) < 1e-11 and abs(Dv - Db) < 1e-11
        assert Pv >= Dv - 1e-12
        gaps.append(Pv - Dv)
    gaps = np.array(gaps)
    # monotone down to the round-off floor of the FP64 energies (~1e-10 here)
    above = gaps[:-1] > 1e-9
    assert np.all(np.diff(gaps)[above] <= 0), np.diff(gaps)[above].max()
    assert gaps[-1] / energies(prob, u, p, P)[0] < 1e-9


def test_dual_is_min_of_lagrangian():
    rng = np.random.default_rng(4)
    keys = [(0, 0, 0, 0), (0, 1, 0, 0), (0, 0, 0, 1)]
    f, w = random_fw(rng, 3, 0.7)
    g = grid_from_blocks(keys, f, w)
    prob = PDProblem(g)
    N = 3 * BLOCK_VOXELS
    q = rng.standard_normal((3, N))
    q = q / np.maximum(1, np.sqrt((q ** 2).sum(0)))
    _, D = energies(prob, np.zeros(N), q, P)
    om, ff, ww = prob.om, prob.f, prob.w

    def L(u):
        return np.sum(prob.grad(u) * q) + 0.5 * P.lam * np.sum(np.where(om, ww * (u - ff) ** 2, 0))
    ustar = np.where(om, ff + prob.div(q) / (P.lam * np.where(om, ww, 1)), 0.0)
    assert abs(L(ustar) - D) < 1e-9 * (1 + abs(D))
    for _ in range(5):
        du = rng.standard_normal(N) * om
        assert L(ustar + 1e-3 * du) > D


def test_weak_duality_random_states():
    rng = np.random.default_rng(6)
    f, w = random_fw(rng, 4, 0.7)
    g = grid_from_blocks(box_keys(2, 2, 1), f, w)
    prob = PDProblem(g)
    N = 4 * BLOCK_VOXELS
    for _ in range(10):
        u = rng.uniform(-1, 1, N)
        q = rng.standard_normal((3, N))
        q = q / np.maximum(1, np.sqrt((q ** 2).sum(0)))
        Pv, Dv = energies(prob, u, q, P)
        assert Pv >= Dv


# ---------------------------------------------------------- isolated regions
def _two_islands(rng, const_f=None):
    keys = [(0, 0, 0, 0), (0, 3, 0, 0)]          # no shared face: two components
    f, w = random_fw(rng, 2, p_omega=0.7)
    if const_f is not None:
        f[:] = const_f
        w[w > 0] = 2.0
    return grid_from_blocks(keys, f, w)


def test_isolated_region_boundary_behaviour():
    rng = np.random.default_rng(7)
    g = _two_islands(rng)
    om = omega(g).reshape(2, BLOCK_VOXELS)
    regularize(g, 150)
    # Omega-bar never changes from its zero start
    assert np.all(g.u[~om] == 0) and np.all(g.u_bar[~om] == 0) and np.all(g.p[:, ~om] == 0)
    # perturbing f and the warm state on Omega-bar leaves Omega bit-identical
    g2 = _two_islands(np.random.default_rng(7))
    g2.f[~om] = rng.uniform(-1, 1, (~om).sum())
    g2.u[~om] = rng.uniform(-1, 1, (~om).sum())
    g2.u_bar[:] = g2.u
    regularize(g2, 150, warm=True)
    assert np.array_equal(g.u[om], g2.u[om]) and np.array_equal(g.p[:, om], g2.p[:, om])
    assert np.array_equal(g2.u[~om], g2.u_bar[~om])   # untouched on Omega-bar


def test_constant_data_stays_put():
    g = _two_islands(np.random.default_rng(8), const_f=0.37)
    om = omega(g).reshape(2, BLOCK_VOXELS)
    regularize(g, 400)
    assert np.all(g.p == 0)
    np.testing.assert_allclose(g.u[om], 0.37, atol=1e-12)
    assert np.all(g.u[~om] == 0)


def _components(g):
    fwd, _ = voxel_neighbours(g)
    om = omega(g)
    N = om.size
    parent = np.arange(N)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for a in range(3):
        for v in np.nonzero(om)[0]:
            n = fwd[a, v]
            if n >= 0 and om[n]:
                ra, rb = find(v), find(n)
                if ra != rb:
                    parent[ra] = rb
    return np.array([find(v) for v in range(N)]), om


def test_weighted_mean_conserved_per_component():
    g = _two_islands(np.random.default_rng(9))
    regularize(g, 6000)
    comp, om = _components(g)
    u, f, w = g.u.reshape(-1), g.f.reshape(-1), g.w.reshape(-1)
    for c in np.unique(comp[om]):
        m = om & (comp == c)
        assert abs(np.sum(w[m] * u[m]) - np.sum(w[m] * f[m])) < 1e-7 * max(1.0, m.sum())


def test_printed_primal_sign_does_not_converge():
    """Reading R7: with the literal u - tau*div p the gap stalls far from zero."""
    g = _tiny_problem(11)
    prob = PDProblem(g)
    N = BLOCK_VOXELS
    z = (np.zeros(N), np.zeros(N), np.zeros((3, N)))
    u1, _, p1 = pd_iterate(prob, *z, 600, P)
    u2, _, p2 = pd_iterate(prob, *z, 600, P, literal_sign=True)
    P1, D1 = energies(prob, u1, p1, P)
    P2, D2 = energies(prob, u2, p2, P)
    assert (P1 - D1) / P1 < 1e-6
    assert (P2 - D2) / P2 > 1e-2


def test_warm_resume_continues_bit_for_bit():
    """A run split in two (the second part started from the stored u, u^ and p) is the
    same iteration as one run of the summed length: the state that carries over is
    (u, u^, p), the relaxed primal included (step 1 of Section III-C starts a run, the
    steps that follow read only that state)."""
    rng = np.random.default_rng(12)
    keys = box_keys(2, 1, 1)
    f, w = random_fw(rng, len(keys), p_omega=0.8)
    whole = grid_from_blocks(keys, f, w)
    regularize(whole, 50)
    split = grid_from_blocks(keys, f, w)
    regularize(split, 30)
    regularize(split, 20, warm=True)
    assert np.array_equal(whole.u, split.u) and np.array_equal(whole.u_bar, split.u_bar)
    assert np.array_equal(whole.p, split.p)
    assert not np.array_equal(split.u, split.u_bar)  # u^ differs from u mid-run
