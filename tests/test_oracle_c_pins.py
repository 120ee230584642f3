"""Pins of the C oracle (oracle/denser_oracle_c.c).

The C oracle restates the numpy oracle's allocation, fusion and primal-dual
iteration in the same operation order, so on every map both reach the same
float64 numbers bit for bit; its energies agree to the summation order.  Beyond
that equality it is pinned on its own, like the numpy oracle, by the two-voxel
TV-L2 closed form, the independent dense-array solve of a fully allocated box,
brute-force energies, the isolated-region behaviour of Section III-B and the
per-component conservation of the weighted mean; and its result does not
depend on the number of threads (Jacobi updates).
"""

import math

import numpy as np
import pytest

from oracle import denser_oracle as O
from oracle import oracle_c as C
from synth.scenes import Camera, Scene, street_scene, tiny_scene
from tests.oracle_helpers import box_keys, grid_from_blocks, intrinsics_of, random_fw
from tests.test_oracle_regularizer_pins import _brute_energies, _dense_solve, _tiny_problem, _to_dense, lin

P = O.Params()


def cmap_of(g, params=P):
    m = C.CMap(params, max(g.n_blocks, 1))
    m.load_blocks(np.array(g.keys, dtype=np.int64).reshape(-1, 4), g.f, g.w)
    return m


def _same_map(snap, g, state=True):
    assert np.array_equal(snap["coords"], g.coords())
    assert np.array_equal(snap["f"], g.f) and np.array_equal(snap["w"], g.w)
    if state:
        assert np.array_equal(snap["u"], g.u) and np.array_equal(snap["u_bar"], g.u_bar)
        assert np.array_equal(snap["p"], g.p)


def test_tiny_pipeline_equals_numpy_oracle_bit_for_bit():
    s = tiny_scene(seed=0)
    d = s.depth_maps()
    K = intrinsics_of(s.camera)
    g = O.run_pipeline(d, K, s.poses, P, 50)
    m = C.run_pipeline(d, K, s.poses, P, 50)
    _same_map(m.snapshot(), g)
    prob = O.PDProblem(g)
    Pn, Dn = O.energies(prob, g.u.reshape(-1), g.p.reshape(3, -1), P)
    Pc, Dc = m.energies()
    assert abs(Pc - Pn) <= 1e-12 * abs(Pn) and abs(Dc - Dn) <= 1e-12 * abs(Pn)


def test_rotated_camera_segment_and_wide_band_equal_numpy():
    """A yawed and pitched camera with fx != fy, segment 3 and the 1 m band of Table I."""
    s = tiny_scene(seed=2, n_frames=2)
    cam = Camera(210.0, 190.0, 64.137, 23.291, 131, 47)
    prm = O.Params(mu=1.0)
    a, b = 0.3, -0.12
    Ry = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    poses = []
    for T in s.poses[:2]:
        T2 = np.array(T, dtype=np.float64)
        T2[:3, :3] = Ry @ Rx
        poses.append(T2)
    sc = Scene(camera=cam, poses=poses, rects=s.rects, boxes=s.boxes, facades=s.facades, d_max=s.d_max,
               noise_sigma=0.02, seed=2)
    d = sc.depth_maps()
    K = intrinsics_of(cam)
    g = O.SparseGrid(prm)
    m = C.CMap(prm, 1 << 14)
    for k in range(2):
        assert m.alloc_blocks(d[k], K, poses[k], 3) == O.alloc_blocks(g, d[k], K, poses[k], 3)
        m.fuse_depth(d[k], K, poses[k], 3)
        O.fuse_depth(g, d[k], K, poses[k], 3)
    assert g.n_blocks > 50
    O.regularize(g, 20)
    m.regularize(20)
    _same_map(m.snapshot(), g)



def test_fuse_into_one_of_two_segments_equals_numpy():
    """The same blocks in segments 0 and 3; a depth map fused into segment 3 leaves
    segment 0 untouched, as in the numpy oracle."""
    s = tiny_scene(seed=1, n_frames=1)
    d = s.depth_maps()
    K = intrinsics_of(s.camera)
    g = O.SparseGrid(P)
    O.alloc_blocks(g, d[0], K, s.poses[0], 3)
    keys = [(0,) + tuple(k[1:]) for k in g.keys] + list(g.keys)
    both = grid_from_blocks(keys)
    m = cmap_of(both)
    O.fuse_depth(both, d[0], K, s.poses[0], 3)
    m.fuse_depth(d[0], K, s.poses[0], 3)
    _same_map(m.snapshot(), both, state=False)
    assert np.all(both.w[:g.n_blocks] == 0) and np.count_nonzero(both.w) > 100

def test_street_frames_equal_numpy():
    s = street_scene(seed=0)
    d = s.depth_maps(range(2))
    K = intrinsics_of(s.camera)
    g = O.SparseGrid(P)
    m = C.CMap(P, 1 << 14)
    for k in range(2):
        O.alloc_blocks(g, d[k], K, s.poses[k])
        O.fuse_depth(g, d[k], K, s.poses[k])
        m.alloc_blocks(d[k], K, s.poses[k])
        m.fuse_depth(d[k], K, s.poses[k])
    _same_map(m.snapshot(), g, state=False)


def test_warm_state_and_thread_count():
    rng = np.random.default_rng(5)
    keys = box_keys(2, 2, 1) + [(0, 5, 5, 5), (1, 0, 0, 0)]
    f, w = random_fw(rng, len(keys), p_omega=0.7)
    g = grid_from_blocks(keys, f, w)
    N = g.n_blocks * 512
    u0 = rng.uniform(-1, 1, N)
    p0 = rng.standard_normal((3, N)) * 0.3
    g.u[:] = u0.reshape(-1, 512)
    g.u_bar[:] = u0.reshape(-1, 512)
    g.p[:] = p0.reshape(3, -1, 512)
    outs = []
    for threads in (1, 3):
        m = cmap_of(g)
        m.set_state(u0, u0, p0)
        m.iterate(40, threads=threads)
        outs.append(m.snapshot())
    O.regularize(g, 40, warm=True)
    for sn in outs:
        _same_map(sn, g)


@pytest.mark.parametrize("f1,f2,w1,w2", [(-0.5, 0.9, 2.0, 3.0), (0.1, 0.6, 2.0, 3.0)])
def test_two_voxel_closed_form(f1, f2, w1, w2):
    lam = P.lam
    f = np.zeros((1, 512))
    w = np.zeros((1, 512))
    a, b = lin(3, 4, 5), lin(4, 4, 5)
    f[0, a], f[0, b], w[0, a], w[0, b] = f1, f2, w1, w2
    m = cmap_of(grid_from_blocks([(0, 0, 0, 0)], f, w))
    m.regularize(4000)
    u = m.snapshot()["u"].reshape(-1)
    sg = math.copysign(1.0, f2 - f1)
    if abs(f2 - f1) > 1 / (lam * w1) + 1 / (lam * w2):
        e1, e2 = f1 + sg / (lam * w1), f2 - sg / (lam * w2)
    else:
        e1 = e2 = (w1 * f1 + w2 * f2) / (w1 + w2)
    assert abs(u[a] - e1) < 1e-10 and abs(u[b] - e2) < 1e-10


def test_dense_box_equivalence():
    rng = np.random.default_rng(12)
    keys = box_keys(2, 2, 2)
    rng.shuffle(keys)
    f, w = random_fw(rng, len(keys), p_omega=0.85)
    g = grid_from_blocks(keys, f, w)
    m = cmap_of(g)
    m.regularize(60)
    sn = m.snapshot()
    ud, pd = _dense_solve(_to_dense(g, g.f, 2, 2, 2), _to_dense(g, g.w, 2, 2, 2), 60, P)
    np.testing.assert_allclose(_to_dense(g, sn["u"], 2, 2, 2), ud, rtol=0, atol=1e-12)
    for a in range(3):
        np.testing.assert_allclose(_to_dense(g, sn["p"][a], 2, 2, 2), pd[a], rtol=0, atol=1e-12)


def test_energies_against_brute_force():
    g = _tiny_problem(seed=13)
    m = cmap_of(g)
    for k in range(3):
        m.iterate(7)
        sn = m.snapshot()
        Pb, Db = _brute_energies(g, sn["u"].reshape(-1), sn["p"].reshape(3, -1), P)
        Pc, Dc = m.energies()
        assert abs(Pc - Pb) < 1e-11 and abs(Dc - Db) < 1e-11
    m.iterate(600)
    Pc, Dc = m.energies()
    assert 0 <= Pc - Dc < 1e-9 * Pc


def test_isolated_regions_and_weighted_mean():
    rng = np.random.default_rng(14)
    keys = [(0, 0, 0, 0), (0, 3, 0, 0)]
    f, w = random_fw(rng, 2, p_omega=0.7)
    g = grid_from_blocks(keys, f, w)
    om = w > 0
    m = cmap_of(g)
    m.regularize(6000)
    sn = m.snapshot()
    assert np.all(sn["u"][~om] == 0) and np.all(sn["p"][:, ~om] == 0)
    # each block is its own component here only if Omega connects it; the sum over the
    # whole of each block's Omega is conserved because no Eq. 3 edge joins the two blocks
    for b in range(2):
        mb = om[b]
        assert abs(np.sum(w[b][mb] * sn["u"][b][mb]) - np.sum(w[b][mb] * f[b][mb])) < 1e-7 * mb.sum()
