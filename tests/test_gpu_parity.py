"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Bars: block keys, block indices, weights and Omega bit-exact; f, u, u_bar and p
within 1e-4 (normalised TSDF units) for float32 storage.
"""

import math

import numpy as np
import pytest

from oracle import denser_oracle as O
from synth.scenes import tiny_scene
from tests.oracle_helpers import box_keys, grid_from_blocks, random_fw
from tests.pipelines import oracle_coords, oracle_K, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
TOL = 1e-4

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import build as B  # noqa: E402
from paper_1604_03734_gb300 import native as N  # noqa: E402

B.build()


@pytest.fixture(scope="module")
def tiny():
    s = tiny_scene(seed=0)
    return s, s.depth_maps()


@pytest.fixture(scope="module")
def tiny_runs(tiny):
    s, d = tiny
    g, news, _ = run_oracle(s, d, 50)
    m, gnews, st = run_gpu(s, d, 50)
    yield g, news, m, gnews, st
    m.close()


def test_tiny_allocation_bit_exact(tiny_runs):
    g, news, m, gnews, _ = tiny_runs
    assert gnews == news
    snap = m.snapshot()
    np.testing.assert_array_equal(snap["coords"], oracle_coords(g))
    assert 250 <= g.n_blocks <= 500


def test_tiny_fusion_parity(tiny_runs):
    g, _, m, _, _ = tiny_runs
    snap = m.snapshot()
    np.testing.assert_array_equal(snap["w"], g.w.astype(np.float32))
    np.testing.assert_array_equal(snap["omega"].astype(bool), g.w > 0)
    assert np.max(np.abs(snap["f"] - g.f)) <= TOL
    assert (g.w > 0).sum() > 50000


def test_tiny_regularize_50_iterations(tiny_runs):
    g, _, m, _, st = tiny_runs
    snap = m.snapshot(dual=True)
    assert st.iters == 50 and st.sweep_launches == 50
    err_u = np.max(np.abs(snap["u"] - g.u))
    err_ub = np.max(np.abs(snap["u_bar"] - g.u_bar))
    err_p = np.max(np.abs(snap["p"] - g.p))
    assert err_u <= TOL and err_ub <= TOL and err_p <= TOL, (err_u, err_ub, err_p)
    prob = O.PDProblem(g)
    P, D = O.energies(prob, g.u.reshape(-1), g.p.reshape(3, -1), g.params)
    assert abs(st.primal - P) <= 1e-5 * abs(P) and abs(st.dual - D) <= 1e-5 * abs(P)


def test_tiny_200_iterations(tiny):
    s, d = tiny
    g, _, _ = run_oracle(s, d, 200)
    m, _, st = run_gpu(s, d, 200)
    snap = m.snapshot(dual=True)
    m.close()
    assert np.max(np.abs(snap["u"] - g.u)) <= TOL
    assert np.max(np.abs(snap["p"] - g.p)) <= TOL


def _load(m, g):
    """Load an oracle map's blocks and fusion state into the context."""
    N.denser_load_blocks(m.ctx, oracle_coords(g), g.f.astype(np.float32), g.w.astype(np.float32))


def test_single_iteration_from_oracle_state(tiny):
    """One sweep from a mid-solve oracle state matches one oracle iteration."""
    s, d = tiny
    g, _, prob = run_oracle(s, d, 20)
    gf = grid_from_blocks(g.keys, g.f.astype(np.float32).astype(np.float64),
                          g.w.astype(np.float32).astype(np.float64))
    u0 = g.u.astype(np.float32)
    ub0 = g.u_bar.astype(np.float32)
    p0 = g.p.astype(np.float32)
    pr = O.PDProblem(gf)
    u1, ub1, p1 = O.pd_iterate(pr, u0.reshape(-1).astype(np.float64), ub0.reshape(-1).astype(np.float64),
                               p0.reshape(3, -1).astype(np.float64), 1, gf.params)
    with N.DenserMap() as m:
        _load(m, g)
        N.denser_load_state(m.ctx, u0, ub0, p0, g.n_blocks)
        st = N.denser_regularize(m.ctx, 1, 0.0, 1)
        snap = m.snapshot(dual=True)
    assert st.iters == 1
    assert np.max(np.abs(snap["u"].reshape(-1) - u1)) <= 2e-6
    assert np.max(np.abs(snap["u_bar"].reshape(-1) - ub1)) <= 4e-6
    assert np.max(np.abs(snap["p"].reshape(3, -1) - p1)) <= 2e-6


def test_energy_reduction_parity(tiny):
    """FP64 energies of a float32 state equal the oracle's on the same values."""
    s, d = tiny
    g, _, _ = run_oracle(s, d, 30)
    u32, p32 = g.u.astype(np.float32), g.p.astype(np.float32)
    gf = grid_from_blocks(g.keys, g.f.astype(np.float32).astype(np.float64),
                          g.w.astype(np.float32).astype(np.float64))
    P, D = O.energies(O.PDProblem(gf), u32.reshape(-1).astype(np.float64),
                      p32.reshape(3, -1).astype(np.float64), gf.params)
    with N.DenserMap() as m:
        _load(m, g)
        N.denser_load_state(m.ctx, u32, u32, p32, g.n_blocks)
        Pg, Dg = N.denser_energy(m.ctx)
    assert abs(Pg - P) <= 1e-12 * abs(P) and abs(Dg - D) <= 1e-12 * abs(P)


def test_dense_box_and_random_omega():
    rng = np.random.default_rng(11)
    keys = box_keys(3, 2, 2, origin=(-1, 4, 2))
    rng.shuffle(keys)
    f, w = random_fw(rng, len(keys), p_omega=0.7)
    f = f.astype(np.float32).astype(np.float64)
    g = grid_from_blocks(keys, f, w)
    O.regularize(g, 80)
    with N.DenserMap() as m:
        _load(m, g)
        N.denser_regularize(m.ctx, 80)
        snap = m.snapshot(dual=True)
    assert np.max(np.abs(snap["u"] - g.u)) <= TOL
    assert np.max(np.abs(snap["p"] - g.p)) <= TOL


def test_isolated_islands_and_edge_neighbours():
    """Blocks touching only along edges or corners, and lone blocks: the Omega-bar
    boundary and the 12-neighbour halo."""
    rng = np.random.default_rng(12)
    keys = [(0, 0, 0, 0), (0, 1, 1, 0), (0, 1, 0, 1), (0, 0, 1, 1), (0, -1, 1, 0), (0, 5, 5, 5),
            (0, 1, 0, 0), (0, 0, -1, 1), (1, 0, 0, 0)]
    f, w = random_fw(rng, len(keys), p_omega=0.75)
    f = f.astype(np.float32).astype(np.float64)
    g = grid_from_blocks(keys, f, w)
    O.regularize(g, 60)
    with N.DenserMap() as m:
        _load(m, g)
        N.denser_regularize(m.ctx, 60)
        snap = m.snapshot(dual=True)
    om = g.w > 0
    assert np.all(snap["u"][~om] == 0) and np.all(snap["p"][:, ~om] == 0)
    assert np.max(np.abs(snap["u"] - g.u)) <= TOL
    assert np.max(np.abs(snap["p"] - g.p)) <= TOL


def test_rotated_camera_and_ragged_image():
    s = tiny_scene(seed=3, n_frames=3, yaw_jitter=0.15, width=131, height=47, focal=90.0)
    d = s.depth_maps()
    g, news, _ = run_oracle(s, d, 25)
    m, gnews, _ = run_gpu(s, d, 25)
    snap = m.snapshot()
    m.close()
    assert gnews == news
    np.testing.assert_array_equal(snap["coords"], oracle_coords(g))
    np.testing.assert_array_equal(snap["w"], g.w.astype(np.float32))
    assert np.max(np.abs(snap["f"] - g.f)) <= TOL
    assert np.max(np.abs(snap["u"] - g.u)) <= TOL


def test_host_and_device_inputs_agree(tiny):
    s, d = tiny
    m1, n1, _ = run_gpu(s, d[:2], 10, device_depth=True)
    m2, n2, _ = run_gpu(s, d[:2], 10, device_depth=False)
    a, b = m1.snapshot(dual=True), m2.snapshot(dual=True)
    m1.close(), m2.close()
    assert n1 == n2
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_segments_and_mu_variant():
    """Two segments in one map never exchange values; a 1.0 m truncation (Table I)."""
    s = tiny_scene(seed=4, n_frames=2)
    d = s.depth_maps()
    prm = O.Params(mu=1.0)
    g = O.SparseGrid(prm)
    K = oracle_K(s.camera)
    with N.DenserMap(mu=1.0) as m:
        cam = s.camera
        Kg = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        for seg in (3, 0):
            for k in range(2):
                assert N.denser_alloc_blocks(m.ctx, d[k], Kg, s.poses[k], seg, count=True) == \
                    O.alloc_blocks(g, d[k], K, s.poses[k], seg)
                N.denser_fuse_depth(m.ctx, d[k], Kg, s.poses[k], seg)
                O.fuse_depth(g, d[k], K, s.poses[k], seg)
        O.regularize(g, 30)
        N.denser_regularize(m.ctx, 30)
        snap = m.snapshot()
    np.testing.assert_array_equal(snap["coords"], oracle_coords(g))
    np.testing.assert_array_equal(snap["w"], g.w.astype(np.float32))
    assert np.max(np.abs(snap["u"] - g.u)) <= TOL
    # the two segments hold identical geometry: identical results
    n = g.n_blocks // 2
    np.testing.assert_array_equal(snap["u"][:n], snap["u"][n:])


def test_gap_stop_rule_and_resume(tiny):
    s, d = tiny
    with N.DenserMap(gap_every=10) as m:
        cam = s.camera
        K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        for k in range(len(d)):
            N.denser_alloc_blocks(m.ctx, d[k], K, s.poses[k])
            N.denser_fuse_depth(m.ctx, d[k], K, s.poses[k])
        gaps = []
        st = N.denser_regularize(m.ctx, 10, 0.0, 0)
        gaps.append(st.gap)
        for _ in range(9):
            st = N.denser_regularize(m.ctx, 10, 0.0, 1)
            gaps.append(st.gap)
        assert all(g >= 0 for g in gaps)
        assert gaps[-1] < 0.2 * gaps[0]
        st = N.denser_regularize(m.ctx, 5000, 1e-3, 0)
        assert st.converged == 1 and st.rel_gap <= 1e-3 and st.iters % 10 == 0 and st.iters < 5000
        assert st.gap_evals == st.iters // 10


def test_edge_cases_empty_and_invalid():
    K = N.intrinsics(100, 100, 16.137, 8.291, 33, 17)
    with N.DenserMap() as m:
        st = N.denser_regularize(m.ctx, 5)           # no blocks at all
        assert st.iters == 5 and st.n_blocks == 0 and st.primal == 0.0
        empty = np.zeros((17, 33), np.float32)
        empty[0, :4] = [np.nan, -1.0, np.inf, -np.inf]
        assert N.denser_alloc_blocks(m.ctx, empty, K, np.eye(4), count=True) == 0
        N.denser_fuse_depth(m.ctx, empty, K, np.eye(4))
        assert N.denser_num_blocks(m.ctx) == 0
        st = N.denser_regularize(m.ctx, 0)
        assert st.iters == 0
        assert N.denser_extract(m.ctx) == 0


def test_error_paths():
    K = N.intrinsics(100, 100, 16.137, 8.291, 33, 17)
    depth = np.full((17, 33), 4.0, np.float32)
    wide = N.intrinsics(10, 10, 16.137, 8.291, 33, 17)   # about 60 blocks in view
    with N.DenserMap(max_blocks=8, hash_slots=16) as m:
        with pytest.raises(N.DenserError) as e:
            N.denser_alloc_blocks(m.ctx, depth, wide, np.eye(4), count=True)
        assert e.value.code in (N.DENSER_ERR_POOL_FULL, N.DENSER_ERR_HASH_FULL)
        N.denser_reset(m.ctx)
        N.denser_sync(m.ctx)  # sticky error cleared
    with N.DenserMap() as m:
        bad = np.eye(4)
        bad[0, 3] = np.nan
        with pytest.raises(N.DenserError) as e:
            N.denser_alloc_blocks(m.ctx, depth, K, bad)
        assert e.value.code == N.DENSER_ERR_INVALID_ARG
        with pytest.raises(N.DenserError):
            N.denser_fuse_depth(m.ctx, depth, K, np.eye(4), segment=127)
        far = np.eye(4)
        far[0, 3] = 1e6   # block coordinates beyond 2^18
        with pytest.raises(N.DenserError) as e:
            N.denser_alloc_blocks(m.ctx, depth, K, far, count=True)
        assert e.value.code == N.DENSER_ERR_RANGE
        N.denser_reset(m.ctx)
        N.denser_alloc_blocks(m.ctx, depth, K, np.eye(4), count=True)
        n = N.denser_num_blocks(m.ctx)
        with pytest.raises(N.DenserError) as e:
            N.denser_extract(m.ctx, coords=np.zeros((max(n - 1, 0), 4), np.int32), capacity_blocks=n - 1)
        assert e.value.code == N.DENSER_ERR_INVALID_ARG
        coords = np.zeros((n, 4), np.int32)
        N.denser_extract(m.ctx, coords=coords, capacity_blocks=n)
        with pytest.raises(N.DenserError) as e:   # duplicates are refused
            N.denser_load_blocks(m.ctx, coords[:1])
        assert e.value.code == N.DENSER_ERR_INVALID_ARG
        assert N.denser_launch_count(m.ctx) > 0


@pytest.mark.parametrize("sched", [(0, 0, 0, 0), (0, 1, 2, 1), (1, 0, 0, 0), (1, 1, 1, 1), (2, 0, 0, 1),
                                   (2, 1, 0, 0), (2, 1, 2, 1), (2, 1, 3, 1), (3, 1, 0, 1), (3, 0, 1, 0),
                                   (4, 1, 0, 1), (4, 0, 2, 0), (5, 0, 0, 1), (5, 1, 2, 0),
                                   (6, 0, 0, 1), (6, 1, 1, 0), (6, 0, 3, 1), (7, 0, 2, 1), (7, 1, 0, 0),
                                   (7, 0, 3, 1), (8, 0, 2, 1), (8, 1, 0, 0), (9, 0, 0, 1), (9, 1, 3, 0)])
def test_schedules_give_identical_iterates(tiny, sched):
    """Every sweep schedule (kernel variant, visiting order, CTAs per SM) computes the
    same Jacobi iterates bit for bit, and matches the oracle."""
    s, d = tiny
    g, _, _ = run_oracle(s, d, 40)
    ref = None
    with N.DenserMap() as m:
        cam = s.camera
        K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        for k in range(len(d)):
            N.denser_alloc_blocks(m.ctx, d[k], K, s.poses[k])
            N.denser_fuse_depth(m.ctx, d[k], K, s.poses[k])
        N.denser_set_schedule(m.ctx, 1, 1, 0, 0)
        N.denser_regularize(m.ctx, 40)
        ref = m.snapshot(dual=True)
        N.denser_set_schedule(m.ctx, *sched)
        assert N.denser_get_schedule(m.ctx) == dict(zip(("sweep_kernel", "order", "ctas_per_sm", "use_graph"), sched))
        N.denser_regularize(m.ctx, 40)
        out = m.snapshot(dual=True)
    for k in ("u", "u_bar", "p"):
        np.testing.assert_array_equal(out[k], ref[k])
    assert np.max(np.abs(out["u"] - g.u)) <= TOL and np.max(np.abs(out["p"] - g.p)) <= TOL


def test_schedule_rejects_bad_fields():
    with N.DenserMap() as m:
        with pytest.raises(N.DenserError):
            N.denser_set_schedule(m.ctx, 10, 0, 0)
        with pytest.raises(N.DenserError):
            N.denser_set_schedule(m.ctx, 1, 0, 9)
        with pytest.raises(N.DenserError):
            N.denser_set_schedule(m.ctx, 1, 0, 0, 2)


def test_integrate_matches_alloc_then_fuse(tiny):
    """denser_integrate (one staging of the depth map) leaves the same map as
    alloc + fuse, for device inputs and for pinned and pageable host inputs (the
    latter through the two copy-stream staging buffers, several frames in flight)."""
    sc, depths = tiny
    cam = sc.camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    ref, _, _ = run_gpu(sc, depths, 0)
    want = ref.snapshot()
    ref.close()
    for kind in ("device", "pinned", "pageable"):
        m = N.DenserMap()
        news = []
        for k in range(len(depths)):
            d = torch.from_numpy(np.ascontiguousarray(depths[k]))
            d = d.cuda() if kind == "device" else (d.pin_memory() if kind == "pinned" else d)
            news.append(N.denser_integrate(m.ctx, d, K, sc.poses[k], 0, count=(k == len(depths) - 1)))
        got = m.snapshot()
        for key in ("coords", "f", "w", "u"):
            np.testing.assert_array_equal(got[key], want[key], err_msg=f"{kind} {key}")
        m.close()


def test_twenty_centimetre_configuration():
    """Table I's 20 cm column: s = 0.2 m, lambda = 0.4, mu = 1.6 m (33 band samples per ray)."""
    sc = tiny_scene(seed=0)
    d = sc.depth_maps()
    prm = O.Params(voxel_size=0.2, mu=1.6, lam=0.4)
    g, news_o, _ = run_oracle(sc, d, 50, params=prm)
    m, news_g, st = run_gpu(sc, d, 50, voxel_size=0.2, mu=1.6, **{"lambda": 0.4})
    snap = m.snapshot(dual=True)
    m.close()
    assert news_g == news_o and st.iters == 50
    np.testing.assert_array_equal(snap["coords"], oracle_coords(g))
    np.testing.assert_array_equal(snap["w"], g.w.astype(np.float32))
    assert np.max(np.abs(snap["f"] - g.f)) <= TOL
    assert np.max(np.abs(snap["u"] - g.u)) <= TOL
    assert np.max(np.abs(snap["p"] - g.p)) <= TOL


def test_checkpoint_and_restore_continue_bit_identically(tiny):
    """Save/restore of the block state: extract everything after 30 iterations, load it
    into a fresh context (same block order), run 20 more; the iterates equal 50
    uninterrupted iterations bit for bit."""
    sc, d = tiny
    m50, _, _ = run_gpu(sc, d, 50)
    want = m50.snapshot(dual=True)
    m50.close()
    m30, _, _ = run_gpu(sc, d, 30)
    s30 = m30.snapshot(dual=True)
    m30.close()
    nb = len(s30["coords"])
    with N.DenserMap() as m:
        N.denser_load_blocks(m.ctx, s30["coords"], s30["f"], s30["w"])
        N.denser_load_state(m.ctx, s30["u"], s30["u_bar"], s30["p"], nb)
        N.denser_regularize(m.ctx, 20, 0.0, 1)
        got = m.snapshot(dual=True)
    for key in ("coords", "f", "w", "u", "u_bar", "p"):
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)
