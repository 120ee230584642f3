"""Full-size driving street (200 depth maps 1241x376, 200 iterations) in the context
configuration bench.py times, checked against the oracle on what it can compute:

  * allocation: the blocks of the first frames bit-exact (keys and indices), and every
    key the oracle finds for later frames present;
  * fusion: 48 sampled blocks fused by the oracle with every frame from the one that
    allocated them on (w bit-exact, f within 1e-4);
  * the batched call the benchmark times (16 maps per launch): the same map, bit for bit;
  * regularisation: from the GPU state after 200 iterations, one more GPU iteration
    equals one oracle iteration on sampled blocks (the update of a block only reads
    its 26-neighbourhood), and the FP64 gap is non-negative.
"""

import numpy as np
import pytest

from oracle import denser_oracle as O
from tests.oracle_helpers import grid_from_blocks
from tests.pipelines import oracle_K

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import native as N  # noqa: E402
from synth.scenes import street_scene  # noqa: E402

TOL = 1e-4


@pytest.fixture(scope="module")
def street():
    s = street_scene(seed=0)
    d = s.depth_maps()
    cam = s.camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    m = N.DenserMap(max_blocks=1 << 17, hash_slots=1 << 20)
    dd = torch.from_numpy(d).cuda()
    news = []   # blocks allocated after each frame
    for k in range(len(d)):
        N.denser_alloc_blocks(m.ctx, dd[k], K, s.poses[k])
        N.denser_fuse_depth(m.ctx, dd[k], K, s.poses[k])
        news.append(N.denser_num_blocks(m.ctx))
    snap = m.snapshot()
    yield s, d, m, snap, news
    m.close()


def test_full_allocation(street):
    s, d, m, snap, news = street
    K = oracle_K(s.camera)
    g = O.SparseGrid(O.Params())
    for k in range(3):
        O.alloc_blocks(g, d[k], K, s.poses[k])
        assert g.n_blocks == news[k]
    np.testing.assert_array_equal(snap["coords"][:g.n_blocks], g.coords().astype(np.int32))
    have = set(map(tuple, snap["coords"].tolist()))
    for k in (57, 123, 199):
        keys = O.frame_block_keys(d[k], K, s.poses[k], O.Params())
        assert keys <= have, len(keys - have)
    assert len(have) == len(snap["coords"]) > 10000


def test_full_fusion_sampled_blocks(street):
    s, d, m, snap, news = street
    rng = np.random.default_rng(0)
    sel = rng.choice(len(snap["coords"]), 48, replace=False)
    g = grid_from_blocks([tuple(c) for c in snap["coords"][sel]])
    K = oracle_K(s.camera)
    # a block exists from the frame that allocated it on: fuse only later frames into it
    born = np.searchsorted(np.array(news), sel, side="right")
    for k in range(len(d)):
        O.fuse_depth(g, d[k], K, s.poses[k], blocks=np.nonzero(born <= k)[0])
    np.testing.assert_array_equal(snap["w"][sel], g.w.astype(np.float32))
    assert np.max(np.abs(snap["f"][sel] - g.f)) <= TOL
    assert g.w.sum() > 0


def test_full_batched_fusion_equals_per_map(street):
    """The benchmark's configuration: all 200 maps through denser_integrate_batch (16 per
    launch) leave the per-map map above bit for bit (coords, f, w), so the oracle checks
    above hold for it too."""
    s, d, m, snap, news = street
    cam = s.camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    with N.DenserMap(max_blocks=1 << 17, hash_slots=1 << 20) as mb:
        n_new = N.denser_integrate_batch(mb.ctx, torch.from_numpy(d).cuda(), K, np.asarray(s.poses[:len(d)]), 0,
                                         count=True)
        got = mb.snapshot()
    assert n_new == news[-1]
    for key in ("coords", "f", "w"):
        np.testing.assert_array_equal(got[key], snap[key], err_msg=key)


def test_full_regularize_step_consistency(street):
    s, d, m, snap, _ = street
    st = N.denser_regularize(m.ctx, 200)
    assert st.gap >= 0 and st.iters == 200
    before = m.snapshot(dual=True)
    N.denser_regularize(m.ctx, 1, 0.0, 1)
    after = m.snapshot(dual=True)
    coords = before["coords"]
    index = {tuple(c): i for i, c in enumerate(coords.tolist())}
    rng = np.random.default_rng(1)
    sample = rng.choice(len(coords), 24, replace=False)
    # sampled blocks first, then their allocated 26-neighbours
    keys = [tuple(coords[i]) for i in sample]
    seen = set(keys)
    for c in list(keys):
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    q = (c[0], c[1] + dx, c[2] + dy, c[3] + dz)
                    if q in index and q not in seen:
                        seen.add(q)
                        keys.append(q)
    rows = [index[k] for k in keys]
    g = grid_from_blocks(keys, before["f"][rows].astype(np.float64), before["w"][rows].astype(np.float64))
    prob = O.PDProblem(g)
    u1, ub1, p1 = O.pd_iterate(prob, before["u"][rows].reshape(-1).astype(np.float64),
                               before["u_bar"][rows].reshape(-1).astype(np.float64),
                               before["p"][:, rows].reshape(3, -1).astype(np.float64), 1, g.params)
    n = len(sample)
    nv = n * 512
    assert np.max(np.abs(after["u"][sample].reshape(-1) - u1[:nv])) <= 2e-6
    assert np.max(np.abs(after["u_bar"][sample].reshape(-1) - ub1[:nv])) <= 4e-6
    assert np.max(np.abs(after["p"][:, sample].reshape(3, -1) - p1[:, :nv])) <= 2e-6
    om = before["omega"].astype(bool)
    assert np.all(after["u"][~om] == 0)
    assert np.all(np.sqrt((after["p"] ** 2).sum(0)) <= 1 + 1e-6)


def test_full_street_200_iterations_against_oracle(street):
    """The whole street in the benchmark's launch configuration (16 maps per batched
    allocation + fusion launch, 200 iterations of the default sweep in the graph loop,
    24 k blocks, so every CTA of the persistent grid takes many blocks in turn) against
    the C oracle's 200-frame, 200-iteration run, element by element on every voxel:
    coords and w bit-exact, f, u, u_bar and p within 1e-4, energies within 1e-5."""
    from oracle import oracle_c as C
    s, d, _, _, _ = street
    cam = s.camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    with N.DenserMap(max_blocks=1 << 17, hash_slots=1 << 20) as mb:
        N.denser_integrate_batch(mb.ctx, torch.from_numpy(d).cuda(), K, np.asarray(s.poses[:len(d)]), 0)
        st = N.denser_regularize(mb.ctx, 200)
        got = mb.snapshot(dual=True)
        Pg, Dg = N.denser_energy(mb.ctx)
    ref = C.run_pipeline(d, oracle_K(cam), s.poses, O.Params(), 200, capacity=1 << 15)
    want = ref.snapshot()
    Po, Do = ref.energies()
    ref.close()
    n = len(want["coords"])
    assert st.iters == 200 and n > 20000 and n * 512 > 4000 * 512
    np.testing.assert_array_equal(got["coords"], want["coords"].astype(np.int32))
    np.testing.assert_array_equal(got["w"], want["w"].astype(np.float32))
    errs = {k: float(np.max(np.abs(got[k] - want[k]))) for k in ("f", "u", "u_bar", "p")}
    print("\nfull street, 200 iterations, max |gpu - oracle|:", errs, "P", Pg, Po, "D", Dg, Do)
    for k, e in errs.items():
        assert e <= TOL, (k, e)
    assert abs(Pg - Po) <= 1e-5 * abs(Po) and abs(Dg - Do) <= 1e-5 * abs(Po)
