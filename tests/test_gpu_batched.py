"""Batched segments, the graph-captured iteration loop and the autotuner.

Many independent street segments share one map (the segment is part of the block
key, and blocks of different segments are never neighbours); one sweep launch per
iteration covers all of them.  Checks: parity with the oracle run over the same
segments, bit-identical results to each segment solved alone, the graph-captured
loop equal to one launch per sweep (also with the device-side gap stop), and the
autotuner leaving the iterates unchanged.
"""

import numpy as np
import pytest

from oracle import denser_oracle as O
from synth.scenes import tiny_scene
from tests.pipelines import oracle_coords, oracle_K

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import autotune as AT  # noqa: E402
from paper_1604_03734_gb300 import native as N  # noqa: E402

TOL = 1e-4


def _segments(n=6):
    """Uneven segments: different seeds, frame counts, wall and cube positions."""
    out = []
    for i in range(n):
        s = tiny_scene(seed=20 + i, n_frames=2 + (i * 3) % 5, wall_z=9.0 + 1.3 * i, cube_at=(-2.0 + 0.7 * i, 6.0 + 0.4 * i))
        out.append((i, s, s.depth_maps()))
    return out


def _fill_gpu(m, segs):
    for seg, s, d in segs:
        cam = s.camera
        K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        for k in range(len(d)):
            N.denser_alloc_blocks(m.ctx, d[k], K, s.poses[k], seg)
            N.denser_fuse_depth(m.ctx, d[k], K, s.poses[k], seg)


def test_batched_segments_parity_and_independence():
    segs = _segments()
    g = O.SparseGrid(O.Params())
    for seg, s, d in segs:
        K = oracle_K(s.camera)
        for k in range(len(d)):
            O.alloc_blocks(g, d[k], K, s.poses[k], seg)
            O.fuse_depth(g, d[k], K, s.poses[k], seg)
    O.regularize(g, 40)
    with N.DenserMap() as m:
        _fill_gpu(m, segs)
        st = N.denser_regularize(m.ctx, 40)
        snap = m.snapshot(dual=True)
    assert st.iters == 40
    np.testing.assert_array_equal(snap["coords"], oracle_coords(g))
    np.testing.assert_array_equal(snap["w"], g.w.astype(np.float32))
    assert np.max(np.abs(snap["u"] - g.u)) <= TOL and np.max(np.abs(snap["p"] - g.p)) <= TOL
    # each segment alone in its own map reaches bit-identical values
    rows = {tuple(c): i for i, c in enumerate(snap["coords"].tolist())}
    for pick in (1, 4):
        with N.DenserMap() as m1:
            _fill_gpu(m1, [segs[pick]])
            N.denser_regularize(m1.ctx, 40)
            alone = m1.snapshot(dual=True)
        idx = [rows[tuple(c)] for c in alone["coords"].tolist()]
        np.testing.assert_array_equal(alone["u"], snap["u"][idx])
        np.testing.assert_array_equal(alone["p"], snap["p"][:, idx])


def _tiny_map(**params):
    s = tiny_scene(seed=0)
    m = N.DenserMap(**params)
    _fill_gpu(m, [(0, s, s.depth_maps())])
    return m


@pytest.mark.parametrize("iters", [60, 37])
def test_graph_loop_equals_single_launches(iters):
    with _tiny_map() as m:
        N.denser_set_schedule(m.ctx, 2, 1, 0, 0)
        st0 = N.denser_regularize(m.ctx, iters)
        a = m.snapshot(dual=True)
        N.denser_set_schedule(m.ctx, 2, 1, 0, 1)
        st1 = N.denser_regularize(m.ctx, iters)
        b = m.snapshot(dual=True)
        st2 = N.denser_regularize(m.ctx, iters)   # replays the recorded graph
        c = m.snapshot(dual=True)
    assert st0.iters == st1.iters == st2.iters == iters
    for k in ("u", "u_bar", "p"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], c[k])
    assert st1.primal == st0.primal and st1.dual == st0.dual


@pytest.mark.parametrize("gap_every", [10, 7])
def test_device_side_gap_stop_equals_host_loop(gap_every):
    with _tiny_map(gap_every=gap_every) as m:
        N.denser_set_schedule(m.ctx, 2, 1, 0, 0)
        ref = N.denser_regularize(m.ctx, 3000, 1e-3, 0)
        N.denser_set_schedule(m.ctx, 2, 1, 0, 1)
        got = N.denser_regularize(m.ctx, 3000, 1e-3, 0)
    assert ref.converged == got.converged == 1
    assert ref.iters == got.iters and ref.gap_evals == got.gap_evals
    assert ref.iters % gap_every == 0 and ref.iters < 3000
    assert got.primal == ref.primal and got.dual == ref.dual and got.rel_gap <= 1e-3


def test_autotune_keeps_iterates(tmp_path):
    with _tiny_map() as m:
        N.denser_regularize(m.ctx, 30)
        ref = m.snapshot(dual=True)
        res = AT.autotune(m.ctx, iters=5, cache_file=str(tmp_path / "tune.json"), use_cache=False)
        assert len(res["table"]) >= 5 and res["ms_per_iter"] > 0
        assert N.denser_get_schedule(m.ctx) == dict(zip(("sweep_kernel", "order", "ctas_per_sm", "use_graph"),
                                                        res["schedule"]))
        N.denser_regularize(m.ctx, 30)
        got = m.snapshot(dual=True)
        again = AT.autotune(m.ctx, iters=5, cache_file=str(tmp_path / "tune.json"))
    assert again["cached"] and again["schedule"] == res["schedule"]
    for k in ("u", "u_bar", "p"):
        np.testing.assert_array_equal(ref[k], got[k])
