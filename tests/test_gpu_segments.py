"""The batched-segments workload: 64 independent street segments of lengths uniform in
50-500 m (seeds 1-64, 36 193 depth maps, 3.95 M blocks) fused into one map with
the segment as part of the block key, then regularised together (one sweep launch per
iteration over every segment, the loop as one CUDA graph, the autotuner's schedule),
as the benchmark runs it.  Blocks of different segments are never neighbours, so each
segment's result is that of the segment alone: the three shortest segments (149, 172
and 175 maps) are fused and iterated 200 times by the C oracle and compared on every
voxel (coords and w bit-exact; f, u, u_bar and p within 1e-4).
"""

import numpy as np
import pytest

from oracle import denser_oracle as O
from synth.scenes import segment_scenes, street_depth_maps
from tests.pipelines import oracle_K

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import autotune as AT  # noqa: E402
from paper_1604_03734_gb300 import native as N  # noqa: E402

TOL = 1e-4


def test_batched_segments_against_oracle():
    import os
    from oracle import oracle_c as C
    scenes = segment_scenes()
    frames = [len(s.poses) for s in scenes]
    specs = [(s.seed, n * 0.5) for s, n in zip(scenes, frames)]
    check = sorted(range(len(scenes)), key=lambda i: frames[i])[:3]
    cam = scenes[0].camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    total_m = sum(length for _, length in specs)
    max_blocks = int(np.ceil(290.0 * total_m / 1024.0)) * 1024
    kept = {i: np.zeros((frames[i], cam.height, cam.width), np.float32) for i in check}
    workers = max(1, min(16, os.cpu_count() or 1))
    with N.DenserMap(max_blocks=max_blocks, hash_slots=1 << 23) as m:
        batch, seg_of_batch, first = [], None, 0
        for i, k, d in street_depth_maps(specs, workers=workers):
            if i in kept:
                kept[i][k] = d
            if seg_of_batch is not None and (i != seg_of_batch or len(batch) == N.DENSER_MAX_BATCH):
                N.denser_integrate_batch(m.ctx, torch.from_numpy(np.stack(batch)).cuda(), K,
                                         np.asarray(scenes[seg_of_batch].poses[first:first + len(batch)]),
                                         seg_of_batch)
                first = 0 if i != seg_of_batch else first + len(batch)
                batch = []
            seg_of_batch = i
            batch.append(d)
        N.denser_integrate_batch(m.ctx, torch.from_numpy(np.stack(batch)).cuda(), K,
                                 np.asarray(scenes[seg_of_batch].poses[first:first + len(batch)]), seg_of_batch)
        nb = N.denser_num_blocks(m.ctx)
        assert nb > 3_500_000
        tune = AT.autotune(m.ctx, 0, iters=10, use_cache=False)
        st = N.denser_regularize(m.ctx, 200)
        assert st.iters == 200 and st.n_blocks == nb
        coords = torch.empty((nb, 4), dtype=torch.int32, device="cuda")
        N.denser_extract(m.ctx, coords, None, None, None, None, nb)
        rows = torch.nonzero(torch.isin(coords[:, 0], torch.tensor(check, dtype=torch.int32, device="cuda")))[:, 0]
        got = {"coords": coords[rows].cpu().numpy()}
        del coords
        buf = torch.empty((nb, 512), dtype=torch.float32, device="cuda")
        for key in ("f", "w", "u"):
            N.denser_extract(m.ctx, **{key: buf}, capacity_blocks=nb)
            got[key] = buf[rows].cpu().numpy()
        N.denser_extract_dual(m.ctx, buf, None, nb)
        got["u_bar"] = buf[rows].cpu().numpy()
        del buf
        p = torch.empty((3, nb, 512), dtype=torch.float32, device="cuda")
        N.denser_extract_dual(m.ctx, None, p, nb)
        got["p"] = p[:, rows].cpu().numpy()
        del p
    torch.cuda.empty_cache()
    print(f"\n64 segments: {nb} blocks, autotuned schedule {tune['schedule']}; checked segments {check}")
    seg = got["coords"][:, 0]
    for i in check:
        s = scenes[i]
        ref = C.run_pipeline(kept[i], oracle_K(cam), s.poses, O.Params(), 200, segment=i, capacity=1 << 16)
        want = ref.snapshot()
        ref.close()
        sel = seg == i
        np.testing.assert_array_equal(got["coords"][sel], want["coords"].astype(np.int32))
        np.testing.assert_array_equal(got["w"][sel], want["w"].astype(np.float32))
        errs = {k: float(np.max(np.abs(got[k][sel] - want[k]))) for k in ("f", "u", "u_bar")}
        errs["p"] = float(np.max(np.abs(got["p"][:, sel] - want["p"])))
        print(f"segment {i} ({frames[i]} maps, {int(sel.sum())} blocks): max |gpu - oracle| {errs}")
        for k, e in errs.items():
            assert e <= TOL, (i, k, e)
