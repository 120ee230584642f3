"""Surface extraction through the C ABI against the oracle (oracle/surface_oracle.py).

Inputs are loaded into the map with denser_load_blocks / denser_load_state, so both
sides see the same f, w, u (u rounded to the storage precision on the host first).
The triangle count, order and vertex ids must match exactly; vertex positions agree
within the float32 evaluation error, |x32 - x64| <= 2^-21 (|x| + s).

At full size (a synthetic 100 m street, ~28 k blocks) the oracle recomputes sampled
blocks one by one from each block and its seven upper neighbours, and every block's
triangle range comes from block_first.
"""

import numpy as np
import pytest

from oracle import denser_oracle as O
from oracle import surface_oracle as S
from synth import maps, scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import native as N  # noqa: E402

from tests.pipelines import run_oracle  # noqa: E402

N.lib()
S_VOX = 0.1


def storage_round(u, precision):
    if precision == N.DENSER_FP16:
        return u.astype(np.float16).astype(np.float32)
    if precision == N.DENSER_BF16:
        return torch.from_numpy(u).to(torch.bfloat16).to(torch.float32).numpy()
    return u.astype(np.float32)


def load_map(coords, f, w, u, precision=N.DENSER_FP32, voxel_size=S_VOX):
    m = N.DenserMap(precision=precision, voxel_size=voxel_size, max_blocks=max(64, len(coords) + 8))
    N.denser_load_blocks(m.ctx, np.ascontiguousarray(coords, np.int32), np.ascontiguousarray(f, np.float32),
                         np.ascontiguousarray(w, np.float32))
    N.denser_load_state(m.ctx, np.ascontiguousarray(u, np.float32), None, None, len(coords))
    return m


def gpu_surface(m):
    nb = N.denser_num_blocks(m.ctx)
    first = np.zeros(nb + 1, np.int64)
    n = N.denser_extract_surface(m.ctx, block_first=first)
    pos = np.zeros((n, 3, 3), np.float32)
    ids = np.zeros((n, 3), np.int64)
    if n:
        assert N.denser_extract_surface(m.ctx, pos, ids, n, first) == n
    return pos, ids, first


def assert_same_mesh(pos, ids, ref_pos, ref_ids, s=S_VOX):
    assert pos.shape[0] == ref_pos.shape[0]
    np.testing.assert_array_equal(ids, ref_ids)
    tol = 2.0 ** -21 * (np.abs(ref_pos) + s)
    err = np.abs(pos.astype(np.float64) - ref_pos)
    assert np.all(err <= tol), float(np.max(err / tol))


@pytest.mark.parametrize("precision", [N.DENSER_FP32, N.DENSER_FP16, N.DENSER_BF16])
@pytest.mark.parametrize("seed", [0, 1])
def test_random_map_parity(seed, precision):
    coords, f, w, u = maps.random_map(seed)
    u = storage_round(u, precision)
    m = load_map(coords, f, w, u, precision)
    pos, ids, first = gpu_surface(m)
    ref_pos, ref_ids = S.extract_surface([tuple(c) for c in coords], u, w > 0, S_VOX)
    assert len(ref_pos) > 100
    assert_same_mesh(pos, ids, ref_pos, ref_ids)
    # block_first: per-block ranges that add up and follow the output order
    assert first[0] == 0 and first[-1] == len(pos) and np.all(np.diff(first) >= 0)
    for b in range(len(coords)):
        sub_pos, sub_ids = S.extract_surface([tuple(c) for c in coords], u, w > 0, S_VOX, blocks=[b])
        assert first[b + 1] - first[b] == len(sub_pos)
    m.close()


def test_oracle_pipeline_parity():
    """The tiny street regularised by the oracle (50 iterations), meshed on both sides."""
    sc = scenes.tiny_scene(0)
    depths = sc.depth_maps()
    g, _, _ = run_oracle(sc, depths, 50)
    coords = g.coords().astype(np.int32)
    u = g.u.astype(np.float32)
    m = load_map(coords, g.f, g.w, u)
    pos, ids, _ = gpu_surface(m)
    ref_pos, ref_ids = S.extract_surface(g.keys, u, O.omega(g).reshape(-1, 512), S_VOX)
    assert len(ref_pos) > 1000
    assert_same_mesh(pos, ids, ref_pos, ref_ids)
    m.close()


def test_outputs_capacity_and_memory_kinds():
    coords, f, w, u = maps.random_map(2)
    m = load_map(coords, f, w, u)
    pos, ids, first = gpu_surface(m)
    n = len(pos)
    # device outputs give the same bytes
    dpos = torch.zeros((n, 3, 3), dtype=torch.float32, device="cuda")
    dids = torch.zeros((n, 3), dtype=torch.int64, device="cuda")
    dfirst = torch.zeros(len(coords) + 1, dtype=torch.int64, device="cuda")
    assert N.denser_extract_surface(m.ctx, dpos, dids, n, dfirst) == n
    np.testing.assert_array_equal(dpos.cpu().numpy(), pos)
    np.testing.assert_array_equal(dids.cpu().numpy(), ids)
    np.testing.assert_array_equal(dfirst.cpu().numpy(), first)
    # positions only, ids only
    p2 = np.zeros_like(pos)
    assert N.denser_extract_surface(m.ctx, p2, None, n) == n
    np.testing.assert_array_equal(p2, pos)
    i2 = np.zeros_like(ids)
    assert N.denser_extract_surface(m.ctx, None, i2, n) == n
    np.testing.assert_array_equal(i2, ids)
    # too small a capacity: the prefix is written, the error says so, the count is exact
    cap = n // 3
    p3 = np.zeros((cap, 3, 3), np.float32)
    i3 = np.zeros((cap, 3), np.int64)
    with pytest.raises(N.DenserError) as e:
        N.denser_extract_surface(m.ctx, p3, i3, cap)
    assert e.value.code == N.DENSER_ERR_TOO_LARGE
    np.testing.assert_array_equal(p3, pos[:cap])
    np.testing.assert_array_equal(i3, ids[:cap])
    with pytest.raises(N.DenserError):
        N.denser_extract_surface(m.ctx, p3, i3, -1)
    m.close()


def test_empty_and_unobserved_maps():
    m = N.DenserMap()
    first = np.full(1, 7, np.int64)
    assert N.denser_extract_surface(m.ctx, block_first=first) == 0 and first[0] == 0
    m.close()
    coords, f, w, u = maps.random_map(3)
    m = load_map(coords, f, np.zeros_like(w), u)  # nothing observed: no cube is meshed
    assert N.denser_extract_surface(m.ctx) == 0
    m.close()
    m = load_map(coords, f, w, np.abs(u) + 0.5)  # all positive: no crossing
    assert N.denser_extract_surface(m.ctx) == 0
    m.close()


def test_fullsize_street_sampled():
    coords, f, w, u = maps.street_map(0)
    m = load_map(coords, f, w, u)
    pos, ids, first = gpu_surface(m)
    nb = len(coords)
    assert nb > 20000 and len(pos) > 300_000
    # the same id is the same vertex, bit for bit
    flat_ids, order = np.unique(ids.reshape(-1), return_inverse=True)
    fp = pos.reshape(-1, 3)
    ref = np.zeros((len(flat_ids), 3), np.float32)
    ref[order] = fp
    np.testing.assert_array_equal(ref[order], fp)
    # sampled blocks against the oracle on the block and its seven upper neighbours
    index = {tuple(c): b for b, c in enumerate(coords.tolist())}
    rng = np.random.default_rng(4)
    om = w > 0
    checked = 0
    for b in rng.choice(nb, 48, replace=False):
        seg, bx, by, bz = coords[b]
        sub = [int(b)]
        for code in range(1, 8):
            k = (seg, bx + (code & 1), by + ((code >> 1) & 1), bz + ((code >> 2) & 1))
            if k in index:
                sub.append(index[k])
        keys = [tuple(coords[i]) for i in sub]
        rp, ri = S.extract_surface(keys, u[sub], om[sub], S_VOX, blocks=[0])
        # map sub-map block indices back to the full map's
        sub_arr = np.array(sub, np.int64)
        ri = (sub_arr[(ri // 8) // 512] * 512 + (ri // 8) % 512) * 8 + ri % 8
        lo, hi = first[b], first[b + 1]
        assert hi - lo == len(rp)
        assert_same_mesh(pos[lo:hi], ids[lo:hi], rp, ri)
        checked += len(rp)
    assert checked > 1000
    m.close()
