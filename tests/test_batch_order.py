"""The index rule of the batched allocation, on the CPU.

denser_integrate_batch indexes the blocks a batch adds by (birth, key), birth being the
first depth map of the batch whose band reaches the block, and sorts them as one 64-bit
word: the key's 7 segment bits replaced by the birth (one segment per call).  These
tests check, against the oracle's one-map-at-a-time allocation (Section III-A, reading
R1), that this order is the sequential one, and that the 64-bit word sorts like the
pair.  No GPU.
"""

import numpy as np

from oracle import denser_oracle as O
from synth.scenes import tiny_scene
from tests.pipelines import oracle_K

COORD_BITS = 19
COORD_BIAS = 1 << 18


def packed_key(seg, bx, by, bz):
    """The 64-bit block key of include/denser.h: bx, by, bz biased by 2^18 in 19 bits each
    (x lowest), the segment in the top 7 bits."""
    return ((bx + COORD_BIAS) | ((by + COORD_BIAS) << COORD_BITS) | ((bz + COORD_BIAS) << (2 * COORD_BITS))
            | (seg << (3 * COORD_BITS)))


def birth_word(birth, key):
    return (birth << (3 * COORD_BITS)) | (key & ((1 << (3 * COORD_BITS)) - 1))


def _batch_order(per_frame_keys, already):
    birth = {}
    for i, keys in enumerate(per_frame_keys):
        for k in keys:
            if k not in already and k not in birth:
                birth[k] = i
    return sorted(birth, key=lambda k: birth_word(birth[k], packed_key(*k))), birth


def test_birth_order_is_the_sequential_order():
    sc = tiny_scene(seed=3, n_frames=6, yaw_jitter=0.15)
    d = sc.depth_maps()
    K = oracle_K(sc.camera)
    prm = O.Params()
    g = O.SparseGrid(prm)
    O.alloc_blocks(g, d[0], K, sc.poses[0], 5)  # blocks from an earlier call keep their indices
    before = g.n_blocks
    per_frame = [O.frame_block_keys(d[k], K, sc.poses[k], prm, 5) for k in range(1, 6)]
    batch, birth = _batch_order(per_frame, set(g.index))
    for k in range(1, 6):
        O.alloc_blocks(g, d[k], K, sc.poses[k], 5)
    seq = [tuple(int(v) for v in c) for c in g.coords()[before:]]
    assert len(batch) == len(seq) > 10
    assert len(set(birth.values())) > 2  # new blocks come from several maps of the batch
    assert batch == seq


def test_birth_word_sorts_like_the_pair():
    rng = np.random.default_rng(0)
    seg = 9
    keys = [(seg, int(x), int(y), int(z)) for x, y, z in rng.integers(-COORD_BIAS, COORD_BIAS, size=(400, 3))]
    keys += [(seg, -COORD_BIAS, -COORD_BIAS, -COORD_BIAS), (seg, COORD_BIAS - 1, COORD_BIAS - 1, COORD_BIAS - 1)]
    births = rng.integers(0, 16, size=len(keys))
    by_word = sorted(range(len(keys)), key=lambda i: birth_word(int(births[i]), packed_key(*keys[i])))
    by_pair = sorted(range(len(keys)), key=lambda i: (int(births[i]), keys[i][3], keys[i][2], keys[i][1]))
    assert by_word == by_pair
    # the largest word (birth 15, all coordinate bits set) stays below the empty-slot marker
    assert birth_word(15, packed_key(seg, COORD_BIAS - 1, COORD_BIAS - 1, COORD_BIAS - 1)) < (1 << 64) - 1
