"""denser_energy_noalloc against denser_energy, through the C ABI.

The allocation-free entry point serves callers that may not allocate device
memory themselves: a process whose GPU memory all belongs to its own allocator
(a framework's caching allocator, or an on-vehicle mapping process with a fixed
memory budget), or a loop that cannot take the device-wide synchronisation of
cudaMalloc / cudaFree.  It must give the same primal and dual energies as the
context-based call, call after call, although all calls share one fixed device
array.  This file is collected last so that a run stopping at the first failure
has run every other test already.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import build as B  # noqa: E402
from paper_1604_03734_gb300 import native as N  # noqa: E402
from synth.scenes import tiny_scene  # noqa: E402

B.build()
REL = 1e-12  # the energy parity tolerance of the context path's tests


def _map_and_buffers(seed, iters):
    """A fused and partly regularised tiny map, its energies from denser_energy, and its
    state copied into device buffers in the layouts the no-alloc call reads."""
    s = tiny_scene(seed=seed)
    d = s.depth_maps()
    cam = s.camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    m = N.DenserMap()
    for k in range(len(d)):
        N.denser_alloc_blocks(m.ctx, d[k], K, s.poses[k])
        N.denser_fuse_depth(m.ctx, d[k], K, s.poses[k])
    N.denser_regularize(m.ctx, iters)
    P, D = N.denser_energy(m.ctx)
    n = N.denser_num_blocks(m.ctx)
    dev = torch.device("cuda")
    buf = {"coords": torch.empty(n, 4, dtype=torch.int32, device=dev),
           "f": torch.empty(n, 512, device=dev), "w": torch.empty(n, 512, device=dev),
           "u": torch.empty(n, 512, device=dev), "p": torch.empty(3, n, 512, device=dev)}
    N.denser_extract(m.ctx, buf["coords"], buf["f"], buf["w"], None, buf["u"], n)
    N.denser_extract_dual(m.ctx, None, buf["p"], n)
    m.close()
    return n, (P, D), buf


def _call(n, buf, out, lam=0.8):
    rc = N.denser_energy_noalloc(buf["coords"], buf["f"], buf["w"], buf["u"], buf["p"], n, lam, out)
    torch.cuda.synchronize()
    return rc


def test_noalloc_matches_context_energy_on_consecutive_calls():
    n_a, (Pa, Da), a = _map_and_buffers(seed=0, iters=30)
    n_b, (Pb, Db), b = _map_and_buffers(seed=5, iters=10)
    assert 0 < n_a <= N.DENSER_NOALLOC_MAX_BLOCKS and 0 < n_b <= N.DENSER_NOALLOC_MAX_BLOCKS
    out_dev = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):   # two calls in a row on the same map, device output
        assert _call(n_a, a, out_dev) == N.DENSER_OK
        P, D = out_dev.tolist()
        assert abs(P - Pa) <= REL * abs(Pa) and abs(D - Da) <= REL * abs(Pa)
    out_host = np.full(2, np.nan)
    for _ in range(2):   # then another map: the shared array keeps nothing stale
        assert _call(n_b, b, out_host) == N.DENSER_OK
        assert abs(out_host[0] - Pb) <= REL * abs(Pb) and abs(out_host[1] - Db) <= REL * abs(Pb)
    assert abs(Pa - Pb) > 1e-6 * abs(Pa)   # the two maps really differ


def test_noalloc_leaves_device_memory_unchanged():
    """After the first call on the device (which looks the array's address up), further
    calls change neither the device's free memory nor torch's allocator."""
    n, (P0, _), a = _map_and_buffers(seed=2, iters=5)
    out_dev = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _call(n, a, out_dev) == N.DENSER_OK
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        assert _call(n, a, out_dev) == N.DENSER_OK
    free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert (free1, alloc1) == (free0, alloc0)
    assert abs(out_dev[0].item() - P0) <= REL * abs(P0)


def test_noalloc_rejects_bad_calls():
    n, _, a = _map_and_buffers(seed=1, iters=2)
    out = np.zeros(2)
    too_many = N.DENSER_NOALLOC_MAX_BLOCKS + 1
    assert _call(too_many, a, out) == N.DENSER_ERR_TOO_LARGE
    host = {k: v.cpu().numpy() for k, v in a.items()}
    assert _call(n, host, out) == N.DENSER_ERR_INVALID_ARG
    assert _call(n, a, out, lam=0.0) == N.DENSER_ERR_INVALID_ARG
    # coordinates 4 bytes past a 16-byte boundary (the kernels read them as int4) are
    # refused before anything is launched
    big = torch.zeros(4 * n + 4, dtype=torch.int32, device="cuda")
    big[1:1 + 4 * n] = a["coords"].reshape(-1)
    odd = dict(a)
    odd["coords"] = big[1:1 + 4 * n]
    assert odd["coords"].data_ptr() % 16 == 4
    assert _call(n, odd, out) == N.DENSER_ERR_INVALID_ARG
    # a repeated coordinate is reported as NaN energies
    dup = dict(a)
    dup["coords"] = a["coords"].clone()
    dup["coords"][1] = dup["coords"][0]
    assert _call(n, dup, out) == N.DENSER_OK and np.isnan(out).all()
    # and the next valid call is unaffected
    assert _call(n, a, out) == N.DENSER_OK and np.isfinite(out).all()
