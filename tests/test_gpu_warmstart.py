"""Warm-start network kernels against the FP64 oracle (oracle/net_oracle.py).  The
forward and data-gradient convolutions run on tcgen05 (tensor memory accumulators),
the weight gradient on mma.sync.

Per layer, on BF16-representable inputs (so that only the FP32 accumulation differs
from the oracle): forward convolution, data gradient and weight/bias gradient to a
relative 1e-5 of the largest entry; the loss to 1e-6.  The whole network (BF16
activations between layers) against the FP64 network: outputs and every layer's
gradients within 5e-2 relative (the rounding of activations to 8 mantissa bits).
Training with the library's Adam lowers the loss.
"""

import numpy as np
import pytest

from oracle import net_oracle as NO

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_03734_gb300 import native as N  # noqa: E402
from paper_1604_03734_gb300 import warmstart as WS  # noqa: E402

N.lib()


def bf16_round(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def to_ours(x):
    """[n, C, 10, 10, 10] -> [n, 1000, 16] (channels zero-padded to 16)."""
    n, c = x.shape[:2]
    out = np.zeros((n, 1000, 16))
    out[:, :, :c] = x.transpose(0, 2, 3, 4, 1).reshape(n, 1000, c)
    return out


def from_ours(y, c):
    n = y.shape[0]
    return y[:, :, :c].reshape(n, 10, 10, 10, c).transpose(0, 4, 1, 2, 3)


def w_ours(W):
    """[co, ci, 3, 3, 3] -> [27, 16, 16] (tap = dx + 3 dy + 9 dz)."""
    co, ci = W.shape[:2]
    out = np.zeros((27, 16, 16))
    out[:, :co, :ci] = W.transpose(2, 3, 4, 0, 1).reshape(27, co, ci)
    return out


def dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda").to(dtype).contiguous()


@pytest.fixture(scope="module")
def layer_case():
    rng = np.random.default_rng(0)
    n = 3
    x = bf16_round(rng.standard_normal((n, 16, 10, 10, 10)))
    W = bf16_round(rng.standard_normal((16, 16, 3, 3, 3)) * 0.1)
    b = rng.standard_normal(16).astype(np.float32).astype(np.float64)
    return n, x, W, b


def test_conv3_forward_layer(layer_case):
    n, x, W, b = layer_case
    y = torch.empty(n, 1000, 16, device="cuda")
    yb = torch.empty(n, 1000, 16, dtype=torch.bfloat16, device="cuda")
    N.denser_conv3(dev(to_ours(x), torch.bfloat16), dev(w_ours(W), torch.bfloat16), dev(b), 0, yb, y, n)
    ref = NO.conv3d_same(x, W, b)
    got = from_ours(y.cpu().numpy().astype(np.float64), 16)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    # ReLU and the BF16 copy
    N.denser_conv3(dev(to_ours(x), torch.bfloat16), dev(w_ours(W), torch.bfloat16), dev(b), 1, yb, y, n)
    got = from_ours(y.cpu().numpy().astype(np.float64), 16)
    assert np.max(np.abs(got - np.maximum(ref, 0))) <= 1e-5 * np.max(np.abs(ref))
    np.testing.assert_array_equal(yb.float().cpu().numpy(), y.to(torch.bfloat16).float().cpu().numpy())
    assert N.denser_net_check() == N.DENSER_OK   # every tensor-core wait completed


def test_conv3_pipelined_samples():
    """Several samples per CTA (700 samples; the grid has two CTAs per SM), so that each
    CTA restages its planes and reuses its tensor-memory columns sample after sample:
    sampled outputs (the first and last samples, and ones spread through every CTA's
    turn) against the FP64 oracle at the per-layer tolerance, and two calls bit-equal."""
    rng = np.random.default_rng(5)
    n = 700
    x = bf16_round(rng.standard_normal((n, 16, 10, 10, 10)))
    W = bf16_round(rng.standard_normal((16, 16, 3, 3, 3)) * 0.1)
    b = rng.standard_normal(16).astype(np.float32).astype(np.float64)
    xd, wd, bd = dev(to_ours(x), torch.bfloat16), dev(w_ours(W), torch.bfloat16), dev(b)
    y = torch.empty(n, 1000, 16, device="cuda")
    y2 = torch.empty_like(y)
    N.denser_conv3(xd, wd, bd, 1, None, y, n)
    N.denser_conv3(xd, wd, bd, 1, None, y2, n)
    assert N.denser_net_check() == N.DENSER_OK
    assert torch.equal(y, y2)
    idx = np.unique(np.concatenate([[0, 1, n - 1, n - 2], rng.choice(n, 24, replace=False)]))
    ref = np.maximum(NO.conv3d_same(x[idx], W, b), 0)
    got = from_ours(y[torch.as_tensor(idx, device="cuda")].cpu().numpy().astype(np.float64), 16)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_conv3_gradients_layer(layer_case):
    n, x, W, b = layer_case
    rng = np.random.default_rng(1)
    dz = bf16_round(rng.standard_normal((n, 16, 10, 10, 10)))
    dx_ref, dW_ref, db_ref = NO.conv3d_same_backward(x, W, dz)
    w32 = dev(w_ours(W))
    wf = torch.empty(27, 16, 16, dtype=torch.bfloat16, device="cuda")
    wb = torch.empty_like(wf)
    N.denser_pack_weights(w32, wf, wb)
    np.testing.assert_array_equal(wf.float().cpu().numpy(), w_ours(W).astype(np.float32))
    dx = torch.empty(n, 1000, 16, device="cuda")
    N.denser_conv3(dev(to_ours(dz), torch.bfloat16), wb, None, 0, None, dx, n)
    got = from_ours(dx.cpu().numpy().astype(np.float64), 16)
    assert np.max(np.abs(got - dx_ref)) <= 1e-5 * np.max(np.abs(dx_ref))
    dw = torch.zeros(27, 16, 16, device="cuda")
    db = torch.zeros(16, device="cuda")
    N.denser_conv3_wgrad(dev(to_ours(x), torch.bfloat16), dev(to_ours(dz), torch.bfloat16), dw, db, n)
    assert np.max(np.abs(dw.cpu().numpy() - w_ours(dW_ref))) <= 1e-5 * np.max(np.abs(dW_ref))
    assert np.max(np.abs(db.cpu().numpy() - db_ref)) <= 1e-5 * np.max(np.abs(db_ref))
    # gradients accumulate
    N.denser_conv3_wgrad(dev(to_ours(x), torch.bfloat16), dev(to_ours(dz), torch.bfloat16), dw, db, n)
    assert np.max(np.abs(dw.cpu().numpy() - 2 * w_ours(dW_ref))) <= 2e-5 * np.max(np.abs(dW_ref))


def test_relu_backward_and_loss():
    rng = np.random.default_rng(2)
    n = 2
    h = dev(bf16_round(rng.standard_normal((n, 1000, 16))), torch.bfloat16)
    dh = dev(bf16_round(rng.standard_normal((n, 1000, 16))), torch.bfloat16)
    dz = torch.empty_like(dh)
    N.denser_relu_backward(dh, h, dz, dh.numel())
    np.testing.assert_array_equal(dz.float().cpu().numpy(), np.where(h.float().cpu().numpy() > 0,
                                                                       dh.float().cpu().numpy(), 0))
    out = rng.standard_normal((n, 1000, 16)).astype(np.float32)
    tgt = rng.standard_normal((n, 4, 512)).astype(np.float32)
    mk = (rng.random((n, 4, 512)) < 0.6).astype(np.float32)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dout = torch.empty(n, 1000, 16, dtype=torch.bfloat16, device="cuda")
    N.denser_net_loss(dev(out), dev(tgt), dev(mk), dout, loss, n)
    o = from_ours(out.astype(np.float64), 4)[:, :, 1:-1, 1:-1, 1:-1]
    t = tgt.astype(np.float64).reshape(n, 4, 8, 8, 8)
    L, dref = NO.loss(o, t, mk.astype(np.float64).reshape(n, 4, 8, 8, 8))
    assert abs(loss.item() - L) <= 1e-6 * L
    full = np.zeros((n, 4, 10, 10, 10))
    full[:, :, 1:-1, 1:-1, 1:-1] = dref
    got = from_ours(dout.float().cpu().numpy().astype(np.float64), 4)
    assert np.max(np.abs(got - full)) <= 1e-2 * np.max(np.abs(full))


def test_network_against_fp64_oracle():
    rng = np.random.default_rng(3)
    n = 4
    params = NO.init_params(5)
    x = np.zeros((n, 2, 10, 10, 10))
    x[:, 0] = rng.uniform(-1, 1, (n, 10, 10, 10))
    x[:, 1] = rng.uniform(0, 0.8, (n, 10, 10, 10))
    x = bf16_round(x)
    tgt = rng.standard_normal((n, 4, 8, 8, 8)) * 0.5
    mk = (rng.random((n, 4, 8, 8, 8)) < 0.7).astype(float)
    out_ref, acts = NO.forward(params, x)
    _, dout = NO.loss(out_ref, tgt, mk)
    grads_ref = NO.backward(params, acts, dout)

    net = WS.WarmStartNet(seed=0)
    sd = {}
    for i, (W, b) in enumerate(params):
        sd[f"layer{i}"] = np.concatenate([w_ours(W).astype(np.float32).reshape(-1),
                                          np.pad(b, (0, 16 - b.size)).astype(np.float32)])
    net.load_state_dict(sd)
    out, gacts = net.forward(dev(to_ours(x), torch.bfloat16))
    got = from_ours(out.cpu().numpy().astype(np.float64), 4)[:, :, 1:-1, 1:-1, 1:-1]
    assert np.max(np.abs(got - out_ref)) <= 5e-2 * np.max(np.abs(out_ref))
    t_ours = dev(tgt.reshape(n, 4, 512))
    m_ours = dev(mk.reshape(n, 4, 512))
    loss, dout_g = net.loss_and_grad(out, t_ours, m_ours)
    grads = net.backward(gacts, dout_g)
    for li in range(4):
        dW_ref, db_ref = grads_ref[li]
        g = grads[li].cpu().numpy()
        dW = g[:27 * 256].reshape(27, 16, 16)
        rel = np.linalg.norm(dW - w_ours(dW_ref)) / np.linalg.norm(dW_ref)
        assert rel <= 5e-2, (li, rel)
        co = db_ref.size
        assert np.linalg.norm(g[27 * 256:][:co] - db_ref) <= 5e-2 * np.linalg.norm(db_ref) + 1e-9
        # padded channels carry no gradient, so their weights stay zero
        assert np.all(dW[:, co:, :] == 0) and np.all(g[27 * 256:][co:] == 0)


def test_training_lowers_loss():
    data = WS.make_training_set(seeds=[100], variants_per_seed=6, iters=400)
    x, t, m = data
    assert x.shape[0] > 1500
    net = WS.WarmStartNet(seed=1)
    hist = WS.train(net, data, epochs=4, batch=128, lr=2e-3)
    assert hist[-1] < 0.6 * hist[0], hist


def test_warm_start_gain_and_same_fixed_point():
    """What the trained network gains over the plain method on held-out scenes: fewer
    iterations (and less time, inference included) to a relative gap of 1e-4, towards the
    same solution."""
    data = WS.make_training_set(seeds=list(range(100, 112)), variants_per_seed=8, iters=4000)
    net = WS.WarmStartNet(seed=0)
    WS.train(net, data, epochs=12, batch=256, lr=2e-3)
    ev = WS.evaluate(net, range(200, 204))
    print("\nwarm start:", ev)
    assert ev["all_converged"]
    assert ev["iters_warm"] <= 0.97 * ev["iters_cold"], ev
    # both starts reach the same fixed point (up to the gap tolerance)
    sc = WS.scene_variant(201, 0)
    sols = []
    for use_net in (False, True):
        m = WS.solved_map([sc], 0)
        if use_net:
            net.warm_start(m.ctx)
        st = N.denser_regularize(m.ctx, 40000, 1e-6, 1 if use_net else 0)
        assert st.converged
        sols.append(m.snapshot())
        m.close()
    om = sols[0]["omega"].astype(bool)
    du = np.abs(sols[0]["u"] - sols[1]["u"])[om]
    assert du.mean() <= 1e-3 and du.max() <= 5e-2, (du.mean(), du.max())


def _oracle_params_of(npz):
    """The committed network's FP32 master weights in the oracle's layout
    W [co, ci, dz, dy, dx] (tap dx + 3 dy + 9 dz of [27][16 out][16 in]) and biases."""
    params = []
    for i, (cin, cout) in enumerate(zip(NO.CHANNELS[:-1], NO.CHANNELS[1:])):
        v = npz[f"layer{i}"].astype(np.float64)
        W = v[:27 * 256].reshape(3, 3, 3, 16, 16).transpose(3, 4, 0, 1, 2)[:cout, :cin]
        params.append((W, v[27 * 256:][:cout]))
    return params


@pytest.mark.parametrize("seed", [200, 201, 202])
def test_warm_started_path_against_oracle(seed):
    """The warm-started path (gather, network, warm start, then the plain iteration to a
    relative gap of 1e-4) against the oracle's warm-started path on a held-out scene: the
    oracle fuses the scene itself, runs the same trained network in FP64 with the stored
    BF16 weights, inputs and hidden activations, applies the warm start and iterates in
    FP64.  u on Omega within 5e-3 of the oracle right after the warm start, after 200
    iterations and at the iteration where the GPU reached the gap; div p is printed."""
    from oracle import denser_oracle as O
    from oracle import oracle_c as C
    from tests.oracle_helpers import grid_from_blocks
    from tests.pipelines import oracle_K
    net = WS.load_default()
    assert net is not None
    params = _oracle_params_of(dict(np.load(WS.WEIGHTS)))
    sc = WS.scene_variant(seed, 0)
    ref = C.run_pipeline(sc.depth_maps(), oracle_K(sc.camera), sc.poses, O.Params(), 0)
    rs = ref.snapshot()
    g = grid_from_blocks([tuple(c) for c in rs["coords"]], rs["f"], rs["w"])
    prob = O.PDProblem(g)
    om = prob.om.reshape(-1, 512)
    # the dual goes on every Eq. 3 edge (network trained on p) or on the block's inner edges
    # only (trained on div p), as the network's apply mode says
    edges = O.edge_mask(prob.om, prob.fwd).reshape(3, -1, 512)
    if net.dual_mode == 2:
        edges = edges & NO.inner_edges(om)
    out = NO.forward_stored(params, NO.gather(rs["coords"], rs["f"], rs["w"]))
    ref.set_state(*NO.warm_state(out, om, edges))

    m = WS.solved_map([sc], 0)
    net.warm_start(m.ctx)
    results = []

    def compare(label):
        got = m.snapshot(dual=True)
        want = ref.snapshot()
        np.testing.assert_array_equal(got["coords"], want["coords"].astype(np.int32))
        du = np.abs(got["u"].astype(np.float64) - want["u"])[om]
        dv = np.abs(prob.div(got["p"].reshape(3, -1).astype(np.float64)) - prob.div(want["p"].reshape(3, -1)))
        results.append((label, float(du.max()), float(du.mean()), float(dv[prob.om].max())))
        return float(du.max())

    e0 = compare("warm start")
    N.denser_regularize(m.ctx, 200, 0.0, 1)
    ref.iterate(200)
    e1 = compare("200 iterations")
    st = N.denser_regularize(m.ctx, 20000, 1e-4, 1)
    ref.iterate(st.iters)
    e2 = compare(f"gap 1e-4 ({200 + st.iters} iterations)")
    P, D = ref.energies()
    m.close()
    ref.close()
    print(f"\nseed {seed}: max|u - u_oracle| / mean / max|div p - div p_oracle|:", results,
          f"oracle rel gap {(P - D) / abs(P):.2e}")
    assert st.converged and (P - D) / abs(P) <= 1.5e-4
    assert max(e0, e1, e2) <= 5e-3, results


def test_divergence_loss_and_targets_against_oracle():
    """denser_net_loss_div (loss and BF16 gradient) and denser_net_targets_div (from a map's
    own state) against the FP64 definitions of oracle/net_oracle.py; apply mode 2 keeps p
    on the inner edges only."""
    rng = np.random.default_rng(30)
    n = 3
    om = rng.random((n, 512)) < 0.75
    tgt = NO.targets_div(rng.uniform(-1, 1, (n, 512)), rng.standard_normal((3, n, 512)) * 0.5, om)
    out4 = rng.standard_normal((n, 4, 512)) * 0.5
    L_ref, g_ref = NO.loss_div(out4, tgt, WS.U_WEIGHT, WS.DIV_WEIGHT)
    grid = np.zeros((n, 4, 10, 10, 10))
    grid[:, :, 1:-1, 1:-1, 1:-1] = out4.reshape(n, 4, 8, 8, 8)
    out = to_ours(grid)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dout = torch.empty(n, 1000, 16, dtype=torch.bfloat16, device="cuda")
    N.denser_net_loss_div(dev(out), dev(tgt), WS.U_WEIGHT, WS.DIV_WEIGHT, dout, loss, n)
    assert abs(loss.item() - L_ref) <= 1e-5 * L_ref
    got = from_ours(dout.float().cpu().numpy().astype(np.float64), 4)
    assert np.all(got[:, :, 0] == 0) and np.all(got[:, :, :, 0] == 0) and np.all(got[:, :, :, :, 9] == 0)
    g = got[:, :, 1:-1, 1:-1, 1:-1].reshape(n, 4, 512)
    assert np.max(np.abs(g - g_ref)) <= 1e-2 * np.max(np.abs(g_ref))
    # targets from a regularised map's own state
    from synth.scenes import tiny_scene
    s = tiny_scene(seed=0)
    d = s.depth_maps()
    cam = s.camera
    K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    with N.DenserMap() as m:
        for k in range(len(d)):
            N.denser_integrate(m.ctx, torch.from_numpy(np.ascontiguousarray(d[k])).cuda(), K, s.poses[k], 0)
        N.denser_regularize(m.ctx, 50)
        snap = m.snapshot(dual=True)
        nb = len(snap["coords"])
        t = torch.empty(nb, 6, 512, device="cuda")
        N.denser_net_targets_div(m.ctx, None, nb, t)
        want = NO.targets_div(snap["u"].astype(np.float64), snap["p"].astype(np.float64), snap["omega"].astype(bool))
        got_t = t.cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(got_t[:, [1, 3, 4, 5]], want[:, [1, 3, 4, 5]])
        assert np.max(np.abs(got_t[:, [0, 2]] - want[:, [0, 2]])) <= 1e-6
        # apply mode 2: p on the inner edges (projected), 0 on the edges crossing a block face
        outs = torch.from_numpy(rng.standard_normal((nb, 1000, 16)).astype(np.float32) * 0.3).cuda()
        N.denser_net_apply(m.ctx, None, nb, outs, 2)
        st = m.snapshot(dual=True)
    e_in = NO.inner_edges(snap["omega"].astype(bool))
    assert np.all(st["p"][~e_in] == 0)
    o = outs.cpu().numpy().reshape(nb, 10, 10, 10, 16)[:, 1:-1, 1:-1, 1:-1, 1:4].reshape(nb, 512, 3)
    q = np.where(e_in, o.transpose(2, 0, 1), 0.0)
    q = q / np.maximum(1.0, np.sqrt((q ** 2).sum(0)))[None]
    assert np.max(np.abs(st["p"] - q)) <= 1e-6
