"""Pins of the warm-start network's oracle: the convolution against a library
correlation, and every gradient against central finite differences (rel 1e-6)."""

import numpy as np
import pytest

from oracle import net_oracle as NO


def test_conv_matches_library_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 6, 5, 7))
    W = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = NO.conv3d_same(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(ndimage.correlate(x[n, c], W[o, c], mode="constant", cval=0.0) for c in range(3))
            np.testing.assert_allclose(y[n, o], ref, rtol=0, atol=1e-12)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 2, 4, 5, 4))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    g = rng.standard_normal((2, 3, 4, 5, 4))
    dx, dW, db = NO.conv3d_same_backward(x, W, g)
    L = lambda x_, W_, b_: float(np.sum(NO.conv3d_same(x_, W_, b_) * g))
    h = 1e-6
    for arr, grad in ((x, dx), (W, dW), (b, db)):
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]:
            old = arr[idx]
            arr[idx] = old + h
            lp = L(x, W, b)
            arr[idx] = old - h
            lm = L(x, W, b)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_network_gradients_finite_differences():
    rng = np.random.default_rng(2)
    params = NO.init_params(3)
    x = rng.standard_normal((2, 2, 10, 10, 10))
    target = rng.standard_normal((2, 4, 8, 8, 8))
    mask = (rng.random((2, 4, 8, 8, 8)) < 0.7).astype(float)
    out, acts = NO.forward(params, x)
    _, dout = NO.loss(out, target, mask)
    grads = NO.backward(params, acts, dout)

    def total():
        o, _ = NO.forward(params, x)
        return NO.loss(o, target, mask)[0]
    h = 1e-6
    for li in (0, 3):
        W, b = params[li]
        dW, db = grads[li]
        for idx in [tuple(rng.integers(0, s) for s in W.shape) for _ in range(6)]:
            old = W[idx]
            W[idx] = old + h
            lp = total()
            W[idx] = old - h
            lm = total()
            W[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dW[idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, dW[idx])
        j = int(rng.integers(0, b.shape[0]))
        old = b[j]
        b[j] = old + h
        lp = total()
        b[j] = old - h
        lm = total()
        b[j] = old
        assert abs((lp - lm) / (2 * h) - db[j]) <= 1e-6 * max(1.0, abs(db[j]))


def test_output_is_centre_and_padding_is_zero():
    params = NO.init_params(4)
    x = np.zeros((1, 2, 10, 10, 10))
    out, acts = NO.forward(params, x)
    assert out.shape == (1, 4, 8, 8, 8)
    # zero input: every activation is the bias chain, constant over the grid
    for a in acts[1:]:
        assert np.allclose(a, a[:, :, :1, :1, :1])


# ------------------------------------------------- warm start on a map
def test_bf16_is_nearest_with_ties_to_even():
    """Against the definition: every BF16 value is a float32 whose low 16 bits are zero;
    the nearest one is chosen, ties to the one with an even last bit."""
    rng = np.random.default_rng(20)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-8, 8, 2000),
                        # exact halfway points between neighbouring BF16 values
                        (np.arange(256, 512) + 0.5) / 256.0, -(np.arange(256, 512) + 0.5) / 128.0])
    got = NO.bf16(x)
    for xi, gi in zip(x, got):
        b = int(np.array([xi], np.float32).view(np.uint32)[0]) & 0xFFFF0000
        cands = [np.array([b + k * 65536], np.uint32).view(np.float32)[0].astype(np.float64)
                 for k in (-1, 0, 1) if 0 <= b + k * 65536 < 2 ** 32]
        dist = [abs(c - xi) for c in cands]
        best = min(dist)
        near = [c for c, d in zip(cands, dist) if d == best]
        if len(near) == 2:   # a tie: the even one
            near = [c for c in near if (np.array([c], np.float32).view(np.uint32)[0] >> 16) % 2 == 0]
        assert gi == near[0], (xi, gi, near)


def test_gather_against_voxel_lookup():
    """Every cell of the 10^3 grid equals the voxel at that global position, found by its
    block key (floor division of the global voxel index by 8), or 0 where absent."""
    rng = np.random.default_rng(21)
    keys = [(0, 0, 0, 0), (0, 1, 0, 0), (0, 0, -1, 0), (0, 1, 1, 1), (0, -1, -1, -1), (2, 0, 0, 1), (0, 0, 0, 1)]
    f = rng.uniform(-1, 1, (len(keys), 512))
    w = rng.integers(0, 6, (len(keys), 512)).astype(float)
    x = NO.gather(keys, f, w)
    index = {k: i for i, k in enumerate(keys)}
    for s, (seg, bx, by, bz) in enumerate(keys):
        for gz in range(10):
            for gy in range(10):
                for gx in range(10):
                    i, j, k = 8 * bx + gx - 1, 8 * by + gy - 1, 8 * bz + gz - 1
                    b = index.get((seg, i // 8, j // 8, k // 8))
                    if b is None:
                        want = (0.0, 0.0)
                    else:
                        l = i % 8 + 8 * (j % 8) + 64 * (k % 8)
                        want = (f[b, l] if w[b, l] > 0 else 0.0, w[b, l] / (w[b, l] + 8.0))
                    assert x[s, 0, gz, gy, gx] == NO.bf16(want[0]) and x[s, 1, gz, gy, gx] == NO.bf16(want[1])


def test_forward_stored_wiring_and_rounding():
    """With weights that keep every activation exactly representable (one power-of-two
    centre tap per channel) the stored network equals the exact one; with random weights
    every hidden activation it produces is a BF16 value and the output stays within the
    rounding's reach of the exact network."""
    n = 2
    rng = np.random.default_rng(22)
    x = NO.bf16(rng.uniform(-1, 1, (n, 2, 10, 10, 10)))
    params = []
    for cin, cout in zip(NO.CHANNELS[:-1], NO.CHANNELS[1:]):
        W = np.zeros((cout, cin, 3, 3, 3))
        for co in range(cout):
            W[co, co % cin, 1, 1, 1] = 2.0 ** -(co % 3)
        params.append((W, np.zeros(cout)))
    exact, _ = NO.forward(params, x)
    np.testing.assert_array_equal(NO.forward_stored(params, x), exact)
    params = NO.init_params(3)
    got = NO.forward_stored(params, x)
    ref, acts = NO.forward([(NO.bf16(W), b) for W, b in params], x)
    assert np.max(np.abs(got - ref)) <= 0.05 * np.max(np.abs(ref))
    h = NO.bf16(x)
    for W, b in params[:-1]:
        h = NO.bf16(np.maximum(NO.conv3d_same(h, NO.bf16(W), b), 0.0))
        assert np.array_equal(h, NO.bf16(h))



def test_forward_stored_rounding_closed_forms():
    """Centre taps only, so every voxel runs the chain on its own value x; worked out by
    hand: a last-layer weight 1 + 2^-9 is stored as 1 (2^-9 is below half an ulp of BF16
    at 1, 2^-8), so x = 1 gives 1; an activation (1 + 2^-7)^2 = 1 + 2^-6 + 2^-14 is stored
    as 1 + 2^-6; the last layer's output keeps every bit."""

    def chain(w_first, w_last):
        params = []
        for li, (cin, cout) in enumerate(zip(NO.CHANNELS[:-1], NO.CHANNELS[1:])):
            W = np.zeros((cout, cin, 3, 3, 3))
            W[0, 0, 1, 1, 1] = w_first if li == 0 else (w_last if li == len(NO.CHANNELS) - 2 else 1.0)
            params.append((W, np.zeros(cout)))
        return params

    def run(params, x):
        xin = np.zeros((1, 2, 10, 10, 10))
        xin[:, 0] = x
        return NO.forward_stored(params, xin)[0, 0]

    a = 1.0 + 2.0 ** -7
    assert np.all(run(chain(1.0, 1.0 + 2.0 ** -9), 1.0) == 1.0)                 # weight rounded
    assert np.all(run(chain(a, 1.0), a) == 1.0 + 2.0 ** -6)                     # activation rounded
    assert np.all(run(chain(1.0, a), a) == 1.0 + 2.0 ** -6 + 2.0 ** -14)        # output kept

def test_warm_state_masks_and_projection():
    rng = np.random.default_rng(23)
    n = 3
    out = rng.standard_normal((n, 4, 8, 8, 8)) * 1.5
    om = rng.random((n, 512)) < 0.7
    edges = (rng.random((3, n, 512)) < 0.6) & om[None]
    u, ub, p = NO.warm_state(out, om, edges)
    o = out.reshape(n, 4, 512)
    assert np.all(u[~om] == 0) and np.array_equal(u[om], np.clip(o[:, 0][om], -1, 1)) and np.array_equal(u, ub)
    assert np.all(p[~edges] == 0)
    nrm = np.sqrt((p ** 2).sum(0))
    assert np.all(nrm <= 1 + 1e-15)
    q = np.where(edges, o[:, 1:].transpose(1, 0, 2), 0.0)
    qn = np.sqrt((q ** 2).sum(0))
    inside = qn <= 1
    assert np.array_equal(p[:, inside], q[:, inside])
    np.testing.assert_allclose(p[:, ~inside] * qn[~inside], q[:, ~inside], rtol=1e-15, atol=1e-15)


def test_inner_divergence_brute_force_and_adjoint():
    """The inner divergence against a per-voxel loop of its definition, and against the
    inner forward difference through the adjoint identity <grad u, p> = -<u, div p>."""
    rng = np.random.default_rng(24)
    n = 3
    om = rng.random((n, 512)) < 0.7
    e = NO.inner_edges(om)
    p = rng.standard_normal((3, n, 512))
    d = NO.inner_divergence(p, e)
    for b in range(n):
        for l in range(512):
            lc = (l % 8, (l // 8) % 8, l // 64)
            want = 0.0
            for a, st in enumerate((1, 8, 64)):
                if lc[a] < 7 and om[b, l] and om[b, l + st]:
                    want += p[a, b, l]
                if lc[a] > 0 and om[b, l - st] and om[b, l]:
                    want -= p[a, b, l - st]
            assert abs(d[b, l] - want) < 1e-12
    u = rng.standard_normal((n, 512))
    g = np.zeros((3, n, 512))
    for a, st in enumerate((1, 8, 64)):
        nxt = np.zeros_like(u)
        idx = np.arange(512)
        ok = (np.array([(l % 8, (l // 8) % 8, l // 64)[a] for l in idx]) < 7)
        nxt[:, ok] = u[:, idx[ok] + st]
        g[a] = np.where(e[a], nxt - u, 0.0)
    assert abs(np.sum(g * p) + np.sum(u * d)) < 1e-10


def test_loss_div_gradient_by_finite_differences():
    rng = np.random.default_rng(25)
    n = 2
    om = rng.random((n, 512)) < 0.75
    tgt = NO.targets_div(rng.uniform(-1, 1, (n, 512)), rng.standard_normal((3, n, 512)) * 0.5, om)
    out = rng.standard_normal((n, 4, 512)) * 0.5
    L, g = NO.loss_div(out, tgt, 6.0, 2.0)
    for _ in range(40):
        i, c, l = rng.integers(n), rng.integers(4), rng.integers(512)
        h = 1e-6
        o1, o2 = out.copy(), out.copy()
        o1[i, c, l] += h
        o2[i, c, l] -= h
        fd = (NO.loss_div(o1, tgt, 6.0, 2.0)[0] - NO.loss_div(o2, tgt, 6.0, 2.0)[0]) / (2 * h)
        assert abs(fd - g[i, c, l]) <= 1e-6 * max(1.0, abs(fd)), (i, c, l, fd, g[i, c, l])
    # only Omega counts: outputs and targets off Omega change neither the loss nor the
    # gradient, which is zero there for u
    o3, t3 = out.copy(), tgt.copy()
    o3[:, 0][~om] += rng.standard_normal((~om).sum())
    t3[:, 0][~om] += 1.0
    L3, g3 = NO.loss_div(o3, t3, 6.0, 2.0)
    assert L3 == L and np.array_equal(g3, g) and np.all(g[:, 0][~om] == 0)
    # targets of the exact state give zero loss
    u, p = rng.uniform(-1, 1, (n, 512)), rng.standard_normal((3, n, 512))
    t = NO.targets_div(u, p, om)
    exact = np.concatenate([np.where(om, u, 0)[:, None], p.transpose(1, 0, 2)], axis=1)
    assert NO.loss_div(exact, t, 6.0, 2.0)[0] < 1e-20
