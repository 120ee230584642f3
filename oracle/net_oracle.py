"""CPU FP64 oracle of the warm-start network -- TEST INFRASTRUCTURE ONLY.

The network maps one fused block with its one-voxel halo (10^3 voxels, channels
f and a normalised weight) to a starting point for the primal-dual iteration of
Section III-C on the block's 8^3 voxels (channels u, p_x, p_y, p_z): four 3^3
convolutions with zero ("same") padding over the 10^3 grid, ReLU after the first
three, the centre 8^3 of the last one as the output.  The paper has no such
network; it only fixes what the output is used for (u, p of Section III-C).

Only tests/ and bench.py's reference leg may import this module.  It shares no
code with the CUDA path.  Layout here: x [n, C, 10, 10, 10] (z, y, x order) and
W [Cout, Cin, 3, 3, 3] (dz, dy, dx), cross-correlation as in every deep-learning
framework:  y[co, z, y, x] = b[co] + sum W[co, ci, dz, dy, dx] x[ci, z+dz-1, y+dy-1, x+dx-1].
"""

from __future__ import annotations

import numpy as np

CHANNELS = (2, 16, 16, 16, 4)
GRID = 10


def conv3d_same(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Zero-padded 3^3 cross-correlation, summed tap by tap."""
    n, ci, D, H, Wd = x.shape
    xp = np.zeros((n, ci, D + 2, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((n, W.shape[0], D, H, Wd)) + b[None, :, None, None, None]
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, :, dz:dz + D, dy:dy + H, dx:dx + Wd]
                y += np.einsum("oc,nczyx->nozyx", W[:, :, dz, dy, dx], patch)
    return y


def conv3d_same_backward(x, W, dy):
    """Gradients of conv3d_same with respect to x, W and b, given dL/dy."""
    n, ci, D, H, Wd = x.shape
    xp = np.zeros((n, ci, D + 2, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for dz in range(3):
        for dy_ in range(3):
            for dx in range(3):
                patch = xp[:, :, dz:dz + D, dy_:dy_ + H, dx:dx + Wd]
                dW[:, :, dz, dy_, dx] = np.einsum("nozyx,nczyx->oc", dy, patch)
                dxp[:, :, dz:dz + D, dy_:dy_ + H, dx:dx + Wd] += np.einsum("oc,nozyx->nczyx", W[:, :, dz, dy_, dx], dy)
    db = dy.sum(axis=(0, 2, 3, 4))
    return dxp[:, :, 1:-1, 1:-1, 1:-1], dW, db


def init_params(seed: int = 0):
    """He-style initial weights, zero biases; layer l maps CHANNELS[l] -> CHANNELS[l+1]."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(CHANNELS[:-1], CHANNELS[1:]):
        W = rng.standard_normal((cout, cin, 3, 3, 3)) * np.sqrt(2.0 / (27 * cin))
        params.append((W, np.zeros(cout)))
    return params


def forward(params, x):
    """Returns (output [n, 4, 8, 8, 8], activations for backward)."""
    acts = [x]
    h = x
    for li, (W, b) in enumerate(params):
        z = conv3d_same(h, W, b)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    return h[:, :, 1:-1, 1:-1, 1:-1], acts


def loss(out, target, mask):
    """Mean over samples of the masked squared error: sum mask (out - target)^2 / n."""
    d = (out - target) * mask
    return float(np.sum(d * d) / out.shape[0]), 2.0 * d * mask / out.shape[0]


def backward(params, acts, dout):
    """Gradients [(dW, db)] of the network given dL/d(output) on the centre 8^3."""
    n = dout.shape[0]
    dh = np.zeros((n, CHANNELS[-1], GRID, GRID, GRID))
    dh[:, :, 1:-1, 1:-1, 1:-1] = dout
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        if li < len(params) - 1:
            dh = dh * (acts[li + 1] > 0)        # through the ReLU
        dx, dW, db = conv3d_same_backward(acts[li], W, dh)
        grads[li] = (dW, db)
        dh = dx
    return grads


# ------------------------------------------------- the warm start on a map
def bf16(x) -> np.ndarray:
    """Nearest BF16 value (8 significant bits, ties to even) of float64 x: the storage
    type of the network's weights, inputs and hidden activations."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def gather(keys, f, w, blocks=None) -> np.ndarray:
    """Network inputs of the listed blocks (default: all), [n, 2, 10, 10, 10] (z, y, x):
    channel 0 = f where w > 0, channel 1 = w / (w + 8), on the block and its one-voxel
    halo taken from the 26 neighbouring blocks of the same segment, 0 where a block is
    absent; both rounded to BF16.  keys: (segment, bx, by, bz) per block index; f, w
    [nb, 512] with voxel l = lx + 8 ly + 64 lz."""
    index = {tuple(int(v) for v in k): i for i, k in enumerate(keys)}
    blocks = range(len(keys)) if blocks is None else blocks
    out = np.zeros((len(blocks), 2, GRID, GRID, GRID))
    f3 = np.asarray(f, dtype=np.float64).reshape(-1, 8, 8, 8)   # [b, lz, ly, lx]
    w3 = np.asarray(w, dtype=np.float64).reshape(-1, 8, 8, 8)
    for s, b in enumerate(blocks):
        seg, bx, by, bz = (int(v) for v in keys[b])
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    nb = index.get((seg, bx + ox, by + oy, bz + oz))
                    if nb is None:
                        continue
                    # grid coordinate g = 1 + local + 8 * offset, kept where 0 <= g < 10
                    zs = [(1 + l + 8 * oz, l) for l in range(8) if 0 <= 1 + l + 8 * oz < GRID]
                    ys = [(1 + l + 8 * oy, l) for l in range(8) if 0 <= 1 + l + 8 * oy < GRID]
                    xs = [(1 + l + 8 * ox, l) for l in range(8) if 0 <= 1 + l + 8 * ox < GRID]
                    gz, lz = zip(*zs)
                    gy, ly = zip(*ys)
                    gx, lx = zip(*xs)
                    ix = np.ix_(lz, ly, lx)
                    wv = w3[nb][ix]
                    out[s, 0][np.ix_(gz, gy, gx)] = np.where(wv > 0, f3[nb][ix], 0.0)
                    out[s, 1][np.ix_(gz, gy, gx)] = wv / (wv + 8.0)
    return bf16(out)


def forward_stored(params, x):
    """The network as stored: BF16 weights and inputs, float64 sums, each hidden
    activation (after its ReLU) rounded to BF16; the last layer's output unrounded.
    Returns the centre 8^3 of the output, [n, 4, 8, 8, 8]."""
    h = bf16(x)
    for li, (W, b) in enumerate(params):
        z = conv3d_same(h, bf16(W), np.asarray(b, dtype=np.float64))
        h = bf16(np.maximum(z, 0.0)) if li < len(params) - 1 else z
    return h[:, :, 1:-1, 1:-1, 1:-1]


def warm_state(out, omega, edges):
    """The starting point a prediction gives the iteration of Section III-C: u = the
    prediction clamped to [-1, 1] on Omega and 0 elsewhere, u_bar = u, p_a = the
    prediction on the Eq. 3 edges along axis a and 0 elsewhere, then projected onto the
    unit ball (the constraint |p| <= 1 of the dual).  out [n, 4, 8, 8, 8] (z, y, x);
    omega [n, 512] and edges [3, n, 512] boolean, voxel l = lx + 8 ly + 64 lz.  Returns
    (u [n, 512], u_bar, p [3, n, 512])."""
    n = out.shape[0]
    o = np.asarray(out, dtype=np.float64).reshape(n, 4, 512)
    u = np.where(omega, np.clip(o[:, 0], -1.0, 1.0), 0.0)
    p = np.where(edges, o[:, 1:].transpose(1, 0, 2), 0.0)
    nrm = np.sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2])
    p = p / np.maximum(1.0, nrm)[None]
    return u, u.copy(), p


# ------------------------------------------- the divergence-trained warm start
def inner_edges(omega):
    """Inner Eq. 3 edge masks of each block, [3, n, 512]: voxel l and l + a both in Omega
    and l + a inside the same block (l_a < 7)."""
    om = np.asarray(omega, dtype=bool).reshape(-1, 8, 8, 8)       # [b, lz, ly, lx]
    e = np.zeros((3,) + om.shape, dtype=bool)
    e[0][..., :-1] = om[..., :-1] & om[..., 1:]
    e[1][:, :, :-1, :] = om[:, :, :-1, :] & om[:, :, 1:, :]
    e[2][:, :-1] = om[:, :-1] & om[:, 1:]
    return e.reshape(3, -1, 512)


def inner_divergence(p, edges):
    """Divergence of p [3, n, 512] over the inner edges only (Eq. 4, the negative adjoint of
    the masked forward difference, with the edges that cross a block face left out)."""
    d = np.zeros(p.shape[1:])
    q = np.where(edges, p, 0.0).reshape(3, -1, 8, 8, 8)
    out = np.zeros(q.shape[1:])
    for a, ax in enumerate((3, 2, 1)):             # x, y, z axes of [b, lz, ly, lx]
        back = np.zeros_like(q[a])
        sl_dst = [slice(None)] * 4
        sl_src = [slice(None)] * 4
        sl_dst[ax], sl_src[ax] = slice(1, None), slice(None, -1)
        back[tuple(sl_dst)] = q[a][tuple(sl_src)]
        out = out + (q[a] - back)
    d[:] = out.reshape(d.shape)
    return d


def targets_div(u, p, omega):
    """[n, 6, 512]: u on Omega, Omega, the inner divergence of p on Omega, the inner edges."""
    om = np.asarray(omega, dtype=bool).reshape(-1, 512)
    e = inner_edges(om)
    t = np.zeros((om.shape[0], 6, 512))
    t[:, 0] = np.where(om, np.asarray(u).reshape(-1, 512), 0.0)
    t[:, 1] = om
    t[:, 2] = np.where(om, inner_divergence(np.asarray(p).reshape(3, -1, 512), e), 0.0)
    t[:, 3:6] = e.transpose(1, 0, 2)
    return t


def loss_div(out, target, wu, wd):
    """Mean over samples of sum_Omega [wu (u - u*)^2 + wd (div p - div p*)^2] for outputs
    out [n, 4, 512] (u, p_x, p_y, p_z on the block) and targets [n, 6, 512]; returns (loss,
    d loss / d out [n, 4, 512])."""
    n = out.shape[0]
    om = target[:, 1] != 0
    e = (target[:, 3:6] != 0).transpose(1, 0, 2)
    ru = np.where(om, out[:, 0] - target[:, 0], 0.0)
    dv = inner_divergence(out[:, 1:4].transpose(1, 0, 2), e)
    rd = np.where(om, dv - target[:, 2], 0.0)
    loss = float(np.sum(wu * ru * ru + wd * rd * rd) / n)
    g = np.zeros_like(out)
    g[:, 0] = 2.0 * wu * ru / n
    # d div / d p_a(l) = +1 at l and -1 at l + a (for an inner edge): the gradient is the
    # negative inner forward difference of the residual, masked to the edges
    r3 = rd.reshape(-1, 8, 8, 8)
    for a, ax in enumerate((3, 2, 1)):
        nxt = np.zeros_like(r3)
        sl_dst = [slice(None)] * 4
        sl_src = [slice(None)] * 4
        sl_dst[ax], sl_src[ax] = slice(None, -1), slice(1, None)
        nxt[tuple(sl_dst)] = r3[tuple(sl_src)]
        g[:, 1 + a] = np.where(e[a], 2.0 * wd * (rd - nxt.reshape(-1, 512)) / n, 0.0)
    return loss, g
