"""Learned warm start for the primal-dual solver: network, training and use.

A 4-layer 3^3 convolutional network (2 -> 16 -> 16 -> 16 -> 4 channels) reads a fused
block with its one-voxel halo (f and w / (w + 8) on 10^3 voxels) and predicts the
block's converged (u, p_x, p_y, p_z).  Those predictions, masked to Omega and to the
edges of Eq. 3 and projected onto |p| <= 1, replace the zero start of Section III-C;
the plain primal-dual iteration then runs from there, so it stays the arbiter of the
result (same fixed point, same gap test).

Every product and update runs in the library's kernels (tensor-core BF16 convolutions
with FP32 accumulation, Adam in FP32); torch only holds the buffers.
"""

from __future__ import annotations

import math

import numpy as np

from . import native as N

C = 16          # channels as computed (inputs and outputs zero-padded to 16)
GV = 1000       # voxels of the 10^3 grid
CHANNELS = (2, 16, 16, 16, 4)


def _torch():
    import torch
    return torch


class WarmStartNet:
    """Parameters and training state of the network, on one CUDA device."""

    def __init__(self, seed: int = 0, device=None):
        torch = _torch()
        self.device = torch.device(device or "cuda")
        rng = np.random.default_rng(seed)
        self.w32, self.b32 = [], []
        for cin, cout in zip(CHANNELS[:-1], CHANNELS[1:]):
            w = np.zeros((27, C, C), np.float32)
            w[:, :cout, :cin] = rng.standard_normal((27, cout, cin)) * math.sqrt(2.0 / (27 * cin))
            self.w32.append(torch.tensor(w, device=self.device))
            self.b32.append(torch.zeros(C, device=self.device))
        self.step = 0
        self.m = [torch.zeros(27 * C * C + C, device=self.device) for _ in self.w32]
        self.v = [torch.zeros(27 * C * C + C, device=self.device) for _ in self.w32]
        self.params = [torch.cat([w.reshape(-1), b]) for w, b in zip(self.w32, self.b32)]
        # how a prediction's dual is applied (denser_net_apply): 1 on every Eq. 3 edge (the
        # network trained on p), 2 on the block's inner edges (trained on div p)
        self.dual_mode = 1
        self._views()
        self.pack()

    def _views(self):
        self.w32 = [p[:27 * C * C].view(27, C, C) for p in self.params]
        self.b32 = [p[27 * C * C:] for p in self.params]

    def pack(self):
        torch = _torch()
        self.wf = [torch.empty(27, C, C, dtype=torch.bfloat16, device=self.device) for _ in self.params]
        self.wb = [torch.empty(27, C, C, dtype=torch.bfloat16, device=self.device) for _ in self.params]
        for w, f, b in zip(self.w32, self.wf, self.wb):
            N.denser_pack_weights(w, f, b)

    # ------------------------------------------------------------ passes
    def forward(self, x):
        """x BF16 [n, 1000, 16] -> (out FP32 [n, 1000, 16], activations for backward)."""
        torch = _torch()
        n = x.shape[0]
        acts = [x]
        h = x
        out = torch.empty(n, GV, C, device=self.device)
        for li in range(4):
            last = li == 3
            y = None if last else torch.empty(n, GV, C, dtype=torch.bfloat16, device=self.device)
            N.denser_conv3(h, self.wf[li], self.b32[li], 0 if last else 1, y, out if last else None, n)
            if not last:
                acts.append(y)
                h = y
        return out, acts

    def backward(self, acts, dout):
        """Gradients (flat FP32 per layer, same layout as params) given dL/dout (BF16)."""
        torch = _torch()
        n = dout.shape[0]
        grads = [torch.zeros_like(p) for p in self.params]
        dz = dout
        for li in range(3, -1, -1):
            g = grads[li]
            N.denser_conv3_wgrad(acts[li], dz, g[:27 * C * C], g[27 * C * C:], n)
            if li > 0:
                dh = torch.empty(n, GV, C, dtype=torch.bfloat16, device=self.device)
                N.denser_conv3(dz, self.wb[li], None, 0, dh, None, n)
                dz = torch.empty_like(dh)
                N.denser_relu_backward(dh, acts[li], dz, dh.numel())
        return grads

    def loss_and_grad(self, out, target, mask):
        torch = _torch()
        n = out.shape[0]
        dout = torch.empty(n, GV, C, dtype=torch.bfloat16, device=self.device)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        N.denser_net_loss(out, target, mask, dout, loss, n)
        return loss, dout

    def loss_and_grad_div(self, out, target):
        """Divergence loss (denser_net_loss_div) for targets [n, 6, 512]."""
        torch = _torch()
        n = out.shape[0]
        dout = torch.empty(n, GV, C, dtype=torch.bfloat16, device=self.device)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        N.denser_net_loss_div(out, target, U_WEIGHT, DIV_WEIGHT, dout, loss, n)
        return loss, dout

    def train_step(self, x, target, mask, lr=1e-3):
        out, acts = self.forward(x)
        if mask is None:
            loss, dout = self.loss_and_grad_div(out, target)
        else:
            loss, dout = self.loss_and_grad(out, target, mask)
        grads = self.backward(acts, dout)
        self.step += 1
        for p, g, m, v in zip(self.params, grads, self.m, self.v):
            N.denser_adam(p, g, m, v, p.numel(), lr, 0.9, 0.999, 1e-8, self.step)
        for w, f, b in zip(self.w32, self.wf, self.wb):
            N.denser_pack_weights(w, f, b)
        return loss

    # -------------------------------------------------------- save / load
    def state_dict(self):
        sd = {f"layer{i}": p.detach().cpu().numpy() for i, p in enumerate(self.params)}
        sd["dual_mode"] = np.array(self.dual_mode, dtype=np.int32)
        return sd

    def load_state_dict(self, sd):
        torch = _torch()
        for i in range(4):
            self.params[i].copy_(torch.as_tensor(sd[f"layer{i}"], device=self.device))
        self.dual_mode = int(sd["dual_mode"]) if "dual_mode" in sd else 1
        self._views()
        self.pack()

    # ----------------------------------------------------------- use
    def warm_start(self, ctx, chunk: int = 4096, stream=None, dual: bool = True):
        """Writes the network's prediction into every block of the map (p = 0 when
        ``dual`` is False); follow with denser_regularize(..., start=1)."""
        torch = _torch()
        nb = N.denser_num_blocks(ctx, stream)
        for first in range(0, nb, chunk):
            n = min(chunk, nb - first)
            blocks = torch.arange(first, first + n, dtype=torch.int32, device=self.device)
            x = torch.empty(n, GV, C, dtype=torch.bfloat16, device=self.device)
            N.denser_net_gather(ctx, blocks, n, x, stream)
            out, _ = self.forward(x)
            N.denser_net_apply(ctx, blocks, n, out, self.dual_mode if dual else 0, stream)


# ------------------------------------------------------------ training data
def scene_variant(seed: int, variant: int):
    """A tiny-workload scene with randomised wall distance, cube position, pose jitter
    and frame count (drawn from the seed and the variant number)."""
    from synth.scenes import tiny_scene
    rng = np.random.default_rng([seed, variant, 3])
    return tiny_scene(seed=seed * 1000 + variant, n_frames=int(rng.integers(2, 6)),
                      yaw_jitter=float(rng.uniform(0.0, 0.12)), wall_z=float(rng.uniform(9.0, 16.0)),
                      cube_at=(float(rng.uniform(-4.0, 3.0)), float(rng.uniform(5.0, 8.5))))


def solved_map(scenes, iters: int, gap_tol: float = 0.0, **params):
    """One map holding every scene as its own segment (at most 127), fused and solved."""
    m = N.DenserMap(max_blocks=max(4096, 700 * len(scenes)), gap_every=10, **params)
    for seg, s in enumerate(scenes):
        cam = s.camera
        K = N.intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
        for k, d in enumerate(s.depth_maps()):
            N.denser_alloc_blocks(m.ctx, d, K, s.poses[k], seg)
            N.denser_fuse_depth(m.ctx, d, K, s.poses[k], seg)
    if iters > 0:
        N.denser_regularize(m.ctx, iters, gap_tol, 0)
    return m


# Loss weights of u and p: the squared distance in the metric of the Chambolle-Pock
# analysis, |u - u*|^2 / tau + |p - p*|^2 / sigma (tau = 1/6, sigma = 0.5).  The
# divergence loss weighs (div p - div p*)^2 by DIV_WEIGHT instead of the p term: p* is
# unique only up to a divergence-free part, which a regression on p cannot predict.
U_WEIGHT, P_WEIGHT = 6.0, 2.0
DIV_WEIGHT = 2.0


def make_training_set(seeds, variants_per_seed: int, iters: int = 8000, gap_tol: float = 1e-7, per_map: int = 64,
                      div: bool = False):
    """(x BF16 [n, 1000, 16], target, mask) from the plain solver on scene variants of the
    given seeds.  p loss: target FP32 [n, 4, 512] and mask FP32 [n, 4, 512] carrying the
    loss weights; divergence loss (div): target FP32 [n, 6, 512] of denser_net_targets_div
    and mask None."""
    torch = _torch()
    xs, ts, ms = [], [], []
    jobs = [(s, v) for s in seeds for v in range(variants_per_seed)]
    for i in range(0, len(jobs), per_map):
        scenes = [scene_variant(s, v) for s, v in jobs[i:i + per_map]]
        m = solved_map(scenes, iters, gap_tol)
        nb = N.denser_num_blocks(m.ctx)
        blocks = torch.arange(nb, dtype=torch.int32, device="cuda")
        x = torch.empty(nb, GV, C, dtype=torch.bfloat16, device="cuda")
        N.denser_net_gather(m.ctx, blocks, nb, x)
        if div:
            t = torch.empty(nb, 6, 512, device="cuda")
            N.denser_net_targets_div(m.ctx, blocks, nb, t)
            mk = None
        else:
            t = torch.empty(nb, 4, 512, device="cuda")
            mk = torch.empty(nb, 4, 512, device="cuda")
            N.denser_net_targets(m.ctx, blocks, nb, t, mk, U_WEIGHT, P_WEIGHT)
        xs.append(x), ts.append(t), ms.append(mk)
        m.close()
    return torch.cat(xs), torch.cat(ts), (None if div else torch.cat(ms))


def train(net: WarmStartNet, data, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0, log=None):
    torch = _torch()
    x, t, mk = data
    n = x.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    history = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(x.device)
        tot = torch.zeros(1, dtype=torch.float64, device=x.device)
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            tot += net.train_step(x[idx].contiguous(), t[idx].contiguous(),
                                  None if mk is None else mk[idx].contiguous(), lr) * batch
        history.append(float(tot.item()) / max(1, (n // batch) * batch))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.5f}")
    return history


def time_to_gap(scene, net: WarmStartNet | None, gap_tol: float = 1e-4, max_iters: int = 20000, dual: bool = True):
    """Device time (ms, CUDA events) and iterations to reach gap_tol from a cold start or
    from the network's warm start (inference included)."""
    torch = _torch()
    m = solved_map([scene], 0)
    N.denser_regularize(m.ctx, 10, 0.0, 0)  # records the graph loop shape, builds tables
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    if net is not None:
        net.warm_start(m.ctx, dual=dual)
        st = N.denser_regularize(m.ctx, max_iters, gap_tol, 1)
    else:
        st = N.denser_regularize(m.ctx, max_iters, gap_tol, 0)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m.close()
    return ms, st.iters, st.rel_gap, st.converged


def evaluate(net: WarmStartNet, seeds, gap_tol: float = 1e-4):
    """Mean time (ms, inference included) and iterations to gap_tol on held-out scenes,
    cold start against warm start."""
    rows = []
    seeds = list(seeds)
    # one untimed cold and warm solve first: the first inference of a process loads the
    # network's kernels and the framework's allocator state (tens of milliseconds)
    if seeds:
        time_to_gap(scene_variant(seeds[0], 0), None, gap_tol)
        time_to_gap(scene_variant(seeds[0], 0), net, gap_tol)
    for seed in seeds:
        sc = scene_variant(seed, 0)
        cold = time_to_gap(sc, None, gap_tol)
        warm = time_to_gap(sc, net, gap_tol)
        rows.append((cold, warm))
    out = {"scenes": len(rows), "gap_tol": gap_tol,
           "ms_cold": float(np.mean([r[0][0] for r in rows])), "ms_warm": float(np.mean([r[1][0] for r in rows])),
           "iters_cold": float(np.mean([r[0][1] for r in rows])), "iters_warm": float(np.mean([r[1][1] for r in rows])),
           "all_converged": all(r[0][3] and r[1][3] for r in rows)}
    out["speedup_time"] = out["ms_cold"] / out["ms_warm"]
    out["speedup_iters"] = out["iters_cold"] / out["iters_warm"]
    return out


WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__file__), "weights", "warmstart.npz")


def load_default(device=None):
    """The network trained by ``main`` on seeds 100-199 (8 variants each), or None."""
    import os
    if not os.path.exists(WEIGHTS):
        return None
    net = WarmStartNet(seed=0, device=device)
    net.load_state_dict(dict(np.load(WEIGHTS)))
    return net


def main(argv=None):
    """python -m paper_1604_03734_gb300.warmstart OUT.npz [--seeds 100:200] [--variants 4]
    [--epochs 30] [--loss div|p]: trains the network on scene variants of the given seeds
    and saves it."""
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("out")
    ap.add_argument("--seeds", default="100:200")
    ap.add_argument("--variants", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--eval-seeds", default="200:220")
    ap.add_argument("--loss", default="div", choices=["div", "p"],
                    help="div: u and the inner divergence of p (applied on inner edges); p: u and p")
    ap.add_argument("--iters", type=int, default=8000, help="iterations of the plain solves that make the targets")
    args = ap.parse_args(argv)
    a, b = (int(v) for v in args.seeds.split(":"))
    data = make_training_set(list(range(a, b)), args.variants, iters=args.iters, div=args.loss == "div")
    net = WarmStartNet(seed=0)
    net.dual_mode = 2 if args.loss == "div" else 1
    n_ep = args.epochs
    for ep in range(n_ep):
        lr = 2e-3 if ep < 0.4 * n_ep else (1e-3 if ep < 0.75 * n_ep else 3e-4)
        loss = train(net, data, epochs=1, lr=lr, seed=ep)[0]
        print(f"epoch {ep}: lr {lr:g} loss {loss:.4f}", flush=True)
    np.savez(args.out, **net.state_dict())
    a, b = (int(v) for v in args.eval_seeds.split(":"))
    import json
    print(json.dumps({"samples": int(data[0].shape[0]), **evaluate(net, range(a, b))}))


if __name__ == "__main__":
    main()
