"""CPU oracle of stereo depth-map estimation -- TEST INFRASTRUCTURE ONLY.

Section IV estimates each depth map by minimising a data term built on the Census
Transform Signature plus an affine (TGV) regulariser whose gradient is shaped by an
image-driven diffusion tensor (Section IV-A to IV-C; lambda, alpha1, alpha2, beta,
gamma from Table I).  The paper follows a cited variational method and fixes no
window size, disparity range, optimiser schedule or boundary rule; the readings
taken here:

  D1  rectified pair, intensities in [0, 1]; the reference image is I_R and
      rho(d, x, y) compares I_L(x + d, y) with I_R(x, y) (Section IV-A), so the
      disparity lives on I_R's grid, d >= 0, depth z = f B / d;
  D2  Census window 9 x 7 (width x height): a 62-bit signature, bit b (row-major over
      the window, the centre skipped) set when that neighbour is darker than the
      centre; pixels beyond the image repeat the edge.  (A 5 x 5 window, 24 bits, left
      a third of the street pair's pixels more than 3 px off after regularisation:
      too few bits to tell 256 candidate disparities apart);
  D3  data cost C(x, y, delta) = Hamming(sig_L(x + delta, y), sig_R(x, y)) / 62 for
      integer delta in [0, D); 1 where x + delta falls off the image;
  D4  T = exp(-gamma |grad I|^beta) n n^T + n_perp n_perp^T with n = grad I / |grad I|
      (= I + (e - 1) n n^T), the identity where grad I = 0; grad I of the reference
      image by forward differences;
  D5  the non-convex data term is decoupled from the regulariser by an auxiliary
      field a: E_theta = lambda sum C(a) + sum (d - a)^2 / (2 theta) + TGV_T(d), with
      TGV_T(d) = min_w alpha1 sum |T grad d - w| + alpha2 sum |grad w|; the outer loop
      alternates the a-step (per pixel, exhaustive over integer delta, ties to the
      smallest) and the d-step (iterations of a primal-dual method on the convex
      TGV_T-L2 problem), theta shrinking by a constant factor per outer step; start:
      d = the a-step with no coupling (winner takes all), w = p = q = 0;
  D6  d-step: Chambolle-Pock on K (d, w) = (T grad d - w, grad w), duals p (|p| <= alpha1)
      and q (2 x 2, Frobenius |q| <= alpha2), tau = sigma = 1/sqrt(12) (||K||^2 <= 12),
      over-relaxation 1;
  D7  forward differences, zero across the last column / row; div = -grad^T;
  D8  the a-step is the argmin of D5's per-pixel energy over integer delta, evaluated in
      float64 like every other quantity here (ties to the smallest delta).  The paper
      fixes no precision.  A pixel whose best candidate beats another candidate by less
      than the rounding bound of a float32 evaluation of the two energies is flagged as a
      near tie: there a float32 implementation may pick either, so a comparison holds the
      unflagged pixels to the exact decision and counts the flagged ones.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It shares no code with the CUDA path.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

RX, RY = 4, 3  # Census window half-width and half-height: 9 x 7
BITS = (2 * RX + 1) * (2 * RY + 1) - 1  # 62, the centre skipped


@dataclass(frozen=True)
class StereoParams:
    """Table I's 2D column (lambda, alpha1, alpha2, beta, gamma) and this reading's
    schedule (D5, D6)."""
    max_disp: int = 64
    lam: float = 0.5
    alpha1: float = 1.0
    alpha2: float = 5.0
    beta: float = 1.0
    gamma: float = 4.0
    theta0: float = 2.0
    theta_decay: float = 0.5
    outer: int = 8
    inner: int = 80


# ----------------------------------------------------------------- Census (D2, D3)
def census(I) -> np.ndarray:
    """62-bit Census signatures [H, W] (uint64) of image I."""
    I = np.asarray(I, dtype=np.float32)
    H, W = I.shape
    ys = np.arange(H)[:, None]
    xs = np.arange(W)[None, :]
    sig = np.zeros((H, W), dtype=np.uint64)
    b = 0
    for dy in range(-RY, RY + 1):
        for dx in range(-RX, RX + 1):
            if dx == 0 and dy == 0:
                continue
            nb = I[np.clip(ys + dy, 0, H - 1), np.clip(xs + dx, 0, W - 1)]
            sig |= (nb < I).astype(np.uint64) << np.uint64(b)
            b += 1
    return sig


def popcount(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)
    return np.unpackbits(x.view(np.uint8).reshape(x.shape + (8,)), axis=-1).sum(axis=-1).astype(np.int64)


def hamming_volume(sigL, sigR, D) -> np.ndarray:
    """Hamming distances h[delta, y, x] = |sig_L(x + delta, y) xor sig_R(x, y)|, BITS where
    x + delta is off the image (D3 before the division by BITS)."""
    H, W = sigR.shape
    h = np.full((D, H, W), BITS, dtype=np.int64)
    for d in range(D):
        if d < W:
            h[d, :, : W - d] = popcount(sigL[:, d:] ^ sigR[:, : W - d])
    return h


# ------------------------------------------------------------- tensor (D4)
def grad(u):
    """Forward differences (D7): [2, H, W]."""
    g = np.zeros((2,) + u.shape)
    g[0, :, :-1] = u[:, 1:] - u[:, :-1]
    g[1, :-1, :] = u[1:, :] - u[:-1, :]
    return g


def div(p):
    """-grad^T of a vector field p [2, H, W] (D7)."""
    px, py = p[0], p[1]
    dx = np.zeros_like(px)
    dx[:, 0] = px[:, 0]
    dx[:, 1:-1] = px[:, 1:-1] - px[:, :-2]
    dx[:, -1] = -px[:, -2]
    dy = np.zeros_like(py)
    dy[0, :] = py[0, :]
    dy[1:-1, :] = py[1:-1, :] - py[:-2, :]
    dy[-1, :] = -py[-2, :]
    return dx + dy


def diffusion_tensor(I, gamma, beta) -> np.ndarray:
    """T [2, 2, H, W] of D4."""
    g = grad(np.asarray(I, dtype=np.float64))
    mag = np.sqrt(g[0] ** 2 + g[1] ** 2)
    e = np.exp(-gamma * mag ** beta)
    with np.errstate(invalid="ignore", divide="ignore"):
        nx = np.where(mag > 0, g[0] / mag, 0.0)
        ny = np.where(mag > 0, g[1] / mag, 0.0)
    T = np.zeros((2, 2) + mag.shape)
    T[0, 0] = 1.0 + (e - 1.0) * nx * nx
    T[0, 1] = T[1, 0] = (e - 1.0) * nx * ny
    T[1, 1] = 1.0 + (e - 1.0) * ny * ny
    return T


def apply_T(T, v):
    return np.stack([T[0, 0] * v[0] + T[0, 1] * v[1], T[1, 0] * v[0] + T[1, 1] * v[1]])


# ------------------------------------------------------------- steps (D5, D6, D8)
def assign(hvol, d, lam, theta, with_flags: bool = False):
    """a-step (D5, D8): argmin over integer delta in [0, D) of
        E(delta) = lam h(delta) / BITS + (d - delta)^2 / (2 theta)
    in float64, ties to the smallest delta; theta = inf drops the coupling (winner takes
    all on the Hamming distance, an exact integer comparison).  hvol is the Hamming volume
    [D, H, W], or a pair (sig_L, sig_R, D) to compute it delta by delta.

    With ``with_flags`` also returns the near-tie flags: for finite theta, a pixel is
    flagged when some other candidate's energy exceeds the best one's by at most
    B(best) + B(other), B(k) = 2^-20 (lam h(k) / BITS + (d - k)^2 / (2 theta)), sixteen
    times the relative rounding error a float32 evaluation of the sum of the two terms
    can make (a product, a difference, a square and a sum, each rounded once)."""
    if isinstance(hvol, tuple):
        sigL, sigR, D = hvol
        H, W = sigR.shape

        def h_of(k):
            h = np.full((H, W), BITS, dtype=np.int64)
            if k < W:
                h[:, : W - k] = popcount(sigL[:, k:] ^ sigR[:, : W - k])
            return h
    else:
        D = hvol.shape[0]

        def h_of(k):
            return hvol[k]
    d64 = np.asarray(d, dtype=np.float32).astype(np.float64)
    coupled = not np.isinf(theta)
    best = np.full(d64.shape, np.inf)
    arg = np.zeros(d64.shape, dtype=np.int64)
    energies = []
    for k in range(D):
        e = lam * h_of(k).astype(np.float64) / BITS
        if coupled:
            dd = d64 - float(k)
            e = e + dd * dd / (2.0 * theta)
        better = e < best
        best = np.where(better, e, best)
        arg = np.where(better, k, arg)
        if with_flags and coupled:
            energies.append(e)
    if not with_flags:
        return arg.astype(np.float64)
    flag = np.zeros(d64.shape, dtype=bool)
    if coupled:
        eps = 2.0 ** -20
        for k, e in enumerate(energies):
            close = (e - best) <= eps * (e + best)
            flag |= close & (arg != k)
    return arg.astype(np.float64), flag


class TGVState:
    """Primal (d, w), relaxed primal (d_bar, w_bar) and dual (p, q) fields of the d-step."""

    def __init__(self, d):
        d = np.asarray(d, dtype=np.float64)
        self.d = d.copy()
        self.d_bar = d.copy()
        self.w = np.zeros((2,) + d.shape)
        self.w_bar = np.zeros((2,) + d.shape)
        self.p = np.zeros((2,) + d.shape)
        self.q = np.zeros((2, 2) + d.shape)


def tgv_iterate(st: TGVState, a, T, theta, alpha1, alpha2, iters):
    """Chambolle-Pock iterations (D6) on min (1/2 theta) |d - a|^2 + alpha1 |T grad d - w|
    + alpha2 |grad w|."""
    tau = sigma = 1.0 / np.sqrt(12.0)
    for _ in range(iters):
        # dual ascent and projection on the balls
        p = st.p + sigma * (apply_T(T, grad(st.d_bar)) - st.w_bar)
        p /= np.maximum(1.0, np.sqrt(p[0] ** 2 + p[1] ** 2) / alpha1)[None]
        gw = np.stack([grad(st.w_bar[0]), grad(st.w_bar[1])])  # q[i, j] pairs with d_j w_i
        q = st.q + sigma * gw
        q /= np.maximum(1.0, np.sqrt((q ** 2).sum(axis=(0, 1))) / alpha2)[None, None]
        st.p, st.q = p, q
        # primal descent: d through the prox of the coupling, w plainly
        d_old, w_old = st.d, st.w
        d_tmp = d_old + tau * div(apply_T(T, p))
        d = (d_tmp + (tau / theta) * a) / (1.0 + tau / theta)
        w = w_old + tau * (p + np.stack([div(q[0]), div(q[1])]))
        st.d, st.w = d, w
        st.d_bar = 2.0 * d - d_old
        st.w_bar = 2.0 * w - w_old
    return st


def tgv_energy(d, w, a, T, theta, alpha1, alpha2):
    """Primal objective of the d-step at (d, w)."""
    r = apply_T(T, grad(d)) - w
    gw = np.stack([grad(w[0]), grad(w[1])])
    return (0.5 / theta) * np.sum((d - a) ** 2) + alpha1 * np.sum(np.sqrt(r[0] ** 2 + r[1] ** 2)) + \
        alpha2 * np.sum(np.sqrt((gw ** 2).sum(axis=(0, 1))))


def estimate(IL, IR, prm: StereoParams = StereoParams(), trace=None):
    """Disparity map on I_R's grid (D1-D8).  ``trace`` (a list) receives (theta, a, d)
    after every outer step."""
    sL, sR = census(IL), census(IR)
    hvol = (sL, sR, prm.max_disp)
    T = diffusion_tensor(IR, prm.gamma, prm.beta)
    d0 = assign(hvol, np.zeros(IR.shape), prm.lam, np.inf)
    st = TGVState(d0)
    theta = prm.theta0
    for _ in range(prm.outer):
        a = assign(hvol, st.d, prm.lam, theta)
        tgv_iterate(st, a, T, theta, prm.alpha1, prm.alpha2, prm.inner)
        if trace is not None:
            trace.append((theta, a.copy(), st.d.copy()))
        theta *= prm.theta_decay
    return st.d
