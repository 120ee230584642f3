"""Pins of the stereo oracle (oracle/stereo_oracle.py) to facts that do not come from it:

* Census signatures (9 x 7 window) against a bit-by-bit loop, invariance under a monotone change of
  intensity (the property Section IV-A names), zero for a flat window;
* Hamming costs: zero at the true shift of an exactly shifted pair, popcount against
  Python's bit count;
* div = -grad^T against the dense transpose of the gradient's matrix;
* the diffusion tensor's eigenpairs (numpy.linalg.eigh): exp(-gamma |grad I|^beta)
  along grad I, 1 across;
* the a-step: no coupling is the first argmin of the cost (numpy), strong coupling
  rounds d to the nearest integer (ties to the smaller);
* the a-step's switching point between two candidates against its closed form;
* the d-step converges to the minimiser of the same convex problem solved as a
  quadratic programme by scipy (trust-constr) on a two-row image, and its iterates keep the
  contraction properties of Chambolle-Pock with over-relaxation 1 in the method's metric;
* the whole estimate recovers an exact integer shift, and the synthetic street pair's
  true disparity (generator geometry) to sub-pixel median error.
"""

import numpy as np
import pytest

from oracle import stereo_oracle as S
from synth.scenes import tiny_scene

optimize = pytest.importorskip("scipy.optimize")


def test_census_bit_by_bit_and_invariance():
    rng = np.random.default_rng(0)
    I = rng.random((7, 9)).astype(np.float32)
    sig = S.census(I)
    H, W = I.shape
    for y in range(H):
        for x in range(W):
            bits, b = 0, 0
            for dy in range(-3, 4):
                for dx in range(-4, 5):
                    if dx == 0 and dy == 0:
                        continue
                    yy, xx = min(max(y + dy, 0), H - 1), min(max(x + dx, 0), W - 1)
                    if I[yy, xx] < I[y, x]:
                        bits |= 1 << b
                    b += 1
            assert sig[y, x] == bits
    J = (I.astype(np.float64) ** 2 * 0.7 + 0.2 * I + 0.05).astype(np.float32)  # increasing on [0, 1]
    assert np.array_equal(S.census(J), sig)
    assert np.all(S.census(np.full((5, 6), 0.3, np.float32)) == 0)
    assert S.BITS == 62


def test_hamming_zero_at_the_true_shift():
    rng = np.random.default_rng(1)
    IR = rng.random((12, 40)).astype(np.float32)
    shift = 7
    IL = np.zeros_like(IR)
    IL[:, shift:] = IR[:, :-shift]           # I_L(x + shift) = I_R(x)
    IL[:, :shift] = rng.random((12, shift))
    h = S.hamming_volume(S.census(IL), S.census(IR), 16)
    inner = (slice(3, -3), slice(4, 40 - shift - 4))
    assert np.all(h[shift][inner] == 0)
    assert np.all(h[:, :, -1][1:] == S.BITS)  # off the image for delta >= 1 at the last column
    x = rng.integers(0, 1 << 62, size=50, dtype=np.uint64)
    assert np.array_equal(S.popcount(x), [bin(int(v)).count("1") for v in x])


def test_div_is_minus_grad_transpose():
    H, W = 4, 5
    n = H * W
    G = np.zeros((2 * n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        G[:, i] = S.grad(e.reshape(H, W)).reshape(-1)
    rng = np.random.default_rng(2)
    p = rng.normal(size=(2, H, W))
    np.testing.assert_allclose(S.div(p).reshape(-1), -(G.T @ p.reshape(-1)), atol=1e-12)


def test_diffusion_tensor_eigenpairs():
    rng = np.random.default_rng(3)
    I = rng.random((6, 7))
    T = S.diffusion_tensor(I, 4.0, 1.0)
    g = S.grad(I)
    for y in range(6):
        for x in range(7):
            M = T[:, :, y, x]
            vals, vecs = np.linalg.eigh(M)
            mag = np.hypot(g[0, y, x], g[1, y, x])
            e = np.exp(-4.0 * mag)
            if mag == 0:
                np.testing.assert_allclose(M, np.eye(2), atol=1e-15)
                continue
            np.testing.assert_allclose(sorted(vals), sorted([e, 1.0]), atol=1e-12)
            v = vecs[:, np.argmin(np.abs(vals - e))]
            n = np.array([g[0, y, x], g[1, y, x]]) / mag
            assert abs(abs(v @ n) - 1.0) < 1e-10


def test_assign_limits():
    rng = np.random.default_rng(4)
    h = rng.integers(0, S.BITS + 1, size=(20, 5, 6))
    a = S.assign(h, rng.random((5, 6)) * 19, 0.5, np.inf)
    np.testing.assert_array_equal(a, np.argmin(h, axis=0))
    d = np.array([[3.2, 7.5, 0.49, 12.51, 18.0]])
    hz = np.zeros((20, 1, 5), dtype=np.int64)
    np.testing.assert_array_equal(S.assign(hz, d, 0.5, 1e-3), [[3, 7, 0, 13, 18]])


def test_assign_switching_point_closed_form():
    """Two candidates, delta = 0 with Hamming cost h0 and delta = 1 with h1: by D5 the
    a-step moves to 1 exactly when (d^2 - (d - 1)^2) / (2 theta) > lam (h1 - h0) / 62,
    i.e. above d* = 1/2 + theta lam (h1 - h0) / 62 (worked out by hand from D5's energy,
    which fixes the factor 1/(2 theta) of the coupling)."""
    lam = 0.5
    cases = [(2.0, 31), (0.5, 62), (1.0, 12), (4.0, -20), (0.25, 0)]  # theta, h1 - h0
    for theta, dh in cases:
        h0 = 30
        h = np.array([[[h0, h0]], [[h0 + dh, h0 + dh]]], dtype=np.int64)  # [D = 2, 1, 2]
        d_star = 0.5 + theta * lam * dh / S.BITS
        d = np.array([[d_star - 1e-3, d_star + 1e-3]])
        a, flag = S.assign(h, d, lam, theta, with_flags=True)
        np.testing.assert_array_equal(a, [[0.0, 1.0]], err_msg=str((theta, dh)))
        assert not flag.any()


def test_tgv_steps_shrink_in_the_primal_dual_metric():
    """D6 is Chambolle-Pock with over-relaxation 1: with x = (d, w) and y = (p, q), the
    pairs v_k = (x_k, y_{k+1}) follow a proximal-point iteration in the metric
    M = [[I/tau, -K^T], [-K, I/sigma]], positive semidefinite since sigma tau ||K||^2 <= 1
    (He and Yuan's reading of the method).  Its resolvent is firmly nonexpansive in M, so
    the step lengths |v_{k+1} - v_k|_M never grow, checked with the ball constraints
    active (small alpha1, alpha2) on random data; and the distance |v_k - v*|_M to any
    saddle point v* never grows, checked where v* = 0 is one: no data term (theta
    infinite) and balls too large to bind.  Leaving out the over-relaxation of d or of w
    makes the distance grow in the second case."""
    tau = sigma = 1.0 / np.sqrt(12.0)
    for seed in range(3):
        rng = np.random.default_rng(40 + seed)
        H, W = 5, 6
        T = S.diffusion_tensor(rng.random((H, W)), 4.0, 1.0)
        a = rng.random((H, W)) * 5.0
        st = S.TGVState(rng.random((H, W)) * 5.0)
        xs, ys = [(st.d.copy(), st.w.copy())], []
        for _ in range(200):
            S.tgv_iterate(st, a, T, 0.7, 0.05, 0.1, 1)
            xs.append((st.d.copy(), st.w.copy()))
            ys.append((st.p.copy(), st.q.copy()))

        def m_norm2(dd, dw, dp, dq):
            r = S.apply_T(T, S.grad(dd)) - dw
            gw = np.stack([S.grad(dw[0]), S.grad(dw[1])])
            return ((np.sum(dd * dd) + np.sum(dw * dw)) / tau + (np.sum(dp * dp) + np.sum(dq * dq)) / sigma
                    - 2.0 * (np.sum(r * dp) + np.sum(gw * dq)))

        steps = np.array([m_norm2(xs[k + 1][0] - xs[k][0], xs[k + 1][1] - xs[k][1],
                                  ys[k + 1][0] - ys[k][0], ys[k + 1][1] - ys[k][1]) for k in range(len(ys) - 1)])
        assert np.all(steps >= -1e-12), steps.min()
        assert np.all(steps[1:] <= steps[:-1] * (1.0 + 1e-9) + 1e-18), np.max(steps[1:] / steps[:-1])
        assert steps[-1] < 1e-3 * steps[0]

        # the bilinear case: (d, w, p, q) = 0 is a saddle point
        st = S.TGVState(rng.standard_normal((H, W)))
        zero = np.zeros((H, W))
        x_prev = (st.d.copy(), st.w.copy())
        dist = []
        for _ in range(300):
            S.tgv_iterate(st, zero, T, np.inf, 1e12, 1e12, 1)
            dist.append(m_norm2(x_prev[0], x_prev[1], st.p, st.q))  # v_k = (x_k, y_{k+1})
            x_prev = (st.d.copy(), st.w.copy())
        dist = np.array(dist)
        assert np.all(dist[1:] <= dist[:-1] * (1.0 + 1e-9)), np.max(dist[1:] / dist[:-1])


def qp_tgv_1d(a, theta, alpha1, alpha2):
    """min (1/2 theta) |d - a|^2 + alpha1 sum |D d - w| + alpha2 sum |D w| with the
    forward difference D (zero at the last entry), as a smooth QP with slacks."""
    n = len(a)
    Dm = np.zeros((n, n))
    for i in range(n - 1):
        Dm[i, i], Dm[i, i + 1] = -1.0, 1.0
    nv = 4 * n  # d, w, s, t

    def f(x):
        d, s, t = x[:n], x[2 * n:3 * n], x[3 * n:]
        return 0.5 / theta * np.sum((d - a) ** 2) + alpha1 * s.sum() + alpha2 * t.sum()

    def jac(x):
        g = np.zeros(nv)
        g[:n] = (x[:n] - a) / theta
        g[2 * n:3 * n] = alpha1
        g[3 * n:] = alpha2
        return g

    A = []
    for sgn in (1.0, -1.0):
        blk = np.zeros((n, nv))
        blk[:, :n] = -sgn * Dm
        blk[:, n:2 * n] = sgn * np.eye(n)
        blk[:, 2 * n:3 * n] = np.eye(n)
        A.append(blk)  # s >= sgn (D d - w)
        blk = np.zeros((n, nv))
        blk[:, n:2 * n] = -sgn * Dm
        blk[:, 3 * n:] = np.eye(n)
        A.append(blk)  # t >= sgn D w
    A = np.vstack(A)
    x0 = np.concatenate([a, np.zeros(n), np.abs(Dm @ a) + 1, np.ones(n)])
    hess = np.zeros((nv, nv))
    hess[:n, :n] = np.eye(n) / theta
    res = optimize.minimize(f, x0, jac=jac, hess=lambda x: hess, method="trust-constr",
                            constraints=[optimize.LinearConstraint(A, 0.0, np.inf)],
                            options={"gtol": 1e-12, "xtol": 1e-14, "maxiter": 20000})
    assert res.status in (1, 2), res.message
    return res.x[:n]


def test_tgv_step_matches_qp():
    a1 = np.array([0.0, 0.3, 0.6, 0.9, 1.2, 1.5, 4.0, 4.1, 3.9, 4.2, 4.0, 4.1])
    theta, al1, al2 = 0.5, 0.4, 1.5
    d_qp = qp_tgv_1d(a1, theta, al1, al2)
    a = np.stack([a1, a1])  # two identical rows: no y-gradient, the same minimiser per row
    T = S.diffusion_tensor(np.ones((2, 12)), 4.0, 1.0)  # flat image: identity
    st = S.TGVState(a)
    S.tgv_iterate(st, a, T, theta, al1, al2, 40000)
    np.testing.assert_allclose(st.d[0], d_qp, atol=2e-5)
    np.testing.assert_allclose(st.d[1], d_qp, atol=2e-5)
    # the ramp is kept, unlike TV: its interior second differences stay near zero
    assert np.max(np.abs(np.diff(st.d[0][:6], 2))) < 1e-3


def smooth_texture(rng, shape):
    """Random texture blurred by a 3 x 3 box (white noise has 4% local extrema, whose
    all-zero / all-one signatures match anything alike)."""
    z = rng.random((shape[0] + 2, shape[1] + 2))
    out = sum(z[i:i + shape[0], j:j + shape[1]] for i in range(3) for j in range(3)) / 9.0
    return out.astype(np.float32)


def test_integer_shift_is_recovered():
    rng = np.random.default_rng(5)
    IR = smooth_texture(rng, (24, 64))
    shift = 9
    IL = smooth_texture(rng, (24, 64))
    IL[:, shift:] = IR[:, :-shift]
    d = S.estimate(IL, IR, S.StereoParams(max_disp=24))
    inner = np.abs(d[4:-4, 5:64 - shift - 5] - shift)
    assert np.median(inner) < 0.01 and (inner < 0.05).mean() > 0.99, (np.median(inner), (inner < 0.05).mean())


def test_synthetic_street_pair_against_ground_truth():
    sc = tiny_scene(0)
    IL, IR, dt, _ = sc.stereo_pair(0)
    d = S.estimate(IL, IR, S.StereoParams(max_disp=32))
    v = dt > 0
    err = np.abs(d - dt)[v]
    assert np.median(err) < 0.02 and (err > 3).mean() < 0.03, (np.median(err), (err > 3).mean())


def test_estimate_composes_the_pinned_stages():
    """D5 as a schedule of the stages pinned above: winner-takes-all start from the
    Census costs of (I_L, I_R), the tensor of the reference image I_R, then per outer
    step an a-step at the current theta and `inner` d-step iterations with (alpha1,
    alpha2) in that order, theta shrinking by theta_decay.  The recorded trace matches
    the stages run one by one, bit for bit."""
    rng = np.random.default_rng(6)
    IR = smooth_texture(rng, (10, 24))
    IL = smooth_texture(rng, (10, 24))
    IL[:, 3:] = IR[:, :-3]
    prm = S.StereoParams(max_disp=8, outer=3, inner=7, alpha1=0.7, alpha2=3.0, theta0=1.5, theta_decay=0.4)
    trace = []
    d = S.estimate(IL, IR, prm, trace=trace)
    h = S.hamming_volume(S.census(IL), S.census(IR), prm.max_disp)
    T = S.diffusion_tensor(IR, prm.gamma, prm.beta)
    st = S.TGVState(np.argmin(h, axis=0).astype(np.float64))  # no coupling: first argmin
    theta = prm.theta0
    assert len(trace) == prm.outer
    for th, a_got, d_got in trace:
        assert th == theta
        a = S.assign(h, st.d, prm.lam, theta)
        S.tgv_iterate(st, a, T, theta, prm.alpha1, prm.alpha2, prm.inner)
        assert np.array_equal(a_got, a) and np.array_equal(d_got, st.d)
        theta *= prm.theta_decay
    assert np.array_equal(d, st.d)
