"""The square root of the primal energy's per-voxel term (regularize.cu, energy_sqrt), on
the CPU: a single-precision reciprocal square root r within 2 ulps, s0 = x r rounded to
single precision, then one step of Heron's method in float64,
s1 = s0 + (x - s0^2) r / 2 (each operation rounded as the kernel's fused multiply-adds
round it).  Over the range of squared gradients the energy sees, and with r moved by up to
two ulps either way, s1 stays within 2^-40 of sqrt(x) relative: far below the 1e-12
relative tolerance of the energies against the oracle.  No GPU."""

import math

import numpy as np
import pytest

F32 = np.float32


def fma64(a, b, c):
    """float64 fma(a, b, c): the exact value (rational arithmetic), rounded once."""
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def heron(x, ulps):
    xf = F32(x)
    r = F32(1.0 / math.sqrt(float(xf)))
    for _ in range(abs(ulps)):
        r = np.nextafter(r, F32(np.inf) if ulps > 0 else F32(-np.inf))
    s0 = float(F32(xf * r))
    return fma64(0.5 * float(r), fma64(-s0, s0, x), s0)


@pytest.mark.parametrize("ulps", [-2, -1, 0, 1, 2])
def test_heron_step_relative_error(ulps):
    rng = np.random.default_rng(11 + ulps)
    xs = np.concatenate([10.0 ** rng.uniform(-29, 3, 400), rng.uniform(0, 12, 200)])
    xs = xs[xs > 1e-30]
    worst = 0.0
    for x in xs:
        s = heron(float(x), ulps)
        worst = max(worst, abs(s - math.sqrt(x)) / math.sqrt(x))
    assert worst <= 2.0 ** -40, worst
