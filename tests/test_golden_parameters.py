"""The method constants against the paper's parameter table (Table I), stored as the
fixture tests/golden/table1_parameters.txt: the oracle's defaults and the library's
defaults (host calls, no GPU)."""

import os

import pytest

from oracle import denser_oracle as O
from oracle import stereo_oracle as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_parameters.txt")


def table():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            name, col, val = line.split()
            out[(name, col)] = float(val)
    return out


def test_oracle_defaults_are_table_one():
    t = table()
    p = O.Params()
    assert p.voxel_size == 0.1
    assert p.lam == t[("lambda_3d", "10cm")]
    assert p.sigma == t[("sigma_p", "-")] and p.theta == t[("theta", "-")]
    assert abs(p.tau - t[("tau", "-")]) < 1e-15
    # the truncation band: Table I's 1.0 m is a parameter; the synthetic workloads use 0.3 m
    assert t[("mu_3d", "10cm")] == 1.0 and O.Params(mu=1.0).mu == 1.0
    sp = S.StereoParams()
    assert (sp.lam, sp.alpha1, sp.alpha2, sp.beta, sp.gamma) == (
        t[("lambda_2d", "-")], t[("alpha1", "-")], t[("alpha2", "-")], t[("beta", "-")], t[("gamma", "-")])


def test_library_defaults_are_table_one():
    native = pytest.importorskip("paper_1604_03734_gb300.native")
    from paper_1604_03734_gb300 import build
    build.build()
    t = table()
    p = native.denser_default_params()
    assert p.lambda_ == t[("lambda_3d", "10cm")] and p.sigma == t[("sigma_p", "-")]
    assert p.theta == t[("theta", "-")] and abs(p.tau - t[("tau", "-")]) < 1e-15
    sp = native.denser_stereo_default_params()
    for field, key in (("lambda_", "lambda_2d"), ("alpha1", "alpha1"), ("alpha2", "alpha2"), ("beta", "beta"),
                       ("gamma", "gamma")):
        assert getattr(sp, field) == pytest.approx(t[(key, "-")], rel=0, abs=0)

