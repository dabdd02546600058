"""Pins of the oracle's tangent model with coupled producers (bottom-hole
pressure unknown, Sec. 2.2 Well Modeling): against central finite differences
of the oracle's own bordered-Newton simulation, and against the fixed-BHP
producer's tangent when a BHP-controlled coupled producer without gravity is
that producer (the residuals coincide exactly)."""
import copy

import numpy as np
import pytest

import isc_inputs as inp
from oracle import adjoint, model


def _case(control=inp.CTRL_TOTAL_RATE, target=8.0):
    return inp.with_coupled_producer(inp.small_box(3, 2, 2), control, target, 4.6e6), [10.0, 40.0]


def _L(case, dts, lnk, Ea, lnA):
    c = adjoint.param_case(case, lnk, Ea, lnA)
    us, bs, cs = adjoint.trajectory_coupled(c, dts, tol=1e-12)
    return adjoint.loss_coupled(c, dts, us, bs)


@pytest.mark.parametrize("which", ["lnk", "kinetics"])
def test_coupled_tangent_matches_central_differences(which):
    case, dts = _case()
    rng = np.random.default_rng({"lnk": 11, "kinetics": 12}[which])
    n, nr = case.n, case.reactions["nr"]
    v_lnk = rng.standard_normal(n) if which == "lnk" else np.zeros(n)
    v_Ea = rng.standard_normal(nr) * 1e3 if which == "kinetics" else np.zeros(nr)
    v_lnA = rng.standard_normal(nr) if which == "kinetics" else np.zeros(nr)
    us, bs, cs = adjoint.trajectory_coupled(case, dts, tol=1e-12)
    L0 = adjoint.loss_coupled(case, dts, us, bs)
    assert L0 > 0
    # the rate control holds at every converged step
    for u, b in zip(us[1:], bs[1:]):
        assert abs(model.well_equations(case, u, b)[0]) <= 1e-9 * 8.0
    d = adjoint.tangent_coupled(case, dts, us, bs, cs, v_lnk, v_Ea, v_lnA)
    h = 1e-5
    Ea0, lnA0 = case.reactions["Ea"], np.log(case.reactions["A"])
    Lp = _L(case, dts, h * v_lnk, Ea0 + h * v_Ea, lnA0 + h * v_lnA)
    Lm = _L(case, dts, -h * v_lnk, Ea0 - h * v_Ea, lnA0 - h * v_lnA)
    fd = (Lp - Lm) / (2 * h)
    assert d == pytest.approx(fd, rel=1e-5, abs=1e-9 * abs(L0))


def test_bhp_controlled_coupled_tangent_is_the_fixed_bhp_tangent():
    base = inp.small_box(3, 2, 2)
    base.fluid = dict(base.fluid)
    base.fluid["gravity"] = 0.0
    target = [w for w in base.wells if w.kind == inp.WELL_BHP_PRODUCER][0].target
    coupled = inp.with_coupled_producer(base, inp.CTRL_BHP, target, target)
    dts = [10.0, 40.0]
    rng = np.random.default_rng(13)
    n, nr = base.n, base.reactions["nr"]
    v_lnk, v_Ea, v_lnA = rng.standard_normal(n), rng.standard_normal(nr) * 1e3, rng.standard_normal(nr)
    us0, cs0 = adjoint.trajectory(base, dts, tol=1e-12)
    us1, bs1, cs1 = adjoint.trajectory_coupled(coupled, dts, tol=1e-12)
    assert np.all(np.concatenate(bs1) == target)
    L0 = adjoint.loss(base, dts, us0)
    L1 = adjoint.loss_coupled(coupled, dts, us1, bs1)
    assert L1 == pytest.approx(L0, rel=1e-10)
    d0 = adjoint.tangent(base, dts, us0, cs0, v_lnk, v_Ea, v_lnA)
    d1 = adjoint.tangent_coupled(coupled, dts, us1, bs1, cs1, v_lnk, v_Ea, v_lnA)
    assert d1 == pytest.approx(d0, rel=1e-8)
