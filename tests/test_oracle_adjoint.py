"""Pin of the oracle's tangent model of the time loop: dL/dtheta . v against
central finite differences of the oracle simulation itself (the paper gives
no sensitivities; the loss is the cumulative oil production)."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import adjoint


def _box():
    case = inp.small_box(3, 2, 2)
    return case, [10.0, 40.0, 160.0]


def _L(case, dts, lnk, Ea, lnA):
    c = adjoint.param_case(case, lnk, Ea, lnA)
    us, cs = adjoint.trajectory(c, dts, tol=1e-11)
    return adjoint.loss(c, dts, us)


@pytest.mark.parametrize("which", ["lnk", "Ea", "lnA", "all"])
def test_tangent_matches_central_differences(which):
    case, dts = _box()
    rng = np.random.default_rng({"lnk": 1, "Ea": 2, "lnA": 3, "all": 4}[which])
    n, nr = case.n, case.reactions["nr"]
    v_lnk = rng.standard_normal(n) if which in ("lnk", "all") else np.zeros(n)
    v_Ea = rng.standard_normal(nr) * 1e3 if which in ("Ea", "all") else np.zeros(nr)
    v_lnA = rng.standard_normal(nr) if which in ("lnA", "all") else np.zeros(nr)
    us, cs = adjoint.trajectory(case, dts, tol=1e-11)
    L0 = adjoint.loss(case, dts, us)
    assert L0 > 0
    d = adjoint.tangent(case, dts, us, cs, v_lnk, v_Ea, v_lnA)
    h = 1e-5
    Ea0, lnA0 = case.reactions["Ea"], np.log(case.reactions["A"])
    Lp = _L(case, dts, h * v_lnk, Ea0 + h * v_Ea, lnA0 + h * v_lnA)
    Lm = _L(case, dts, -h * v_lnk, Ea0 - h * v_Ea, lnA0 - h * v_lnA)
    fd = (Lp - Lm) / (2 * h)
    assert d == pytest.approx(fd, rel=1e-5, abs=1e-9 * abs(L0))
