"""Determinism: the same Newton step run twice from the same state gives the
same bits (state, residual norms, Krylov counts), in every precision and with
either preconditioner. The sweeps and the factorisation hand pencils to
whichever warp claims them first, so this also checks that no result depends
on that order (the reductions have a fixed order)."""
import numpy as np
import pytest

import isc_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Simulator():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator as S
    return S


@pytest.mark.parametrize("prec,precision", [("bilu0", "fp64"), ("bilu0", "mixed"), ("bilu0", "mixed_fgmres"),
                                            ("cpr", "fp64"), ("cpr", "mixed_fgmres")])
def test_newton_step_is_bitwise_repeatable(Simulator, prec, precision):
    case = inp.config(2)                 # field 60x60x20, 1,200 pencils
    g = Simulator(case, prec=prec, precision=precision, tol_lin=1e-6)
    g.init_equilibrium()
    u0, c0 = g.get_state()
    runs = []
    for _ in range(3):
        g.set_state(u0, c0)
        info = g.newton_step(case.dt0)
        u, c = g.get_state()
        runs.append((info.krylov_iterations, info.krylov_rel_residual, info.norm, u, c))
    for r in runs[1:]:
        assert r[:3] == runs[0][:3]
        assert np.array_equal(r[3], runs[0][3]) and np.array_equal(r[4], runs[0][4])
    g.close()


def test_large_grid_apply_is_bitwise_repeatable(Simulator):
    """On a grid where the pair sweeps' warps take several pencil pairs each
    (2 x 160 x 100: 8,000 pairs), the ILU(0) apply of the same vector is the
    same bits every time."""
    case = inp.field_case(2, 160, 100, 0, 9, "field 2x160x100", inp.DAY, 4)
    g = Simulator(case)
    g.init_equilibrium()
    g.assemble(case.dt0)
    g.decouple()
    g.build_preconditioner()
    x = np.random.default_rng(4).standard_normal((8, case.n))
    z = g.precond_apply(x)
    for _ in range(3):
        assert np.array_equal(g.precond_apply(x), z)
    g.close()
