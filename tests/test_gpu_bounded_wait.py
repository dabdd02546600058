"""Failure detection without a GPU fault: a sweep whose neighbour value never
arrives (its producer pencil is skipped) ends its wait by the iteration limit,
reports ISC_ERR_TIMEOUT through the kernel's status word, and the CUDA context
stays usable for the next calls."""
import time

import numpy as np
import pytest

import isc_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import isc
    return isc


def test_wait_runs_out_and_the_context_survives(lib):
    t0 = time.perf_counter()
    st = lib.check_bounded_wait()
    elapsed = time.perf_counter() - t0
    assert lib.STATUS.get(st) == "device wait timed out", st
    assert elapsed < 60.0
    # the device still works: a reciprocal check and a small solve
    y, z = lib.check_reciprocal(np.array([3.0, -7.5]))
    assert np.allclose(y, z)
    case = inp.small_box(3, 2, 2)
    sim = lib.Simulator(case)
    sim.init_equilibrium()
    info = sim.newton_step(case.dt0)
    assert info.krylov_rel_residual <= 1e-6
    sim.close()
