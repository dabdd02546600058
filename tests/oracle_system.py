"""Linear systems built by the oracle alone (test helper): its residual and
Jacobian (Sec. 3.1) at seeded random states, and their Gauss-Jordan decoupling
(Sec. 3.2). GPU stages are fed these through isc_set_system, so that no oracle
input ever comes from the CUDA path."""
import isc_inputs as inp
from oracle import linalg, model


def assembled(case, seed_a, seed_b, dt=100.0):
    """(rowptr, col, J, F) with F (8, N): the oracle's system at state b with
    the accepted state a (random states of the workload's ranges)."""
    a = inp.random_state(case, seed_a)
    b = inp.random_state(case, seed_b)
    acc = model.old_accumulation(case, a["u"], a["coke"])
    F = model.residual(case, b["u"], a["coke"], acc, dt)
    rp, col, J = model.jacobian(case, b["u"], a["coke"], acc, dt)
    return rp, col, J, F


def decoupled(case, seed_a, seed_b, dt=100.0):
    """(rowptr, col, J, F, Jd, Fd): the assembled system and its decoupling
    (Jd with unit diagonal blocks, Fd (8, N))."""
    rp, col, J, F = assembled(case, seed_a, seed_b, dt)
    vd, rd = linalg.gauss_jordan_decouple(rp, col, J, F.T.copy())
    return rp, col, J, F, vd, rd.T.copy()


def initial_decoupled(case, dt):
    """(rowptr, col, Jd, Fd): the oracle's decoupled system at the case's
    flash-consistent initial state (ignited cells included) for step size dt."""
    from oracle import sim
    u0, c0 = sim.initial_state(case)
    acc = model.old_accumulation(case, u0, c0)
    F = model.residual(case, u0, c0, acc, dt)
    rp, col, J = model.jacobian(case, u0, c0, acc, dt)
    vd, rd = linalg.gauss_jordan_decouple(rp, col, J, F.T.copy())
    return rp, col, vd, rd.T.copy()
