"""GPU discrete adjoint (isc_adjoint) against the oracle's tangent-linear
model (an independent, forward-mode algorithm) element by element on a small
box, against central finite differences of the GPU time loop itself on the
40x40x10 adjoint workload, and for the properties the checkpointing must keep
(bit-exact recomputation, loss independent of the gradient request)."""
import numpy as np
import pytest

import isc_inputs as inp
from oracle import adjoint

pytestmark = pytest.mark.gpu

BOX_DTS = [10.0, 40.0, 160.0]


def _sim(case, **kw):
    pytest.importorskip("torch")
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator
    opts = dict(tol_newton=1e-10, tol_lin=1e-10, maxit_newton=40)
    opts.update(kw)
    return Simulator(case, **opts)


@pytest.fixture(scope="module")
def box():
    case = inp.small_box(4, 3, 2)
    us, cs = adjoint.trajectory(case, BOX_DTS, tol=1e-11)
    return case, us, cs


def test_loss_and_full_gradient_match_oracle_tangent(box):
    case, us, cs = box
    n, nr = case.n, int(case.reactions["nr"])
    g = _sim(case)
    g.init_equilibrium()
    L, gk, ge, ga, info = g.adjoint(BOX_DTS, checkpoint_every=2, tol_adjoint=1e-12)
    assert info["recomputed_steps"] == 2
    L0 = adjoint.loss(case, BOX_DTS, us)
    assert L == pytest.approx(L0, rel=1e-8)
    # every component through a unit direction of the tangent model
    ref_k = np.array([adjoint.tangent(case, BOX_DTS, us, cs, np.eye(n)[i], np.zeros(nr), np.zeros(nr))
                      for i in range(n)])
    ref_e = np.array([adjoint.tangent(case, BOX_DTS, us, cs, np.zeros(n), np.eye(nr)[r], np.zeros(nr))
                      for r in range(nr)])
    ref_a = np.array([adjoint.tangent(case, BOX_DTS, us, cs, np.zeros(n), np.zeros(nr), np.eye(nr)[r])
                      for r in range(nr)])
    for got, ref in ((gk, ref_k), (ge, ref_e), (ga, ref_a)):
        scale = np.abs(ref).max()
        assert scale > 0
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-8 * scale)
    g.close()


def test_gradient_with_heat_loss_matches_oracle_tangent():
    """The same comparison with heat loss to the overburden and underburden switched
    on (Sec. 2.1): the loss term enters every step's Jacobian (the temperature
    column of the energy row), which the reverse sweep transposes."""
    case = inp.with_heat_loss(inp.small_box(4, 3, 2))
    us, cs = adjoint.trajectory(case, BOX_DTS, tol=1e-11)
    n, nr = case.n, int(case.reactions["nr"])
    g = _sim(case)
    g.init_equilibrium()
    L, gk, ge, ga, info = g.adjoint(BOX_DTS, checkpoint_every=2, tol_adjoint=1e-12)
    assert L == pytest.approx(adjoint.loss(case, BOX_DTS, us), rel=1e-8)
    ref_k = np.array([adjoint.tangent(case, BOX_DTS, us, cs, np.eye(n)[i], np.zeros(nr), np.zeros(nr))
                      for i in range(n)])
    ref_e = np.array([adjoint.tangent(case, BOX_DTS, us, cs, np.zeros(n), np.eye(nr)[r], np.zeros(nr))
                      for r in range(nr)])
    for got, ref in ((gk, ref_k), (ge, ref_e)):
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-8 * scale)
    # the loss changes the trajectory: the gradient differs from the one without it
    us0, cs0 = adjoint.trajectory(inp.small_box(4, 3, 2), BOX_DTS, tol=1e-11)
    assert not np.allclose(adjoint.loss(inp.small_box(4, 3, 2), BOX_DTS, us0), L, rtol=1e-9)
    g.close()


def test_checkpointing_recomputes_bit_exactly(box):
    case, _, _ = box
    g = _sim(case)
    res = []
    for K in (1, 2, 3):
        g.init_equilibrium()
        res.append(g.adjoint(BOX_DTS, checkpoint_every=K, tol_adjoint=1e-12))
    for L, gk, ge, ga, info in res[1:]:
        assert L == res[0][0]
        np.testing.assert_array_equal(gk, res[0][1])
        np.testing.assert_array_equal(ge, res[0][2])
        np.testing.assert_array_equal(ga, res[0][3])
    # the loss does not depend on the gradient request, and the handle ends at
    # the final state of the same loop run step by step
    g.init_equilibrium()
    L_only, *_ = g.adjoint(BOX_DTS, checkpoint_every=2, gradient=False)
    assert L_only == res[0][0]
    u_adj, c_adj = g.get_state()
    g.init_equilibrium()
    for dt in BOX_DTS:
        g.timestep(dt)
    u_ts, c_ts = g.get_state()
    np.testing.assert_array_equal(u_adj, u_ts)
    np.testing.assert_array_equal(c_adj, c_ts)
    g.close()


def test_parameters_change_the_loop_like_the_oracle(box):
    """isc_set_parameters scales k and WI and replaces E_a, A as the oracle's
    parameterised case does: the perturbed loss matches the oracle's."""
    case, _, _ = box
    n, nr = case.n, int(case.reactions["nr"])
    rng = np.random.default_rng(5)
    lnk = 0.3 * rng.standard_normal(n)
    Ea = case.reactions["Ea"] * (1 + 0.01 * rng.standard_normal(nr))
    lnA = np.log(case.reactions["A"]) + 0.1 * rng.standard_normal(nr)
    g = _sim(case)
    g.set_parameters(lnk, Ea, lnA)
    lk2, Ea2, lnA2 = g.get_parameters()
    np.testing.assert_array_equal(lk2, lnk)
    np.testing.assert_array_equal(Ea2, Ea)
    np.testing.assert_array_equal(lnA2, lnA)
    g.init_equilibrium()
    L, *_ = g.adjoint(BOX_DTS, gradient=False)
    c = adjoint.param_case(case, lnk, Ea, lnA)
    us, _ = adjoint.trajectory(c, BOX_DTS, tol=1e-11)
    assert L == pytest.approx(adjoint.loss(c, BOX_DTS, us), rel=1e-8)
    g.close()


def test_autograd_function_returns_the_adjoint_gradient(box):
    """forward runs the loss only; backward runs the reverse sweep (the
    transposed solves) and gives the gradient of the one-call isc_adjoint bit
    for bit."""
    torch = pytest.importorskip("torch")
    from paper_1811_11992_gb300.autograd import oil_production
    case, _, _ = box
    g = _sim(case)
    lk0, Ea0, lnA0 = g.get_parameters()
    lk = torch.tensor(lk0, requires_grad=True)
    Ea = torch.tensor(Ea0, requires_grad=True)
    lnA = torch.tensor(lnA0, requires_grad=True)
    L = oil_production(g, BOX_DTS, lk, Ea, lnA, checkpoint_every=2, tol_adjoint=1e-12)
    assert L.grad_fn.info["krylov_iterations_adjoint"] == 0          # no transposed solve yet
    (2.0 * L).backward()
    assert L.grad_fn.info_backward["krylov_iterations_adjoint"] > 0
    g.init_equilibrium()
    L2, gk, ge, ga, _ = g.adjoint(BOX_DTS, checkpoint_every=2, tol_adjoint=1e-12)
    assert L.item() == L2
    np.testing.assert_array_equal(lk.grad.numpy(), 2.0 * gk)
    np.testing.assert_array_equal(Ea.grad.numpy(), 2.0 * ge)
    np.testing.assert_array_equal(lnA.grad.numpy(), 2.0 * ga)
    g.close()


def test_split_adjoint_repeats_and_refuses_a_changed_model(box):
    from paper_1811_11992_gb300 import isc
    case, _, _ = box
    g = _sim(case)
    g.init_equilibrium()
    L, info = g.adjoint_forward(BOX_DTS, checkpoint_every=2, tol_adjoint=1e-12)
    a = g.adjoint_backward()
    b = g.adjoint_backward()           # the last segment is recomputed the second time
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    g.init_equilibrium()
    L2, gk, ge, ga, _ = g.adjoint(BOX_DTS, checkpoint_every=2, tol_adjoint=1e-12)
    assert L == L2
    np.testing.assert_array_equal(a[0], gk)
    np.testing.assert_array_equal(a[1], ge)
    lk0, Ea0, lnA0 = g.get_parameters()
    g.set_parameters(lk0, Ea0, lnA0)
    with pytest.raises(isc.IscError) as err:
        g.adjoint_backward()
    assert err.value.status == -11
    g.close()


def test_adjoint_workload_central_differences():
    """40x40x10, 20 steps, checkpoints every 5: the adjoint directional
    derivative against central differences with a relative step of 1e-6 on 20
    seeded directions: 14 in all parameters, 3 in E_a alone and 3 in ln A
    alone (the ln k part dominates the mixed directions and would hide an
    error in the reaction gradients). The step is relative to each
    parameter's magnitude (E_a, ln A); the ln k multipliers are zero, so
    their step is 1e-6 in ln k itself."""
    case = inp.config(4)
    n, nr = case.n, int(case.reactions["nr"])
    dts = inp.adjoint_steps(case)
    torch = pytest.importorskip("torch")
    from paper_1811_11992_gb300.autograd import oil_production
    # the differences divide the loss's solver error by 2h = 2e-6: the time loop is
    # converged tightly (Newton 1e-10, linear 1e-10) so that this error stays far below
    # the 1e-4 being checked
    g = _sim(case, tol_newton=1e-10, tol_lin=1e-10, maxit_lin=3000, maxit_newton=40)
    lk0, Ea0, lnA0 = g.get_parameters()
    # the gradient through torch.autograd.grad: forward = the loss, backward = the reverse sweep
    params = [torch.tensor(v, requires_grad=True) for v in (lk0, Ea0, lnA0)]
    Lt = oil_production(g, dts, *params, checkpoint_every=5, tol_adjoint=1e-10)
    gk, ge, ga = (t.numpy() for t in torch.autograd.grad(Lt, params))
    L = Lt.item()
    assert L > 0 and Lt.grad_fn.info_backward["recomputed_steps"] == 15
    rng = np.random.default_rng(2024)
    h = 1e-6
    rows = []
    for d in range(20):
        group = "all" if d < 14 else ("Ea" if d < 17 else "lnA")
        vk = rng.standard_normal(n) * (group == "all")
        ve = Ea0 * rng.standard_normal(nr) * (group in ("all", "Ea"))
        va = np.abs(lnA0) * rng.standard_normal(nr) * (group in ("all", "lnA"))
        ad = gk @ vk + ge @ ve + ga @ va
        Ls = []
        for sgn in (1.0, -1.0):
            g.set_parameters(lk0 + sgn * h * vk, Ea0 + sgn * h * ve, lnA0 + sgn * h * va)
            g.init_equilibrium()
            Ls.append(g.adjoint(dts, checkpoint_every=5, gradient=False)[0])
        fd = (Ls[0] - Ls[1]) / (2 * h)
        rows.append((group, ad, fd, abs(fd - ad) / max(abs(ad), abs(fd))))
    g.set_parameters(lk0, Ea0, lnA0)
    g.close()
    worst = max(r[3] for r in rows)
    assert worst < 1e-4, rows
