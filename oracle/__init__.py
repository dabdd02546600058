"""Plain FP64 CPU oracle of the in-situ-combustion Newton step (arXiv 1811.11992).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA product path never calls it and shares no code with it.

Modules
-------
model   per-cell properties (Sec. 2.2), the discrete residual (Sec. 3.1) and the
        Jacobian as the exact derivative of that residual (complex-step
        differentiation, so no hand-written derivative is shared with anything).
linalg  Gauss-Jordan decoupling with partial pivoting (Sec. 3.2), textbook block
        ILU(0), GMRES(m), BiCGSTAB, BSR helpers.
sim     the Newton linearise-decouple-solve-update step with the paper's
        saturation safeguard (Sec. 2.2, "Phase Equilibrium"), the time step loop
        and the initial-state recipe.
cpr     the CPR-PF two-stage preconditioner (Sec. 4, Example 2): aggregation
        multigrid on the decoupled pressure matrix, then block ILU(0).
adjoint the tangent-linear model of the time loop's cumulative oil production
        (sensitivities; not in the paper).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
values printed in the paper, closed forms, invariants or library routines,
except the full combustion-tube trajectory, which is "parity unpinned" beyond
those invariants (the paper's STARS comparison exists only as figures).
"""
