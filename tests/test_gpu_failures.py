"""Failure paths of the solver, made on the host or by a bounded device wait.

No test faults, traps or hangs the GPU: bad inputs are rejected on the host, a
singular pivot is detected and reported, non-convergence is reported, and the
bounded wait of the preconditioner apply is made to run out by a test switch
(the copy engine issues nothing), after which the context is used again.
"""
import numpy as np
import pytest

import vesselmesh as vm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1810_04289_gb300 import fsi  # noqa: E402

MAT = dict(rho_f=1.05, mu_f=0.035, rho_s=1.2, E_s=3.0e6, nu_s=0.45, eta_s=0.0)


def tube():
    return vm.tube_config("tube-12x8x4")


def test_singular_pivot_is_reported():
    # a wall-tagged node that belongs to no tet has empty displacement rows:
    # its 7x7 pivot block is singular and the ILU reports it
    m = vm.box_mesh(1, 1.0, domain=1)
    m.tets = m.tets[:1].copy()
    m.tet_domain = m.tet_domain[:1].copy()      # tags kept from the 6-tet box on purpose
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=1))
    y = np.zeros((m.n_nodes, 7))
    S.set_state(y, t=0.0)
    S.jacobian(y)
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_pc_apply(S.ctx, S.vec(np.ones((m.n_nodes, 7))), S.vec())
    assert e.value.status == 5


def test_newton_iteration_limit_leaves_state_unchanged():
    m = tube()
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(newton_maxit=1, newton_rtol=1e-14, newton_atol=1e-300,
                                                   n_subdomains=4))
    y0 = vm.poiseuille_state(m)
    S.set_state(y0, t=0.0)
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_step(S.ctx)
    assert e.value.status == 7
    y, t = S.state()
    assert t == 0.0 and np.array_equal(y, y0)
    # the context still works
    S2 = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4))
    S2.set_state(y0, t=0.0)
    assert S2.step().converged == 1


def test_nonfinite_state_is_reported():
    m = tube()
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4))
    y0 = vm.poiseuille_state(m)
    y0[5, 2] = np.nan
    S.set_state(y0, t=0.0)
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_step(S.ctx)
    assert e.value.status == 10


def test_gmres_iteration_limit():
    m = tube()
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4, gmres_rtol=1e-12, gmres_maxit=3))
    y0 = vm.poiseuille_state(m)
    S.set_state(y0, t=0.0)
    S.jacobian(y0)
    F = S.vec(S.residual(y0))
    x = S.vec()
    st = fsi.fsi_linear_solve(S.ctx, F, x, raise_on_divergence=False)
    assert st.converged == 0 and st.rnorm < st.rnorm0
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_linear_solve(S.ctx, F, x)
    assert e.value.status == 6


def test_bounded_wait_runs_out_and_context_stays_usable():
    m = tube()
    y0 = vm.poiseuille_state(m)
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4, precision=1, fault_test=1))
    S.set_state(y0, t=0.0)
    S.jacobian(y0)
    r = S.vec(np.ones((m.n_nodes, 7)))
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_pc_apply(S.ctx, r, S.vec())
    assert e.value.status == 9
    # the device and the library are still usable afterwards
    T = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4, precision=1))
    T.set_state(y0, t=0.0)
    assert T.step().converged == 1


def test_state_checkpoint_resume_is_bitwise():
    m = tube()
    y0 = vm.poiseuille_state(m)
    A = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4))
    A.set_state(y0, t=0.0)
    A.step()
    A.step()
    ya, ta = A.state()
    # resume a fresh context from the checkpoint of step 1 and redo step 2
    B = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4))
    B.set_state(y0, t=0.0)
    B.step()
    y1, t1 = B.state()
    C = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4))
    C.set_state(y1, y0, y0, t=t1)
    C.step()
    yc, tc = C.state()
    assert tc == ta and np.array_equal(yc, ya)
