"""Failure paths of the library on a GPU, each made to happen without a fault: a tensor-core wait
that runs out (the test hook ms_options.tc_wait_test makes every CTA wait, bounded, on a barrier that
nothing arrives at), a non-finite right-hand side, and an iteration cap that is too small.  After each,
the context stays usable and a normal call on the same device gives the right answer.  Also the
initial guess of ms_solve_rhs."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402
from paper_2608_26875_b300 import _native as nat  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.fixture(scope="module")
def case():
    wl = syn.small_case(901, 12, 8, omega=3.0, nrhs=4)
    return wl, dev(syn.random_coeffs(902, wl.M, wl.p, 4))


def test_tensor_core_wait_that_runs_out_reports_timeout(case):
    wl, x = case
    hooked = P.Solver.from_workload(wl, tensor_cores=True, tc_wait_test=2000)    # 2 ms per CTA
    with pytest.raises(P.MsError) as e:
        hooked.apply(x, prec=P.MS_PREC_FP32)
    assert e.value.status == nat.MS_ERR_TIMEOUT
    # the flag was read and cleared: the FP64 operator (no tensor-core kernels) still runs on the handle
    y64 = hooked.apply(x, prec=P.MS_PREC_FP64)
    # the context is usable: a normal handle on the same device gives the FP32 result
    good = P.Solver.from_workload(wl, tensor_cores=True)
    y32 = good.apply(x, prec=P.MS_PREC_FP32)
    assert float(torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64)) < 1e-5


def test_timeout_inside_a_solve_is_reported(case):
    wl, _ = case
    hooked = P.Solver.from_workload(wl, tensor_cores=True, tc_wait_test=500)
    with pytest.raises(P.MsError) as e:
        hooked.solve(wl.inc_kind, wl.inc_angle, tol=1e-8, prec=P.MS_PREC_FP32)
    assert e.value.status == nat.MS_ERR_TIMEOUT


@pytest.mark.parametrize("prec", [P.MS_PREC_FP64, P.MS_PREC_FP32])
def test_non_finite_right_hand_side_is_refused(case, prec):
    wl, _ = case
    s = P.Solver.from_workload(wl)
    b = s.rhs(wl.inc_kind, wl.inc_angle)
    b[3, 1, 2, 1] = complex(float("nan"), 0.0)
    with pytest.raises(P.MsError) as e:
        s.solve_rhs(b, tol=1e-10, prec=prec)
    assert e.value.status == nat.MS_ERR_NONFINITE


def test_iteration_cap_returns_not_converged_with_residuals(case):
    wl, _ = case
    s = P.Solver.from_workload(wl, max_iters=3)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-12, prec=P.MS_PREC_FP64)
    assert info["status"] == nat.MS_NOT_CONVERGED
    assert info["iterations"] <= 3 and info["max_rel_residual"] > 1e-12
    assert torch.isfinite(torch.view_as_real(g)).all()


def test_solve_rhs_matches_solve_and_uses_the_initial_guess(case):
    wl, _ = case
    s = P.Solver.from_workload(wl)
    g1, _ = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-12, prec=P.MS_PREC_FP64)
    b = s.rhs(wl.inc_kind, wl.inc_angle)
    g2, info2 = s.solve_rhs(b, tol=1e-12, prec=P.MS_PREC_FP64)
    assert float(torch.linalg.norm(g2 - g1) / torch.linalg.norm(g1)) < 1e-10
    # started from the solution, the refinement stops at its first residual check
    g3, info3 = s.solve_rhs(b, tol=1e-10, prec=P.MS_PREC_FP32, x0=g1)
    assert info3["status"] == 0 and info3["iterations"] == 0 and info3["refinements"] == 0
    assert float(torch.linalg.norm(g3 - g1) / torch.linalg.norm(g1)) < 1e-12
