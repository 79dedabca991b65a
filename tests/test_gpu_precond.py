"""Group-block Jacobi preconditioner (ms_options.precond_group): right preconditioning of the block
GMRES with the inverses of I - S~ T~ over groups of nearby particles.  The preconditioned solves reach
the oracle's dense-LU solution to the solver bars (FP64 1e-10, mixed 1e-8) for discs and for star
prototypes, in fewer block iterations than the unpreconditioned ones, and the adjoint system (through
ms_grad) gives the same gradient."""
import numpy as np
import pytest

import synthetic as syn
from oracle import system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402


def rel(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


@pytest.mark.parametrize("group", [3, 8, 64])
def test_preconditioned_solve_matches_oracle_lu(group):
    wl = syn.small_case(941, 24, 6, omega=3.0, nrhs=7)
    ref = system.Problem(wl)
    want = ref.solve_lu(ref.rhs(wl.inc_kind, wl.inc_angle))
    s = P.Solver.from_workload(wl, precond_group=group)
    for prec, tol, bar in ((P.MS_PREC_FP64, 1e-12, 1e-10), (P.MS_PREC_FP32, 1e-10, 1e-8),
                           (P.MS_PREC_BF16, 1e-10, 1e-8)):
        g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=tol, prec=prec)
        assert info["status"] == 0, (prec, info)
        assert rel(g.cpu().numpy(), want) <= bar, prec


def test_preconditioner_cuts_block_iterations_at_the_workload_density():
    wl = syn.config3_discs(M=400, nrhs=32)
    wl.p = 8
    plain = P.Solver.from_workload(wl, restart=300)
    pre = P.Solver.from_workload(wl, restart=300, precond_group=12)
    a, ia = plain.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP64)
    b, ib = pre.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP64)
    assert ia["status"] == 0 and ib["status"] == 0
    print(f"block GMRES iterations: {ia['iterations']} plain, {ib['iterations']} with 12-particle groups")
    assert ib["iterations"] < ia["iterations"]
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) <= 1e-8
    c, ic = pre.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP32)
    assert ic["status"] == 0
    assert float(torch.linalg.norm(c - a) / torch.linalg.norm(a)) <= 1e-8


def test_full_block_of_dependent_columns_converges():
    """64 plane waves on a system of 364 unknowns: the block Krylov space closes after a few block
    iterations and the residual blocks become rank-deficient; the solver deflates them and converges."""
    wl = syn.small_case(932, 14, 6, omega=2.5, nrhs=64)
    ref = system.Problem(wl)
    want = ref.solve_lu(ref.rhs(wl.inc_kind, wl.inc_angle))
    for group in (0, 6):
        s = P.Solver.from_workload(wl, precond_group=group)
        for prec, tol, bar in ((P.MS_PREC_FP64, 1e-12, 1e-10), (P.MS_PREC_FP32, 1e-10, 1e-8)):
            g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=tol, prec=prec)
            assert info["status"] == 0, (group, prec, info)
            assert rel(g.cpu().numpy(), want) <= bar, (group, prec)


def test_preconditioned_gradient_matches_plain():
    """ms_grad solves the forward system and the adjoint one (A~^H, preconditioned by P^{-H})."""
    wl = syn.config3_discs(M=120, nrhs=4)
    wl.p = 6
    rx = np.stack([np.linspace(-8, 8, 16), np.full(16, -0.5)], axis=1)
    rng = np.random.default_rng(5)
    w = torch.as_tensor(rng.normal(size=(wl.nrhs, 16, 2)) + 1j * rng.normal(size=(wl.nrhs, 16, 2)), device="cuda")
    out = []
    for group in (0, 10):
        s = P.Solver.from_workload(wl, precond_group=group)
        g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP64)
        assert info["status"] == 0, (group, info)
        gc, gr, go, gi = s.grad(wl.inc_kind, wl.inc_angle, g, w, rx, tol=1e-9, prec=P.MS_PREC_FP64)
        assert gi["status"] == 0, (group, gi)
        out.append((gc.cpu().numpy(), gr.cpu().numpy(), go))
    for a, b in zip(out[0][:2], out[1][:2]):
        assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(a)
    assert abs(out[0][2] - out[1][2]) <= 1e-7 * abs(out[0][2])
