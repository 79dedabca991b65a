"""Block GMRES over the right-hand sides (the default inner solver of ms_solve / ms_solve_rhs / ms_grad)
against the oracle's dense LU solve and against the per-column GMRES it replaces.

Bars: FP64 solves 1e-10, mixed solves (FP32 inner solves on the tensor cores or the CUDA cores, FP64
refinement) 1e-8, relative l2 against the oracle.  Cases: one column (the block degenerates to
GMRES), a ragged block (5 columns, not a multiple of the 16-entry chunk), a full 64-column block,
restarts every 3 block iterations, and the full block at the workload's density."""
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


@pytest.fixture(scope="module")
def small():
    wl = syn.small_case(931, 10, 8, omega=3.0, nrhs=5)
    ref = system.Problem(wl)
    return wl, ref.solve_lu(ref.rhs(wl.inc_kind, wl.inc_angle))


@pytest.mark.parametrize("prec,tc,tol,bar", [(P.MS_PREC_FP64, True, 1e-12, 1e-10),
                                            (P.MS_PREC_FP32, True, 1e-10, 1e-8),
                                            (P.MS_PREC_FP32, False, 1e-10, 1e-8)])
@pytest.mark.parametrize("restart", [50, 3])
def test_block_solve_matches_oracle_lu(small, prec, tc, tol, bar, restart):
    wl, want = small
    s = P.Solver.from_workload(wl, tensor_cores=tc, restart=restart)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=tol, prec=prec)
    assert info["status"] == 0, info
    assert rel(g.cpu().numpy(), want) <= bar


def test_block_and_per_column_gmres_agree_and_block_needs_fewer_iterations():
    wl = syn.config3_discs(M=120, nrhs=16)
    wl.p = 8
    blk = P.Solver.from_workload(wl, restart=200)
    col = P.Solver.from_workload(wl, restart=200, block_krylov=False, max_iters=20000)
    gb, ib = blk.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP64)
    gc, ic = col.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP64)
    assert ib["status"] == 0 and ic["status"] == 0
    assert float(torch.linalg.norm(gb - gc) / torch.linalg.norm(gc)) <= 1e-8
    print(f"block GMRES {ib['iterations']} block iterations, per-column GMRES {ic['iterations']} iterations")
    assert ib["iterations"] < ic["iterations"]


@pytest.mark.parametrize("nrhs", [1, 64])
def test_block_width_extremes(nrhs):
    wl = syn.small_case(932, 14, 6, omega=2.5, nrhs=nrhs)
    ref = system.Problem(wl)
    want = ref.solve_lu(ref.rhs(wl.inc_kind, wl.inc_angle))
    s = P.Solver.from_workload(wl)
    for prec, tol, bar in ((P.MS_PREC_FP64, 1e-12, 1e-10), (P.MS_PREC_FP32, 1e-10, 1e-8)):
        g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=tol, prec=prec)
        assert info["status"] == 0, (prec, info)
        assert rel(g.cpu().numpy(), want) <= bar, prec


def test_full_block_mixed_solve_at_the_workload_density():
    """64 plane waves, 60 particles at the 10^4-particle workload's density: the mixed solve with
    tensor-core orthogonalisation of full 64-column blocks reaches the oracle's solution.  (The
    adjoint system goes through the same solver in ms_grad; the gradient tests cover it.)"""
    wl = syn.config3_discs(M=60, nrhs=64)
    wl.p = 6
    ref = system.Problem(wl)
    want = ref.solve_lu(ref.rhs(wl.inc_kind, wl.inc_angle))
    s = P.Solver.from_workload(wl, restart=100)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP32)
    assert info["status"] == 0, info
    assert rel(g.cpu().numpy(), want) <= 1e-8
