"""Captured CUDA graphs of the operator (ms_options.cuda_graph, the default): replaying the captured
kernel sequence gives the same bits as plain launches, for every precision, part selection and the
adjoint, across repeated calls, interleaved column counts and a workspace that grows (which rebuilds
the graphs)."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.fixture(scope="module")
def pair():
    wl = syn.config3_discs(M=400, nrhs=8)
    wl.p = 8
    return wl, P.Solver.from_workload(wl, cuda_graph=True), P.Solver.from_workload(wl, cuda_graph=False)


@pytest.mark.parametrize("prec", [P.MS_PREC_FP64, P.MS_PREC_FP32, P.MS_PREC_BF16])
def test_graph_replay_is_bitwise_equal_to_plain_launches(pair, prec):
    wl, g, d = pair
    for nrhs, seed in ((4, 1), (16, 2), (4, 3), (16, 4)):        # the second 16 reuses the rebuilt graphs
        x = dev(syn.random_coeffs(970 + seed, wl.M, wl.p, nrhs))
        for _ in range(2):
            assert torch.equal(g.apply(x, prec=prec), d.apply(x, prec=prec))
            assert torch.equal(g.apply_adjoint(x, prec=prec), d.apply_adjoint(x, prec=prec))
        for parts in (P.MS_PART_T_NEAR | P.MS_PART_S, P.MS_PART_R, P.MS_PART_T_FAR):
            assert torch.equal(g.operator(x, parts, prec=prec), d.operator(x, parts, prec=prec))


def test_graph_solves_match_plain_solves(pair):
    """Same iterations, status and bits with and without graphs (a capped run: the replayed operator
    must not change a single iterate, converged or not)."""
    wl = pair[0]
    g = P.Solver.from_workload(wl, cuda_graph=True, max_iters=60)
    d = P.Solver.from_workload(wl, cuda_graph=False, max_iters=60)
    for prec, tol in ((P.MS_PREC_FP64, 1e-12), (P.MS_PREC_FP32, 1e-10)):
        a, ia = g.solve(wl.inc_kind, wl.inc_angle, tol=tol, prec=prec)
        b, ib = d.solve(wl.inc_kind, wl.inc_angle, tol=tol, prec=prec)
        assert ia["status"] == ib["status"]
        assert ia["iterations"] == ib["iterations"]
        assert torch.equal(a, b)
