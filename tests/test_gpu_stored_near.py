"""Stored near-pair operator (ms_options.store_near): the 3xTF32 tensor-core tiles of the near-field
Graf sum (Sec. 4.2) are generated once at setup and streamed from device memory by the bulk-copy
pipeline in every application.  The multiplies see the same operand bits in the same order as the
generating kernel, so every FP32 result is bitwise equal to the generated path's; the FP64 and BF16
paths do not use the stored tiles at all."""
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
def pair():
    wl = syn.config3_discs(M=600, nrhs=8)
    wl.p = 8
    s = P.Solver.from_workload(wl, store_near=4)
    g = P.Solver.from_workload(wl)
    return wl, s, g


def test_tiles_are_stored_within_the_budget(pair):
    wl, s, g = pair
    nb = s.near_stored_bytes()
    assert nb > 0 and nb <= 4e9
    assert g.near_stored_bytes() == 0
    # every near tile stores (n rows rounded to 16) x (chunks of 32 real K) x 4 bytes x hi, lo, per wave
    nc = 2 * wl.p + 1
    assert nb % (2 * 2 * 16 * 32 * 4) == 0
    # at least the near pairs' own operator: per ordered pair and wave nc rows x 2 nc real K entries,
    # 4 bytes, hi and lo
    assert s.near_pairs > 0
    assert nb >= 2 * s.near_pairs * nc * (2 * nc) * 4 * 2


@pytest.mark.parametrize("nrhs", [1, 7, 64])
def test_stored_apply_is_bitwise_equal_to_generated(pair, nrhs):
    wl, s, g = pair
    x = dev(syn.random_coeffs(1200 + nrhs, wl.M, wl.p, nrhs))
    assert torch.equal(s.operator(x, P.MS_PART_T_NEAR, prec=P.MS_PREC_FP32),
                       g.operator(x, P.MS_PART_T_NEAR, prec=P.MS_PREC_FP32))
    assert torch.equal(s.apply(x, prec=P.MS_PREC_FP32), g.apply(x, prec=P.MS_PREC_FP32))
    for prec in (P.MS_PREC_FP64, P.MS_PREC_BF16):
        assert torch.equal(s.apply(x, prec=prec), g.apply(x, prec=prec))
    assert torch.equal(s.apply_adjoint(x, prec=P.MS_PREC_FP32), g.apply_adjoint(x, prec=P.MS_PREC_FP32))


def test_stored_solve_matches_generated(pair):
    """A capped mixed solve: the same iterates, status and bits from the stored and generated tiles."""
    wl = pair[0]
    s = P.Solver.from_workload(wl, store_near=4, max_iters=40)
    g = P.Solver.from_workload(wl, max_iters=40)
    a, ia = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP32)
    b, ib = g.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP32)
    assert ia["status"] == ib["status"]
    assert ia["iterations"] == ib["iterations"]
    assert torch.equal(a, b)


def test_budget_below_the_tiles_leaves_them_generated():
    wl = syn.config3_discs(M=3000, nrhs=4)
    wl.p = 12
    s = P.Solver.from_workload(wl, store_near=1)
    big = P.Solver.from_workload(wl, store_near=64)
    nb = big.near_stored_bytes()
    assert nb > 1e9                      # the 1 GB budget is too small for these tiles
    assert s.near_stored_bytes() == 0
    x = dev(syn.random_coeffs(1300, wl.M, wl.p, 4))
    assert torch.equal(s.operator(x, P.MS_PART_T_NEAR, prec=P.MS_PREC_FP32),
                       big.operator(x, P.MS_PART_T_NEAR, prec=P.MS_PREC_FP32))


def test_autotune_rebuilds_the_stored_tiles():
    wl = syn.config3_discs(M=800, nrhs=4)
    wl.p = 8
    s = P.Solver.from_workload(wl, store_near=4)
    leaf, rows, _ = s.autotune(nrhs=16, prec=P.MS_PREC_FP32)
    assert s.near_stored_bytes() > 0
    ref = P.Solver.from_workload(wl, leaf_target=leaf)
    x = dev(syn.random_coeffs(1400, wl.M, wl.p, 16))
    assert torch.equal(s.operator(x, P.MS_PART_T_NEAR, prec=P.MS_PREC_FP32),
                       ref.operator(x, P.MS_PART_T_NEAR, prec=P.MS_PREC_FP32))


def test_stored_pipeline_reports_a_timeout():
    """The stored-tile kernel takes the same bounded-wait failure path (test hook: every CTA waits,
    bounded, on a barrier that nothing arrives at) and the call returns MS_ERR_TIMEOUT."""
    wl = syn.config3_discs(M=300, nrhs=2)
    wl.p = 6
    s = P.Solver.from_workload(wl, store_near=2, tc_wait_test=500)
    assert s.near_stored_bytes() > 0
    x = dev(syn.random_coeffs(1500, wl.M, wl.p, 2))
    with pytest.raises(P.MsError) as e:
        s.operator(x, P.MS_PART_T_NEAR, prec=P.MS_PREC_FP32)
    assert e.value.status == nat.MS_ERR_TIMEOUT
