"""The benchmarked mat-vec at full size, in the launch configuration bench.py times: 10^4 particles
(half discs, half stars of 32 prototypes), p = 20, the adapted 4800-node contour, 64 right-hand sides
(bench.py's rank-0 input), FMM with 10 particles per leaf, FP32 operator on the tensor cores.  The
star tables are the oracle's Nystrom matrices.

* Sampled outputs (3 targets spread over the particle order, two of them stars, 3 of the 64 columns)
  against the FP64 oracle's mat-vec at those targets, for the FP64 GPU path (bar 1e-10, ten times the
  bar of the smaller FMM tests) and the FP32 tensor-core path.
* Every output of the FP32 tensor-core mat-vec against the FP64 GPU mat-vec.

FP32 bar: the tensor-core bar of the smaller cases, 1.6e-4 in the scaled norm (8 x the 2e-5 of FP32
on the CUDA cores, for the 2^-21 relative error of a 3xTF32 product against 2^-24).  The contractions
at full size are longer than in any smaller case (4800 nodes x 10^4 particles), but their error
grows like the square root of the length for independent roundings, and the measured errors are
printed so that the margin is on record.  Outputs must also be finite.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import nystrom, system
from oracle.media import Layered

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402

TARGETS = [0, 4321, 9999]
COLS = [0, 31, 63]
FULL_FP32_BAR = 1.6e-4


def tau(wl):
    """Order scale (k_b R_m / 2)^|n| / |n|! per (m, b, n): the natural size of outgoing coefficients."""
    L = Layered(wl.media, wl.omega)
    n = np.abs(np.arange(-wl.p, wl.p + 1))
    lg = np.array([math.lgamma(k + 1) for k in n])
    out = np.empty((wl.M, 2, 2 * wl.p + 1))
    for b, k in ((0, L.kp_l), (1, L.ks_l)):
        out[:, b, :] = np.exp(n[None, :] * np.log(k * wl.radius[:, None] / 2) - lg[None, :])
    return out[..., None]


def scaled_err(got, want, t):
    return (np.abs(got - want) / t).max() / (np.abs(want) / t).max()


def rel_l2(got, want):
    return np.linalg.norm(got - want) / np.linalg.norm(want)


@pytest.fixture(scope="module")
def full():
    wl = syn.config3()
    assert (wl.M, wl.p) == (10000, 20) and wl.proto[4321] >= 0 and wl.proto[9999] >= 0
    tabs = nystrom.workload_tables(wl)
    x = syn.random_coeffs(1000, wl.M, wl.p, 64)
    s = P.Solver.from_workload(wl, proto_S=tabs, leaf_target=10, tensor_cores=True)
    assert s.n_nodes == 4800 and s.fmm_levels >= 4
    xd = torch.as_tensor(x, device="cuda")
    y32 = s.apply(xd, prec=P.MS_PREC_FP32).cpu().numpy()
    y64 = s.apply(xd, prec=P.MS_PREC_FP64).cpu().numpy()
    s.close()
    del xd
    ref = system.Problem(wl, proto_S=tabs)
    want = ref.matvec(np.ascontiguousarray(x[..., COLS]), targets=TARGETS)
    return wl, y32, y64, want


def test_full_size_fp64_matches_oracle_on_sampled_targets(full):
    wl, _, y64, want = full
    got, t = y64[TARGETS][..., COLS], tau(wl)[TARGETS]
    assert rel_l2(got, want) <= 1e-10
    assert scaled_err(got, want, t) <= 1e-10


def test_full_size_fp32_tensor_cores_matches_oracle_on_sampled_targets(full):
    wl, y32, _, want = full
    got, t = y32[TARGETS][..., COLS], tau(wl)[TARGETS]
    e1, e2 = rel_l2(got, want), scaled_err(got, want, t)
    print(f"full size FP32 tensor cores vs oracle: relative l2 {e1:.3e}, scaled {e2:.3e}")
    assert e1 <= FULL_FP32_BAR and e2 <= FULL_FP32_BAR


def test_full_size_fp32_tensor_cores_matches_fp64_everywhere(full):
    wl, y32, y64, _ = full
    assert np.isfinite(y32).all() and np.isfinite(y64).all()
    e1, e2 = rel_l2(y32, y64), scaled_err(y32, y64, tau(wl))
    print(f"full size FP32 tensor cores vs FP64 everywhere: relative l2 {e1:.3e}, scaled {e2:.3e}")
    assert e1 <= FULL_FP32_BAR and e2 <= FULL_FP32_BAR


def test_fp32_far_field_on_the_physical_right_hand_side():
    """The FP32 FMM (5 levels, box orders up to a few hundred on the coarse levels) against the FP64 one
    on the plane-wave right-hand side b = S a0, whose coefficients follow the physical decay with the
    order -- the input the mixed solve's inner iterations see -- at the FP32 tensor-core bar."""
    wl = syn.config3_discs(M=10000, nrhs=8)
    s = P.Solver.from_workload(wl)
    assert s.fmm_levels >= 5
    b = s.rhs(wl.inc_kind[:8], wl.inc_angle[:8])
    y64 = s.operator(b, P.MS_PART_T_FAR, prec=P.MS_PREC_FP64)
    y32 = s.operator(b, P.MS_PART_T_FAR, prec=P.MS_PREC_FP32)
    e = float(torch.linalg.norm(y64 - y32) / torch.linalg.norm(y64))
    print(f"FP32 far field on b: relative error {e:.2e}")
    assert e <= FULL_FP32_BAR
