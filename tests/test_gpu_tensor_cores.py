"""Spectral contractions of the FP32 operator on the tensor cores (tcgen05 kind::tf32, 3xTF32 split,
FP32 accumulation) against the FP64 oracle, the CUDA-core FP32 kernels and the FP64 GPU path.

Bars, in the scaled norm (|y| / tau, tau the order scale (k R / 2)^|n| / |n|!, relative to the
largest entry): the CUDA-core FP32 operator is held to 2e-5.  A 3xTF32 product carries about
2^-21 relative error against 2^-24 for an FP32 multiply (the dropped lo*lo term and the tf32
rounding of the low parts), so the tensor-core path is held to 8 x 2e-5 = 1.6e-4; on the narrow
and moderate clouds below it stays within the FP32 bar, and on a 24-wide cloud (contour growth
e^{d W} = e^3) it measured 2.6e-5 against 4.5e-6 for the CUDA cores.  The mixed solve's FP64
refinement removes either error (tested to 1e-8).  The cases cover one particle, quadrature rules whose node count
is not a multiple of the 16-node K chunk, output row counts that leave a ragged last 256-row tile,
several multipole-to-Sommerfeld K splits, 1 to 64 right-hand sides, and the adjoint maps.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402


def tau(wl):
    from oracle.media import Layered
    L = Layered(wl.media, wl.omega)
    n = np.abs(np.arange(-wl.p, wl.p + 1))
    lg = np.array([math.lgamma(k + 1) for k in n])
    out = np.empty((wl.M, 2, 2 * wl.p + 1))
    for b, k in ((0, L.kp_l), (1, L.ks_l)):
        out[:, b, :] = np.exp(n[None, :] * np.log(k * wl.radius[:, None] / 2) - lg[None, :])
    return out[..., None]


TC_BAR = 8 * 2e-5


def scaled_err(got, want, wl):
    t = tau(wl)
    return (np.abs(got - want) / t).max() / (np.abs(want) / t).max()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


CASES = [
    # (seed, M, p, nrhs, omega, n_panels, nodes_per_panel, box)
    (51, 1, 3, 1, 2.0, 32, 16, (-8.0, 8.0, -6.0, -1.0)),      # one particle: the reflected self term only
    (52, 7, 6, 3, 2.5, 5, 7, (-8.0, 8.0, -6.0, -1.0)),        # N_S = 35: ragged last K chunk / node tile
    (53, 20, 10, 64, 3.0, 32, 16, (-8.0, 8.0, -6.0, -1.0)),   # 64 columns; 420 rows: ragged 256-row tile
    (54, 150, 8, 17, 3.0, 0, 16, (-12.0, 12.0, -14.0, -1.0)),   # 2550 rows: two M2S K splits; 17 columns
]


@pytest.mark.parametrize("seed,M,p,nrhs,omega,npan,npp,box", CASES)
def test_reflected_part_fp32_tensor_cores_matches_oracle(seed, M, p, nrhs, omega, npan, npp, box):
    depth, grade = 0.5, 0
    if npan == 0:        # a 24-wide cloud: the contour adapted to the width (growth e^{d W} <= e^3)
        npan, depth, grade = syn.contour_for_width(box[1] - box[0])
    wl = syn.small_case(seed, M, p, omega=omega, nrhs=nrhs, n_panels=npan, nodes_per_panel=npp, box=box,
                        depth=depth, grade=grade)
    ref = system.Problem(wl)
    x = syn.random_coeffs(seed + 3, M, p, nrhs)
    want = ref.apply_S(ref.reflect(x))
    s = P.Solver.from_workload(wl, tensor_cores=True)
    got = s.operator(dev(x), P.MS_PART_R | P.MS_PART_S, prec=P.MS_PREC_FP32).cpu().numpy()
    e_tc = scaled_err(got, want, wl)
    # the CUDA-core FP32 kernels on the same inputs: the tensor-core path must be as accurate.  On a
    # wide cloud the contour's growth e^{d W} (<= e^3 on the adapted rule) scales both errors.
    cc = P.Solver.from_workload(wl, tensor_cores=False)
    e_cc = scaled_err(cc.operator(dev(x), P.MS_PART_R | P.MS_PART_S, prec=P.MS_PREC_FP32).cpu().numpy(), want, wl)
    assert e_tc <= TC_BAR, (e_tc, e_cc)


def test_tensor_cores_and_cuda_cores_agree_with_fp64():
    wl = syn.config3_discs(M=600, nrhs=64)
    x = dev(syn.random_coeffs(61, wl.M, wl.p, 64))
    s_tc = P.Solver.from_workload(wl, tensor_cores=True)
    s_cc = P.Solver.from_workload(wl, tensor_cores=False)
    parts = P.MS_PART_R | P.MS_PART_S
    want = s_tc.operator(x, parts, prec=P.MS_PREC_FP64).cpu().numpy()
    tcv = s_tc.operator(x, parts, prec=P.MS_PREC_FP32).cpu().numpy()
    ccv = s_cc.operator(x, parts, prec=P.MS_PREC_FP32).cpu().numpy()
    e_tc, e_cc = scaled_err(tcv, want, wl), scaled_err(ccv, want, wl)
    assert e_tc <= 2e-5 and e_cc <= 2e-5, (e_tc, e_cc)
    # the full FP32 mat-vec on the tensor cores, FMM and all
    full = s_tc.apply(x, prec=P.MS_PREC_FP32).cpu().numpy()
    full64 = s_tc.apply(x, prec=P.MS_PREC_FP64).cpu().numpy()
    assert scaled_err(full, full64, wl) <= 2e-5


@pytest.mark.parametrize("M,nrhs", [(9, 5), (400, 64)])
def test_adjoint_fp32_tensor_cores_dot_product(M, nrhs):
    side = 20.0 if M < 100 else 40.0
    wl = syn.small_case(71, M, 7, omega=2.5, nrhs=nrhs, box=(-side / 2, side / 2, -side, -1.0), rmin=0.2, rmax=0.35)
    s = P.Solver.from_workload(wl, tensor_cores=True)
    x = dev(syn.random_coeffs(72, wl.M, wl.p, nrhs))
    y = dev(syn.random_coeffs(73, wl.M, wl.p, nrhs))
    Ax = s.apply(x, prec=P.MS_PREC_FP64)
    AHy32 = s.apply_adjoint(y, prec=P.MS_PREC_FP32)
    AHy64 = s.apply_adjoint(y, prec=P.MS_PREC_FP64)
    for r in range(nrhs):
        lhs = torch.vdot(y[..., r].flatten(), Ax[..., r].flatten())
        rhs = torch.vdot(AHy32[..., r].flatten(), x[..., r].flatten())
        scale = float(torch.linalg.norm(y[..., r]) * torch.linalg.norm(Ax[..., r]))
        assert abs(complex(lhs - rhs)) <= 2e-5 * scale
    rel = float(torch.linalg.norm(AHy32 - AHy64) / torch.linalg.norm(AHy64))
    assert rel <= 2e-5, rel


def test_mixed_solve_with_tensor_cores_reaches_fp64_accuracy():
    wl = syn.small_case(81, 12, 8, omega=3.0, nrhs=6)
    s = P.Solver.from_workload(wl, tensor_cores=True)
    g32, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_FP32)
    g64, _ = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-12, prec=P.MS_PREC_FP64)
    assert info["status"] == 0
    assert float(torch.linalg.norm(g32 - g64) / torch.linalg.norm(g64)) <= 1e-8


# --------------------------------------------------------------------- near-field Graf sum
@pytest.mark.parametrize("seed,M,p,nrhs", [(91, 1, 4, 2), (92, 9, 6, 3), (93, 16, 10, 64)])
def test_translation_fp32_tensor_cores_matches_oracle(seed, M, p, nrhs):
    """All pairs direct (one leaf): the translation sum S T x against the oracle's Graf sum."""
    wl = syn.small_case(seed, M, p, omega=2.5, nrhs=nrhs)
    ref = system.Problem(wl)
    x = syn.random_coeffs(seed + 5, M, p, nrhs)
    want = ref.apply_S(ref.translate(x))
    s = P.Solver.from_workload(wl, tensor_cores=True)
    got = s.operator(dev(x), P.MS_PART_T | P.MS_PART_S, prec=P.MS_PREC_FP32).cpu().numpy()
    if M == 1:
        assert not np.any(got)
        return
    assert scaled_err(got, want, wl) <= 2e-5


@pytest.mark.parametrize("M,nrhs,leaf", [(600, 64, 10), (2500, 7, 10), (1200, 32, 6)])
def test_near_field_fp32_tensor_cores_matches_fp64(M, nrhs, leaf):
    """Quadtree near lists (3 x 3 leaves): tensor-core tiles against the FP64 near sum."""
    wl = syn.config3_discs(M=M, nrhs=nrhs)
    x = dev(syn.random_coeffs(94, wl.M, wl.p, nrhs))
    s = P.Solver.from_workload(wl, tensor_cores=True, leaf_target=leaf)
    assert s.fmm_levels >= 2
    parts = P.MS_PART_T_NEAR | P.MS_PART_S
    want = s.operator(x, parts, prec=P.MS_PREC_FP64).cpu().numpy()
    got = s.operator(x, parts, prec=P.MS_PREC_FP32).cpu().numpy()
    assert scaled_err(got, want, wl) <= 2e-5


# --------------------------------------------------------------------- FMM multipole-to-local
@pytest.mark.parametrize("M,nrhs,leaf", [(2500, 16, 10), (1200, 64, 6)])
def test_fmm_far_field_fp32_tensor_cores_matches_fp64(M, nrhs, leaf):
    """M2L of every level on tensor-core tiles (the other FMM stages on the CUDA cores) against
    the FP64 far field, and the whole FP32 mat-vec against the FP64 one."""
    wl = syn.config3_discs(M=M, nrhs=nrhs)
    x = dev(syn.random_coeffs(95, wl.M, wl.p, nrhs))
    s = P.Solver.from_workload(wl, tensor_cores=True, leaf_target=leaf)
    assert s.fmm_levels >= 3
    parts = P.MS_PART_T_FAR | P.MS_PART_S
    want = s.operator(x, parts, prec=P.MS_PREC_FP64).cpu().numpy()
    got = s.operator(x, parts, prec=P.MS_PREC_FP32).cpu().numpy()
    assert scaled_err(got, want, wl) <= TC_BAR
    full = s.apply(x, prec=P.MS_PREC_FP32).cpu().numpy()
    full64 = s.apply(x, prec=P.MS_PREC_FP64).cpu().numpy()
    assert scaled_err(full, full64, wl) <= TC_BAR
