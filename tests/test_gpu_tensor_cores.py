"""Spectral contractions of the FP32 operator on the tensor cores (tcgen05 kind::tf32, 3xTF32 split,
FP32 accumulation) against the FP64 oracle, the CUDA-core FP32 kernels and the FP64 GPU path.

The bar is the FP32 operator's: 2e-5 of the largest entry in the scaled norm (|y| / tau, tau the
order scale (k R / 2)^|n| / |n|!).  The cases cover one particle, quadrature rules whose node count
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


def scaled_err(got, want, wl):
    t = tau(wl)
    return (np.abs(got - want) / t).max() / (np.abs(want) / t).max()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


CASES = [
    # (seed, M, p, nrhs, omega, n_panels, nodes_per_panel)
    (51, 1, 3, 1, 2.0, 32, 16),      # one particle: the reflected self term only
    (52, 7, 6, 3, 2.5, 5, 7),        # N_S = 35 nodes: ragged last K chunk of S2L, ragged node tile of M2S
    (53, 20, 10, 64, 3.0, 32, 16),   # full 64-column block; 420 rows: ragged 256-row S2L tile
    (54, 150, 8, 17, 3.0, 20, 16),   # 2550 rows: two M2S K splits; 17 columns
]


@pytest.mark.parametrize("seed,M,p,nrhs,omega,npan,npp", CASES)
def test_reflected_part_fp32_tensor_cores_matches_oracle(seed, M, p, nrhs, omega, npan, npp):
    wl = syn.small_case(seed, M, p, omega=omega, nrhs=nrhs, n_panels=npan, nodes_per_panel=npp,
                        box=(-8.0, 8.0, -6.0, -1.0))
    ref = system.Problem(wl)
    x = syn.random_coeffs(seed + 3, M, p, nrhs)
    want = ref.apply_S(ref.reflect(x))
    s = P.Solver.from_workload(wl, tensor_cores=True)
    got = s.operator(dev(x), P.MS_PART_R | P.MS_PART_S, prec=P.MS_PREC_FP32).cpu().numpy()
    assert scaled_err(got, want, wl) <= 2e-5


def test_tensor_cores_and_cuda_cores_agree_with_fp64():
    wl = syn.config3(M=600, nrhs=64)
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
    wl = syn.small_case(71, M, 7, omega=2.5, nrhs=nrhs, box=(-10.0, 10.0, -9.0, -1.0), rmin=0.2, rmax=0.35)
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
