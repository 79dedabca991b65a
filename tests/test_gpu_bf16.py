"""The BF16-split precision variant (MS_PREC_BF16): the tensor-core contractions of the operator on bf16
hi/lo operands, three products, FP32 accumulation; everything else as the FP32 path.

Bar: the CUDA-core FP32 operator is held to 2e-5 in the scaled norm (sums of ~10^3 products with
2^-24 relative rounding); a 3-product bf16 split carries about 2^-16 relative error per product,
2^8 times more, so the BF16 operator is held to 256 x 2e-5 = 5e-3 (measured errors are printed).  The
mixed solve's FP64 refinement removes that error: BF16 solves are held to the same 1e-8 as FP32 ones."""
import numpy as np
import pytest

import synthetic as syn
from oracle import nystrom, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402
from paper_2608_26875_b300 import _native as nat  # noqa: E402
from test_gpu_tensor_cores import scaled_err  # noqa: E402

BF16_BAR = 256 * 2e-5


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("parts", ["near", "far", "refl", "all"])
def test_bf16_operator_parts_against_fp64(parts):
    wl = syn.config3_discs(M=600, nrhs=64)
    x = dev(syn.random_coeffs(951, wl.M, wl.p, 64))
    s = P.Solver.from_workload(wl, leaf_target=6)
    sel = {"near": P.MS_PART_T_NEAR | P.MS_PART_S, "far": P.MS_PART_T_FAR | P.MS_PART_S,
           "refl": P.MS_PART_R | P.MS_PART_S}
    if parts == "all":
        want = s.apply(x, prec=P.MS_PREC_FP64).cpu().numpy()
        got = s.apply(x, prec=P.MS_PREC_BF16).cpu().numpy()
        tf = s.apply(x, prec=P.MS_PREC_FP32).cpu().numpy()
    else:
        want = s.operator(x, sel[parts], prec=P.MS_PREC_FP64).cpu().numpy()
        got = s.operator(x, sel[parts], prec=P.MS_PREC_BF16).cpu().numpy()
        tf = s.operator(x, sel[parts], prec=P.MS_PREC_FP32).cpu().numpy()
    e, e32 = scaled_err(got, want, wl), scaled_err(tf, want, wl)
    print(f"BF16-split {parts}: scaled error {e:.3e} (3xTF32 {e32:.3e})")
    assert e <= BF16_BAR
    if parts == "near":
        # the near part is all tensor-core contraction, so the coarser split shows; the far and reflected
        # parts' error is set by their FP32 CUDA-core stages and FP32 tables, the same for both splits
        assert e > e32


def test_bf16_star_apply_against_oracle():
    wl = syn.config3(M=60, nrhs=16, Q=2)
    tabs = nystrom.workload_tables(wl)
    ref = system.Problem(wl, proto_S=tabs)
    x = syn.random_coeffs(952, wl.M, wl.p, 16)
    want = ref.matvec(x)
    s = P.Solver.from_workload(wl, proto_S=tabs)
    e = scaled_err(s.apply(dev(x), prec=P.MS_PREC_BF16).cpu().numpy(), want, wl)
    print(f"BF16-split apply with stars: scaled error {e:.3e}")
    assert e <= BF16_BAR


def test_bf16_mixed_solve_reaches_the_oracle_solution():
    wl = syn.small_case(953, 12, 8, omega=3.0, nrhs=6)
    ref = system.Problem(wl)
    want = ref.solve_lu(ref.rhs(wl.inc_kind, wl.inc_angle))
    s = P.Solver.from_workload(wl)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-10, prec=P.MS_PREC_BF16)
    assert info["status"] == 0 and info["refinements"] >= 1, info
    assert np.linalg.norm(g.cpu().numpy() - want) / np.linalg.norm(want) <= 1e-8


def test_bf16_adjoint_dot_product():
    wl = syn.small_case(954, 9, 7, omega=2.5, nrhs=5)
    s = P.Solver.from_workload(wl)
    x = dev(syn.random_coeffs(955, wl.M, wl.p, 5))
    y = dev(syn.random_coeffs(956, wl.M, wl.p, 5))
    Ax = s.apply(x, prec=P.MS_PREC_FP64)
    AHy = s.apply_adjoint(y, prec=P.MS_PREC_BF16)
    for r in range(5):
        lhs = torch.vdot(y[..., r].flatten(), Ax[..., r].flatten())
        rhs = torch.vdot(AHy[..., r].flatten(), x[..., r].flatten())
        scale = float(torch.linalg.norm(y[..., r]) * torch.linalg.norm(Ax[..., r]))
        assert abs(complex(lhs - rhs)) <= BF16_BAR * scale


def test_bf16_needs_the_tensor_cores():
    wl = syn.small_case(957, 4, 5, omega=2.0, nrhs=1)
    s = P.Solver.from_workload(wl, tensor_cores=False)
    with pytest.raises(P.MsError) as e:
        s.apply(dev(syn.random_coeffs(958, wl.M, wl.p, 1)), prec=P.MS_PREC_BF16)
    assert e.value.status == nat.MS_ERR_UNSUPPORTED
