"""The launch-shape autotuner (ms_autotune): it picks among the candidate FMM leaf levels and
multipole-to-Sommerfeld split sizes, the tuned handle still applies the same operator (FMM against the
direct sum, FP32 on the tensor cores within the 3xTF32 bar), and a second handle of the same sizes
adopts the cached choice."""
import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402
from test_gpu_tensor_cores import TC_BAR, scaled_err  # noqa: E402


def test_autotune_keeps_the_operator_and_caches_its_choice():
    wl = syn.config3_discs(M=2500, nrhs=16)
    s = P.Solver.from_workload(wl)
    leaf, rows, ms = s.autotune(16, P.MS_PREC_FP32)
    print(f"autotune: leaf target {leaf}, {rows} rows per split, {ms:.2f} ms per application")
    assert rows in (1024, 2048, 4096, 8192) and leaf >= 1 and ms > 0 and s.fmm_levels >= 2
    x = torch.as_tensor(syn.random_coeffs(981, wl.M, wl.p, 16), device="cuda")
    direct = P.Solver.from_workload(wl, use_fmm=False).apply(x, prec=P.MS_PREC_FP64).cpu().numpy()
    assert scaled_err(s.apply(x, prec=P.MS_PREC_FP64).cpu().numpy(), direct, wl) <= 1e-11
    assert scaled_err(s.apply(x, prec=P.MS_PREC_FP32).cpu().numpy(), direct, wl) <= TC_BAR
    s2 = P.Solver.from_workload(wl)
    leaf2, rows2, _ = s2.autotune(16, P.MS_PREC_FP32)
    assert (leaf2, rows2) == (leaf, rows)


@pytest.mark.parametrize("prec", [P.MS_PREC_FP32, P.MS_PREC_BF16])
def test_tensor_peak_microkernel(prec):
    """The project tcgen05 rate kernel: a positive, repeatable rate, bf16 about twice tf32 per flop."""
    tf1, _ = P.tensor_peak(prec, 20000)
    tf2, _ = P.tensor_peak(prec, 20000)
    print(f"tensor peak, {'tf32' if prec == P.MS_PREC_FP32 else 'bf16'}: {tf1:.1f} / {tf2:.1f} TFLOP/s")
    assert tf1 > 50 and abs(tf1 - tf2) <= 0.2 * max(tf1, tf2)
