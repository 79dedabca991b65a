"""3D path (include/ms3_b300.h; Sec. 6) against the 3D oracle (oracle/layered3d.py) on the same polar
rule: the free-space translation (scalar addition theorem on the Cartesian components on the GPU,
projection on a sphere in the oracle), the interface-reflected part, the whole mat-vec, the plane-wave
right-hand side and the solve, for rigid and traction-free spheres; and sampled targets of the
500-sphere workload.  Bars: relative l2 1e-10 for the parts and the mat-vec (FP64 throughout), 1e-9
for the solve against the oracle's dense LU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import synthetic as syn  # noqa: E402
from oracle import layered3d as L3  # noqa: E402
from oracle import sph3d as S3  # noqa: E402

import paper_2608_26875_b300 as P  # noqa: E402
from paper_2608_26875_b300 import _native as nat  # noqa: E402

RULE = dict(n_r=32, n_theta=16, n_panels=2, t_max=12.0, alpha=0.5, beta=1.0)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def scaled_random(seed, M, p, nrhs):
    """Outgoing coefficients decaying with the order like the solutions do (0.3^n)."""
    rng = np.random.default_rng(seed)
    nmn, nl, tot = S3.sizes(p)
    n, _ = S3.orders(p)
    f = np.concatenate([0.3 ** n[1:], 0.3 ** n[1:], 0.3 ** n])
    return (rng.normal(size=(M, tot, nrhs)) + 1j * rng.normal(size=(M, tot, nrhs))) * f[None, :, None]


@pytest.fixture(scope="module", params=[4, 6])
def case(request):
    p = request.param
    wl = syn.spheres3d(M=5, seed=71, box=(-2.0, 2.0, -2.0, 2.0, -3.5, -1.0), bc="alternate")
    md = L3.Media3(wl.media.lam_u, wl.media.mu_u, wl.media.lam_l, wl.media.mu_l, wl.omega)
    ref = L3.Problem3(md, wl.centres, wl.radius, wl.bc, p, ntheta_proj=40, **RULE)
    gpu = P.Solver3(wl.centres, wl.radius, wl.bc, wl.media, wl.omega, p, **RULE)
    return wl, p, ref, gpu


def test_parts_and_matvec_match_oracle(case):
    wl, p, ref, gpu = case
    x = scaled_random(90 + p, wl.M, p, 3)
    xd = torch.as_tensor(x, device="cuda")
    t = gpu.operator(xd, nat.MS3_PART_T).cpu().numpy()
    assert rel(t, ref.translate(x)) <= 1e-10
    r = gpu.operator(xd, nat.MS3_PART_R).cpu().numpy()
    assert rel(r, ref.layered(x)) <= 1e-10
    y = gpu.apply(xd).cpu().numpy()
    assert rel(y, ref.matvec(x)) <= 1e-10


def test_rhs_and_solve_match_oracle(case):
    wl, p, ref, gpu = case
    kinds, th, ph = [0, 1, 2, 1], [0.3, 0.6, 0.2, 1.2], [0.1, 1.0, 2.5, -0.7]
    b = gpu.rhs(kinds, th, ph).cpu().numpy()
    want_b = ref.rhs(list(zip(kinds, th, ph)))
    assert rel(b, want_b) <= 1e-12
    g, info = gpu.solve(kinds, th, ph, tol=1e-12)
    assert info["status"] == 0, info
    want = ref.solve_lu(want_b)
    assert rel(g.cpu().numpy(), want) <= 1e-9
    gm, im = gpu.solve(kinds, th, ph, tol=1e-10, prec=P.MS_PREC_FP32)      # FP32 inner solves, FP64 refinement
    assert im["status"] == 0 and im["refinements"] >= 2, im
    assert rel(gm.cpu().numpy(), want) <= 1e-8


def test_fp32_operator_against_fp64(case):
    """The FP32 tables and arithmetic: relative l2 against the FP64 operator at the FP32 bar 2e-5 (FP32
    entries and accumulation; the coefficient block's orders span many decades, so the bar is on the
    whole block)."""
    wl, p, ref, gpu = case
    x = torch.as_tensor(scaled_random(300 + p, wl.M, p, 5), device="cuda")
    a = gpu.apply(x, prec=P.MS_PREC_FP64)
    b = gpu.apply(x, prec=P.MS_PREC_FP32)
    e = float(torch.linalg.norm(a - b) / torch.linalg.norm(a))
    print(f"3D FP32 operator p = {p}: relative error {e:.2e}")
    assert e <= 2e-5


def test_single_column_and_ragged_blocks(case):
    wl, p, ref, gpu = case
    for nrhs in (1, 17):
        x = scaled_random(200 + nrhs, wl.M, p, nrhs)
        y = gpu.apply(torch.as_tensor(x, device="cuda")).cpu().numpy()
        assert rel(y, ref.matvec(x)) <= 1e-10


def test_full_size_translation_on_sampled_targets():
    """The 500-sphere workload (p = 8): free-space part at two targets against the oracle's projection
    of the field of all 499 other spheres."""
    wl = syn.spheres3d()
    p = wl.p
    md = L3.Media3(wl.media.lam_u, wl.media.mu_u, wl.media.lam_l, wl.media.mu_l, wl.omega)
    gpu = P.Solver3(wl.centres, wl.radius, wl.bc, wl.media, wl.omega, p, n_r=8, n_theta=8, n_panels=1)
    x = scaled_random(5, wl.M, p, 2)
    t = gpu.operator(torch.as_tensor(x, device="cuda"), nat.MS3_PART_T).cpu().numpy()
    assert np.isfinite(t).all()
    for m in (0, wl.M // 2):
        others = [l for l in range(wl.M) if l != m]
        dmin = min(np.linalg.norm(wl.centres[l] - wl.centres[m]) for l in others)
        want = S3.translate(p, md.kp_l, md.ks_l, wl.centres[others], x[others], wl.centres[m], 0.5 * dmin, 40)
        assert rel(t[m], want) <= 1e-10
