"""GPU adjoint (ms_apply_adjoint) and adjoint gradient (ms_grad) against the oracle.

* Dot-product test: <A x, y> = <x, A^H y> to round-off, with and without the FMM.
* ms_grad against the oracle's adjoint gradient (itself pinned to central differences of the
  oracle loss) on the same seeded case: relative 1e-8 on centres and radii, 1e-6 on omega (both
  sides take the omega derivative by central differences, h = 1e-6 omega).
* ms_grad against central differences (h = 1e-6) of the GPU's own FP64 forward loss on a larger
  case (direct Graf sum), the FMM gradient against the direct-sum gradient on one geometry, and
  the gradient through torch.autograd.
"""
import copy

import numpy as np
import pytest

import synthetic as syn
from oracle import adjoint

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402
from paper_2608_26875_b300.autograd import scattered_fields  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("case", ["small", "fmm"])
def test_adjoint_dot_product(case):
    if case == "small":
        wl = syn.small_case(501, 7, 6, omega=2.5, nrhs=3)
    else:
        wl = syn.config3_discs(M=1500, nrhs=3)
    s = P.Solver.from_workload(wl)
    x = dev(syn.random_coeffs(502, wl.M, wl.p, 3))
    y = dev(syn.random_coeffs(503, wl.M, wl.p, 3))
    Ax = s.apply(x)
    AHy = s.apply_adjoint(y)
    for r in range(3):
        lhs = torch.vdot(y[..., r].flatten(), Ax[..., r].flatten())      # <y, A x>
        rhs = torch.vdot(AHy[..., r].flatten(), x[..., r].flatten())     # <A^H y, x>
        scale = torch.linalg.norm(y[..., r]) * torch.linalg.norm(Ax[..., r])
        assert abs(complex(lhs - rhs)) <= 1e-11 * float(scale), (r, complex(lhs), complex(rhs))


def test_gradient_matches_oracle_adjoint():
    wl = syn.small_case(401, 3, 5, omega=2.0, nrhs=2)      # the case the oracle adjoint is pinned on
    rx = wl.receivers[::6]
    rng = np.random.default_rng(0)
    d = 0.1 * (rng.standard_normal((2, rx.shape[0], 2)) + 1j * rng.standard_normal((2, rx.shape[0], 2)))
    L, gc_or, gr_or, gw_or = adjoint.gradient(wl, wl.inc_kind, wl.inc_angle, rx, d)
    s = P.Solver.from_workload(wl)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-13, prec=P.MS_PREC_FP64)
    u = s.fields(g, rx)
    w = (u - dev(d)).contiguous()
    gc, gr, gw, ginfo = s.grad(wl.inc_kind, wl.inc_angle, g, w, rx, tol=1e-13)
    assert ginfo["status"] == 0
    gc, gr = gc.cpu().numpy(), gr.cpu().numpy()
    assert np.abs(gc - gc_or).max() <= 1e-8 * np.abs(gc_or).max(), (gc, gc_or)
    assert np.abs(gr - gr_or).max() <= 1e-8 * np.abs(gr_or).max(), (gr, gr_or)
    assert abs(gw - gw_or) <= 1e-6 * abs(gw_or), (gw, gw_or)


def test_mixed_precision_gradient_matches_oracle_adjoint():
    """The mixed form: forward solve and transposed solve with FP32 inner solves (tensor cores) inside
    FP64 refinement to 1e-11, against the oracle's FP64 adjoint gradient; held to the mixed path's
    1e-8 (relative to the largest entry of each gradient)."""
    wl = syn.small_case(401, 3, 5, omega=2.0, nrhs=2)
    rx = wl.receivers[::6]
    rng = np.random.default_rng(0)
    d = 0.1 * (rng.standard_normal((2, rx.shape[0], 2)) + 1j * rng.standard_normal((2, rx.shape[0], 2)))
    L, gc_or, gr_or, gw_or = adjoint.gradient(wl, wl.inc_kind, wl.inc_angle, rx, d)
    s = P.Solver.from_workload(wl, tensor_cores=True)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-11, prec=P.MS_PREC_FP32)
    assert info["status"] == 0 and info["refinements"] >= 1
    w = (s.fields(g, rx) - dev(d)).contiguous()
    gc, gr, gw, ginfo = s.grad(wl.inc_kind, wl.inc_angle, g, w, rx, tol=1e-11, prec=P.MS_PREC_FP32)
    assert ginfo["status"] == 0 and ginfo["refinements"] >= 1
    gc, gr = gc.cpu().numpy(), gr.cpu().numpy()
    assert np.abs(gc - gc_or).max() <= 1e-8 * np.abs(gc_or).max(), (gc, gc_or)
    assert np.abs(gr - gr_or).max() <= 1e-8 * np.abs(gr_or).max(), (gr, gr_or)
    assert abs(gw - gw_or) <= 1e-6 * abs(gw_or), (gw, gw_or)


def _gpu_loss(wl, rx, d, **kw):
    s = P.Solver.from_workload(wl, **kw)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-13, prec=P.MS_PREC_FP64)
    assert info["status"] == 0, info          # central differences need converged solves
    u = s.fields(g, rx).cpu().numpy()
    return 0.5 * float(np.sum(np.abs(u - d) ** 2))


def _fd_case(M, side, seed=7):
    """Rigid discs R ~ U[0.2, 0.5] spread thinly enough that GMRES reaches 1e-13 quickly."""
    npan, depth, grade = syn.contour_for_width(side)
    wl = syn.small_case(400 + M, M, 10, omega=2.0, nrhs=2, box=(-side / 2, side / 2, -side, -1.0),
                        rmin=0.2, rmax=0.5, mixed_bc=False, n_panels=npan, depth=depth, grade=grade)
    rx = wl.receivers[::2]
    rng = np.random.default_rng(seed)
    d = 0.05 * (rng.standard_normal((2, rx.shape[0], 2)) + 1j * rng.standard_normal((2, rx.shape[0], 2)))
    return wl, rx, d


def _grad(wl, rx, d, tol=1e-13, **kw):
    s = P.Solver.from_workload(wl, **kw)
    g, info = s.solve(wl.inc_kind, wl.inc_angle, tol=tol, prec=P.MS_PREC_FP64)
    assert info["status"] == 0, info
    u = s.fields(g, rx)
    gc, gr, gw, ginfo = s.grad(wl.inc_kind, wl.inc_angle, g, (u - dev(d)).contiguous(), rx, tol=tol)
    assert ginfo["status"] == 0, ginfo
    return gc.cpu().numpy(), gr.cpu().numpy(), gw, s


def test_gradient_matches_gpu_central_differences():
    """Direct Graf sum (no tree): adjoint gradient vs central differences of the GPU FP64 loss."""
    wl, rx, d = _fd_case(40, 40.0)
    gc, gr, gw, _ = _grad(wl, rx, d, use_fmm=False)
    h = 1e-6
    for m, axis in ((0, 0), (7, 1), (21, 0), (39, 1)):
        wp, wm = copy.deepcopy(wl), copy.deepcopy(wl)
        wp.centres = wl.centres.copy(); wp.centres[m, axis] += h
        wm.centres = wl.centres.copy(); wm.centres[m, axis] -= h
        fd = (_gpu_loss(wp, rx, d, use_fmm=False) - _gpu_loss(wm, rx, d, use_fmm=False)) / (2 * h)
        assert abs(gc[m, axis] - fd) <= 1e-6 * np.abs(gc).max(), (m, axis, gc[m, axis], fd)
    for m in (3, 30):
        wp, wm = copy.deepcopy(wl), copy.deepcopy(wl)
        wp.radius = wl.radius.copy(); wp.radius[m] += h
        wm.radius = wl.radius.copy(); wm.radius[m] -= h
        fd = (_gpu_loss(wp, rx, d, use_fmm=False) - _gpu_loss(wm, rx, d, use_fmm=False)) / (2 * h)
        assert abs(gr[m] - fd) <= 1e-6 * np.abs(gr).max(), (m, gr[m], fd)


def test_gradient_with_fmm_matches_direct_sum():
    """The FMM's position derivatives (L2P for targets, the adjoint P2M for sources) against the
    gradient of the direct Graf sum on the same geometry."""
    wl, rx, d = _fd_case(300, 110.0)
    gcf, grf, gwf, s = _grad(wl, rx, d, tol=1e-11, leaf_target=8)
    assert s.fmm_levels >= 3
    gcd, grd, gwd, _ = _grad(wl, rx, d, tol=1e-11, use_fmm=False)
    assert np.abs(gcf - gcd).max() <= 1e-8 * np.abs(gcd).max()
    assert np.abs(grf - grd).max() <= 1e-8 * np.abs(grd).max()
    assert abs(gwf - gwd) <= 1e-6 * abs(gwd)


def test_autograd_function_backward():
    wl = syn.small_case(404, 4, 5, omega=2.0, nrhs=2)
    rx = wl.receivers[::4]
    c = torch.tensor(wl.centres, dtype=torch.float64, requires_grad=True)
    r = torch.tensor(wl.radius, dtype=torch.float64, requires_grad=True)
    om = torch.tensor(wl.omega, dtype=torch.float64, requires_grad=True)
    d = torch.zeros((2, rx.shape[0], 2), dtype=torch.complex128, device="cuda")
    u = scattered_fields(c, r, om, wl.bc, wl.media, wl.p, wl.inc_kind, wl.inc_angle, rx, tol=1e-13)
    loss = 0.5 * (u - d).abs().pow(2).sum()
    loss.backward()
    s = P.Solver.from_workload(wl)
    g, _ = s.solve(wl.inc_kind, wl.inc_angle, tol=1e-13)
    w = s.fields(g, rx)
    gc, gr, gw, _ = s.grad(wl.inc_kind, wl.inc_angle, g, w.contiguous(), rx, tol=1e-13)
    np.testing.assert_allclose(c.grad.numpy(), gc.cpu().numpy(), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(r.grad.numpy(), gr.cpu().numpy(), rtol=1e-9, atol=1e-12)
    assert float(om.grad) == pytest.approx(gw, rel=1e-6)
