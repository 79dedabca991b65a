"""Star particles on the GPU (Sec. 4.3: prototype scattering matrices with rotated copies; Sec. 7:
the star family r(t) = a (1 + 0.2 cos 5t)) against the FP64 oracle.

The prototype tables are the oracle's Nystrom matrices (oracle.nystrom.workload_tables), passed to
both sides as inputs.  Bars as in test_gpu_tensor_cores: the scaled norm (|y| / tau, tau the order
scale (k R / 2)^|n| / |n|!, relative to the largest entry), 1e-11 for FP64, 2e-5 for FP32 on the
CUDA cores, 1.6e-4 for 3xTF32 on the tensor cores; solves 1e-10 (FP64) and 1e-8 (mixed form)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import nystrom, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_2608_26875_b300 as P  # noqa: E402
from test_gpu_tensor_cores import TC_BAR, scaled_err  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def rel(got, want):
    return np.linalg.norm(got - want) / np.linalg.norm(want)


@pytest.fixture(scope="module")
def mixed():
    """150 particles of the 10^4-particle recipe (half discs, half stars, p = 20, 4 sizes x 2 BCs),
    16 columns: every prototype table is a full 82 x 82 Nystrom matrix."""
    wl = syn.config3(M=150, nrhs=16, Q=4)
    tabs = nystrom.workload_tables(wl)
    ref = system.Problem(wl, proto_S=tabs)
    x = syn.random_coeffs(701, wl.M, wl.p, 16)
    return wl, tabs, x, ref.matvec(x)


def test_stars_fp64_apply_matches_oracle(mixed):
    wl, tabs, x, want = mixed
    s = P.Solver.from_workload(wl, proto_S=tabs)
    got = s.apply(dev(x), prec=P.MS_PREC_FP64).cpu().numpy()
    assert rel(got, want) <= 1e-12 and scaled_err(got, want, wl) <= 1e-11


@pytest.mark.parametrize("tc,bar", [(True, TC_BAR), (False, 2e-5)])
def test_stars_fp32_apply_matches_oracle(mixed, tc, bar):
    wl, tabs, x, want = mixed
    s = P.Solver.from_workload(wl, proto_S=tabs, tensor_cores=tc)
    got = s.apply(dev(x), prec=P.MS_PREC_FP32).cpu().numpy()
    e = scaled_err(got, want, wl)
    print(f"stars FP32 apply, tensor cores {tc}: scaled error {e:.3e}")
    assert e <= bar


@pytest.mark.parametrize("nrhs", [1, 7, 64])
def test_star_scattering_apply_alone(nrhs):
    """S~ a~ through the operator-parts view (S applied to the reflected part of a one-particle
    cloud, so that the prototype apply dominates), for 1, 7 and 64 columns, both precisions."""
    wl = syn.config3(M=40, nrhs=nrhs, Q=2)
    tabs = nystrom.workload_tables(wl)
    ref = system.Problem(wl, proto_S=tabs)
    x = syn.random_coeffs(702, wl.M, wl.p, nrhs)
    want = ref.apply_S(ref.reflect(x))
    for tc, prec, bar in ((True, P.MS_PREC_FP64, 1e-11), (True, P.MS_PREC_FP32, TC_BAR),
                          (False, P.MS_PREC_FP32, 2e-5)):
        s = P.Solver.from_workload(wl, proto_S=tabs, tensor_cores=tc)
        got = s.operator(dev(x), P.MS_PART_R | P.MS_PART_S, prec=prec).cpu().numpy()
        assert scaled_err(got, want, wl) <= bar, (tc, prec)


def test_stars_adjoint_matches_the_dense_oracle_matrix():
    """ms_apply_adjoint against A^H from the oracle's assembled matrix (star and disc particles)."""
    wl = syn.config3(M=14, nrhs=3, Q=2)
    wl.p = 6
    tabs = nystrom.workload_tables(wl)
    ref = system.Problem(wl, proto_S=tabs)
    A = ref.assemble()
    y = syn.random_coeffs(703, wl.M, wl.p, 3)
    want = (A.conj().T @ y.reshape(A.shape[0], -1)).reshape(y.shape)
    s = P.Solver.from_workload(wl, proto_S=tabs)
    got = s.apply_adjoint(dev(y), prec=P.MS_PREC_FP64).cpu().numpy()
    assert rel(got, want) <= 1e-12
    for tc in (True, False):
        st = P.Solver.from_workload(wl, proto_S=tabs, tensor_cores=tc)
        assert rel(st.apply_adjoint(dev(y), prec=P.MS_PREC_FP32).cpu().numpy(), want) <= 2e-5


def test_stars_solve_fp64_and_mixed_match_oracle_lu():
    wl = syn.config3(M=12, nrhs=4, Q=2)
    wl.p = 10
    tabs = nystrom.workload_tables(wl)
    ref = system.Problem(wl, proto_S=tabs)
    want = ref.solve_lu(ref.rhs(wl.inc_kind, wl.inc_angle))
    s = P.Solver.from_workload(wl, proto_S=tabs)
    for prec, tol, bar in ((P.MS_PREC_FP64, 1e-12, 1e-10), (P.MS_PREC_FP32, 1e-10, 1e-8)):
        got, info = s.solve(wl.inc_kind, wl.inc_angle, tol=tol, prec=prec)
        assert info["status"] == 0, (prec, info)
        assert rel(got.cpu().numpy(), want) <= bar, prec


def test_prototype_shared_by_particles_of_different_radii():
    """Two particles use one table with different enclosing radii: their scales differ from the
    prototype's reference scales, which the row and column factors carry as exact powers of two."""
    wl = syn.small_case(704, 5, 8, omega=3.0, nrhs=6)
    wl.radius = np.array([0.48, 0.36, 0.5, 0.6, 0.42])
    tab = nystrom.scattering_matrix(nystrom.StarCurve(0.35, 0.07, 5), 1, nystrom.Host(2.0, 1.0, 3.0), 8, N=96)
    proto = np.array([0, 0, -1, 0, -1])
    ref = system.Problem(wl, proto_S=tab[None], proto_index=proto)
    x = syn.random_coeffs(705, wl.M, wl.p, 6)
    want = ref.matvec(x)
    s = P.Solver(wl.centres, wl.radius, wl.bc, wl.media, wl.omega, wl.p, proto=proto, rotation=wl.rotation,
                 proto_S=tab[None])
    assert scaled_err(s.apply(dev(x), prec=P.MS_PREC_FP64).cpu().numpy(), want, wl) <= 1e-11
    assert scaled_err(s.apply(dev(x), prec=P.MS_PREC_FP32).cpu().numpy(), want, wl) <= TC_BAR


def test_config2_stars_apply_sampled_targets():
    """1000 stars (p = 16, omega = 4, 32 prototypes): the full mat-vec on sampled targets."""
    wl = syn.config2()
    tabs = nystrom.workload_tables(wl)
    x = syn.random_coeffs(81, wl.M, wl.p, 2)
    s = P.Solver.from_workload(wl, proto_S=tabs)
    ref = system.Problem(wl, proto_S=tabs)
    targets = [0, 1, 137, 500, 998, 999]
    want = ref.matvec(x, targets=targets)
    got = s.apply(dev(x), prec=P.MS_PREC_FP64).cpu().numpy()[targets]
    assert rel(got, want) <= 1e-11
    got32 = s.apply(dev(x), prec=P.MS_PREC_FP32).cpu().numpy()[targets]
    assert rel(got32, want) <= TC_BAR
