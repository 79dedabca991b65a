"""Point-source incidence (ms_rhs_point, Sec. 7.2), upper-layer fields (ms_fields_upper) and the
time-reversal matrix (ms_time_reversal, Sec. 7.5) on the GPU against the oracle.

Bars: right-hand sides and fields 1e-12 / 1e-10 relative l2 (FP64 throughout); the response matrix
1e-9 against the oracle's dense-LU version and symmetric (reciprocity) to 1e-9; the eigenvalues of
conj(F)^T F against numpy's on the returned F to 1e-10 of the largest; the mixed-precision matrix 1e-7
against the FP64 one (solves refined to 1e-10)."""
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


def rel(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def _mirror(n, radius=6.0):
    th = np.linspace(0, np.pi, n + 2)[1:-1]
    return np.stack([radius * np.cos(th), radius * np.sin(th)], 1)


@pytest.fixture(scope="module")
def case():
    wl = syn.small_case(22, 3, 5, omega=3.0, nrhs=1)
    wl.centres = np.array([[2.5, -2.0], [-0.5, -3.5], [-3.0, -2.5]])
    wl.radius = np.array([0.3, 0.36, 0.25])
    wl.bc = np.array([0, 1, 1])
    wl.rotation = np.array([0.0, 0.8, 0.0])
    tab = nystrom.scattering_matrix(nystrom.StarCurve(0.3, 0.06, 5), 1, nystrom.Host(2.0, 1.0, 3.0), 5, N=192)
    proto = np.array([-1, 0, -1])
    ref = system.Problem(wl, proto_S=tab[None], proto_index=proto)
    s = P.Solver(wl.centres, wl.radius, wl.bc, wl.media, wl.omega, wl.p, proto=proto, rotation=wl.rotation,
                 proto_S=tab[None], n_panels=wl.n_panels, nodes_per_panel=wl.nodes_per_panel)
    return wl, ref, s


def test_point_source_rhs_matches_oracle(case):
    wl, ref, s = case
    src = np.array([[-3.0, 3.0], [1.0, 2.0], [0.5, 4.0]])
    force = np.array([[np.cos(np.pi / 4), np.sin(np.pi / 4)], [1.0, 0.0], [0.0, 1.0]])
    got = s.rhs_point(src, force).cpu().numpy()
    assert rel(got, ref.point_rhs(src, force)) <= 1e-12


def test_upper_fields_match_oracle(case):
    wl, ref, s = case
    g = syn.random_coeffs(961, wl.M, wl.p, 3) * 1e-2
    rx = np.stack([np.linspace(-5, 5, 11), np.linspace(0.5, 3.0, 11)], 1)
    got = s.fields_upper(torch.as_tensor(g, device="cuda"), rx).cpu().numpy()
    want = ref.upper_field(g, rx[:, 0], rx[:, 1]).transpose(0, 2, 1)
    assert rel(got, want) <= 1e-10


def test_receivers_of_upper_fields_must_lie_above_the_interface(case):
    wl, _, s = case
    g = torch.zeros((wl.M, 2, wl.nc, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(P.MsError) as e:
        s.fields_upper(g, np.array([[0.0, 1.0], [0.0, -0.5]]))
    assert e.value.status == nat.MS_ERR_RECEIVER_INSIDE


def test_time_reversal_matrix_matches_oracle_and_is_reciprocal(case):
    wl, ref, s = case
    mirror = _mirror(10)
    F, ev, V, info = s.time_reversal(mirror, tol=1e-12)
    Fo, evo = ref.time_reversal(mirror)
    assert info["status"] == 0
    assert rel(F, Fo) <= 1e-9
    assert np.abs(F - F.T).max() <= 1e-9 * np.abs(F).max()
    T = F.conj().T @ F
    want = np.sort(np.linalg.eigvalsh(T))[::-1]
    assert np.abs(ev - want).max() <= 1e-10 * want[0]
    assert np.abs(ev - evo).max() <= 1e-8 * evo[0]
    # eigenvectors: T v_k = lambda_k v_k, orthonormal
    assert np.abs(T @ V - V * ev[None, :]).max() <= 1e-10 * want[0]
    assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() <= 1e-10
    # mixed precision: FP32 inner solves, FP64 refinement
    F32, _, _, info32 = s.time_reversal(mirror, tol=1e-10, prec=P.MS_PREC_FP32)
    assert info32["status"] == 0 and rel(F32, F) <= 1e-7


def test_three_small_rigid_particles_give_six_significant_eigenvalues():
    wl = syn.small_case(21, 3, 3, omega=8.0, nrhs=1)
    wl.centres = np.array([[3.0, -2.0], [0.0, -4.0], [-3.0, -6.0]])
    wl.radius = np.full(3, 0.02)
    wl.bc = np.zeros(3, np.int32)
    wl.n_panels = 64
    s = P.Solver.from_workload(wl)
    _, ev, _, info = s.time_reversal(_mirror(30), tol=1e-10)
    assert info["status"] == 0
    assert ev[5] > 100 * ev[6]
