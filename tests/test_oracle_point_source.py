"""Pins of the oracle's point-source incidence (Sec. 7.2), upper-layer fields and time-reversal matrix
(Sec. 7.5): the downgoing spectrum of an upper-layer point force against the fundamental solution,
the transmitted field's local expansions against the fundamental solution when both layers are the
same, continuity of the scattered field across the interface, elastodynamic reciprocity of the
mirror's response matrix (F = F^T), and the eigenvalue count of the time-reversal operator for small
rigid particles (two significant eigenvalues per particle, as the paper reports)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import nystrom, sommerfeld, system, waves


def test_point_force_downgoing_spectrum_is_the_upper_fundamental_solution():
    wl = syn.small_case(11, 3, 6, omega=2.0, nrhs=1)
    P = system.Problem(wl)
    L = P.L
    z = np.array([-1.0, 3.0])
    q = np.array([np.cos(0.7), np.sin(0.7)])
    IP, IS = sommerfeld.point_force_downgoing(P.xi, L, z, q)
    X, Y = np.array([0.0, -2.0, 1.5, 0.4]), np.array([1.0, 0.5, 1.2, 0.1])
    u1, u2, _ = sommerfeld.upper_downgoing_field(P.xi, P.W, L, IP, IS, X, Y)
    want = nystrom.fundamental(np.stack([X, Y], 1) - z, nystrom.Host(L.lam_u, L.mu_u, L.omega)) @ q
    assert np.abs(np.stack([u1, u2], 1) - want).max() < 1e-10 * np.abs(want).max()


def test_transmitted_point_force_in_identical_layers_is_the_free_field():
    """With the same medium on both sides nothing is reflected: the local expansion of the transmitted
    field about a particle reproduces Phi(x, z) q near it (Jacobi-Anger to order 12)."""
    wl = syn.small_case(11, 3, 12, omega=2.0, nrhs=1, media=syn.Media(2.0, 1.0, 2.0, 1.0))
    P = system.Problem(wl)
    z = np.array([-1.0, 2.5])
    q = np.array([np.cos(0.7), np.sin(0.7)])
    a0 = P.point_source_local([z], [q])
    h = nystrom.Host(2.0, 1.0, 2.0)
    for m in range(3):
        th = np.linspace(0, 2 * np.pi, 7, endpoint=False)
        X, Y = 0.3 * np.cos(th), 0.3 * np.sin(th)
        v1, v2, _ = waves.field_of_coeffs("J", a0[m, 0, :, 0], a0[m, 1, :, 0], wl.p, h.kp, h.ks, X, Y)
        want = nystrom.fundamental(np.stack([X + P.centres[m, 0], Y + P.centres[m, 1]], 1) - z, h) @ q
        assert np.abs(np.stack([v1, v2], 1) - want).max() < 1e-9 * np.abs(want).max()


def test_scattered_field_is_continuous_across_the_interface():
    """Lower-layer representation (direct multipole sums plus the reflected field) against the upper-layer
    one (the transmitted spectra) on y = 0, for a solved plane-wave problem."""
    wl = syn.small_case(12, 3, 6, omega=2.0, nrhs=2)
    P = system.Problem(wl)
    gam = P.solve_lu(P.rhs(wl.inc_kind, wl.inc_angle))
    X = np.linspace(-4, 4, 9)
    lo = P.scattered_field(gam, X, np.zeros_like(X))
    up = P.upper_field(gam, X, np.zeros_like(X))
    assert np.abs(lo - up).max() < 1e-8 * np.abs(lo).max()


def _mirror(n, radius=6.0):
    th = np.linspace(0, np.pi, n + 2)[1:-1]
    return np.stack([radius * np.cos(th), radius * np.sin(th)], 1)


@pytest.fixture(scope="module")
def mixed_case():
    """Two discs and one rotated traction-free star, 10 mirror points."""
    wl = syn.small_case(22, 3, 5, omega=3.0, nrhs=1)
    wl.centres = np.array([[2.5, -2.0], [-0.5, -3.5], [-3.0, -2.5]])
    wl.radius = np.array([0.3, 0.36, 0.25])
    wl.bc = np.array([0, 1, 1])
    wl.rotation = np.array([0.0, 0.8, 0.0])
    # (N = 192: the Nystrom matrix's discretisation error, not the method, would otherwise set the asymmetry)
    tab = nystrom.scattering_matrix(nystrom.StarCurve(0.3, 0.06, 5), 1, nystrom.Host(2.0, 1.0, 3.0), 5, N=192)
    P = system.Problem(wl, proto_S=tab[None], proto_index=np.array([-1, 0, -1]))
    return P, _mirror(10)


def test_response_matrix_is_reciprocal(mixed_case):
    """Reciprocity of the layered medium with particles: the field scattered at mirror point i under the
    force e_d at point j, component c, equals the one at point j under e_c at point i, component d."""
    P, mirror = mixed_case
    F, _ = P.time_reversal(mirror)
    assert np.abs(F).max() > 0
    assert np.abs(F - F.T).max() < 1e-11 * np.abs(F).max()


def test_planted_point_force_sign_breaks_reciprocity(mixed_case, monkeypatch):
    P, mirror = mixed_case
    orig = sommerfeld.point_force_downgoing

    def bad(xi, L, z, q):
        ip, is_ = orig(xi, L, z, q)
        return ip, -is_

    monkeypatch.setattr(sommerfeld, "point_force_downgoing", bad)
    F, _ = P.time_reversal(mirror)
    assert np.abs(F - F.T).max() > 1e-3 * np.abs(F).max()


def test_three_small_rigid_particles_give_six_significant_eigenvalues():
    """Sec. 7.5: each small rigid particle contributes two significant eigenvalues of T = conj(F)^T F."""
    wl = syn.small_case(21, 3, 3, omega=8.0, nrhs=1)
    wl.centres = np.array([[3.0, -2.0], [0.0, -4.0], [-3.0, -6.0]])
    wl.radius = np.full(3, 0.02)
    wl.bc = np.zeros(3, np.int32)
    wl.n_panels = 64
    P = system.Problem(wl)
    _, ev = P.time_reversal(_mirror(16))
    assert ev[5] > 100 * ev[6]
