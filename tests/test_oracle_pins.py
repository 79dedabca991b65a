"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against the paper's printed values, a closed-form
identity evaluated independently (scipy Bessel routines, direct field sums), a physical
conservation law or a second derivation, chosen so that a dropped term, a sign or index
error or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import special

import synthetic as syn
from oracle import disc, graf, sommerfeld, system, waves
from oracle.media import Layered, wavenumbers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
L_STD = Layered(syn.MEDIA_STD, 2.0)


def test_wavenumbers_match_paper_printed_values():
    """Sec. 7 preamble prints kp, ks, kp', ks' for omega = 2 pi and the default Lame constants."""
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_wavenumbers.txt"))
    for lam, mu, om, kp, ks in rows:
        got = wavenumbers(lam, mu, om)
        assert got[0] == pytest.approx(kp, rel=1e-14)
        assert got[1] == pytest.approx(ks, rel=1e-14)


@pytest.mark.parametrize("n", [0, 1, -1, 5, -7, 20, 33, -40, 60])
def test_bessel_and_hankel_against_mpmath(n):
    """The oracle's J_n and H_n^(1) (every Graf entry, multipole and local expansion goes through
    them) against mpmath at 30 digits, over the orders and arguments k d of the direct sums
    (|n| <= 2p = 40 at p = 20, k d up to ~10^3).  J is compared against the envelope |H_n|, so
    that an argument near a zero of J does not count as a large relative error."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for x in (0.3, 1.0, 2.7, 9.0, 20.0, 39.5, 150.0, 1200.0):
        h_ref = complex(mpmath.hankel1(n, x))
        j_ref = complex(mpmath.besselj(n, x))
        assert abs(complex(waves.Z("H", n, x)) - h_ref) <= 1e-12 * abs(h_ref), (n, x)
        assert abs(complex(waves.Z("J", n, x)) - j_ref) <= 1e-12 * abs(h_ref), (n, x)


@pytest.mark.parametrize("k", [0.7, 2.0, 6.0])
def test_graf_translation_pointwise(k):
    """Sec. 4.2: the local expansion T gamma about x_m reproduces the outgoing potential of
    particle l evaluated directly with Hankel functions."""
    p, P = 8, 50
    xl = np.array([0.3, -2.0])
    xm = np.array([2.1, -4.5])
    rng = np.random.default_rng(0)
    g = rng.standard_normal(2 * p + 1) + 1j * rng.standard_normal(2 * p + 1)
    a = graf.translation_matrix(p, k, xm, xl, p_out=P) @ g
    for t in np.linspace(0, 2 * np.pi, 9)[:-1]:
        x = xm + 0.5 * np.array([math.cos(t), math.sin(t)])
        dl = x - xl
        direct = sum(g[j + p] * special.hankel1(j, k * np.hypot(*dl)) * np.exp(1j * j * math.atan2(dl[1], dl[0]))
                     for j in range(-p, p + 1))
        dm = x - xm
        loc = sum(a[i + P] * special.jv(i, k * np.hypot(*dm)) * np.exp(1j * i * math.atan2(dm[1], dm[0]))
                  for i in range(-P, P + 1))
        assert abs(direct - loc) <= 1e-12 * abs(direct)


def test_graf_all_sources_matches_pairwise():
    p = 5
    rng = np.random.default_rng(3)
    centres = rng.uniform(-5, 5, (6, 2))
    T = graf.translation_all_sources(p, 1.3, centres[0], centres)
    assert np.all(T[0] == 0)
    for l in range(1, 6):
        np.testing.assert_allclose(T[l], graf.translation_matrix(p, 1.3, centres[0], centres[l]), rtol=1e-14)


def test_sommerfeld_identity_som1():
    """Sec. 3 som1: (i/4) H_0(k|x-x0|) = (1/4pi) int e^{-s|y-y0|}/s e^{i xi (x-x0)} dxi on the contour."""
    xi, W = sommerfeld.contour(64, 16, 40.0)
    for k, dx, dy in ((1.0, 0.7, 1.2), (2.0, -1.5, -0.9), (3.0, 2.0, 2.5)):
        s = sommerfeld.branch_s(xi, k)
        quad = (W * np.exp(-s * abs(dy)) / s * np.exp(1j * xi * dx)).sum() / (4 * np.pi)
        assert abs(quad - 0.25j * special.hankel1(0, k * math.hypot(dx, dy))) < 1e-9


@pytest.mark.parametrize("n", [0, 1, -1, 3, -5, 10])
def test_multipole_to_sommerfeld_pts1(n):
    """Sec. 5.4 pts1 as quadrature on the contour equals H_n(k r) e^{i n theta} evaluated by scipy."""
    xi, W = sommerfeld.contour(64, 16, 40.0)
    k, xm, ym, x, y = 1.0, 0.4, -1.3, 1.1, -0.2
    s = sommerfeld.branch_s(xi, k)
    integ = ((-1.0) ** n / (1j * np.pi)) * np.exp(s * (ym - y)) / s * np.exp(1j * xi * (x - xm)) \
        * ((s - xi) / (1j * k)) ** n
    quad = (W * integ).sum()
    ex = special.hankel1(n, k * math.hypot(x - xm, y - ym)) * np.exp(1j * n * math.atan2(y - ym, x - xm))
    assert abs(quad - ex) <= 1e-8 * abs(ex)


def test_m2s_reproduces_particle_field_above_centre():
    """m2s amplitudes: the upgoing plane-wave sum equals the direct outgoing field (sed1/sed2)."""
    xi, W = sommerfeld.contour(64, 16, 40.0)
    p = 4
    rng = np.random.default_rng(5)
    centres = np.array([[0.2, -1.5]])
    gam = (rng.standard_normal((1, 2, 2 * p + 1, 1)) + 1j * rng.standard_normal((1, 2, 2 * p + 1, 1)))
    U_P, U_S = sommerfeld.m2s(xi, L_STD, centres, gam)
    X = np.array([-0.5, 0.4, 1.0])
    Y = np.array([-0.3, -0.1, 0.0])
    sp, ss = sommerfeld.branch_s(xi, L_STD.kp_l), sommerfeld.branch_s(xi, L_STD.ks_l)
    e_p = W * U_P[:, 0] * np.exp(1j * xi * X[:, None] - sp * Y[:, None])
    e_s = W * U_S[:, 0] * np.exp(1j * xi * X[:, None] - ss * Y[:, None])
    u1 = (1j * xi * e_p + ss * e_s).sum(-1)
    u2 = (-sp * e_p + 1j * xi * e_s).sum(-1)
    d1, d2, _ = waves.field_of_coeffs("H", gam[0, 0, :, 0], gam[0, 1, :, 0], p, L_STD.kp_l, L_STD.ks_l,
                                      X - centres[0, 0], Y - centres[0, 1])
    np.testing.assert_allclose(u1, d1, rtol=1e-8, atol=1e-8 * np.abs(d1).max())
    np.testing.assert_allclose(u2, d2, rtol=1e-8, atol=1e-8 * np.abs(d2).max())


def test_jacobi_anger_on_contour_nodes():
    """Sec. 5.3 ja/stm: e^{i xi X + s Y} = sum_n i^n q^n J_n(k r) e^{i n theta}, q = (xi - s)/k, at contour nodes."""
    xi, _ = sommerfeld.contour(32, 16, 20.0)
    k, X, Y = 1.0, 0.08, -0.05
    r, th = math.hypot(X, Y), math.atan2(Y, X)
    n = np.arange(-80, 81)
    for q_i in (3, 100, 255, 256, 400, 508):
        x0 = xi[q_i]
        s = sommerfeld.branch_s(x0, k)
        q = (x0 - s) / k
        rhs = np.sum((1j ** n) * q ** n * special.jv(n, k * r) * np.exp(1j * n * th))
        lhs = np.exp(1j * x0 * X + s * Y)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_branch_has_nonnegative_real_part_and_limiting_absorption():
    xi, _ = sommerfeld.contour(32, 16, 20.0)
    for k in (1.0, 2.0, 6.0):
        s = sommerfeld.branch_s(xi, k)
        assert np.all(s.real >= 0)
        np.testing.assert_allclose(s * s, xi * xi - k * k, rtol=1e-12, atol=1e-12)
        # real propagating xi: s = -i sqrt(k^2 - xi^2)
        assert sommerfeld.branch_s(0.5 * k, k) == pytest.approx(-1j * math.sqrt(0.75) * k)


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("R", [0.2, 0.5, 1.3])
def test_disc_scattering_matrix_boundary_condition(bc, R):
    """Sec. 4.1: incoming + S(incoming) satisfies the rigid (u = 0) or traction-free (sigma r-hat = 0)
    condition on r = R; the field is evaluated with Cartesian derivative recurrences (DLMF 10.6)
    and the traction of Sec. 2, independently of the polar formulas used to build S."""
    p = 12
    L = L_STD
    S = disc.disc_smatrix(p, L.kp_l, L.ks_l, R, bc, L.lam_l, L.mu_l)
    rng = np.random.default_rng(int(R * 10) + bc)
    a = (rng.standard_normal((2, 2 * p + 1)) + 1j * rng.standard_normal((2, 2 * p + 1)))
    out = np.einsum("nij,jn->in", S, a)
    th = np.linspace(0, 2 * np.pi, 50, endpoint=False)
    X, Y = R * np.cos(th), R * np.sin(th)
    ui1, ui2, gi = waves.field_of_coeffs("J", a[0], a[1], p, L.kp_l, L.ks_l, X, Y)
    uo1, uo2, go = waves.field_of_coeffs("H", out[0], out[1], p, L.kp_l, L.ks_l, X, Y)
    if bc == 0:
        scale = max(np.abs(ui1).max(), np.abs(ui2).max())
        assert np.abs(ui1 + uo1).max() < 1e-12 * scale
        assert np.abs(ui2 + uo2).max() < 1e-12 * scale
    else:
        g = [[gi[i][j] + go[i][j] for j in range(2)] for i in range(2)]
        t1, t2 = waves.traction(g, np.cos(th), np.sin(th), L.lam_l, L.mu_l)
        s1, s2 = waves.traction(gi, np.cos(th), np.sin(th), L.lam_l, L.mu_l)
        scale = max(np.abs(s1).max(), np.abs(s2).max())
        assert np.abs(t1).max() < 1e-11 * scale
        assert np.abs(t2).max() < 1e-11 * scale


def test_reflection_two_routes_agree():
    """The paper's A_xi / b1 / b2 / eee1 route (Sec. 3, 5.3, 5.4) and the plane-wave continuity
    route give the same interface-reflected local expansions."""
    wl = syn.small_case(7, 3, 6, omega=2.0)
    P = system.Problem(wl)
    gam = syn.random_coeffs(3, P.M, P.p, 2)
    a1 = sommerfeld.layered_apply(P.xi, P.W, P.L, P.centres, gam)
    a2 = sommerfeld.layered_apply_paper(P.xi, P.W, P.L, P.centres, gam)
    assert np.linalg.norm(a1 - a2) <= 1e-12 * np.linalg.norm(a1)


def test_reflection_vanishes_for_identical_media():
    L = Layered(syn.Media(2.0, 1.0, 2.0, 1.0), 2.0)
    xi, _ = sommerfeld.contour(8, 8, 20.0)
    for x in list(xi[::5]) + [0.3 + 0j, 1.7 + 0j]:
        assert np.abs(sommerfeld.reflection_plane_wave(x, L)).max() < 1e-13


@pytest.mark.parametrize("xi0", [0.05, 0.5, 0.95])
@pytest.mark.parametrize("U", [(1.0, 0.0), (0.0, 1.0), (0.3, -0.7j)])
def test_interface_energy_balance(xi0, U):
    """Time-averaged vertical energy flux Im(conj(u).T_y u) of the incident wave equals the sum
    over reflected and transmitted waves when all four waves propagate (|xi| < min k)."""
    L = L_STD
    x = complex(xi0, 0)

    def flux(kind, d, lam, mu, amp):
        u = amp * sommerfeld._pw(kind, x, d)
        return np.imag(np.vdot(u, sommerfeld._traction_y(u, x, d, lam, mu)))

    D, E = sommerfeld.interface_solve(x, L, U=U)
    sp, ss = sommerfeld.branch_s(x, L.kp_l), sommerfeld.branch_s(x, L.ks_l)
    spu, ssu = sommerfeld.branch_s(x, L.kp_u), sommerfeld.branch_s(x, L.ks_u)
    fin = flux("P", -sp, L.lam_l, L.mu_l, U[0]) + flux("S", -ss, L.lam_l, L.mu_l, U[1])
    fr = flux("P", sp, L.lam_l, L.mu_l, D[0]) + flux("S", ss, L.lam_l, L.mu_l, D[1])
    ft = flux("P", -spu, L.lam_u, L.mu_u, E[0]) + flux("S", -ssu, L.lam_u, L.mu_u, E[1])
    assert fin > 0 and fr <= 0 and ft > 0
    assert abs(fin + fr - ft) < 1e-13 * fin


@pytest.mark.parametrize("kind", [0, 1])
def test_normal_incidence_matches_impedance_formulas(kind):
    """Background field of the right-hand side at normal incidence: a plane P (S) wave from the
    upper layer reflects and transmits with the one-dimensional displacement coefficients
    R = (Z_u - Z_l)/(Z_u + Z_l), T = 2 Z_u/(Z_u + Z_l), Z = rho c = sqrt(lam + 2 mu) (sqrt(mu)) at
    rho = 1, and converts into no wave of the other type."""
    L = L_STD
    xi, D, E, I = sommerfeld.plane_wave_incidence(kind, math.pi / 2, L)
    assert abs(xi) < 1e-15
    if kind == 0:
        zu, zl = math.sqrt(L.lam_u + 2 * L.mu_u), math.sqrt(L.lam_l + 2 * L.mu_l)
        ku, kl = L.kp_u, L.kp_l
        # y-displacements at y = 0: incident -1, reflected i ku E_P, transmitted -i kl D_P
        inc, refl, trans = -1.0, 1j * ku * E[0], -1j * kl * D[0]
        other = (D[1], E[1])
    else:
        zu, zl = math.sqrt(L.mu_u), math.sqrt(L.mu_l)
        ku, kl = L.ks_u, L.ks_l
        # x-displacements at y = 0: incident 1, reflected -i ku E_S, transmitted i kl D_S
        inc, refl, trans = 1.0, -1j * ku * E[1], 1j * kl * D[1]
        other = (D[0], E[0])
    assert abs(refl / inc - (zu - zl) / (zu + zl)) < 1e-14
    assert abs(trans / inc - 2 * zu / (zu + zl)) < 1e-14
    assert max(abs(o) for o in other) < 1e-15


@pytest.mark.parametrize("kind,deg", [(0, 60.0), (0, 80.0), (1, 75.0), (1, 85.0)])
def test_incidence_from_above_energy_balance(kind, deg):
    """Oblique plane wave from the upper layer, angles at which all four scattered waves
    propagate: the downward energy flux of the incident wave equals the upward flux of the
    reflected P and S waves plus the downward flux of the transmitted ones (mode conversion
    included)."""
    L = L_STD
    xi, D, E, I = sommerfeld.plane_wave_incidence(kind, math.radians(deg), L)
    assert abs(xi) < min(L.kp_u, L.ks_u, L.kp_l, L.ks_l)

    def flux(k, d, lam, mu, amp):
        u = amp * sommerfeld._pw(k, xi, d)
        return np.imag(np.vdot(u, sommerfeld._traction_y(u, xi, d, lam, mu)))

    sp, ss = sommerfeld.branch_s(xi, L.kp_l), sommerfeld.branch_s(xi, L.ks_l)
    spu, ssu = sommerfeld.branch_s(xi, L.kp_u), sommerfeld.branch_s(xi, L.ks_u)
    f_inc = flux("P", spu, L.lam_u, L.mu_u, I[0]) + flux("S", ssu, L.lam_u, L.mu_u, I[1])
    f_ref = flux("P", -spu, L.lam_u, L.mu_u, E[0]) + flux("S", -ssu, L.lam_u, L.mu_u, E[1])
    f_tr = flux("P", sp, L.lam_l, L.mu_l, D[0]) + flux("S", ss, L.lam_l, L.mu_l, D[1])
    assert f_inc < 0 and f_ref >= 0 and f_tr < 0
    assert abs(E[1 - kind]) > 1e-3 and abs(D[1 - kind]) > 1e-3      # oblique: both wave types appear
    assert abs(f_inc + f_ref - f_tr) < 1e-13 * abs(f_inc)


@pytest.fixture(scope="module")
def solved_small():
    wl = syn.small_case(11, 3, 14, omega=2.0, nrhs=2)
    P = system.Problem(wl)
    b = P.rhs(wl.inc_kind, wl.inc_angle)
    x, it = P.solve_gmres(b, tol=1e-13)
    return wl, P, b, x


def test_solved_system_satisfies_particle_boundary_conditions(solved_small):
    """Total field (background + every particle's outgoing field + interface reflection), summed
    directly on each particle's boundary, meets its boundary condition to truncation error."""
    wl, P, b, x = solved_small
    worst = 0.0
    for m in range(P.M):
        res, sc = P.boundary_residual(x, wl.inc_kind, wl.inc_angle, m, 32)
        worst = max(worst, np.abs(res).max() / np.abs(sc).max())
    assert worst < 1e-6


def test_boundary_residual_decays_with_order():
    res = []
    for p in (6, 10):
        wl = syn.small_case(11, 3, p, omega=2.0, nrhs=1)
        P = system.Problem(wl)
        x, _ = P.solve_gmres(P.rhs(wl.inc_kind, wl.inc_angle), tol=1e-13)
        r, s = P.boundary_residual(x, wl.inc_kind, wl.inc_angle, 0, 32)
        res.append(np.abs(r).max() / np.abs(s).max())
    assert res[1] < 1e-2 * res[0]


def test_interface_continuity_of_assembled_field(solved_small):
    """Particle-induced field: lower side (direct multipole sums + downgoing Sommerfeld field) and
    upper side (upgoing Sommerfeld field) agree in displacement and traction on y = 0 (Sec. 3)."""
    wl, P, b, x = solved_small
    X = np.linspace(-3, 3, 7)
    Y = np.zeros_like(X)
    _, (E_P, E_S) = P.interface_amplitudes(x[..., :1])
    us, gs = P.scattered_field(x[..., :1], X, Y, with_gradient=True)
    u1, u2, gu = sommerfeld.upgoing_upper_field(P.xi, P.W, P.L, E_P[:, 0], E_S[:, 0], X, Y)
    lo = np.stack([us[0][0], us[0][1]])
    assert np.abs(lo - np.stack([u1, u2])).max() < 1e-8 * np.abs(lo).max()
    tl = np.stack(waves.traction(gs[0], 0.0, 1.0, P.L.lam_l, P.L.mu_l))
    tu = np.stack(waves.traction(gu, 0.0, 1.0, P.L.lam_u, P.L.mu_u))
    assert np.abs(tl - tu).max() < 1e-8 * np.abs(tl).max()


def _betti_on_circles(P, gam, rho=0.6, npts=128):
    """Betti's reciprocal form I_k = circle integral of u^A . t^B - u^B . t^A (outward normal of the
    circle) around each of the two centres, for the layered scattered fields of two states given as
    the two columns of gam."""
    out = []
    for m in range(2):
        th = np.linspace(0, 2 * np.pi, npts, endpoint=False)
        nx, ny = np.cos(th), np.sin(th)
        us, gs = P.scattered_field(gam, P.centres[m, 0] + rho * nx, P.centres[m, 1] + rho * ny,
                                   with_gradient=True)
        tA = waves.traction(gs[0], nx, ny, P.L.lam_l, P.L.mu_l)
        tB = waves.traction(gs[1], nx, ny, P.L.lam_l, P.L.mu_l)
        f = us[0][0] * tB[0] + us[0][1] * tB[1] - us[1][0] * tA[0] - us[1][1] * tA[1]
        out.append(f.sum() * 2 * np.pi * rho / npts)
    return out


@pytest.fixture(scope="module")
def two_sources():
    wl = syn.small_case(21, 2, 5, omega=2.0, nrhs=2)
    wl.centres = np.array([[-1.5, -2.5], [1.2, -3.1]])
    wl.radius = np.array([0.3, 0.3])
    P = system.Problem(wl)
    rng = np.random.default_rng(5)
    gam = np.zeros((2, 2, 2 * wl.p + 1, 2), complex)
    for m in range(2):          # state A: particle 0 radiates alone; state B: particle 1
        gam[m, :, :, m] = rng.standard_normal((2, 2 * wl.p + 1)) + 1j * rng.standard_normal((2, 2 * wl.p + 1))
    return P, gam


def test_layered_field_is_reciprocal(two_sources):
    """Elastodynamic reciprocity (Betti) in the welded two-layer medium.  Two states are each the
    field of one radiating particle: its outgoing multipoles plus the interface-reflected Sommerfeld
    field.  Betti's form vanishes over the region outside two small circles around the sources:
    displacement and traction are continuous across the interface and both states radiate.  So
    the two circle integrals cancel, though each is O(1).  A transposed 2x2 reflection (P->S read
    as S->P), a flipped order index or x-phase in the multipole-to-Sommerfeld map, or a wrong P/S
    normalisation there breaks the cancellation."""
    P, gam = two_sources
    I1, I2 = _betti_on_circles(P, gam)
    assert abs(I1) > 1.0
    assert abs(I1 + I2) < 1e-11 * abs(I1)


def test_planted_reflection_transpose_is_caught_by_reciprocity(two_sources, monkeypatch):
    P, gam = two_sources
    R = P.reflection_table()
    monkeypatch.setattr(P, "reflection_table", lambda: np.ascontiguousarray(np.transpose(R, (0, 2, 1))))
    I1, I2 = _betti_on_circles(P, gam)
    assert abs(I1 + I2) > 1e-4 * abs(I1)


def _manufactured_case(p=10, delta=0.15):
    """Three discs (rigid, traction-free, rigid), each holding a P + S point source at distance delta
    from its centre.  The exact scattered field u_ex is the sources' free-space field (H_0 potentials
    summed directly) plus its interface reflection, taken from the monopole spectral form (som1) and
    the 2x2 plane-wave reflection.  The boundary data of u_ex (displacement on rigid circles,
    traction on traction-free ones) are fitted by outgoing waves f^m on each circle.  Then
    gamma = f + S (T + R) gamma has the exact solution whose field is u_ex: by uniqueness of the
    exterior problem the solver, through Graf translations, pts1 at every order, Jacobi-Anger and
    the scattering matrices, must reproduce a field built from none of them."""
    wl = syn.small_case(31, 3, p, omega=2.0, nrhs=1)
    wl.centres = np.array([[-2.0, -2.0], [0.5, -3.0], [2.5, -1.8]])
    wl.radius = np.full(3, 0.5)
    wl.bc = np.array([0, 1, 0])
    P = system.Problem(wl)
    L = P.L
    rng = np.random.default_rng(7)
    ph = rng.uniform(0, 2 * np.pi, 3)
    z = P.centres + delta * np.stack([np.cos(ph), np.sin(ph)], 1)
    amp = rng.standard_normal((3, 2)) + 1j * rng.standard_normal((3, 2))
    sp, ss = sommerfeld.branch_s(P.xi, L.kp_l), sommerfeld.branch_s(P.xi, L.ks_l)
    # som1: H_0(k |x - z|) = sum_q W_q e^{s z_y - i xi z_x} / (i pi s) e^{i xi x - s y} above the source
    U_P = sum(amp[m, 0] * np.exp(sp * z[m, 1] - 1j * P.xi * z[m, 0]) / (1j * np.pi * sp) for m in range(3))
    U_S = sum(amp[m, 1] * np.exp(ss * z[m, 1] - 1j * P.xi * z[m, 0]) / (1j * np.pi * ss) for m in range(3))
    R = P.reflection_table()
    D_P = R[:, 0, 0] * U_P + R[:, 0, 1] * U_S
    D_S = R[:, 1, 0] * U_P + R[:, 1, 1] * U_S

    def u_ex(X, Y):
        u1, u2, g = sommerfeld.downgoing_field(P.xi, P.W, L, D_P, D_S, X, Y)
        g = [[g[i][j] for j in range(2)] for i in range(2)]
        for m in range(3):
            a, b, gg = waves.field_of_coeffs("H", [amp[m, 0]], [amp[m, 1]], 0, L.kp_l, L.ks_l,
                                             X - z[m, 0], Y - z[m, 1])
            u1, u2 = u1 + a, u2 + b
            g = [[g[i][j] + gg[i][j] for j in range(2)] for i in range(2)]
        return u1, u2, g

    nc = 2 * p + 1
    f = np.zeros((3, 2, nc, 1), complex)
    th = np.linspace(0, 2 * np.pi, 96, endpoint=False)
    nx, ny = np.cos(th), np.sin(th)

    def trace(u1, u2, g, bc):
        return np.concatenate([u1, u2] if bc == 0 else waves.traction(g, nx, ny, L.lam_l, L.mu_l))

    for m in range(3):
        X, Y = P.centres[m, 0] + P.radius[m] * nx, P.centres[m, 1] + P.radius[m] * ny
        data = trace(*u_ex(X, Y), P.bc[m])
        cols = []
        for b in range(2):
            for j in range(nc):
                c = np.zeros((2, nc), complex)
                c[b, j] = 1.0
                cols.append(trace(*waves.field_of_coeffs("H", c[0], c[1], p, L.kp_l, L.ks_l,
                                                         X - P.centres[m, 0], Y - P.centres[m, 1]), P.bc[m]))
        A = np.stack(cols, 1)
        cn = np.linalg.norm(A, axis=0)                # orders differ by many decades at k R < 1
        sol = np.linalg.lstsq(A / cn, data, rcond=None)[0] / cn
        # the fit leaves the data's modes above p (about 1e-6 here); they decay like (R/r)^n away from the circle
        assert np.abs(A @ sol - data).max() < 1e-4 * np.abs(data).max()
        f[m, :, :, 0] = sol.reshape(2, nc)
    Xr = np.concatenate([np.linspace(-4, 4, 9), [-0.8, 1.5, 0.0]])
    Yr = np.concatenate([np.full(9, -0.5), [-2.6, -2.2, -4.5]])
    return P, f, Xr, Yr, u_ex


def test_manufactured_solution_from_interior_sources():
    P, f, X, Y, u_ex = _manufactured_case()
    gam = P.solve_lu(f)
    got = P.scattered_field(gam, X, Y)[0]
    e1, e2, _ = u_ex(X, Y)
    want = np.stack([e1, e2])
    assert np.abs(got - want).max() < 1e-8 * np.abs(want).max()


def test_planted_s2l_sign_is_caught_by_manufactured_solution(monkeypatch):
    orig = sommerfeld.s2l
    monkeypatch.setattr(sommerfeld, "s2l", lambda *a, **k: -orig(*a, **k))
    with pytest.raises(AssertionError):
        test_manufactured_solution_from_interior_sources()


def test_gmres_matches_dense_lu():
    wl = syn.small_case(12, 3, 6, omega=2.0, nrhs=2)
    P = system.Problem(wl)
    b = P.rhs(wl.inc_kind, wl.inc_angle)
    x, _ = P.solve_gmres(b, tol=1e-13)
    xl = P.solve_lu(b)
    assert np.linalg.norm(x - xl) <= 1e-11 * np.linalg.norm(xl)
    assert np.linalg.norm(P.matvec(x) - b) <= 1e-12 * np.linalg.norm(b)


def test_rotated_prototype_matrix_of_a_disc_is_invariant():
    """Rotating a disc prototype (Sec. 4.3 basis rotation) leaves its scattering matrix unchanged,
    and rotating a dense prototype by 2 pi is the identity map."""
    wl = syn.small_case(13, 2, 5)
    P = system.Problem(wl)
    S0 = P.dense_S(0)
    P2 = system.Problem(wl, proto_S=S0[None], proto_index=np.array([0, 0]))
    np.testing.assert_allclose(P2.dense_S(0), S0, atol=1e-15)
    P2.rotation = np.array([2 * np.pi, 1.0])
    rng = np.random.default_rng(1)
    Sr = rng.standard_normal(S0.shape) + 1j * rng.standard_normal(S0.shape)
    P3 = system.Problem(wl, proto_S=Sr[None], proto_index=np.array([0, 0]))
    P3.rotation = np.array([2 * np.pi, 0.0])
    np.testing.assert_allclose(P3.dense_S(0), Sr, atol=1e-12)


# --------------------------------------------------------------------- planted mistakes
# A plausible slip in the oracle must fail one of the pins above; these plant one at a time.

def test_planted_graf_index_flip_is_caught(monkeypatch):
    orig = graf.translation_matrix

    def flipped(p, k, xm, xl, p_out=None):
        return orig(p, k, xl, xm, p_out)          # x_l - x_m instead of x_m - x_l
    monkeypatch.setattr(graf, "translation_matrix", flipped)
    with pytest.raises(AssertionError):
        test_graf_translation_pointwise(2.0)


def test_planted_branch_sign_is_caught(monkeypatch):
    orig = sommerfeld.branch_s
    monkeypatch.setattr(sommerfeld, "branch_s", lambda xi, k: np.conj(orig(xi, k)))
    with pytest.raises(AssertionError):
        test_multipole_to_sommerfeld_pts1(3)


def test_planted_traction_term_drop_is_caught(monkeypatch):
    orig = disc.mode_matrix

    def dropped(kind, n, kp, ks, R, bc, lam, mu):
        return orig(kind, n, kp, ks, R, bc, 0.0, mu)     # lambda term dropped
    monkeypatch.setattr(disc, "mode_matrix", dropped)
    with pytest.raises(AssertionError):
        test_disc_scattering_matrix_boundary_condition(1, 0.5)


# --------------------------------------------------------------------- wide particle clouds
def _graded_rule(width, L):
    npan, depth, grade = syn.contour_for_width(width)
    return sommerfeld.contour(npan, 16, 20.0, depth, grade, (L.kp_u, L.ks_u, L.kp_l, L.ks_l))


@pytest.mark.parametrize("dx,dy", [(140.0, 2.0), (75.0, 3.5), (20.0, 2.2)])
def test_graded_rule_reproduces_som1_at_large_separation(dx, dy):
    """som1 (Sec. 3) on the shallow graded rule chosen for a cloud of width 143, against the closed
    form (i/4) H_0(k r) evaluated by scipy."""
    L = Layered(syn.MEDIA_STD, 6.0)
    xi, W = _graded_rule(143.0, L)
    for k in (L.kp_l, L.ks_l):
        s = sommerfeld.branch_s(xi, k)
        quad = (W * np.exp(-s * dy) / s * np.exp(1j * xi * dx)).sum() / (4 * np.pi)
        ex = 0.25j * special.hankel1(0, k * math.hypot(dx, dy))
        assert abs(quad - ex) <= 1e-9 * abs(ex)


def test_graded_rule_reproduces_pts1_high_order_at_large_separation():
    L = Layered(syn.MEDIA_STD, 6.0)
    xi, W = _graded_rule(143.0, L)
    k, xm, x, y = L.ks_l, -60.0, 70.0, 0.0
    # high orders need a deeper source for the integrand to decay by |t| = t_max = 20
    for n, ym in ((0, -1.4), (7, -1.4), (-13, -8.0), (20, -8.0)):
        s = sommerfeld.branch_s(xi, k)
        integ = ((-1.0) ** n / (1j * np.pi)) * np.exp(s * (ym - y)) / s * np.exp(1j * xi * (x - xm)) \
            * ((s - xi) / (1j * k)) ** n
        ex = special.hankel1(n, k * math.hypot(x - xm, y - ym)) * np.exp(1j * n * math.atan2(y - ym, x - xm))
        assert abs((W * integ).sum() - ex) <= 1e-8 * abs(ex)


def test_paper_contour_is_unusable_for_wide_clouds():
    """Reading A20: with the paper's depth 1/2 and 512 nodes, e^{i xi dx} grows like e^{dx/2} on the
    contour and its oscillation is unresolved; som1 at dx = 50 is off by orders of magnitude."""
    L = Layered(syn.MEDIA_STD, 6.0)
    xi, W = sommerfeld.contour(32, 16, 20.0)
    k, dx, dy = L.ks_l, 50.0, 2.0
    s = sommerfeld.branch_s(xi, k)
    quad = (W * np.exp(-s * dy) / s * np.exp(1j * xi * dx)).sum() / (4 * np.pi)
    ex = 0.25j * special.hankel1(0, k * math.hypot(dx, dy))
    assert abs(quad - ex) > 1.0 * abs(ex)
