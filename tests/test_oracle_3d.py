"""Pins of the 3D oracle (oracle/sph3d.py, oracle/layered3d.py; Sec. 6) against what the mathematics
fixes: orthonormality and the addition theorem of the spherical harmonics, finite differences of the
harmonics and of the wave functions' curls, the exponential itself for the plane-wave coefficients
(real and complex directions), boundary conditions on spheres, the local expansion reproducing the
sources' field, the polar Sommerfeld quadrature of the paper's spectral representation reproducing the
outgoing field above a particle, zero reflection between identical half-spaces, energy balance at
propagating nodes, and the boundary residual of solved multi-sphere systems falling with the order."""

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import layered3d as L3
from oracle import sph3d as S

KP, KS, LAM, MU = 1.0, 2.0, 2.0, 1.0          # lower layer of the 3D workload at omega = 2


def _sph(th, ph):
    return np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])


def test_harmonics_orthonormal_conjugate_and_addition_theorem():
    p = 7
    d, w = S.sphere_rule(12)
    Y = S.ylm(p, d)
    assert abs(np.einsum("k,ki,kj->ij", w, Y.conj(), Y) - np.eye(S.nlm(p))).max() < 1e-13
    assert abs(Y.conj() - Y[:, S.neg_m(p)]).max() < 1e-15
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=3), rng.normal(size=3)
    a, b = a / np.linalg.norm(a), b / np.linalg.norm(b)
    Ya, Yb = S.ylm(p, a), S.ylm(p, b)
    n, _ = S.orders(p)
    for k in range(p + 1):
        sel = n == k
        assert abs((Ya[sel] * Yb[sel].conj()).sum() - (2 * k + 1) / (4 * np.pi) * eval_legendre(k, a @ b)) < 1e-14


def test_surface_gradient_against_differences():
    p, h = 6, 1e-6
    for th, ph in ((0.7, 1.3), (2.2, -0.4)):
        G = S.grad_ylm(p, _sph(th, ph))
        dth = (S.ylm(p, _sph(th + h, ph)) - S.ylm(p, _sph(th - h, ph))) / (2 * h)
        dph = (S.ylm(p, _sph(th, ph + h)) - S.ylm(p, _sph(th, ph - h))) / (2 * h)
        eth = np.array([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
        eph = np.array([-np.sin(ph), np.cos(ph), 0.0])
        Gn = dth[:, None] * eth[None] + (dph / np.sin(th))[:, None] * eph[None]
        assert abs(G - Gn).max() < 1e-8


@pytest.mark.parametrize("kind", ["h", "j"])
def test_wave_functions_are_gradient_and_curls(kind):
    """L = grad(z Y), M = curl(x z Y), N = curl M / (i ks), by central differences."""
    p, h = 5, 1e-5
    x0 = np.array([0.7, -0.4, 0.55])
    E = np.eye(3)

    def scal(x, k):
        r = np.linalg.norm(x)
        z, _ = S.radial(p, k * r, kind)
        n, _ = S.orders(p)
        return z[n] * S.ylm(p, x / r)

    def curl(f):
        J = np.stack([(f(x0 + h * E[i]) - f(x0 - h * E[i])) / (2 * h) for i in range(3)], axis=-1)
        return np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], axis=-1)

    N, M, L = S.vswf(p, KP, KS, x0, kind)
    Lf = np.stack([(scal(x0 + h * E[i], KP) - scal(x0 - h * E[i], KP)) / (2 * h) for i in range(3)], axis=-1)
    scale = np.abs(L).max()
    assert abs(L - Lf).max() < 1e-8 * scale
    Mf = curl(lambda x: scal(x, KS)[:, None] * x[None, :])
    assert abs(M - Mf[1:]).max() < 1e-8 * np.abs(M).max()
    Nf = curl(lambda x: S.vswf(p, KP, KS, x, kind)[1]) / (1j * KS)
    assert abs(N - Nf).max() < 1e-7 * np.abs(N).max()


@pytest.mark.parametrize("complex_dir", [False, True])
def test_paper_plane_wave_coefficients_reproduce_the_wave(complex_dir):
    """Sec. 6.3: the coefficients a, b, c expand e^{i ks x.d} (d x pol) x d + e^{i kp x.d} (d.pol) d; with
    a complex direction (an evanescent wave below the interface) by analytic continuation."""
    rng = np.random.default_rng(1)
    if complex_dir:
        lam, th = 2.9, 0.8
        d = np.array([lam * np.cos(th), lam * np.sin(th), -np.sqrt(KS * KS - lam * lam + 0j)]) / KS
    else:
        d = np.array([0.3, 0.5, -0.8])
        d = d / np.linalg.norm(d)
    pol = rng.normal(size=3) + 1j * rng.normal(size=3)
    c = S.plane_wave_coeffs(22, KP, d, pol)
    for x in (np.array([0.2, 0.1, -0.3]), np.array([-0.35, 0.2, 0.1])):
        u = S.field(22, KP, KS, x, c, "j")
        ud = np.exp(1j * KS * (x @ d)) * np.cross(np.cross(d, pol), d) + np.exp(1j * KP * (x @ d)) * (d @ pol) * d
        assert abs(u - ud).max() < 1e-13 * max(1.0, abs(ud).max())


def test_planted_plane_wave_sign_fails():
    """The pin above catches a flipped sign of the M-coefficient b."""
    d = np.array([0.3, 0.5, -0.8]) / np.linalg.norm([0.3, 0.5, -0.8])
    pol = np.array([0.2, -1.0, 0.4], dtype=complex)
    c = S.plane_wave_coeffs(16, KP, d, pol)
    nmn = S.sizes(16)[0]
    c[nmn:2 * nmn] *= -1
    x = np.array([0.2, 0.1, -0.3])
    u = S.field(16, KP, KS, x, c, "j")
    ud = np.exp(1j * KS * (x @ d)) * np.cross(np.cross(d, pol), d) + np.exp(1j * KP * (x @ d)) * (d @ pol) * d
    assert abs(u - ud).max() > 1e-2


def _traction(u, x, normal, h=1e-5):
    E = np.eye(3)
    J = np.stack([(u(x + h * E[i]) - u(x - h * E[i])) / (2 * h) for i in range(3)], axis=-1)
    sig = LAM * np.trace(J) * np.eye(3) + MU * (J + J.T)
    return sig @ normal


@pytest.mark.parametrize("bc", [0, 1])
def test_sphere_matrices_satisfy_the_boundary_condition(bc):
    """Rigid: u = 0; traction-free: sigma n = 0 (stress by central differences), per mode on r = R."""
    p, R = 4, 0.45
    nmn, nl, tot = S.sizes(p)
    Sn = S.sphere_smatrix(p, KP, KS, LAM, MU, R, bc)
    d, _ = S.sphere_rule(4)
    for j in (0, 3, nmn + 3, 2 * nmn, 2 * nmn + 5, tot - 1):
        a = np.zeros(tot, complex)
        a[j] = 1.0
        g = S.apply_sphere_S(p, Sn, a)

        def u(x):
            return S.field(p, KP, KS, x, a, "j") + S.field(p, KP, KS, x, g, "h")
        for x in R * d[::5]:
            if bc == 0:
                assert abs(u(x)).max() < 1e-12
            else:
                assert abs(_traction(u, x, x / R)).max() < 1e-7


def test_planted_traction_term_fails():
    """Dropping the mu (n x curl) term of the N traction breaks the traction-free condition."""
    p, R = 3, 0.45
    nmn, nl, tot = S.sizes(p)
    orig = S._traction_coeffs

    def planted(n, kp, ks, lam, mu, R_, kind):
        tNr, tNg, tM, tLr, tLg = orig(n, kp, ks, lam, mu, R_, kind)
        z, _ = S.radial(n, ks * R_, kind)
        return tNr, tNg + 1j * ks * mu * z[n], tM, tLr, tLg
    try:
        S._traction_coeffs = planted
        Sn = S.sphere_smatrix(p, KP, KS, LAM, MU, R, 1)
    finally:
        S._traction_coeffs = orig
    a = np.zeros(tot, complex)
    a[2] = 1.0
    g = S.apply_sphere_S(p, Sn, a)
    x = R * np.array([0.3, 0.5, -0.8]) / np.linalg.norm([0.3, 0.5, -0.8])
    t = _traction(lambda y: S.field(p, KP, KS, y, a, "j") + S.field(p, KP, KS, y, g, "h"), x, x / R)
    assert abs(t).max() > 1e-3


def test_translation_reproduces_the_sources_field():
    """Local coefficients by projection on a sphere about the target, evaluated inside it, against the
    outgoing fields of two sources summed directly."""
    rng = np.random.default_rng(3)
    p, P = 4, 18
    src = np.array([[0.0, 0.0, 0.0], [2.1, 0.4, -0.3]])
    tgt = np.array([1.3, -0.4, 0.7])
    nmn, nl, tot = S.sizes(p)
    nmnP, nlP, totP = S.sizes(P)
    gs = []
    for _ in range(2):
        g = rng.normal(size=tot) + 1j * rng.normal(size=tot)
        gp = np.zeros(totP, complex)
        gp[:nmn], gp[nmnP:nmnP + nmn], gp[2 * nmnP:2 * nmnP + nl] = g[:nmn], g[nmn:2 * nmn], g[2 * nmn:]
        gs.append(gp)
    a = S.translate(P, KP, KS, src, gs, tgt, 0.35, 26)
    for off in (np.array([0.1, 0.15, -0.12]), np.array([-0.2, 0.05, 0.1])):
        x = tgt + off
        u_loc = S.field(P, KP, KS, x - tgt, a, "j")
        u_dir = sum(S.field(P, KP, KS, x - c, g, "h") for c, g in zip(src, gs))
        assert abs(u_loc - u_dir).max() < 1e-10 * abs(u_dir).max()


def test_spectral_representation_of_outgoing_waves():
    """Sec. 6.2: the upgoing amplitudes of the paper's formulas, summed on a converged polar rule,
    reproduce the outgoing field of each family above the particle."""
    md = L3.Media3(1.0, 0.5, LAM, MU, 2.0)
    p = 4
    nmn, nl, tot = S.sizes(p)
    rng = np.random.default_rng(4)
    g = rng.normal(size=tot) + 1j * rng.normal(size=tot)
    c0 = np.array([0.0, 0.0, -3.0])
    P3 = L3.Problem3(md, [c0], [0.4], [0], p, n_r=400, n_theta=96, t_max=30.0, alpha=0.6, beta=1.0, n_panels=20)
    eP, _, _ = L3.basis(md.kp_l, P3.lam, P3.th, True)
    eS, vS, hS = L3.basis(md.ks_l, P3.lam, P3.th, True)
    X = np.array([0.3, -0.2, -1.5])
    fp = P3.W * np.exp(1j * md.kp_l * (X @ eP.T))
    fs = P3.W * np.exp(1j * md.ks_l * (X @ eS.T))
    for blk in (slice(0, nmn), slice(nmn, 2 * nmn), slice(2 * nmn, tot)):
        gg = np.zeros(tot, complex)
        gg[blk] = g[blk]
        U = P3.m2s(gg[None])
        u = (np.einsum("q,q,qi->i", fp, U[:, 0], eP) + np.einsum("q,q,qi->i", fs, U[:, 1], vS)
             + np.einsum("q,q,qi->i", fs, U[:, 2], hS))
        ud = S.field(p, md.kp_l, md.ks_l, X - c0, gg, "h")
        assert abs(u - ud).max() < 1e-10 * abs(ud).max()


def test_reflection_zero_between_identical_layers_and_energy_balance():
    md_same = L3.Media3(LAM, MU, LAM, MU, 2.0)
    lam = np.array([0.3, 0.7, 1.5, 2.5, 0.2 - 0.1j])
    th = np.array([0.3, 1.1, 2.0, -0.5, 0.9])
    assert abs(L3.reflection(md_same, lam, th)).max() < 1e-14
    Dt = L3.transmission_of_incident(md_same, 1, 0.5, 0.7)[2]          # an SV wave passes unchanged
    assert abs(Dt - np.array([0.0, 1.0, 0.0])).max() < 1e-14
    md = L3.Media3(1.0, 0.5, LAM, MU, 2.0)
    lam = np.array([0.3, 0.7, 0.95])
    th = np.array([0.2, 1.0, 2.5])
    R = L3.reflection(md, lam, th)
    wv = L3._waves(md, lam, th)
    for q in range(3):
        A = np.zeros((6, 6), complex)
        for i in range(3):
            A[:3, i], A[3:, i] = wv["ld"][0][i][q], wv["ld"][1][i][q]
            A[:3, 3 + i], A[3:, 3 + i] = -wv["uu"][0][i][q], -wv["uu"][1][i][q]
        for j in range(3):
            U = np.eye(3)[j]
            sol = np.linalg.solve(A, -np.concatenate([wv["lu"][0][j][q], wv["lu"][1][j][q]]))
            assert abs(sol[:3] - R[q] @ U).max() < 1e-13

            def F(name, amps):
                return sum(L3.flux_z(amps[i] * wv[name][0][i][q], amps[i] * wv[name][1][i][q], md.omega)
                           for i in range(3))
            fin, fr, ft = F("lu", U), F("ld", sol[:3]), F("uu", sol[3:])
            assert fin > 0 and fr <= 0 and ft > 0
            assert abs(fin + fr - ft) < 1e-13 * fin


def test_solved_system_boundary_residual_falls_with_the_order():
    """Three rigid spheres below the interface, three plane waves from above (P, SV, SH): the total
    field (transmitted incident + outgoing + reflected, each evaluated directly) on the spheres."""
    md = L3.Media3(1.0, 0.5, LAM, MU, 2.0)
    c = np.array([[0.0, 0.0, -2.0], [1.6, 0.3, -2.5], [-0.4, 1.5, -3.0]])
    R = np.array([0.4, 0.35, 0.45])
    inc = [(0, 0.4, 0.3), (1, 0.6, 1.0), (2, 0.3, 2.0)]
    res = []
    for p in (4, 6, 8):
        P3 = L3.Problem3(md, c, R, [0] * 3, p, n_r=32, n_theta=16, t_max=12.0, alpha=0.5, beta=1.0, n_panels=2,
                         ntheta_proj=16)
        g = P3.solve_lu(P3.rhs(inc))
        d, _ = S.sphere_rule(4)
        worst = 0.0
        for r in range(3):
            for m in range(3):
                X = c[m] + R[m] * d
                worst = max(worst, abs(P3.incident_field(*inc[r], X) + P3.scattered_field(g[..., r], X)).max())
        res.append(worst)
    assert res[1] < 0.1 * res[0] and res[2] < res[1] and res[2] < 1e-4, res


def test_projection_translation_against_the_addition_theorem_series():
    """The projection (sph3d.translate) against the scalar addition theorem for the compressional part,
    written independently: h_n Y_n^m about the source = sum 4 pi i^{nu-n+q} h_q(k d) Y_q^{m-mu}(d^) G
    j_nu Y_nu^mu about the target, G = int Y_n^m conj(Y_nu^mu) conj(Y_q^{m-mu}) by sphere quadrature."""
    p, kp = 4, KP
    nmn, nl, tot = S.sizes(p)
    rng = np.random.default_rng(11)
    g = np.zeros(tot, complex)
    g[2 * nmn:] = rng.normal(size=nl) + 1j * rng.normal(size=nl)     # compressional part only
    src, tgt = np.array([0.2, -0.1, -2.0]), np.array([1.3, -0.4, -2.6])
    d = tgt - src
    dn = np.linalg.norm(d)
    P2 = 2 * p
    dirs, w = S.sphere_rule(24)
    Y = S.ylm(P2, dirs)
    hq, _ = S.radial(P2, kp * dn, "h")
    Yd = S.ylm(P2, d / dn)
    want = np.zeros(nl, complex)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            for nu in range(p + 1):
                for mu in range(-nu, nu + 1):
                    s = 0
                    for q in range(abs(n - nu), n + nu + 1, 2):
                        if abs(m - mu) > q:
                            continue
                        G = np.sum(w * Y[:, S.idx(n, m)] * Y[:, S.idx(nu, mu)].conj() * Y[:, S.idx(q, m - mu)].conj())
                        s += 4 * np.pi * 1j ** (nu - n + q) * hq[q] * Yd[S.idx(q, m - mu)] * G
                    want[S.idx(nu, mu)] += s * g[2 * nmn + S.idx(n, m)]
    got = S.translate(p, KP, KS, [src], [g], tgt, 0.5 * dn)
    assert abs(got[2 * nmn:] - want).max() < 1e-11 * abs(want).max()
    assert abs(got[:2 * nmn]).max() < 1e-11 * abs(want).max()
