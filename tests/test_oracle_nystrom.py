"""Pins of the oracle's non-circular particles (Sec. 4.3) and of its whole coupled formulation.

Each test ties oracle.nystrom, oracle.layered_bie or the adaptive Sommerfeld quadrature to something
other than itself: closed-form quadrature moments, central differences of the fundamental solution,
its small-argument series, the closed-form disc scattering matrix, an exact exterior solution from a
point force inside a star, the paper's two coefficient formulas (S7, S10) against each other, the
solver on a rotated boundary, a brute-force boundary integral solve of three stars with the layered
Green's function, and adaptive Gauss-Kronrod quadrature of the contour integral.  Planted mistakes
show that the checks see the errors they are meant to see."""
import numpy as np
import pytest

import synthetic as syn
from oracle import disc, layered_bie, nystrom, sommerfeld, system, waves

H4 = nystrom.Host(2.0, 1.0, 4.0)      # the lower layer of the workloads at omega = 4
H6 = nystrom.Host(2.0, 1.0, 6.0)


# ----------------------------------------------------------------------------- quadrature weights

@pytest.mark.parametrize("m", [0, 1, 4, 9, 15])
def test_kress_log_weights_exact_on_trig_polynomials(m):
    """int_0^{2pi} ln(4 sin^2(tau/2)) cos(m tau) dtau = -2 pi / m (m >= 1), 0 (m = 0)."""
    N = 32
    R = nystrom.kress_log_weights(N)
    t = 2 * np.pi * np.arange(N) / N
    for i in (0, 5):
        got = sum(R[(i - j) % N] * np.cos(m * t[j]) for j in range(N))
        want = 0.0 if m == 0 else -2 * np.pi / m * np.cos(m * t[i])
        assert abs(got - want) < 1e-12


@pytest.mark.parametrize("m", [-15, -3, 0, 1, 7])
def test_hilbert_weights_exact_on_trig_polynomials(m):
    """(1/2pi) PV int cot((tau - t)/2) e^{i m tau} dtau = i sign(m) e^{i m t}."""
    N = 32
    T = nystrom.hilbert_weights(N)
    t = 2 * np.pi * np.arange(N) / N
    for i in (0, 11):
        got = sum(T[(i - j) % N] * np.exp(1j * m * t[j]) for j in range(N))
        assert abs(got - 1j * np.sign(m) * np.exp(1j * m * t[i])) < 1e-12


# ----------------------------------------------------------------------------- kernels

def test_traction_kernel_matches_central_differences_of_phi():
    """The closed-form traction of each column of Phi equals sigma(u) nu built by waves.traction from
    central differences of Phi."""
    z = np.array([0.31, -0.17])
    nu = np.array([0.6, 0.8])
    d = 1e-6
    Jac = np.zeros((2, 2, 2), complex)     # [i, j, k] = d_k Phi_ij
    for k in range(2):
        e = np.zeros(2)
        e[k] = d
        Jac[:, :, k] = (nystrom.fundamental(z + e, H4) - nystrom.fundamental(z - e, H4)) / (2 * d)
    want = np.empty((2, 2), complex)
    for j in range(2):
        g = [[Jac[0, j, 0], Jac[0, j, 1]], [Jac[1, j, 0], Jac[1, j, 1]]]
        want[:, j] = waves.traction(g, nu[0], nu[1], H4.lam, H4.mu)
    got = nystrom.traction_kernel(z, nu, H4)
    assert np.abs(got - want).max() < 1e-8 * np.abs(want).max()


def test_fundamental_solution_solves_navier_off_the_source():
    """mu Lap Phi + (lam + mu) grad div Phi + w^2 Phi = 0 away from y (fourth-order differences)."""
    z0 = np.array([0.4, 0.7])
    d = 1e-3

    def F(dx, dy):
        return nystrom.fundamental(z0 + np.array([dx, dy]), H4)

    def d2(a, b):
        ea = np.eye(2)[a] * d
        eb = np.eye(2)[b] * d
        return (nystrom.fundamental(z0 + ea + eb, H4) - nystrom.fundamental(z0 + ea - eb, H4)
                - nystrom.fundamental(z0 - ea + eb, H4) + nystrom.fundamental(z0 - ea - eb, H4)) / (4 * d * d)

    H = [[d2(a, b) for b in range(2)] for a in range(2)]
    lap = H[0][0] + H[1][1]
    res = np.empty((2, 2), complex)
    for j in range(2):
        for i in range(2):
            gd = H[i][0][0, j] + H[i][1][1, j]          # d_i div of column j
            res[i, j] = H4.mu * lap[i, j] + (H4.lam + H4.mu) * gd + H4.omega ** 2 * F(0, 0)[i, j]
    assert np.abs(res).max() < 1e-5 * H4.omega ** 2 * np.abs(F(0, 0)).max()


def test_log_free_part_of_phi_at_zero_matches_the_series():
    """Phi - (2i/pi) Phi^J ln r tends to c_I I + c_rr r_hat r_hat^T with an O(r^2 ln r) remainder."""
    cI, crr = nystrom.phi_smooth_at_zero(H6)
    errs = []
    for r in (1e-2, 1e-3, 1e-4):
        rh = np.array([np.cos(0.3), np.sin(0.3)])
        z = r * rh
        S = nystrom.fundamental(z, H6) - (2j / np.pi) * nystrom.fundamental(z, H6, "J") * np.log(r)
        errs.append(np.abs(S - (cI * np.eye(2) + crr * np.outer(rh, rh))).max())
    assert errs[2] < 1e-7 and errs[2] < 1e-3 * errs[0]


def test_static_limit_of_the_traction_kernel_is_kelvin():
    """The Cauchy-singular part of the traction kernel is that of the static Kelvin solution: the
    difference is O(r ln r)."""
    nu = np.array([0.6, 0.8])
    # (below r ~ 1e-5 the 1/r^2 terms of the Hankel form cancel to rounding and the check is moot)
    d = [np.abs(nystrom.traction_kernel(r * np.array([0.8, -0.6]), nu, H4)
                - nystrom.kelvin_traction(r * np.array([0.8, -0.6]), nu, H4)).max() for r in (1e-2, 1e-4)]
    k = np.abs(nystrom.kelvin_traction(1e-4 * np.array([0.8, -0.6]), nu, H4)).max()
    assert d[1] < 1e-5 * k and d[1] < 1e-1 * d[0]


# ----------------------------------------------------------------------------- scattering matrices

def _dense_disc(p, h, R, bc):
    nc = 2 * p + 1
    Sd = disc.disc_smatrix(p, h.kp, h.ks, R, bc, h.lam, h.mu)
    S = np.zeros((2, nc, 2, nc), complex)
    for i in range(nc):
        S[:, i, :, i] = Sd[i]
    return S.reshape(2 * nc, 2 * nc)


@pytest.mark.parametrize("bc", [0, 1])
def test_nystrom_on_a_disc_matches_closed_form(bc):
    """A star with a2 = 0 is a disc: the Nystrom matrix (S10 route) equals the closed-form disc S,
    entry by entry relative to each order's own magnitude up to order 20."""
    p = 20
    nc = 2 * p + 1
    S = nystrom.scattering_matrix(nystrom.StarCurve(0.5), bc, H4, p, N=128).reshape(2, nc, 2, nc)
    Sd = disc.disc_smatrix(p, H4.kp, H4.ks, 0.5, bc, H4.lam, H4.mu)
    for i in range(nc):
        assert np.abs(S[:, i, :, i] - Sd[i]).max() <= 1e-12 * np.abs(Sd[i]).max()
    off = S.copy()
    for i in range(nc):
        off[:, i, :, i] = 0
    assert np.abs(off).max() < 1e-14


def test_s7_single_layer_formula_on_a_disc():
    S = nystrom.scattering_matrix(nystrom.StarCurve(0.45), 1, H6, 12, N=128, route="S7")
    assert np.abs(S - _dense_disc(12, H6, 0.45, 1)).max() < 1e-13


STAR = nystrom.StarCurve(0.4, 0.08, 5)


@pytest.mark.parametrize("bc", [0, 1])
def test_star_matrix_converges_spectrally(bc):
    """64 -> 128 -> 256 nodes: the differences fall by orders of magnitude (a wrong diagonal limit or
    Cauchy correction leaves first-order convergence)."""
    S = {N: nystrom.scattering_matrix(STAR, bc, H6, 12, N=N) for N in (64, 128, 256)}
    d1 = np.abs(S[64] - S[256]).max()
    d2 = np.abs(S[128] - S[256]).max()
    assert d2 < 1e-9 and d2 < 1e-3 * d1


@pytest.mark.parametrize("bc", [0, 1])
def test_point_force_inside_a_star_is_reproduced_outside(bc):
    """Exterior problem whose exact solution is the field Phi(x, z0) q of two point forces at z0
    inside the star: with the boundary data of that field, the boundary integral solve reproduces it
    at exterior points (rigid: displacement data, combined layer; traction-free: traction data,
    single layer)."""
    B = nystrom.Boundary(STAR, 192, H6)
    z0 = np.array([0.05, -0.1])
    q = np.array([[1.0, 0.2], [0.3, -1.0]])
    zb = B.x - z0
    data = nystrom.fundamental(zb, H6) @ q if bc == 0 else nystrom.traction_kernel(zb, B.nu, H6) @ q
    phi, cond = nystrom.solve_density(B, bc, data)
    th = np.linspace(0, 2 * np.pi, 11, endpoint=False)
    X, Y = 0.9 * np.cos(th), 0.75 * np.sin(th)
    got = B.potential(phi, X, Y, "C" if bc == 0 else "S")
    want = nystrom.fundamental(np.stack([X, Y], 1) - z0, H6) @ q
    assert cond < 100
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_s7_and_s10_agree_for_a_traction_free_star():
    """Sec. 4.3 gives two routes from the density to the outgoing coefficients: the single-layer
    formula S7 and the projection formula S10 on a circle outside the particle."""
    S10 = nystrom.scattering_matrix(STAR, 1, H6, 12, N=192)
    S7 = nystrom.scattering_matrix(STAR, 1, H6, 12, N=192, route="S7")
    assert np.abs(S7 - S10).max() < 1e-13 * np.abs(S10).max()


@pytest.mark.parametrize("bc", [0, 1])
def test_rotation_phase_matches_the_solver_on_the_rotated_star(bc):
    """Reading A11: the matrix of the copy rotated by phi is e^{-i (n - n') phi} S.  The solver run on
    the rotated boundary fixes the sign: the opposite phase misses by O(0.1)."""
    phi = 0.7
    S0 = nystrom.scattering_matrix(STAR, bc, H6, 10, N=128)
    Sr = nystrom.scattering_matrix(nystrom.StarCurve(0.4, 0.08, 5, rotation=phi), bc, H6, 10, N=128)
    assert np.abs(Sr - nystrom.rotate(S0, 10, phi)).max() < 1e-13
    assert np.abs(Sr - nystrom.rotate(S0, 10, -phi)).max() > 1e-2


def test_problem_dense_s_rotates_prototypes_like_the_rotated_solve():
    """system.Problem.dense_S (the matrix the GPU parity tests use for prototype particles) against
    the Nystrom matrix of the rotated star, with the unrotated matrix as the prototype table."""
    p = 8
    wl = syn.small_case(13, 2, p, omega=6.0)
    wl.rotation = np.array([0.4, 2.2])
    S0 = nystrom.scattering_matrix(STAR, 1, H6, p, N=128)
    P = system.Problem(wl, proto_S=S0[None], proto_index=np.array([0, 0]))
    for m in range(2):
        Sr = nystrom.scattering_matrix(nystrom.StarCurve(0.4, 0.08, 5, rotation=wl.rotation[m]), 1, H6, p, N=128)
        assert np.abs(P.dense_S(m) - Sr).max() < 1e-13


def test_planted_flip_of_the_rotation_phase_is_caught(monkeypatch):
    orig = system.Problem.dense_S

    def flipped(self, m):
        S = orig(self, m)
        n = np.tile(np.arange(-self.p, self.p + 1), 2)
        return S * np.exp(2j * (n[:, None] - n[None, :]) * self.rotation[m])   # e^{+i(n - n') phi}

    monkeypatch.setattr(system.Problem, "dense_S", flipped)
    with pytest.raises(AssertionError):
        test_problem_dense_s_rotates_prototypes_like_the_rotated_solve()


def test_planted_missing_cauchy_correction_is_caught(monkeypatch):
    monkeypatch.setattr(nystrom, "hilbert_weights", lambda N: np.zeros(N))
    with pytest.raises(AssertionError):
        test_point_force_inside_a_star_is_reproduced_outside(1)


def test_combined_layer_stays_well_conditioned_where_the_double_layer_alone_does_not():
    """Reading A22: over the star sizes of the 1000-particle workload (omega = 4, a in [0.3, 0.6]) the
    double layer alone passes near interior Neumann eigenfrequencies; the combined layer does not."""
    worst_dl, worst_cf = 0.0, 0.0
    for a in np.linspace(0.52, 0.55, 7):
        B = nystrom.Boundary(nystrom.StarCurve(a, 0.2 * a, 5), 64, H4)
        I = np.eye(2 * B.N)
        worst_dl = max(worst_dl, np.linalg.cond(0.5 * I + B.double_layer()))
        worst_cf = max(worst_cf, np.linalg.cond(0.5 * I + B.double_layer() - 1j * B.single_layer()))
    assert worst_dl > 1e3 and worst_cf < 50


# ----------------------------------------------------------------------------- whole formulation

def test_point_force_multipole_reproduces_phi():
    g = layered_bie.point_force_coefficients(H4)
    X, Y = np.array([0.7, -0.3, 0.1]), np.array([0.2, 0.5, -0.9])
    for k in range(2):
        u1, u2, _ = waves.field_of_coeffs("H", g[0, :, k], g[1, :, k], 1, H4.kp, H4.ks, X, Y)
        want = nystrom.fundamental(np.stack([X, Y], 1), H4)[:, :, k]
        assert np.abs(np.stack([u1, u2], 1) - want).max() < 1e-14 * np.abs(want).max()


@pytest.fixture(scope="module")
def three_stars():
    wl = syn.small_case(41, 3, 8, omega=3.0, nrhs=1)
    a = np.array([0.35, 0.3, 0.4])
    wl.centres = np.array([[-1.8, -1.7], [1.0, -2.4], [-0.4, -4.4]])
    wl.radius = 1.2 * a
    wl.bc = np.array([0, 1, 0])
    wl.rotation = np.array([0.3, 1.1, 2.0])
    P = system.Problem(wl)
    curves = [nystrom.StarCurve(a[m], 0.2 * a[m], 5, rotation=wl.rotation[m]) for m in range(3)]
    bie = layered_bie.LayeredBIE(P, curves, wl.centres, wl.bc, N=96)
    X = np.concatenate([np.linspace(-4, 4, 9), [0.3, -1.0]])
    Y = np.concatenate([np.full(9, -0.5), [-3.4, -3.1]])
    u = bie.field(bie.solve(int(wl.inc_kind[0]), float(wl.inc_angle[0])), X, Y)
    return wl, a, X, Y, u


def _ms_field(wl, a, X, Y, p):
    h = nystrom.Host(2.0, 1.0, wl.omega)
    wl.p = p
    protos = np.stack([nystrom.scattering_matrix(nystrom.StarCurve(a[m], 0.2 * a[m], 5), wl.bc[m], h, p, N=96)
                       for m in range(3)])
    P = system.Problem(wl, proto_S=protos, proto_index=np.arange(3))
    gam = P.solve_lu(P.rhs(wl.inc_kind, wl.inc_angle))
    return P.scattered_field(gam, X, Y)[0]


def test_multiple_scattering_solve_matches_brute_force_layered_bie(three_stars):
    """Pin T10: three stars (rigid, traction-free, rigid; rotated) below the interface.  The coupled
    multiple-scattering solve (Nystrom scattering matrices, Graf translations, the separable reflected
    operator, plane-wave right-hand side) converges to the brute-force boundary integral solve with
    the layered Green's function as the order p grows: 2e-5, 7e-7, 7e-9 measured at p = 8, 12, 16."""
    wl, a, X, Y, u = three_stars
    e = [np.abs(_ms_field(wl, a, X, Y, p) - u).max() / np.abs(u).max() for p in (8, 16)]
    assert e[1] < 2e-8 and e[1] < 1e-2 * e[0]


def test_planted_transposed_reflection_is_caught_by_the_brute_force_solve(three_stars, monkeypatch):
    wl, a, X, Y, u = three_stars
    orig = system.Problem.reflection_table
    monkeypatch.setattr(system.Problem, "reflection_table",
                        lambda self: np.ascontiguousarray(np.transpose(orig(self), (0, 2, 1))))
    e = np.abs(_ms_field(wl, a, X, Y, 12) - u).max() / np.abs(u).max()
    assert e > 1e-4


def test_fixed_contour_rule_matches_adaptive_gauss_kronrod():
    """Reading A5: the composite Gauss-Legendre rule (32 panels x 16 nodes, depth 1/2) against adaptive
    Gauss-Kronrod quadrature of the same contour integral; and the truncation at t_max = 20 against
    t_max = 40."""
    wl = syn.small_case(7, 3, 8, omega=2.0, nrhs=2)
    P = system.Problem(wl)
    x = syn.random_coeffs(3, wl.M, wl.p, 2)
    fixed = sommerfeld.layered_apply(P.xi, P.W, P.L, P.centres, x)
    ad, err = sommerfeld.layered_apply_adaptive(P.L, P.centres, x)
    scale = np.abs(ad).max()
    assert np.abs(fixed - ad).max() < 1e-12 * scale and err < 1e-11 * scale
    ad40, _ = sommerfeld.layered_apply_adaptive(P.L, P.centres, x, t_max=40.0)
    assert np.abs(ad40 - ad).max() < 1e-9 * scale
