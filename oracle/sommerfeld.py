"""Sommerfeld-integral part of the layered operator (Sec. 3, 5.1, 5.3, 5.4).

Test infrastructure only (see oracle/__init__.py).

Contour (Sec. 5.1): xi(t) = t - i d tanh(t) on [-t_max, t_max], d = 1/2 in the paper.  The
paper uses a trapezoid rule; we use composite Gauss-Legendre panels (reading A5), optionally
graded at the branch points, and the same nodes for every part of the operator.  Weights
W_q = w_q xi'(t_q), xi'(t) = 1 - i d sech^2 t.  The factor e^{i xi (x_m - x_l)} grows like
e^{d |x_m - x_l|} on one half of the contour, so wide particle clouds need a shallower contour
(reading A20).

Branch (Sec. 3 remark, reading A4): s_k(xi) = sqrt(xi^2 - k^2) with Re s >= 0, taken as
-i * sqrt(k^2 - xi^2) with the principal root, which also gives the limiting-absorption
value s = -i sqrt(k^2 - xi^2) on the real propagating interval.

Plane-wave bases used by the textbook route:
  lower, upgoing   P: grad(e^{i xi x - s'_p y}),  S: grad_perp(e^{i xi x - s'_s y})
  lower, downgoing P: grad(e^{i xi x + s'_p y}),  S: grad_perp(e^{i xi x + s'_s y})
  upper, upgoing   P: grad(e^{i xi x - s_p y}),   S: grad_perp(e^{i xi x - s_s y})
  upper, downgoing P: grad(e^{i xi x + s_p y}),   S: grad_perp(e^{i xi x + s_s y})

M2S (Sec. 5.4, pts1 / sed1 / sed2): above a particle centred at (x_l, y_l),
  grad(H_n(k r) e^{in th}) = (-1)^n/(i pi) int grad(e^{i xi x - s y}) e^{s y_l - i xi x_l}/s ((s - xi)/(i k))^n dxi
so the upgoing amplitudes are U_b(xi) = sum_l sum_n gamma^l_{b,n} (-1)^n/(i pi) e^{s y_l - i xi x_l}/s ((s-xi)/(ik))^n.

S2L (Sec. 5.3, Jacobi-Anger ja / stm): about a centre (x_m, y_m),
  e^{i xi x + s y} = e^{i xi x_m + s y_m} sum_n i^n e^{i n phi} J_n(k r_m) e^{i n th_m},
with e^{i phi} := (xi - s)/k, the analytic continuation of phi = arccos(xi/k) (reading A3),
so a downgoing amplitude D_b contributes D_b e^{i xi x_m + s y_m} i^n e^{i n phi} to the local
coefficient of order n.

Reflection: the 2x2 map R(xi): (U_P, U_S) -> (D_P, D_S) is computed two independent ways:
  * plane-wave route: continuity of displacement and of the traction T_y (Sec. 3) across y = 0
    for the four plane waves, solved per node;
  * paper route: the 4x4 system A_xi sigma = b_xi of Sec. 3 (aa), with the particle field's
    spectral displacement b1 and traction b2 of Sec. 5.4 on the right-hand side, then sigma_21,
    sigma_22 mapped to local expansions by eee1 (through c1/c2) of Sec. 5.3.
"""
from __future__ import annotations

import numpy as np

from .media import Layered


def contour(n_panels: int, nodes_per_panel: int, t_max: float, depth: float = 0.5, grade: int = 0,
            branch_points=()):
    """Nodes xi_q and weights W_q = w_q xi'(t_q) of the composite Gauss-Legendre rule on
    xi(t) = t - i depth tanh(t), |t| <= t_max (Sec. 5.1 has depth 1/2).

    Panel edges: -t_max + k (2 t_max / n_panels), k = 0..n_panels; with grade > 0 also each
    branch point c = +-k (k in branch_points) and c +- depth 2^j, j < grade, inside the interval;
    sorted, dropping an edge within 1e-9 of the previous kept one."""
    g, gw = np.polynomial.legendre.leggauss(nodes_per_panel)
    edges = [-t_max + k * (2.0 * t_max / n_panels) for k in range(n_panels + 1)]
    if grade > 0:
        for kb in branch_points:
            for c in (-kb, kb):
                cand = [c] + [c + sg * depth * 2.0 ** j for j in range(grade) for sg in (-1.0, 1.0)]
                edges += [v for v in cand if -t_max < v < t_max]
    kept = []
    for v in sorted(edges):
        if not kept or v - kept[-1] > 1e-9:
            kept.append(v)
    t = []
    w = []
    for a, b in zip(kept[:-1], kept[1:]):
        t.append(0.5 * (b - a) * g + 0.5 * (a + b))
        w.append(0.5 * (b - a) * gw)
    t = np.concatenate(t)
    w = np.concatenate(w)
    xi = t - 1j * depth * np.tanh(t)
    dxi = 1.0 - 1j * depth / np.cosh(t) ** 2
    return xi, w * dxi


def branch_s(xi, k):
    """s = sqrt(xi^2 - k^2) with Re s >= 0 (limiting absorption on the real axis)."""
    xi = np.asarray(xi, dtype=complex)
    return -1j * np.sqrt(k * k - xi * xi)


# ----------------------------------------------------------------------------- plane waves

def _pw(kind: str, xi, d):
    """Displacement amplitude of grad(e^{i xi x + d y}) (kind 'P') or grad_perp(.) (kind 'S')."""
    if kind == "P":
        return np.array([1j * xi, d])
    return np.array([-d, 1j * xi])


def _traction_y(u, xi, d, lam, mu):
    """T_y of a plane wave u e^{i xi x + d y} (Sec. 3: (mu(du1/dy + du2/dx), (lam+2mu) du2/dy + lam du1/dx))."""
    return np.array([mu * (d * u[0] + 1j * xi * u[1]), (lam + 2 * mu) * d * u[1] + lam * 1j * xi * u[0]])


def interface_solve(xi: complex, L: Layered, U=(0.0, 0.0), I=(0.0, 0.0)):
    """Plane-wave route.  Given upgoing lower amplitudes U and downgoing upper amplitudes I
    at horizontal wavenumber xi, return (D, E): downgoing lower and upgoing upper amplitudes
    that make displacement and traction continuous at y = 0."""
    sp_l, ss_l = branch_s(xi, L.kp_l), branch_s(xi, L.ks_l)
    sp_u, ss_u = branch_s(xi, L.kp_u), branch_s(xi, L.ks_u)

    def col(kind, d, lam, mu):
        u = _pw(kind, xi, d)
        return np.concatenate([u, _traction_y(u, xi, d, lam, mu)])

    lo = (L.lam_l, L.mu_l)
    up = (L.lam_u, L.mu_u)
    # unknowns: D_P, D_S (lower, +s y), E_P, E_S (upper, -s y); equation: lower - upper = 0
    A = np.stack([col("P", sp_l, *lo), col("S", ss_l, *lo),
                  -col("P", -sp_u, *up), -col("S", -ss_u, *up)], axis=1)
    rhs = -(U[0] * col("P", -sp_l, *lo) + U[1] * col("S", -ss_l, *lo)) \
        + (I[0] * col("P", sp_u, *up) + I[1] * col("S", ss_u, *up))
    z = np.linalg.solve(A, rhs)
    return z[:2], z[2:]


def reflection_plane_wave(xi: complex, L: Layered):
    """2x2 R with (D_P, D_S) = R (U_P, U_S), plane-wave route."""
    R = np.empty((2, 2), dtype=complex)
    R[:, 0] = interface_solve(xi, L, U=(1.0, 0.0))[0]
    R[:, 1] = interface_solve(xi, L, U=(0.0, 1.0))[0]
    return R


def paper_A(xi: complex, L: Layered):
    """The 4x4 matrix A_xi of Sec. 3 (aa), entry by entry as printed, with one reading.

    Row 2 is the x2-displacement continuity.  The paper prints its lower-layer entry
    lp' - ks'^2/ls' - ls' in column 3 (sigma_21).  The sigma_21 column of the lower spectral
    Green tensor has x2-component i xi (e^{s'_s y} - e^{s'_p y}) / (4 pi omega^2), which vanishes
    at y = 0, while the sigma_22 column has x2-component (ks'^2/s'_s + s'_s - s'_p)/(4 pi omega^2);
    so the entry belongs in column 4 (reading A18).  Every other entry matches the columns of
    the upper and lower spectral Green tensors as printed."""
    ls, lp = branch_s(xi, L.ks_u), branch_s(xi, L.kp_u)
    ls2, lp2 = branch_s(xi, L.ks_l), branch_s(xi, L.kp_l)
    ks, kp, ks2, kp2 = L.ks_u, L.kp_u, L.ks_l, L.kp_l
    lam, mu, lam2, mu2 = L.lam_u, L.mu_u, L.lam_l, L.mu_l
    x2 = xi * xi
    return np.array([
        [ks**2 / ls - x2 / ls + x2 / lp, 0, x2 / ls2 - ks2**2 / ls2 - x2 / lp2, 0],
        [0, ks**2 / ls + ls - lp, 0, lp2 - ks2**2 / ls2 - ls2],   # printed in column 3; see paper_A doc
        [-mu * ks**2, 1j * mu * xi * (ks**2 / ls + 2 * ls - 2 * lp), -mu2 * ks2**2,
         1j * mu2 * xi * (2 * lp2 - 2 * ls2 - ks2**2 / ls2)],
        [1j * xi * (2 * mu * (ls - lp) + lam * kp**2 / lp), -(lam + 2 * mu) * kp**2,
         1j * xi * (2 * mu2 * (lp2 - ls2) - lam2 * kp2**2 / lp2), -(lam2 + 2 * mu2) * kp2**2],
    ], dtype=complex)


# ----------------------------------------------------------------------------- M2S / S2L

def m2s(xi, L: Layered, centres, gamma, chunk: int = 512):
    """Upgoing amplitudes U_P, U_S at every node: arrays (N_S, nrhs) (pts1/sed1/sed2, Sec. 5.4).

    gamma: (M, 2, 2p+1, nrhs) outgoing coefficients (alpha = [:,0], beta = [:,1]).  Particles are
    summed in chunks; each chunk is one matrix product over the orders n."""
    M, _, nc, nrhs = gamma.shape
    p = (nc - 1) // 2
    n = np.arange(-p, p + 1)
    out = []
    for b, k in ((0, L.kp_l), (1, L.ks_l)):
        s = branch_s(xi, k)                                   # (Q,)
        fac = (s - xi) / (1j * k)                             # (Q,)
        powers = ((-1.0) ** n)[None, :] * fac[:, None] ** n[None, :]     # (Q, nc)
        U = np.zeros((xi.size, nrhs), dtype=complex)
        for c0 in range(0, M, chunk):
            c1 = min(M, c0 + chunk)
            cc = centres[c0:c1]
            E = np.exp(s[:, None] * cc[None, :, 1] - 1j * xi[:, None] * cc[None, :, 0])  # (Q, mc)
            E = E / (1j * np.pi * s[:, None])
            g = gamma[c0:c1, b].transpose(1, 0, 2).reshape(nc, -1)           # (nc, mc*nrhs)
            inner = (powers @ g).reshape(xi.size, c1 - c0, nrhs)              # (Q, mc, nrhs)
            U += np.einsum("qm,qmr->qr", E, inner)
        out.append(U)
    return out[0], out[1]


def s2l(xi, W, L: Layered, centres, D_P, D_S, p: int, chunk: int = 512):
    """Local (incoming) coefficients (M, 2, 2p+1, nrhs) of the downgoing field
    int D_P grad(e^{i xi x + s'_p y}) + D_S grad_perp(e^{i xi x + s'_s y}) dxi  (Sec. 5.3, stm)."""
    n = np.arange(-p, p + 1)
    M = centres.shape[0]
    nc = 2 * p + 1
    res = []
    for D, k in ((D_P, L.kp_l), (D_S, L.ks_l)):
        s = branch_s(xi, k)
        eiphi = (xi - s) / k
        powers = (1j ** n)[None, :] * eiphi[:, None] ** n[None, :]       # (Q, nc)
        out = np.empty((M, nc, D.shape[1]), dtype=complex)
        for c0 in range(0, M, chunk):
            c1 = min(M, c0 + chunk)
            cc = centres[c0:c1]
            E = np.exp(1j * xi[:, None] * cc[None, :, 0] + s[:, None] * cc[None, :, 1])  # (Q, mc)
            A = (E * W[:, None])[:, :, None] * powers[:, None, :]                         # (Q, mc, nc)
            out[c0:c1] = (A.reshape(xi.size, -1).T @ D).reshape(c1 - c0, nc, -1)
        res.append(out)
    return np.stack(res, axis=1)


def reflect_nodes(xi, L: Layered, U_P, U_S):
    """(D_P, D_S) = R(xi_q) (U_P, U_S) per node, plane-wave route."""
    D_P = np.empty_like(U_P)
    D_S = np.empty_like(U_S)
    for q in range(xi.size):
        R = reflection_plane_wave(xi[q], L)
        D_P[q] = R[0, 0] * U_P[q] + R[0, 1] * U_S[q]
        D_S[q] = R[1, 0] * U_P[q] + R[1, 1] * U_S[q]
    return D_P, D_S


def layered_apply(xi, W, L: Layered, centres, gamma):
    """Local coefficients of the interface-reflected field generated by gamma (plane-wave route)."""
    U_P, U_S = m2s(xi, L, centres, gamma)
    D_P, D_S = reflect_nodes(xi, L, U_P, U_S)
    p = (gamma.shape[2] - 1) // 2
    return s2l(xi, W, L, centres, D_P, D_S, p)


def layered_apply_adaptive(L: Layered, centres, gamma, t_max: float = 20.0, depth: float = 0.5,
                           epsrel: float = 1e-12):
    """The same reflected operator (R gamma) with the contour integral evaluated by adaptive
    Gauss-Kronrod quadrature (scipy.integrate.quad_vec, 21-point Kronrod rule, error control on the
    vector of every output coefficient) instead of a fixed rule: xi(t) = t - i depth tanh(t) on
    |t| <= t_max (Sec. 5.1), with break points at the branch points +-kp, +-ks of both layers.
    Its difference from the fixed composite rule of `contour` is that rule's discretisation error
    (reading A5).  Returns (local coefficients (M, 2, 2p+1, nrhs), quad_vec's error estimate)."""
    from scipy.integrate import quad_vec
    p = (gamma.shape[2] - 1) // 2
    M = centres.shape[0]

    def f(t):
        xi = np.array([t - 1j * depth * np.tanh(t)])
        dxi = np.array([1.0 - 1j * depth / np.cosh(t) ** 2])
        U_P, U_S = m2s(xi, L, centres, gamma)
        D_P, D_S = reflect_nodes(xi, L, U_P, U_S)
        return s2l(xi, dxi, L, centres, D_P, D_S, p).ravel()

    pts = sorted({s * k for k in (L.kp_u, L.ks_u, L.kp_l, L.ks_l) for s in (-1.0, 1.0) if k < t_max})
    res, err = quad_vec(f, -t_max, t_max, epsrel=epsrel, epsabs=0.0, points=pts, limit=20000)
    return res.reshape(M, 2, 2 * p + 1, gamma.shape[3]), err


def layered_apply_paper(xi, W, L: Layered, centres, gamma, x0: float = 0.0):
    """Same operator by the paper's route: b1/b2 spectral values -> A_xi sigma = b -> eee1.

    b1 gives the spectral displacement (f11, f12) of grad(H_n(kp' r)e^{in th}) and
    (f21, f22) of grad_perp(H_n(ks' r)e^{in th}) at y = 0, scaled by 4 pi omega^2 e^{i xi x0};
    b2 gives their tractions.  Continuity u_1^s - u_2^s = v and T u_1^s - T' u_2^s = T' v
    (rows of aa) put them on the right-hand side.  eee1 maps sigma_21, sigma_22 to local
    coefficients; a quadrature weight W_q multiplies each node (Sec. 5.1)."""
    M, _, nc, nrhs = gamma.shape
    p = (nc - 1) // 2
    n = np.arange(-p, p + 1)
    om2 = L.omega ** 2
    lam2, mu2 = L.lam_l, L.mu_l
    out = np.zeros((M, 2, nc, nrhs), dtype=complex)
    for q in range(xi.size):
        x = xi[q]
        lp2, ls2 = branch_s(x, L.kp_l), branch_s(x, L.ks_l)
        phase = np.exp(1j * x * (x0 - centres[:, 0]))                      # (M,)
        powp = ((-1.0) ** n) * ((lp2 - x) / (1j * L.kp_l)) ** n              # (nc,)
        pows = ((-1.0) ** n) * ((ls2 - x) / (1j * L.ks_l)) ** n
        ep = np.exp(lp2 * centres[:, 1]) * phase
        es = np.exp(ls2 * centres[:, 1]) * phase
        f11 = 4 * om2 * x / lp2 * ep[:, None] * powp[None, :]
        f12 = 4 * om2 * 1j * ep[:, None] * powp[None, :]
        f21 = -4 * om2 * 1j * es[:, None] * pows[None, :]
        f22 = 4 * om2 * x / ls2 * es[:, None] * pows[None, :]
        t11 = mu2 * f11 * (-lp2) + mu2 * f12 * (1j * x)
        t12 = (lam2 + 2 * mu2) * f12 * (-lp2) + lam2 * f11 * (1j * x)
        t21 = mu2 * f21 * (-ls2) + mu2 * f22 * (1j * x)
        t22 = (lam2 + 2 * mu2) * f22 * (-ls2) + lam2 * f21 * (1j * x)
        al = gamma[:, 0]
        be = gamma[:, 1]
        rhs = np.stack([
            np.einsum("mn,mnr->r", f11, al) + np.einsum("mn,mnr->r", f21, be),
            np.einsum("mn,mnr->r", f12, al) + np.einsum("mn,mnr->r", f22, be),
            np.einsum("mn,mnr->r", t11, al) + np.einsum("mn,mnr->r", t21, be),
            np.einsum("mn,mnr->r", t12, al) + np.einsum("mn,mnr->r", t22, be)])
        sig = np.linalg.solve(paper_A(x, L), rhs)                        # (4, nrhs)
        s21, s22 = sig[2], sig[3]
        eiphp = (x - lp2) / L.kp_l
        eiphs = (x - ls2) / L.ks_l
        base = W[q] / (4 * np.pi * om2) * np.exp(1j * x * (centres[:, 0] - x0))   # (M,)
        inp = (1j ** n) * eiphp ** n
        ins = (1j ** n) * eiphs ** n
        cp = (base * np.exp(lp2 * centres[:, 1]))[:, None] * inp[None, :]        # (M, nc)
        cs = (base * np.exp(ls2 * centres[:, 1]))[:, None] * ins[None, :]
        out[:, 0] += cp[:, :, None] * (-1j * x / lp2 * s21 - s22)[None, None, :]
        out[:, 1] += cs[:, :, None] * (s21 - 1j * x / ls2 * s22)[None, None, :]
    return out


# ----------------------------------------------------------------------------- field sums

def downgoing_field(xi, W, L: Layered, D_P, D_S, X, Y):
    """u and grad u of int D_P grad(e^{i xi x + s'_p y}) + D_S grad_perp(e^{i xi x + s'_s y}) dxi.

    D_P, D_S: (Q,) amplitudes for one right-hand side; X, Y: point arrays (lower layer)."""
    X = np.asarray(X, float)[..., None]
    Y = np.asarray(Y, float)[..., None]
    sp, ss = branch_s(xi, L.kp_l), branch_s(xi, L.ks_l)
    ep = W * D_P * np.exp(1j * xi * X + sp * Y)
    es = W * D_S * np.exp(1j * xi * X + ss * Y)
    ix = 1j * xi
    u1 = (ix * ep - ss * es).sum(-1)
    u2 = (sp * ep + ix * es).sum(-1)
    g = [[(ix * ix * ep - ss * ix * es).sum(-1), (ix * sp * ep - ss * ss * es).sum(-1)],
         [(sp * ix * ep + ix * ix * es).sum(-1), (sp * sp * ep + ix * ss * es).sum(-1)]]
    return u1, u2, g


def upgoing_upper_field(xi, W, L: Layered, E_P, E_S, X, Y):
    """u and grad u of int E_P grad(e^{i xi x - s_p y}) + E_S grad_perp(e^{i xi x - s_s y}) dxi (upper layer)."""
    X = np.asarray(X, float)[..., None]
    Y = np.asarray(Y, float)[..., None]
    sp, ss = branch_s(xi, L.kp_u), branch_s(xi, L.ks_u)
    ep = W * E_P * np.exp(1j * xi * X - sp * Y)
    es = W * E_S * np.exp(1j * xi * X - ss * Y)
    ix = 1j * xi
    u1 = (ix * ep + ss * es).sum(-1)
    u2 = (-sp * ep + ix * es).sum(-1)
    g = [[(ix * ix * ep + ss * ix * es).sum(-1), (-ix * sp * ep - ss * ss * es).sum(-1)],
         [(-sp * ix * ep + ix * ix * es).sum(-1), (sp * sp * ep - ix * ss * es).sum(-1)]]
    return u1, u2, g


# ----------------------------------------------------------------------------- incidence

def plane_wave_incidence(kind: int, angle: float, L: Layered):
    """Incident plane wave from the upper layer travelling along d = (cos t, -sin t) (reading A7).

    P-wave u = d e^{i kp d.x} = (1/(i kp)) grad(e^{i kp d.x}); S-wave u = d_perp e^{i ks d.x}
    = (1/(i ks)) grad_perp(e^{i ks d.x}).  Returns (xi, (D_P, D_S), (E_P, E_S), (I_P, I_S)):
    the transmitted (lower, downgoing) and reflected (upper, upgoing) amplitudes of the
    background field of Sec. 7.3 (bplan)."""
    k = L.kp_u if kind == 0 else L.ks_u
    xi = complex(k * np.cos(angle), 0.0)
    I = (1.0 / (1j * k), 0.0) if kind == 0 else (0.0, 1.0 / (1j * k))
    D, E = interface_solve(xi, L, U=(0.0, 0.0), I=I)
    return xi, D, E, I


def point_force_downgoing(xi, L: Layered, z, q):
    """Downgoing plane-wave amplitudes (I_P, I_S) per node of the upper-layer field Phi_u(x, z) q of a
    unit-density point force q at z (z_2 > 0), valid below the source:
        Phi_u(., z) q = -(i/(4 w^2)) [grad (q . grad) H_0(kp r) + grad_perp (q . grad_perp) H_0(ks r)],
    with som1 below the source, H_0(k |x - z|) = (1/(i pi)) int e^{i xi (x - z_1) + s (y - z_2)} / s dxi, so that
    d/dx -> i xi and d/dy -> s.  In the basis grad(e^{i xi x + s_p y}), grad_perp(e^{i xi x + s_s y}):
        I_P = -(i xi q_1 + s_p q_2) e^{-i xi z_1 - s_p z_2} / (4 pi w^2 s_p),
        I_S = -(i xi q_2 - s_s q_1) e^{-i xi z_1 - s_s z_2} / (4 pi w^2 s_s)
    (upper-layer wavenumbers; point sources of Sec. 7.2)."""
    sp, ss = branch_s(xi, L.kp_u), branch_s(xi, L.ks_u)
    w2 = L.omega ** 2
    IP = -(1j * xi * q[0] + sp * q[1]) * np.exp(-1j * xi * z[0] - sp * z[1]) / (4 * np.pi * w2 * sp)
    IS = -(1j * xi * q[1] - ss * q[0]) * np.exp(-1j * xi * z[0] - ss * z[1]) / (4 * np.pi * w2 * ss)
    return IP, IS


def upper_downgoing_field(xi, W, L: Layered, I_P, I_S, X, Y):
    """u and grad u of int I_P grad(e^{i xi x + s_p y}) + I_S grad_perp(e^{i xi x + s_s y}) dxi (upper layer)."""
    X = np.asarray(X, float)[..., None]
    Y = np.asarray(Y, float)[..., None]
    sp, ss = branch_s(xi, L.kp_u), branch_s(xi, L.ks_u)
    ep = W * I_P * np.exp(1j * xi * X + sp * Y)
    es = W * I_S * np.exp(1j * xi * X + ss * Y)
    ix = 1j * xi
    u1 = (ix * ep - ss * es).sum(-1)
    u2 = (sp * ep + ix * es).sum(-1)
    g = [[(ix * ix * ep - ss * ix * es).sum(-1), (ix * sp * ep - ss * ss * es).sum(-1)],
         [(sp * ix * ep + ix * ix * es).sum(-1), (sp * sp * ep + ix * ss * es).sum(-1)]]
    return u1, u2, g


def point_force_transmitted(xi, L: Layered, z, q):
    """Downgoing lower-layer amplitudes (D_P, D_S) per node of the field of the upper-layer point force
    transmitted through the welded interface (the background field of point-source incidence)."""
    IP, IS = point_force_downgoing(xi, L, z, q)
    DP = np.empty_like(IP)
    DS = np.empty_like(IS)
    for k in range(xi.size):
        D, _ = interface_solve(xi[k], L, U=(0.0, 0.0), I=(IP[k], IS[k]))
        DP[k], DS[k] = D
    return DP, DS


def local_expansion_of_plane(xi: complex, D, L: Layered, centres, p: int):
    """Incoming coefficients (M, 2, 2p+1) of D_P grad(e^{i xi x + s'_p y}) + D_S grad_perp(e^{i xi x + s'_s y})
    about every centre, by Jacobi-Anger (Sec. 5.3 ja/stm)."""
    n = np.arange(-p, p + 1)
    out = np.empty((centres.shape[0], 2, 2 * p + 1), dtype=complex)
    for b, k in ((0, L.kp_l), (1, L.ks_l)):
        s = branch_s(xi, k)
        eiphi = (xi - s) / k
        e = np.exp(1j * xi * centres[:, 0] + s * centres[:, 1])
        out[:, b] = D[b] * e[:, None] * ((1j ** n) * eiphi ** n)[None, :]
    return out
