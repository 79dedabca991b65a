"""Nystrom boundary integral solver for one non-circular particle and its scattering matrix (Sec. 4.3).

Test infrastructure only (see oracle/__init__.py).

Equations (Sec. 4.3, bdint).  With the elastic fundamental solution of the host layer (density 1)
    Phi(x, y) = -(i / (4 w^2)) [ grad grad^T H_0(kp r) + grad_perp grad_perp^T H_0(ks r) ],  r = |x - y|,
(equal to (i/(4 mu)) H_0(ks r) I + (i/(4 w^2)) grad grad^T (H_0(ks r) - H_0(kp r)); it solves
mu Lap u + (lam + mu) grad div u + w^2 u = -delta), the scattered field of a particle is written as
  traction-free:  u = S phi,           S phi(x) = int Phi(x, y) phi(y) ds_y,
                  boundary equation  -phi/2 + K' phi = -T u_inc   (traction on the outward normal);
  rigid:          u = (D - i eta S) phi,  D phi(x) = int [T_{nu(y)} Phi(x, y)]^T phi(y) ds_y,
                  boundary equation   phi/2 + K phi - i eta S phi = -u_inc.
The paper states the rigid equation with the double layer alone and assumes it uniquely solvable;
its remark proposes a combined potential where that fails.  Here eta = 1 is always added (reading
A22): the double layer alone is singular at interior Neumann eigenfrequencies of the particle,
which the star sizes of the 1000- and 10^4-particle workloads approach.

Kernel splitting (Kress's product quadrature on 2n equispaced nodes t_j = pi j / n).  Every kernel
k(t, tau) |x'(tau)| is written as
    K1(t, tau) ln(4 sin^2((t - tau)/2)) + B cot((tau - t)/2) + K2(t, tau)
with K1, K2 smooth and B a constant matrix:
  * H_n = J_n + i Y_n and Y_n = (2/pi) J_n ln(z/2) + (poles and a power series), so the coefficient of
    ln r in Phi is L = (2i/pi) Phi^J, Phi^J being Phi with every H_n replaced by J_n (an entire
    function of x - y).  With ln r = ln(4 sin^2((t-tau)/2))/2 + smooth, K1 = (i/pi) Phi^J |x'| for S
    and (i/pi) T Phi^J |x'| for the traction kernels.
  * Near r = 0, Phi = Phi_0 + O(r^2 ln r), where Phi_0 = a ln r I + b r_hat r_hat^T is the static
    (Kelvin) solution, a = -(lam + 3 mu) / (4 pi mu (lam + 2 mu)), b = (lam + mu) / (4 pi mu (lam + 2 mu)).
    Its traction carries the only non-integrable part, c (nu_i z_j - nu_j z_i) / r^2 with
    c = mu / (2 pi (lam + 2 mu)); on the curve this is c (z . tau) / r^2 E, E = [[0, 1], [-1, 0]], so
    B = -(c/2) E for K and K'.
  * The diagonal of K2 is the limit of the remainder, worked out from the small-argument series of
    H_0, H_1, H_2 (DLMF 10.8.2) and from the Taylor expansion of the curve.
Quadrature weights: the log weights R_j of Kress (exact on trigonometric polynomials of degree < n,
the cos(n t) term included), the trapezoid rule for K2, and for the Cauchy part the Hilbert-transform
weights of the trigonometric interpolant, T_j = -(1/n) sum_{m=1}^{n-1} sin(m (t - t_j)) (exact
because (1/2pi) PV int cot((tau - t)/2) e^{i m tau} dtau = i sign(m) e^{i m t}).

Scattering matrix.  Incident fields are the regular basis grad(J_n(kp r) e^{in th}),
grad_perp(J_n(ks r) e^{in th}) about the centre (Sec. 4.3).  The outgoing coefficients of each
scattered field come from
  S10 (the projection formula of the remark in Sec. 4.3): the field on a circle of radius rho outside
      the particle, projected on e^{-i l th} r_hat and e^{-i l th} th_hat, then the 2x2 Hankel mode
      matrix; the paper prints e^{+i l th}, which projects on mode -l (reading A21);
  S7 (the single-layer coefficient formula of Sec. 4.3): alpha_l, beta_l as boundary integrals of the
      density against E_l^k(y) = J_l(k |y|) e^{-i l th(y)} (traction-free particles).
The two must agree for a traction-free particle.  Rotated copies: S' = e^{-i (n - n') phi} S
(reading A11), checked against the solver run on the rotated boundary.
"""
from __future__ import annotations

import functools

import numpy as np
from scipy import special

from .waves import field_of_coeffs, traction

E_ROT = np.array([[0.0, 1.0], [-1.0, 0.0]])


class Host:
    """Lame constants and wavenumbers of the layer holding the particle (density 1, Sec. 2)."""

    def __init__(self, lam: float, mu: float, omega: float):
        self.lam, self.mu, self.omega = float(lam), float(mu), float(omega)
        self.kp = omega / np.sqrt(lam + 2 * mu)
        self.ks = omega / np.sqrt(mu)
        # Kelvin (static) solution constants and the Cauchy coefficient of its traction
        self.a0 = -(lam + 3 * mu) / (4 * np.pi * mu * (lam + 2 * mu))
        self.b0 = (lam + mu) / (4 * np.pi * mu * (lam + 2 * mu))
        self.c0 = mu / (2 * np.pi * (lam + 2 * mu))


# ----------------------------------------------------------------------------- kernels

def _Z(kind, n, x):
    return special.hankel1(n, x) if kind == "H" else special.jv(n, x)


def radial(kind: str, r, h: Host):
    """A1, A1', A2, A2' with Phi = A1(r) I + A2(r) r_hat r_hat^T (Z = H: Phi; Z = J: Phi^J):
    A1 = (i/(4mu)) Z_0(ks r) - (i/(4 w^2 r)) [ks Z_1(ks r) - kp Z_1(kp r)],
    A2 = (i/(4 w^2)) [ks^2 Z_2(ks r) - kp^2 Z_2(kp r)]  (from d_i d_j Z_0(kr) = -k Z_1/r d_ij + k^2 Z_2 r_i r_j).
    Derivatives: (Z_0)' = -k Z_1, (k Z_1(kr)/r)' = -k^2 Z_2(kr)/r, Z_2'(z) = Z_1(z) - 2 Z_2(z)/z."""
    w2 = h.omega ** 2
    kp, ks = h.kp, h.ks
    r = np.asarray(r, float)
    zs, zp = ks * r, kp * r
    s0, s1, s2 = _Z(kind, 0, zs), _Z(kind, 1, zs), _Z(kind, 2, zs)
    p1, p2 = _Z(kind, 1, zp), _Z(kind, 2, zp)
    A1 = 1j / (4 * h.mu) * s0 - 1j / (4 * w2 * r) * (ks * s1 - kp * p1)
    dA1 = -1j * ks / (4 * h.mu) * s1 + 1j / (4 * w2 * r) * (ks ** 2 * s2 - kp ** 2 * p2)
    A2 = 1j / (4 * w2) * (ks ** 2 * s2 - kp ** 2 * p2)
    dA2 = 1j / (4 * w2) * (ks ** 3 * (s1 - 2 * s2 / zs) - kp ** 3 * (p1 - 2 * p2 / zp))
    return np.asarray(A1), np.asarray(dA1), np.asarray(A2), np.asarray(dA2)


def fundamental(z, h: Host, kind: str = "H"):
    """Phi(x, y) (or Phi^J) for z = x - y of shape (..., 2), z != 0: array (..., 2, 2)."""
    r = np.asarray(np.hypot(z[..., 0], z[..., 1]))
    A1, _, A2, _ = radial(kind, r, h)
    rh = z / r[..., None]
    return A1[..., None, None] * np.eye(2) + A2[..., None, None] * rh[..., :, None] * rh[..., None, :]


def traction_of(z, nu, r, dA1, A2, dA2, h: Host):
    """t[..., i, j]: traction component i, on the unit normal nu at x, of column j of
    Phi = A1 I + A2 r_hat r_hat^T as a function of x, z = x - y (Sec. 2 tracdef):
        div_j = (A1' + A2' + A2/r) r_j
        t_ij  = lam div_j nu_i + mu [A1' (r.nu) d_ij + A1' r_i nu_j + 2 A2' (r.nu) r_i r_j
                                     + A2 (2 nu_i r_j + nu_j r_i + d_ij (r.nu) - 4 r_i r_j (r.nu)) / r]."""
    rh = z / r[..., None]
    rn = np.einsum("...k,...k->...", rh, nu)
    I = np.eye(2)
    rr = rh[..., :, None] * rh[..., None, :]
    nr = nu[..., :, None] * rh[..., None, :]          # nu_i r_j
    rnT = rh[..., :, None] * nu[..., None, :]         # r_i nu_j
    div = (dA1 + dA2 + A2 / r)[..., None, None] * nr
    t = h.lam * div + h.mu * (
        (dA1 * rn)[..., None, None] * I + dA1[..., None, None] * rnT + (2 * dA2 * rn)[..., None, None] * rr
        + (A2 / r)[..., None, None] * (2 * nr + np.swapaxes(nr, -1, -2) + rn[..., None, None] * I
                                       - 4 * rn[..., None, None] * rr))
    return t


def traction_kernel(z, nu, h: Host, kind: str = "H"):
    r = np.asarray(np.hypot(z[..., 0], z[..., 1]))
    _, dA1, A2, dA2 = radial(kind, r, h)
    return traction_of(z, nu, r, dA1, A2, dA2, h)


def kelvin_traction(z, nu, h: Host):
    """Traction kernel of the static solution a ln r I + b r_hat r_hat^T (A1' = a / r, A2 = b, A2' = 0)."""
    r = np.asarray(np.hypot(z[..., 0], z[..., 1]))
    return traction_of(z, nu, r, h.a0 / r, np.full_like(r, h.b0), np.zeros_like(r), h)


def phi_smooth_at_zero(h: Host):
    """Limit of Phi - L ln r at r -> 0 without its direction-dependent part: returns (c_I, c_rr) with
    Phi - L ln r -> c_I I + c_rr r_hat r_hat^T.  From H_0(z) = 1 + (2i/pi)(ln(z/2) + g) + ...,
    Y_1(z) = -2/(pi z) + (2/pi) J_1 ln(z/2) - (1 - 2g) z / (2 pi) + ..., Y_2(z) = -4/(pi z^2) - 1/pi + ...
    (g Euler's constant; DLMF 10.8.2)."""
    g = np.euler_gamma
    kp, ks, mu, w2 = h.kp, h.ks, h.mu, h.omega ** 2
    d = ks ** 2 - kp ** 2
    cI = (1j / (4 * mu) - (np.log(ks / 2) + g) / (2 * np.pi * mu) - 1j * d / (8 * w2)
          + (ks ** 2 * np.log(ks / 2) - kp ** 2 * np.log(kp / 2) - (1 - 2 * g) * d / 2) / (4 * np.pi * w2))
    c_rr = d / (4 * np.pi * w2)
    return cI, c_rr


def phiJ_at_zero(h: Host):
    """Phi^J(0) = [i/(4 mu) - i (ks^2 - kp^2) / (8 w^2)] I (J_0(0) = 1, J_1(z)/z -> 1/2, J_2(0) = 0)."""
    return (1j / (4 * h.mu) - 1j * (h.ks ** 2 - h.kp ** 2) / (8 * h.omega ** 2)) * np.eye(2)


# ----------------------------------------------------------------------------- curves

class StarCurve:
    """x(t) = Rot(phi) (a1 + a2 cos(a3 t)) (cos t, sin t), t in [0, 2pi) (the shape family of Sec. 7),
    counter-clockwise; a2 = 0 is a disc of radius a1."""

    def __init__(self, a1: float, a2: float = 0.0, a3: int = 5, rotation: float = 0.0):
        self.a1, self.a2, self.a3, self.rot = float(a1), float(a2), int(a3), float(rotation)

    def enclosing_radius(self):
        return self.a1 + abs(self.a2)

    def eval(self, t):
        """Points x, first and second derivatives in t: three (len(t), 2) arrays."""
        a1, a2, k = self.a1, self.a2, self.a3
        r = a1 + a2 * np.cos(k * t)
        r1 = -a2 * k * np.sin(k * t)
        r2 = -a2 * k * k * np.cos(k * t)
        c, s = np.cos(t), np.sin(t)
        x = np.stack([r * c, r * s], 1)
        dx = np.stack([r1 * c - r * s, r1 * s + r * c], 1)
        ddx = np.stack([r2 * c - 2 * r1 * s - r * c, r2 * s + 2 * r1 * c - r * s], 1)
        cr, sr = np.cos(self.rot), np.sin(self.rot)
        Q = np.array([[cr, -sr], [sr, cr]])
        return x @ Q.T, dx @ Q.T, ddx @ Q.T


# ----------------------------------------------------------------------------- quadrature weights

def kress_log_weights(N: int):
    """R_k, k = 0..N-1 (N = 2n even): int_0^{2pi} ln(4 sin^2((t_i - tau)/2)) f(tau) dtau ~ sum_j R_{(i-j) mod N} f(t_j),
    R_k = -(2 pi / n) sum_{m=1}^{n-1} cos(m t_k) / m - (pi / n^2) cos(n t_k),  t_k = pi k / n."""
    n = N // 2
    tk = np.pi * np.arange(N) / n
    m = np.arange(1, n)
    return -(2 * np.pi / n) * (np.cos(np.outer(tk, m)) / m).sum(1) - (np.pi / n ** 2) * np.cos(n * tk)


def hilbert_weights(N: int):
    """T_k, k = 0..N-1: (1/2pi) PV int_0^{2pi} cot((tau - t_i)/2) f(tau) dtau ~ sum_j T_{(i-j) mod N} f(t_j),
    T_k = -(1/n) sum_{m=1}^{n-1} sin(m t_k)."""
    n = N // 2
    tk = np.pi * np.arange(N) / n
    m = np.arange(1, n)
    return -(1.0 / n) * np.sin(np.outer(tk, m)).sum(1)


# ----------------------------------------------------------------------------- boundary operators

class Boundary:
    """Nodes, normals and the Nystrom matrices S, K, K' of one closed curve with N nodes.

    Unknown vectors have layout (N, 2): node j, Cartesian component c, flattened as 2 j + c."""

    def __init__(self, curve: StarCurve, N: int, h: Host, centre=(0.0, 0.0)):
        if N % 2:
            raise ValueError("N must be even")
        self.curve, self.N, self.h = curve, N, h
        self.t = 2 * np.pi * np.arange(N) / N
        x, dx, ddx = curve.eval(self.t)
        self.x = x + np.asarray(centre, float)
        self.dx, self.ddx = dx, ddx
        self.speed = np.hypot(dx[:, 0], dx[:, 1])
        self.tau = dx / self.speed[:, None]
        self.nu = np.stack([self.tau[:, 1], -self.tau[:, 0]], 1)       # outward for counter-clockwise
        self._S = self._K = self._Kp = None

    # -- pieces
    def _pairs(self):
        N = self.N
        z = self.x[:, None, :] - self.x[None, :, :]
        off = ~np.eye(N, dtype=bool)
        zz = np.where(off[..., None], z, 1.0)                # placeholder on the diagonal
        dt = self.t[:, None] - self.t[None, :]
        lg = np.where(off, np.log(np.where(off, 4 * np.sin(dt / 2) ** 2, 1.0)), 0.0)
        ct = np.where(off, 1.0 / np.tan(np.where(off, -dt / 2, 1.0)), 0.0)    # cot((tau - t)/2)
        return zz, off, lg, ct

    def _assemble(self, K1, K2, B=None):
        N = self.N
        R = kress_log_weights(N)
        idx = (np.arange(N)[:, None] - np.arange(N)[None, :]) % N
        A = R[idx][..., None, None] * K1 + (2 * np.pi / N) * K2
        if B is not None:
            T = hilbert_weights(N)
            A = A + (2 * np.pi * T[idx])[..., None, None] * B
        return A.transpose(0, 2, 1, 3).reshape(2 * N, 2 * N)

    def single_layer(self):
        if self._S is None:
            h = self.h
            zz, off, lg, _ = self._pairs()
            sp = self.speed[None, :, None, None]
            full = fundamental(zz, h, "H") * sp
            K1 = 1j / np.pi * fundamental(zz, h, "J") * sp
            K2 = full - K1 * lg[..., None, None]
            cI, c_rr = phi_smooth_at_zero(h)
            L0 = (2j / np.pi) * phiJ_at_zero(h)
            for i in range(self.N):
                tt = np.outer(self.tau[i], self.tau[i])
                s = self.speed[i]
                K1[i, i] = 1j / np.pi * phiJ_at_zero(h) * s
                K2[i, i] = s * (L0 * np.log(s) + cI * np.eye(2) + c_rr * tt)
            self._S = self._assemble(K1, K2)
        return self._S

    def _diag_traction(self, i):
        """Diagonal limit of the smooth part of K and of K' at node i (the same for both):
        (x''.nu / (2 |x'|)) (c I + 4 mu b tau tau^T) from the bounded Kelvin terms, whose ratio
        (z . nu) / r^2 tends to -+ x''.nu / (2 |x'|^2), and -c E (x'.x'') / (2 |x'|^2) from the Cauchy term
        minus B cot((tau - t)/2)."""
        h = self.h
        s = self.speed[i]
        kn = float(self.ddx[i] @ self.nu[i])
        kt = float(self.ddx[i] @ self.dx[i])
        tt = np.outer(self.tau[i], self.tau[i])
        bounded = (kn / (2 * s)) * (h.c0 * np.eye(2) + 4 * h.mu * h.b0 * tt)
        return bounded - h.c0 * E_ROT * kt / (2 * s * s)

    def adjoint_double_layer(self):
        """K': traction at x (normal nu(x)) of the single layer, principal value."""
        if self._Kp is None:
            h = self.h
            zz, off, lg, ct = self._pairs()
            nu = np.broadcast_to(self.nu[:, None, :], zz.shape)
            sp = self.speed[None, :, None, None]
            full = traction_kernel(zz, nu, h, "H") * sp
            K1 = 1j / np.pi * traction_kernel(zz, nu, h, "J") * sp
            B = -0.5 * h.c0 * E_ROT
            K2 = full - K1 * lg[..., None, None] - ct[..., None, None] * B
            for i in range(self.N):
                K1[i, i] = 0.0
                K2[i, i] = self._diag_traction(i)
            self._Kp = self._assemble(K1, K2, B)
        return self._Kp

    def double_layer(self):
        """K: kernel [T_{nu(y)} Phi(x, y)]^T = -t(x - y, nu(y))^T, principal value."""
        if self._K is None:
            h = self.h
            zz, off, lg, ct = self._pairs()
            nu = np.broadcast_to(self.nu[None, :, :], zz.shape)
            sp = self.speed[None, :, None, None]
            full = -np.swapaxes(traction_kernel(zz, nu, h, "H"), -1, -2) * sp
            K1 = -1j / np.pi * np.swapaxes(traction_kernel(zz, nu, h, "J"), -1, -2) * sp
            B = -0.5 * h.c0 * E_ROT
            K2 = full - K1 * lg[..., None, None] - ct[..., None, None] * B
            for i in range(self.N):
                K1[i, i] = 0.0
                K2[i, i] = self._diag_traction(i)
            self._K = self._assemble(K1, K2, B)
        return self._K

    # -- potentials at points off the boundary (smooth integrands: trapezoid rule)
    def potential(self, phi, X, Y, layer: str, eta: float = 1.0):
        """Field of density phi (N, 2, ncol) at points (X, Y): 'S' single layer, 'C' = D - i eta S.
        Returns (npts, 2, ncol)."""
        P = np.stack([np.ravel(X), np.ravel(Y)], 1)
        z = P[:, None, :] - self.x[None, :, :]
        w = (2 * np.pi / self.N) * self.speed
        G = fundamental(z, self.h, "H")
        if layer == "C":
            nu = np.broadcast_to(self.nu[None, :, :], z.shape)
            G = -np.swapaxes(traction_kernel(z, nu, self.h, "H"), -1, -2) - 1j * eta * G
        return np.einsum("pjab,j,jbc->pac", G, w, phi)

    def potential_gradient(self, phi, X, Y, layer: str, eta: float = 1.0, d: float = 1e-5):
        """Displacement and its Jacobian by central differences of width d (for tractions off the
        boundary in tests only)."""
        X = np.ravel(X)
        Y = np.ravel(Y)
        u = self.potential(phi, X, Y, layer, eta)
        gx = (self.potential(phi, X + d, Y, layer, eta) - self.potential(phi, X - d, Y, layer, eta)) / (2 * d)
        gy = (self.potential(phi, X, Y + d, layer, eta) - self.potential(phi, X, Y - d, layer, eta)) / (2 * d)
        return u, gx, gy


# ----------------------------------------------------------------------------- boundary solves

def solve_density(B: Boundary, bc: int, data, eta: float = 1.0):
    """Density for boundary data (N, 2, ncol): bc = 0 rigid (data = -u_inc on the boundary, combined
    layer), bc = 1 traction-free (data = -T u_inc, single layer)."""
    N = B.N
    I = np.eye(2 * N)
    if bc == 0:
        A = 0.5 * I + B.double_layer() - 1j * eta * B.single_layer()
    else:
        A = -0.5 * I + B.adjoint_double_layer()
    rhs = data.reshape(2 * N, -1)
    return np.linalg.solve(A, rhs).reshape(N, 2, -1), np.linalg.cond(A)


def incident_basis(B: Boundary, p: int, centre=(0.0, 0.0)):
    """Displacement and traction (outward normal) on the boundary of the 2(2p+1) regular basis fields
    grad(J_n(kp r) e^{in th}) (b = 0) and grad_perp(J_n(ks r) e^{in th}) (b = 1) about the centre, in
    the column order (b, n).  Returns two arrays (N, 2, 2nc)."""
    nc = 2 * p + 1
    X = B.x[:, 0] - centre[0]
    Y = B.x[:, 1] - centre[1]
    U = np.empty((B.N, 2, 2 * nc), complex)
    Tr = np.empty((B.N, 2, 2 * nc), complex)
    for b in range(2):
        for i in range(nc):
            c = np.zeros((2, nc), complex)
            c[b, i] = 1.0
            u1, u2, g = field_of_coeffs("J", c[0], c[1], p, B.h.kp, B.h.ks, X, Y)
            t1, t2 = traction(g, B.nu[:, 0], B.nu[:, 1], B.h.lam, B.h.mu)
            U[:, 0, b * nc + i], U[:, 1, b * nc + i] = u1, u2
            Tr[:, 0, b * nc + i], Tr[:, 1, b * nc + i] = t1, t2
    return U, Tr


def project_coefficients(B: Boundary, phi, layer: str, p: int, rho: float, eta: float = 1.0, npts: int = 256,
                         centre=(0.0, 0.0)):
    """S10: outgoing coefficients (2, 2p+1, ncol) of the field of density phi from its values on the
    circle |x - centre| = rho (outside the particle), by the Hankel mode matrix of Sec. 4.3's
    projection formula with the e^{-i l th} projection (reading A21)."""
    th = 2 * np.pi * np.arange(npts) / npts
    X = centre[0] + rho * np.cos(th)
    Y = centre[1] + rho * np.sin(th)
    u = B.potential(phi, X, Y, layer, eta)                  # (npts, 2, ncol)
    ur = np.cos(th)[:, None] * u[:, 0] + np.sin(th)[:, None] * u[:, 1]
    ut = -np.sin(th)[:, None] * u[:, 0] + np.cos(th)[:, None] * u[:, 1]
    kp, ks = B.h.kp, B.h.ks
    out = np.empty((2, 2 * p + 1, phi.shape[2]), complex)
    for i, l in enumerate(range(-p, p + 1)):
        e = np.exp(-1j * l * th)[:, None] / npts            # (1/2pi) int . e^{-i l th} dth
        fr = (e * ur).sum(0)
        ft = (e * ut).sum(0)
        hp = special.hankel1(l, kp * rho)
        hs = special.hankel1(l, ks * rho)
        hpd = 0.5 * kp * (special.hankel1(l - 1, kp * rho) - special.hankel1(l + 1, kp * rho))
        hsd = 0.5 * ks * (special.hankel1(l - 1, ks * rho) - special.hankel1(l + 1, ks * rho))
        M = np.array([[hpd, -1j * l / rho * hs], [1j * l / rho * hp, hsd]])
        out[:, i] = np.linalg.solve(M, np.stack([fr, ft]))
    return out


def single_layer_coefficients(B: Boundary, phi, p: int, centre=(0.0, 0.0)):
    """S7: outgoing coefficients (2, 2p+1, ncol) of the single-layer field of phi,
        [alpha_l; beta_l] = i/(8 w^2) int [[kp (E^p_{l-1} - E^p_{l+1}), -i kp (E^p_{l-1} + E^p_{l+1})],
                                          [i ks (E^s_{l-1} + E^s_{l+1}),  ks (E^s_{l-1} - E^s_{l+1})]] phi ds,
    E^k_l(y) = J_l(k |y|) e^{-i l th(y)}, y relative to the centre."""
    h = B.h
    y = B.x - np.asarray(centre, float)
    ry = np.hypot(y[:, 0], y[:, 1])
    ty = np.arctan2(y[:, 1], y[:, 0])
    w = (2 * np.pi / B.N) * B.speed

    def E(k, l):
        return special.jv(l, k * ry) * np.exp(-1j * l * ty)

    pref = 1j / (8 * h.omega ** 2)
    out = np.empty((2, 2 * p + 1, phi.shape[2]), complex)
    for i, l in enumerate(range(-p, p + 1)):
        pm, pp = E(h.kp, l - 1), E(h.kp, l + 1)
        sm, sp = E(h.ks, l - 1), E(h.ks, l + 1)
        a = h.kp * (pm - pp)[:, None] * phi[:, 0] - 1j * h.kp * (pm + pp)[:, None] * phi[:, 1]
        b = 1j * h.ks * (sm + sp)[:, None] * phi[:, 0] + h.ks * (sm - sp)[:, None] * phi[:, 1]
        out[0, i] = pref * (w[:, None] * a).sum(0)
        out[1, i] = pref * (w[:, None] * b).sum(0)
    return out


def scattering_matrix(curve: StarCurve, bc: int, h: Host, p: int, N: int = 128, rho: float | None = None,
                      eta: float = 1.0, route: str = "S10", return_cond: bool = False):
    """(2nc, 2nc) scattering matrix of the particle, row (b, n) <- column (b', n') (incoming basis
    coefficient to outgoing coefficient), by the Nystrom solve and the S10 projection (route 'S10')
    or, for traction-free particles, the S7 single-layer formula (route 'S7').  rho defaults to
    1.25 times the enclosing radius."""
    B = Boundary(curve, N, h)
    U, Tr = incident_basis(B, p)
    phi, cond = solve_density(B, bc, -U if bc == 0 else -Tr, eta)
    layer = "C" if bc == 0 else "S"
    if route == "S7":
        if bc != 1:
            raise ValueError("S7 is the single-layer formula (traction-free particles)")
        coef = single_layer_coefficients(B, phi, p)
    else:
        rho = 1.25 * curve.enclosing_radius() if rho is None else rho
        coef = project_coefficients(B, phi, layer, p, rho, eta)
    nc = 2 * p + 1
    S = coef.reshape(2 * nc, 2 * nc)
    return (S, cond) if return_cond else S


def rotate(S, p: int, phi: float):
    """Scattering matrix of the copy rotated by phi (reading A11): S'_{(b,n),(b',n')} = e^{-i (n - n') phi} S."""
    n = np.tile(np.arange(-p, p + 1), 2)
    return S * np.exp(-1j * (n[:, None] - n[None, :]) * phi)


@functools.lru_cache(maxsize=256)
def _table(a1: float, a2: float, a3: int, bc: int, lam: float, mu: float, omega: float, p: int, N: int):
    return scattering_matrix(StarCurve(a1, a2, a3), bc, Host(lam, mu, omega), p, N=N)


def workload_tables(wl, N: int = 128):
    """Scattering matrices (Q, 2nc, 2nc) of the star prototypes of a synthetic workload (shapes
    wl.proto_shape, boundary conditions wl.proto_bc) in the lower layer, in their own unrotated frame;
    prototypes no particle uses are left zero."""
    nc = 2 * wl.p + 1
    out = np.zeros((wl.n_proto, 2 * nc, 2 * nc), complex)
    used = set(int(q) for q in np.asarray(wl.proto) if q >= 0)
    for q in sorted(used):
        a1, a2, a3 = wl.proto_shape[q]
        out[q] = _table(float(a1), float(a2), int(a3), int(wl.proto_bc[q]), float(wl.media.lam_l),
                        float(wl.media.mu_l), float(wl.omega), int(wl.p), int(N))
    return out
