"""3D layered multiple scattering (Sec. 6): two welded elastic half-spaces split at z = 0, rigid or
traction-free spheres in the lower one.  The Sommerfeld integrals over (k_x, k_y) run on the polar rule
of Sec. 6.1: k_rho = lambda(t) = t - i alpha tanh(beta t), t in [0, t_max] by Gauss-Legendre, and
N_theta equispaced angles; the spectral field of a particle above it (block B, Sec. 6.2) and the
plane-wave expansion about a particle (block C, Sec. 6.3) are the paper's formulas; the reflection of
each node's upgoing P, SV, SH waves at the interface is solved from the continuity of displacement and
traction (the plane-wave route); the free-space particle-to-particle part is the projection of the
sources' outgoing fields on a sphere about each target (sph3d.translate).

Test infrastructure only (see oracle/__init__.py).

Plane waves at a node (k_x, k_y) = lambda (cos theta, sin theta) (reading A26): in a layer with
wavenumber k, k_z = sqrt(k^2 - lambda^2) with Im k_z >= 0 (the principal root on the contour), unit
directions e_up = (k_x, k_y, k_z)/k and e_down = (k_x, k_y, -k_z)/k (e.e = 1), and polarisations
P: e,  SV: h x e,  SH: h = (-sin theta, cos theta, 0).  A wave of amplitude A is A pol e^{i k e.x}.
"""
from __future__ import annotations

import numpy as np

from . import sph3d as S3


class Media3:
    """Upper (lam, mu) and lower (lam', mu') layers, unit density, frequency omega."""

    def __init__(self, lam_u, mu_u, lam_l, mu_l, omega):
        self.lam_u, self.mu_u, self.lam_l, self.mu_l, self.omega = map(float, (lam_u, mu_u, lam_l, mu_l, omega))
        self.kp_u = omega / np.sqrt(lam_u + 2 * mu_u)
        self.ks_u = omega / np.sqrt(mu_u)
        self.kp_l = omega / np.sqrt(lam_l + 2 * mu_l)
        self.ks_l = omega / np.sqrt(mu_l)


def polar_rule(n_r: int, n_theta: int, t_max: float, alpha: float, beta: float, n_panels: int = 1):
    """Nodes (lambda, theta) and weights W of sum_q W_q f(q) ~ int int f dk_x dk_y = int lambda d lambda d theta:
    composite Gauss-Legendre in t on [0, t_max] (n_panels equal panels of n_r / n_panels nodes),
    lambda(t) = t - i alpha tanh(beta t), W = w_t lambda lambda'(t) 2 pi / n_theta (Sec. 6.1)."""
    per = n_r // n_panels
    g, gw = np.polynomial.legendre.leggauss(per)
    ts, ws = [], []
    for k in range(n_panels):
        a, b = k * t_max / n_panels, (k + 1) * t_max / n_panels
        ts.append(0.5 * (b - a) * g + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * gw)
    t = np.concatenate(ts)
    w = np.concatenate(ws)
    lam = t - 1j * alpha * np.tanh(beta * t)
    dlam = 1.0 - 1j * alpha * beta / np.cosh(beta * t) ** 2
    th = 2.0 * np.pi * np.arange(n_theta) / n_theta
    L, TH = np.meshgrid(lam, th, indexing="ij")
    W = np.outer(w * lam * dlam, np.full(n_theta, 2.0 * np.pi / n_theta))
    return L.reshape(-1), TH.reshape(-1), W.reshape(-1)


def kz(k, lam):
    return np.sqrt(k * k - lam * lam + 0j)


def basis(k, lam, th, up: bool):
    """Unit direction e, SV and SH polarisations (..., 3) of the waves of wavenumber k at the nodes."""
    z = kz(k, lam)
    c, s = np.cos(th), np.sin(th)
    e = np.stack([lam * c, lam * s, (z if up else -z)], axis=-1) / k
    h = np.stack([-s, c, 0.0 * s], axis=-1).astype(complex)
    v = np.cross(h, e)
    return e, v, h


def traction_z(kvec, A, lam, mu):
    """Traction sigma e_z of the plane wave A e^{i k.x}: i [lam (k.A) e_z + mu (k A_z + A k_z)]."""
    kA = np.sum(kvec * A, axis=-1)
    ez = np.zeros_like(A)
    ez[..., 2] = 1.0
    return 1j * (lam * kA[..., None] * ez + mu * (kvec * A[..., 2:3] + A * kvec[..., 2:3]))


def _waves(md: Media3, lam, th):
    """Per node: displacement and traction columns of the nine waves at z = 0:
    lower up (P, SV, SH), lower down (P, SV, SH), upper up (P, SV, SH), upper down (P, SV, SH)."""
    out = {}
    for name, (k, lm, mu, up) in {"lu": (None, md.lam_l, md.mu_l, True), "ld": (None, md.lam_l, md.mu_l, False),
                                  "uu": (None, md.lam_u, md.mu_u, True), "ud": (None, md.lam_u, md.mu_u, False)}.items():
        kp, ks = (md.kp_l, md.ks_l) if name[0] == "l" else (md.kp_u, md.ks_u)
        eP, _, _ = basis(kp, lam, th, up)
        eS, vS, hS = basis(ks, lam, th, up)
        cols_u = [eP, vS, hS]
        kv = [kp * eP, ks * eS, ks * eS]
        cols_t = [traction_z(kv[i], cols_u[i], lm, mu) for i in range(3)]
        out[name] = (cols_u, cols_t)
    return out


def reflection(md: Media3, lam, th):
    """R (nodes, 3, 3): downgoing lower amplitudes (P, SV, SH) for unit upgoing lower ones, with the
    transmitted upgoing upper waves, from continuity of displacement and traction at z = 0."""
    wv = _waves(md, lam, th)
    n = lam.shape[0]
    R = np.zeros((n, 3, 3), dtype=complex)
    for q in range(n):
        A = np.zeros((6, 6), dtype=complex)
        for j in range(3):
            A[:3, j] = wv["ld"][0][j][q]
            A[3:, j] = wv["ld"][1][j][q]
            A[:3, 3 + j] = -wv["uu"][0][j][q]
            A[3:, 3 + j] = -wv["uu"][1][j][q]
        Bm = np.zeros((6, 3), dtype=complex)
        for j in range(3):
            Bm[:3, j] = -wv["lu"][0][j][q]
            Bm[3:, j] = -wv["lu"][1][j][q]
        R[q] = np.linalg.solve(A, Bm)[:3]
    return R


def transmission_of_incident(md: Media3, kind: int, theta_inc: float, phi_inc: float):
    """A plane wave from the upper layer, kind 0 P, 1 SV, 2 SH, travelling in the direction
    (sin t cos f, sin t sin f, -cos t): its horizontal wavenumber lambda (real) and azimuth, and the
    downgoing lower amplitudes (P, SV, SH) of the transmitted field (unit incident amplitude), from the
    same continuity conditions (reflected upper waves upgoing)."""
    k = md.kp_u if kind == 0 else md.ks_u
    lam = np.array([k * np.sin(theta_inc)], dtype=complex)
    th = np.array([phi_inc])
    wv = _waves(md, lam, th)
    A = np.zeros((6, 6), dtype=complex)
    for j in range(3):
        A[:3, j] = wv["ld"][0][j][0]
        A[3:, j] = wv["ld"][1][j][0]
        A[:3, 3 + j] = -wv["uu"][0][j][0]
        A[3:, 3 + j] = -wv["uu"][1][j][0]
    b = np.concatenate([wv["ud"][0][kind][0], wv["ud"][1][kind][0]])
    sol = np.linalg.solve(A, b)
    return lam[0], phi_inc, sol[:3]


def flux_z(u, t, omega):
    """Time-averaged energy flux through a horizontal plane, upward positive: (omega/2) Im(conj(u).t)
    for the traction t = sigma e_z of a field with time factor e^{-i omega t}."""
    return 0.5 * omega * np.imag(np.sum(np.conj(u) * t, axis=-1))


class Problem3:
    """Spheres (centres (M, 3), radii (M,), bc (M,): 0 rigid, 1 traction-free) below z = 0, order p, polar
    rule parameters; the mat-vec y = gamma - S (T + R) gamma and the dense solve."""

    def __init__(self, md: Media3, centres, radii, bc, p: int, n_r=48, n_theta=24, t_max=10.0, alpha=1.0,
                 beta=1.0, n_panels=1, ntheta_proj=40, rho_frac=0.5):
        self.md = md
        self.c = np.asarray(centres, dtype=float)
        self.R = np.asarray(radii, dtype=float)
        self.bc = np.asarray(bc, dtype=int)
        self.p = p
        self.M = len(self.R)
        self.nmn, self.nl, self.tot = S3.sizes(p)
        self.lam, self.th, self.W = polar_rule(n_r, n_theta, t_max, alpha, beta, n_panels)
        self.ntheta_proj = ntheta_proj
        self.rho_frac = rho_frac
        self.Sn = [S3.sphere_smatrix(p, md.kp_l, md.ks_l, md.lam_l, md.mu_l, r, b) for r, b in zip(self.R, self.bc)]
        self._Rt = None

    # ---------------------------------------------------------------- parts
    def apply_S(self, a):
        return np.stack([S3.apply_sphere_S(self.p, self.Sn[m], a[m]) for m in range(self.M)])

    def translate(self, g):
        """Free-space part: local coefficients at every particle of the other particles' outgoing fields."""
        out = np.zeros_like(g, dtype=complex)
        for m in range(self.M):
            others = [l for l in range(self.M) if l != m]
            if not others:
                continue
            # projection sphere: well inside the ball of convergence (radius = the nearest source centre's
            # distance), large enough that j_n(k rho) of the highest order stays far from underflow
            dmin = min(np.linalg.norm(self.c[l] - self.c[m]) for l in others)
            rho = self.rho_frac * dmin
            out[m] = S3.translate(self.p, self.md.kp_l, self.md.ks_l, self.c[others], g[others], self.c[m], rho,
                                  self.ntheta_proj)
        return out

    def _m2s_tables(self):
        if getattr(self, "_m2s_t", None) is None:
            self._m2s_t = self._make_m2s_tables()
        return self._m2s_t

    def _make_m2s_tables(self):
        md, p = self.md, self.p
        n, _ = S3.orders(p)
        eP, _, _ = basis(md.kp_l, self.lam, self.th, True)
        eS, vS, hS = basis(md.ks_l, self.lam, self.th, True)
        zp, zs = kz(md.kp_l, self.lam), kz(md.ks_l, self.lam)
        YP = S3.ylm(p, eP)                                        # (q, nlm)
        GS = S3.grad_ylm(p, eS)                                   # (q, nlm, 3)
        GxS = np.cross(GS, eS[:, None, :])
        cP = ((-1j) ** (n - 1))[None, :] * YP / (2 * np.pi * zp[:, None])
        fS = ((-1j) ** n)[None, :] / (2 * np.pi * md.ks_l * zs[:, None])
        aV = fS * np.einsum("qki,qi->qk", GS, vS)
        bV = fS * np.einsum("qki,qi->qk", GxS, vS)
        aH = fS * np.einsum("qki,qi->qk", GS, hS)
        bH = fS * np.einsum("qki,qi->qk", GxS, hS)
        return cP, aV, bV, aH, bH, zp, zs

    def m2s(self, g):
        """Upgoing lower amplitudes U (nodes, 3[, nrhs]) of all particles' outgoing fields (block B):
        U_P = sum_l e^{-i (k_x x_l + k_y y_l) - i k_z z_l} sum_nm gamma_nm (-i)^{n-1} Y_nm(e_P) / (2 pi k_z),
        U_SV, U_SH = sum_l (same phase, shear k_z) sum_nm (-i)^n / (2 pi k_s k_z)
                     [alpha_nm Grad Y_nm(e_S) + beta_nm Grad Y_nm(e_S) x e_S] . (v, h)."""
        nmn = self.nmn
        cP, aV, bV, aH, bH, zp, zs = self._m2s_tables()
        kx, ky = self.lam * np.cos(self.th), self.lam * np.sin(self.th)
        vec = g.ndim == 3
        G = g if vec else g[..., None]
        U = np.zeros((len(self.lam), 3, G.shape[-1]), dtype=complex)
        for l in range(self.M):
            x, y, z = self.c[l]
            eh = np.exp(-1j * (kx * x + ky * y))
            ep = eh * np.exp(-1j * zp * z)
            es = eh * np.exp(-1j * zs * z)
            al, be, ga = G[l, :nmn], G[l, nmn:2 * nmn], G[l, 2 * nmn:]
            U[:, 0] += ep[:, None] * (cP @ ga)
            U[:, 1] += es[:, None] * (aV[:, 1:] @ al + bV[:, 1:] @ be)
            U[:, 2] += es[:, None] * (aH[:, 1:] @ al + bH[:, 1:] @ be)
        return U if vec else U[..., 0]

    def reflect(self, U):
        if self._Rt is None:
            self._Rt = reflection(self.md, self.lam, self.th)
        return np.einsum("qij,qj...->qi...", self._Rt, U) * self.W.reshape((-1,) + (1,) * (U.ndim - 1))

    def _s2l_tables(self):
        if getattr(self, "_s2l_t", None) is None:
            md, p = self.md, self.p
            eP, _, _ = basis(md.kp_l, self.lam, self.th, False)
            eS, vS, hS = basis(md.ks_l, self.lam, self.th, False)
            self._s2l_t = (S3.plane_wave_coeffs(p, md.kp_l, eP, eP), S3.plane_wave_coeffs(p, md.kp_l, eS, vS),
                           S3.plane_wave_coeffs(p, md.kp_l, eS, hS))
        return self._s2l_t

    def s2l(self, D):
        """Local coefficients at every particle of the downgoing waves sum_q D(q) (weights included): the
        plane-wave expansions of Sec. 6.3 at the down-going directions, times e^{i k e_down . x_m}."""
        md = self.md
        zp, zs = kz(md.kp_l, self.lam), kz(md.ks_l, self.lam)
        CP, CV, CH = self._s2l_tables()
        kx, ky = self.lam * np.cos(self.th), self.lam * np.sin(self.th)
        vec = D.ndim == 3
        Dv = D if vec else D[..., None]
        out = np.zeros((self.M, self.tot, Dv.shape[-1]), dtype=complex)
        for m in range(self.M):
            x, y, z = self.c[m]
            eh = np.exp(1j * (kx * x + ky * y))
            ep = eh * np.exp(-1j * zp * z)
            es = eh * np.exp(-1j * zs * z)
            out[m] = (CP.T @ (ep[:, None] * Dv[:, 0]) + CV.T @ (es[:, None] * Dv[:, 1])
                      + CH.T @ (es[:, None] * Dv[:, 2]))
        return out if vec else out[..., 0]

    def layered(self, g):
        return self.s2l(self.reflect(self.m2s(g)))

    def matvec(self, g):
        """y = gamma - S (T gamma + R gamma), gamma (M, total[, nrhs])."""
        return g - self.apply_S(self.translate(g) + self.layered(g))

    # ---------------------------------------------------------------- incidence and solve
    def incident_local(self, kind: int, theta_inc: float, phi_inc: float):
        """Local coefficients at every particle of the transmitted field of a unit plane wave from above."""
        md, p = self.md, self.p
        lam, th, Dt = transmission_of_incident(md, kind, theta_inc, phi_inc)
        lam_a, th_a = np.array([lam]), np.array([th])
        eP, _, _ = basis(md.kp_l, lam_a, th_a, False)
        eS, vS, hS = basis(md.ks_l, lam_a, th_a, False)
        zp, zs = kz(md.kp_l, lam_a)[0], kz(md.ks_l, lam_a)[0]
        CP = S3.plane_wave_coeffs(p, md.kp_l, eP[0], eP[0])
        CV = S3.plane_wave_coeffs(p, md.kp_l, eS[0], vS[0])
        CH = S3.plane_wave_coeffs(p, md.kp_l, eS[0], hS[0])
        kx, ky = lam * np.cos(th), lam * np.sin(th)
        out = np.zeros((self.M, self.tot), dtype=complex)
        for m in range(self.M):
            x, y, z = self.c[m]
            eh = np.exp(1j * (kx * x + ky * y))
            out[m] = Dt[0] * eh * np.exp(-1j * zp * z) * CP + eh * np.exp(-1j * zs * z) * (Dt[1] * CV + Dt[2] * CH)
        return out

    def incident_field(self, kind: int, theta_inc: float, phi_inc: float, X):
        """The transmitted incident field at points X (..., 3) of the lower layer."""
        md = self.md
        lam, th, Dt = transmission_of_incident(md, kind, theta_inc, phi_inc)
        lam_a, th_a = np.array([lam]), np.array([th])
        eP, _, _ = basis(md.kp_l, lam_a, th_a, False)
        eS, vS, hS = basis(md.ks_l, lam_a, th_a, False)
        X = np.asarray(X, dtype=float)
        fp = np.exp(1j * md.kp_l * (X @ eP[0]))
        fs = np.exp(1j * md.ks_l * (X @ eS[0]))
        return Dt[0] * fp[..., None] * eP[0] + fs[..., None] * (Dt[1] * vS[0] + Dt[2] * hS[0])

    def rhs(self, incidences):
        """b = S a_inc for a list of (kind, theta, phi): (M, total, nrhs)."""
        a = np.stack([self.incident_local(*inc) for inc in incidences], axis=-1)
        return np.stack([np.stack([S3.apply_sphere_S(self.p, self.Sn[m], a[m, :, r]) for r in range(a.shape[-1])],
                                  axis=-1) for m in range(self.M)])

    def dense(self):
        """The system matrix (M total x M total), column by column."""
        n = self.M * self.tot
        A = np.zeros((n, n), dtype=complex)
        E = np.eye(n, dtype=complex).reshape(self.M, self.tot, n)
        for j0 in range(0, n, 64):
            cols = E[:, :, j0:j0 + 64]
            A[:, j0:j0 + cols.shape[-1]] = self.matvec(cols).reshape(n, -1)
        return A

    def solve_lu(self, b):
        """Dense LU solve, equilibrated (columns, then rows, scaled by their largest entries): the
        coefficients of different orders differ by many orders of magnitude."""
        A = self.dense()
        cs = 1.0 / np.maximum(np.abs(A).max(axis=0), 1e-300)
        A = A * cs[None, :]
        rs = 1.0 / np.maximum(np.abs(A).max(axis=1), 1e-300)
        sol = np.linalg.solve(A * rs[:, None], b.reshape(self.M * self.tot, -1) * rs[:, None])
        return (sol * cs[:, None]).reshape(b.shape)

    # ---------------------------------------------------------------- fields
    def reflected_field(self, D, X):
        """Downgoing lower field of amplitudes D (nodes, 3) with weights included, at points X (..., 3)."""
        md = self.md
        eP, _, _ = basis(md.kp_l, self.lam, self.th, False)
        eS, vS, hS = basis(md.ks_l, self.lam, self.th, False)
        X = np.asarray(X, dtype=float)
        fp = np.exp(1j * md.kp_l * (X @ eP.T))                   # (..., q)
        fs = np.exp(1j * md.ks_l * (X @ eS.T))
        return (np.einsum("...q,q,qi->...i", fp, D[:, 0], eP) + np.einsum("...q,q,qi->...i", fs, D[:, 1], vS)
                + np.einsum("...q,q,qi->...i", fs, D[:, 2], hS))

    def scattered_field(self, g, X):
        """Particles' outgoing fields plus their reflection at points X (..., 3) of the lower layer, for
        one coefficient set g (M, total)."""
        X = np.asarray(X, dtype=float)
        u = 0.0
        for l in range(self.M):
            u = u + S3.field(self.p, self.md.kp_l, self.md.ks_l, X - self.c[l], g[l], "h")
        return u + self.reflected_field(self.reflect(self.m2s(g)), X)
