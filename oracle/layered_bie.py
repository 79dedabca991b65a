"""Brute-force boundary integral solve of a few particles with the layered Green's function.

Test infrastructure only (see oracle/__init__.py).

This is the direct method of Sec. 7.1 in a form that needs no scattering matrix, no Graf
translation and no local expansion: every particle boundary carries a single-layer density of the
layered Green's function,
    u_sc(x) = sum_l int_{dD_l} G_L(x, y) phi_l(y) ds_y,     G_L = Phi + G_R,
where Phi is the free-space fundamental solution of the lower layer and G_R(x, y) e_k the
interface-reflected field at x of a unit force e_k at y.  The reflected part is the Sommerfeld
representation of Sec. 5: the force's outgoing potentials are first-order multipoles at y (the
derivatives of H_0 in Phi = -(i/(4 w^2)) (grad grad^T H_0(kp r) + grad_perp grad_perp^T H_0(ks r))),
their upgoing amplitudes come from pts1 (sommerfeld.m2s), the 2x2 reflection per node gives the
downgoing amplitudes, and the downgoing plane waves are summed at x directly (no Jacobi-Anger).
Boundary conditions (Sec. 2): rigid u_sc = -u_inc (a first-kind equation on the self block),
traction-free T u_sc = -T u_inc (-phi/2 + K' phi on the self block); u_inc is the transmitted
plane wave of Sec. 7.3.  The self blocks use the Nystrom matrices of oracle.nystrom; every other
kernel is smooth and summed by the trapezoid rule.

Comparing its receiver fields with the multiple-scattering solve (scattering matrices from
oracle.nystrom, Graf translations, the separable reflected operator) checks the coupled
formulation of Sec. 4-5 as a whole.
"""
from __future__ import annotations

import numpy as np

from . import nystrom, sommerfeld


def point_force_coefficients(h: nystrom.Host):
    """Outgoing coefficients (2, 3, 2) of the free-space field Phi(., y) e_k about y: axis 0 the wave
    (P, S), axis 1 the order n = -1, 0, 1, axis 2 the force direction k.  From
    d_x H_0(kr) = (k/2)(w_{-1} - w_1), d_y H_0(kr) = (ik/2)(w_{-1} + w_1), w_n = H_n(kr) e^{in th}:
    P potential -(i/(4w^2)) d_k H_0(kp r), S potential -(i/(4w^2)) (grad_perp)_k H_0(ks r)."""
    c = 1j / (8 * h.omega ** 2)
    g = np.zeros((2, 3, 2), complex)
    g[0, 0, 0], g[0, 2, 0] = -c * h.kp, c * h.kp                 # force e_x, P wave, n = -1 and 1
    g[0, 0, 1], g[0, 2, 1] = -1j * c * h.kp, -1j * c * h.kp      # force e_y
    g[1, 0, 0], g[1, 2, 0] = 1j * c * h.ks, 1j * c * h.ks
    g[1, 0, 1], g[1, 2, 1] = -c * h.ks, c * h.ks
    return g


def _downgoing_maps(xi, W, L, X, Y):
    """Matrices mapping downgoing amplitudes (D_P, D_S) per node to u and grad u at the points:
    the sum of D_P grad(e^{i xi x + s_p y}) + D_S grad_perp(e^{i xi x + s_s y}) (Sec. 5.3)."""
    sp, ss = sommerfeld.branch_s(xi, L.kp_l), sommerfeld.branch_s(xi, L.ks_l)
    ep = W[None, :] * np.exp(1j * xi[None, :] * X[:, None] + sp[None, :] * Y[:, None])
    es = W[None, :] * np.exp(1j * xi[None, :] * X[:, None] + ss[None, :] * Y[:, None])
    ix = 1j * xi[None, :]
    spb, ssb = sp[None, :], ss[None, :]
    u = [(ix * ep, -ssb * es), (spb * ep, ix * es)]
    g = [[(ix * ix * ep, -ssb * ix * es), (ix * spb * ep, -ssb * ssb * es)],
         [(spb * ix * ep, ix * ix * es), (spb * spb * ep, ix * ssb * es)]]
    return u, g


def reflected_green(P, X, Y, src, nu=None):
    """G_R at targets (X, Y) from unit forces at the points src (ns, 2): array (nt, 2, ns, 2) with
    [i, component; j, source; k, force direction].  With unit normals nu (nt, 2), the traction of
    each column at the targets instead."""
    L = P.L
    h = nystrom.Host(L.lam_l, L.mu_l, L.omega)
    g = point_force_coefficients(h)
    ns = src.shape[0]
    UP = np.empty((P.xi.size, ns, 2), complex)
    US = np.empty((P.xi.size, ns, 2), complex)
    for j in range(ns):
        a, b = sommerfeld.m2s(P.xi, L, src[j:j + 1], g[None])
        UP[:, j], US[:, j] = a, b
    R = P.reflection_table()
    DP = R[:, 0, 0, None, None] * UP + R[:, 0, 1, None, None] * US
    DS = R[:, 1, 0, None, None] * UP + R[:, 1, 1, None, None] * US
    DP = DP.reshape(P.xi.size, -1)
    DS = DS.reshape(P.xi.size, -1)
    u, gr = _downgoing_maps(P.xi, P.W, L, np.asarray(X, float), np.asarray(Y, float))
    nt = len(X)
    if nu is None:
        out = np.stack([u[i][0] @ DP + u[i][1] @ DS for i in range(2)], 1)
    else:
        G = [[gr[i][j][0] @ DP + gr[i][j][1] @ DS for j in range(2)] for i in range(2)]
        from .waves import traction
        t1, t2 = traction(G, nu[:, 0, None], nu[:, 1, None], L.lam_l, L.mu_l)
        out = np.stack([t1, t2], 1)
    return out.reshape(nt, 2, ns, 2)


class LayeredBIE:
    """Boundaries of a few particles (nystrom.StarCurve about each centre), bc 0 rigid / 1 traction-free,
    buried in the lower layer of the problem P (a system.Problem that supplies the medium, the
    contour and the reflection table)."""

    def __init__(self, P, curves, centres, bc, N: int = 128):
        self.P = P
        L = P.L
        self.h = nystrom.Host(L.lam_l, L.mu_l, L.omega)
        self.bnd = [nystrom.Boundary(c, N, self.h, centre=x) for c, x in zip(curves, centres)]
        self.bc = list(bc)
        self.N = N

    def _nodes(self):
        x = np.concatenate([b.x for b in self.bnd])
        nu = np.concatenate([b.nu for b in self.bnd])
        w = np.concatenate([(2 * np.pi / b.N) * b.speed for b in self.bnd])
        return x, nu, w

    def system_matrix(self):
        N, nb = self.N, len(self.bnd)
        x, nu, w = self._nodes()
        h = self.h
        n = N * nb
        A = np.zeros((n, 2, n, 2), complex)
        # interface-reflected part between every pair of nodes (smooth)
        for m in range(nb):
            rows = slice(m * N, (m + 1) * N)
            xm = x[rows]
            GR = reflected_green(self.P, xm[:, 0], xm[:, 1], x, nu=None if self.bc[m] == 0 else nu[rows])
            A[rows] += GR * w[None, None, :, None]
        # free-space part
        for m in range(nb):
            rows = slice(m * N, (m + 1) * N)
            B = self.bnd[m]
            for l in range(nb):
                cols = slice(l * N, (l + 1) * N)
                if l == m:
                    M = B.single_layer() if self.bc[m] == 0 else -0.5 * np.eye(2 * N) + B.adjoint_double_layer()
                    A[rows, :, cols, :] += M.reshape(N, 2, N, 2)
                    continue
                z = B.x[:, None, :] - self.bnd[l].x[None, :, :]
                if self.bc[m] == 0:
                    K = nystrom.fundamental(z, h)
                else:
                    K = nystrom.traction_kernel(z, np.broadcast_to(B.nu[:, None, :], z.shape), h)
                A[rows, :, cols, :] += K.transpose(0, 2, 1, 3) * w[cols][None, None, :, None]
        return A.reshape(2 * n, 2 * n)

    def incident_data(self, kind: int, angle: float):
        """-u_inc on rigid boundaries, -T u_inc on traction-free ones: (n, 2)."""
        L = self.P.L
        xi, D, _, _ = sommerfeld.plane_wave_incidence(kind, angle, L)
        out = []
        for B, bc in zip(self.bnd, self.bc):
            u1, u2, g = sommerfeld.downgoing_field(np.array([xi]), np.array([1.0]), L,
                                                   np.array([D[0]]), np.array([D[1]]), B.x[:, 0], B.x[:, 1])
            if bc == 0:
                out.append(-np.stack([u1, u2], 1))
            else:
                from .waves import traction
                t1, t2 = traction(g, B.nu[:, 0], B.nu[:, 1], L.lam_l, L.mu_l)
                out.append(-np.stack([t1, t2], 1))
        return np.concatenate(out)

    def solve(self, kind: int, angle: float):
        A = self.system_matrix()
        rhs = self.incident_data(kind, angle).reshape(-1)
        return np.linalg.solve(A, rhs).reshape(-1, 2)

    def field(self, phi, X, Y):
        """Scattered displacement (2, npts) at points of the lower layer away from the boundaries."""
        X = np.asarray(X, float)
        Y = np.asarray(Y, float)
        x, nu, w = self._nodes()
        z = np.stack([X, Y], 1)[:, None, :] - x[None, :, :]
        G = nystrom.fundamental(z, self.h).transpose(0, 2, 1, 3) + reflected_green(self.P, X, Y, x)
        return np.einsum("aibk,b,bk->ia", G, w, phi)
