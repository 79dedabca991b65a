"""Assembled multiple-scattering operator, right-hand side, solvers and fields.

Test infrastructure only (see oracle/__init__.py).

System (Sec. 4.2 mul2 with the layered Schur complement of Sec. 5.2, reading A6):
    gamma^m = S_m ( a0^m + sum_{l != m} T^{ml} gamma^l + (R gamma)^m ),
i.e.  y = A gamma = gamma - S (T + R) gamma  and  A gamma = S a0.
T is the direct Graf sum over every ordered pair (no FMM); R is the interface-reflected
operator of Sec. 5.3-5.4 and includes the self term l = m.  Plane-wave right-hand sides
follow Sec. 7.3 (bplan): the transmitted background field expanded about every centre.
Coefficient blocks have layout (M, 2, 2p+1, nrhs): [particle][P or S][order n + p][rhs].
"""
from __future__ import annotations

import numpy as np

from . import disc, graf, sommerfeld
from .media import Layered
from .waves import field_of_coeffs, traction


class Problem:
    def __init__(self, wl, proto_S=None, proto_index=None):
        """wl: a synthetic.Workload.  proto_S (Q, 2nc, 2nc) and proto_index (M,) with -1 for
        closed-form discs (default: wl.proto) give dense prototype scattering matrices, rotated per
        particle by wl.rotation (Sec. 4.3: rotated copies by a rotation of the basis)."""
        self.wl = wl
        self.L = Layered(wl.media, wl.omega)
        self.p = wl.p
        self.nc = 2 * wl.p + 1
        self.centres = np.asarray(wl.centres, float)
        self.radius = np.asarray(wl.radius, float)
        self.bc = np.asarray(wl.bc, int)
        self.M = self.centres.shape[0]
        self.xi, self.W = sommerfeld.contour(wl.n_panels, wl.nodes_per_panel, wl.t_max, wl.depth, wl.grade,
                                             (self.L.kp_u, self.L.ks_u, self.L.kp_l, self.L.ks_l))
        self.proto_S = proto_S
        if proto_index is None and getattr(wl, "proto", None) is not None:
            proto_index = wl.proto
        self.proto_index = np.full(self.M, -1) if proto_index is None else np.asarray(proto_index)
        if (self.proto_index >= 0).any() and proto_S is None:
            raise ValueError("prototype particles need their scattering matrices (proto_S)")
        self.rotation = np.asarray(wl.rotation, float)
        self._disc_S = {}

    # ------------------------------------------------------------------ scattering matrices
    def disc_S(self, m: int):
        key = (round(self.radius[m], 15), int(self.bc[m]))
        if key not in self._disc_S:
            lam, mu = self.L.lam_l, self.L.mu_l
            self._disc_S[key] = disc.disc_smatrix(self.p, self.L.kp_l, self.L.ks_l,
                                                  self.radius[m], int(self.bc[m]), lam, mu)
        return self._disc_S[key]

    def dense_S(self, m: int):
        """(2nc, 2nc) scattering matrix of particle m in the order (b, n)."""
        nc = self.nc
        if self.proto_index[m] < 0:
            Sd = self.disc_S(m)
            S = np.zeros((2, nc, 2, nc), dtype=complex)
            for i in range(nc):
                S[:, i, :, i] = Sd[i]
            return S.reshape(2 * nc, 2 * nc)
        n = np.tile(np.arange(-self.p, self.p + 1), 2)
        ph = np.exp(-1j * (n[:, None] - n[None, :]) * self.rotation[m])
        return self.proto_S[self.proto_index[m]] * ph

    def apply_S(self, a, targets=None):
        """S_m a^m for every particle (or the listed targets): a has shape (len, 2, nc, nrhs)."""
        targets = range(self.M) if targets is None else targets
        out = np.empty_like(a)
        for i, m in enumerate(targets):
            S = self.dense_S(m)
            out[i] = (S @ a[i].reshape(2 * self.nc, -1)).reshape(2, self.nc, -1)
        return out

    # ------------------------------------------------------------------ operator pieces
    def translate(self, gamma, targets=None):
        """(T gamma)^m = sum_{l != m} T^{ml} gamma^l, direct O(M^2) Graf sum (Sec. 4.2)."""
        targets = range(self.M) if targets is None else list(targets)
        out = np.zeros((len(targets), 2, self.nc, gamma.shape[3]), dtype=complex)
        for i, m in enumerate(targets):
            for b, k in ((0, self.L.kp_l), (1, self.L.ks_l)):
                T = graf.translation_all_sources(self.p, k, self.centres[m], self.centres)
                T[m] = 0.0
                # sum over sources l and orders j as one matrix product
                nrhs = gamma.shape[3]
                out[i, b] = T.transpose(1, 0, 2).reshape(self.nc, -1) @ gamma[:, b].reshape(-1, nrhs)
        return out

    def reflection_table(self):
        """R(xi_q) for every node (plane-wave route), computed once per problem."""
        if getattr(self, "_R", None) is None:
            self._R = np.stack([sommerfeld.reflection_plane_wave(x, self.L) for x in self.xi])
        return self._R

    def reflect(self, gamma, targets=None):
        """(R gamma)^m: local coefficients of the interface-reflected field (Sec. 5.3-5.4)."""
        U_P, U_S = sommerfeld.m2s(self.xi, self.L, self.centres, gamma)
        R = self.reflection_table()
        D_P = R[:, 0, 0, None] * U_P + R[:, 0, 1, None] * U_S
        D_S = R[:, 1, 0, None] * U_P + R[:, 1, 1, None] * U_S
        c = self.centres if targets is None else self.centres[list(targets)]
        return sommerfeld.s2l(self.xi, self.W, self.L, c, D_P, D_S, self.p)

    def matvec(self, gamma, targets=None):
        """y = gamma - S (T + R) gamma, optionally only at the listed targets."""
        a = self.translate(gamma, targets) + self.reflect(gamma, targets)
        g = gamma if targets is None else gamma[list(targets)]
        return g - self.apply_S(a, targets)

    # ------------------------------------------------------------------ right-hand side
    def incident_local(self, kinds, angles):
        """Local coefficients a0 (M, 2, nc, nrhs) of the transmitted background field (Sec. 7.3)."""
        cols = []
        for kind, ang in zip(kinds, angles):
            xi, D, _, _ = sommerfeld.plane_wave_incidence(int(kind), float(ang), self.L)
            cols.append(sommerfeld.local_expansion_of_plane(xi, D, self.L, self.centres, self.p))
        return np.stack(cols, axis=-1)

    def rhs(self, kinds, angles):
        """b = S a0 (right-hand side of mul2)."""
        return self.apply_S(self.incident_local(kinds, angles))

    def point_source_local(self, sources, forces):
        """Local coefficients a0 (M, 2, nc, nsrc) of point forces in the upper layer (Sec. 7.2): each
        source's downgoing spectrum transmitted through the interface, expanded about every centre by the
        Sommerfeld-to-local map on the problem's contour."""
        cols = []
        for z, q in zip(np.asarray(sources, float), np.asarray(forces, float)):
            DP, DS = sommerfeld.point_force_transmitted(self.xi, self.L, z, q)
            cols.append(sommerfeld.s2l(self.xi, self.W, self.L, self.centres, DP[:, None], DS[:, None], self.p)[..., 0])
        return np.stack(cols, axis=-1)

    def point_rhs(self, sources, forces):
        """b = S a0 for upper-layer point forces."""
        return self.apply_S(self.point_source_local(sources, forces))

    def time_reversal(self, mirror):
        """Response matrix F of a mirror in the upper layer (Sec. 7.5): column 2j + d is the solve for a
        point force e_d at mirror point j, row 2i + c component c of its scattered field at mirror point i;
        returns F and the eigenvalues of T = conj(F)^T F, descending (dense LU solves)."""
        mirror = np.asarray(mirror, float)
        n = mirror.shape[0]
        src = np.repeat(mirror, 2, axis=0)
        force = np.tile(np.eye(2), (n, 1))
        gam = self.solve_lu(self.point_rhs(src, force))
        u = self.upper_field(gam, mirror[:, 0], mirror[:, 1])        # (2n, 2, n)
        F = u.transpose(2, 1, 0).reshape(2 * n, 2 * n)               # row 2i + c, column 2j + d
        T = F.conj().T @ F
        return F, np.sort(np.linalg.eigvalsh(T))[::-1]

    def upper_field(self, gamma, X, Y):
        """Scattered displacement in the upper layer at (X, Y), Y > 0: the particles' upgoing spectra
        transmitted through the interface (Sec. 3, 5).  Returns (nrhs, 2, npts)."""
        (_, _), (E_P, E_S) = self.interface_amplitudes(gamma)
        out = []
        for r in range(gamma.shape[3]):
            u1, u2, _ = sommerfeld.upgoing_upper_field(self.xi, self.W, self.L, E_P[:, r], E_S[:, r], X, Y)
            out.append(np.stack([u1, u2]))
        return np.stack(out)

    # ------------------------------------------------------------------ solvers
    def solve_gmres(self, b, tol=1e-12, restart=200, maxit=2000):
        """Restarted GMRES (modified Gram-Schmidt, Givens rotations) per right-hand side,
        stopping on ||b - A x|| / ||b|| <= tol (reading A13: zero initial guess)."""
        shape = b.shape
        nrhs = shape[-1]
        x = np.zeros_like(b)
        iters = np.zeros(nrhs, int)
        for r in range(nrhs):
            bb = b[..., r].ravel()
            bn = np.linalg.norm(bb)
            xr = np.zeros_like(bb)
            if bn == 0:
                continue
            total = 0
            while total < maxit:
                res = bb - self.matvec(xr.reshape(shape[:-1] + (1,)))[..., 0].ravel()
                beta = np.linalg.norm(res)
                if beta / bn <= tol:
                    break
                V = [res / beta]
                H = np.zeros((restart + 1, restart), dtype=complex)
                cs = np.zeros(restart, dtype=complex)
                sn = np.zeros(restart, dtype=complex)
                g = np.zeros(restart + 1, dtype=complex)
                g[0] = beta
                j_done = 0
                for j in range(restart):
                    w = self.matvec(V[j].reshape(shape[:-1] + (1,)))[..., 0].ravel()
                    for i in range(j + 1):
                        H[i, j] = np.vdot(V[i], w)
                        w = w - H[i, j] * V[i]
                    H[j + 1, j] = np.linalg.norm(w)
                    V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
                    # earlier rotations G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]]
                    for i in range(j):
                        hi, hn = H[i, j], H[i + 1, j]
                        H[i, j] = np.conj(cs[i]) * hi + np.conj(sn[i]) * hn
                        H[i + 1, j] = -sn[i] * hi + cs[i] * hn
                    den = np.hypot(abs(H[j, j]), abs(H[j + 1, j]))
                    cs[j] = H[j, j] / den if den else 1.0
                    sn[j] = H[j + 1, j] / den if den else 0.0
                    H[j, j] = den
                    H[j + 1, j] = 0.0
                    g[j + 1] = -sn[j] * g[j]
                    g[j] = np.conj(cs[j]) * g[j]
                    total += 1
                    j_done = j + 1
                    if abs(g[j + 1]) / bn <= tol or total >= maxit:
                        break
                y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
                xr = xr + np.stack(V[:j_done], axis=1) @ y
            x[..., r] = xr.reshape(shape[:-1])
            iters[r] = total
        return x, iters

    def assemble(self):
        """Dense matrix of A (N x N, N = M * 2 * nc) by applying the operator to the identity."""
        N = self.M * 2 * self.nc
        E = np.eye(N, dtype=complex).reshape(self.M, 2, self.nc, N)
        return self.matvec(E).reshape(N, N)

    def solve_lu(self, b):
        """Dense LU solve of A gamma = b.  Columns, then rows, of A are scaled to unit 2-norm before
        the factorisation (equilibration; the solution is the same): coefficients of different orders
        differ by tens of decades at p >= 16, and the unscaled matrix's condition number (1e22 at
        p = 16 for three particles) would leave no correct digit."""
        N = self.M * 2 * self.nc
        A = self.assemble()
        cs = 1.0 / np.linalg.norm(A, axis=0)
        A = A * cs[None, :]
        rs = 1.0 / np.linalg.norm(A, axis=1)
        A = A * rs[:, None]
        return (np.linalg.solve(A, rs[:, None] * b.reshape(N, -1)) * cs[:, None]).reshape(b.shape)

    # ------------------------------------------------------------------ fields
    def interface_amplitudes(self, gamma):
        """Downgoing lower (D) and upgoing upper (E) amplitudes per node generated by gamma."""
        U_P, U_S = sommerfeld.m2s(self.xi, self.L, self.centres, gamma)
        D_P = np.empty_like(U_P)
        D_S = np.empty_like(U_S)
        E_P = np.empty_like(U_P)
        E_S = np.empty_like(U_S)
        for q in range(self.xi.size):
            for r in range(U_P.shape[1]):
                D, E = sommerfeld.interface_solve(self.xi[q], self.L, U=(U_P[q, r], U_S[q, r]))
                D_P[q, r], D_S[q, r] = D
                E_P[q, r], E_S[q, r] = E
        return (D_P, D_S), (E_P, E_S)

    def scattered_field(self, gamma, X, Y, with_gradient=False):
        """Scattered displacement in the lower layer at points (X, Y), per right-hand side:
        direct sum of outgoing waves of every particle (Sec. 5 total-field representation)
        plus the interface-reflected Sommerfeld field.  Returns u of shape (nrhs, 2, npts)."""
        X = np.asarray(X, float)
        Y = np.asarray(Y, float)
        nrhs = gamma.shape[3]
        U_P, U_S = sommerfeld.m2s(self.xi, self.L, self.centres, gamma)
        R = self.reflection_table()
        D_P = R[:, 0, 0, None] * U_P + R[:, 0, 1, None] * U_S
        D_S = R[:, 1, 0, None] * U_P + R[:, 1, 1, None] * U_S
        us = []
        gs = []
        for r in range(nrhs):
            u1 = np.zeros(X.shape, complex)
            u2 = np.zeros(X.shape, complex)
            g = [[np.zeros(X.shape, complex) for _ in range(2)] for _ in range(2)]
            for m in range(self.M):
                a, b2, gg = field_of_coeffs("H", gamma[m, 0, :, r], gamma[m, 1, :, r], self.p,
                                            self.L.kp_l, self.L.ks_l,
                                            X - self.centres[m, 0], Y - self.centres[m, 1])
                u1 += a
                u2 += b2
                for i in range(2):
                    for j in range(2):
                        g[i][j] = g[i][j] + gg[i][j]
            a, b2, gg = sommerfeld.downgoing_field(self.xi, self.W, self.L, D_P[:, r], D_S[:, r], X, Y)
            u1 += a
            u2 += b2
            for i in range(2):
                for j in range(2):
                    g[i][j] = g[i][j] + gg[i][j]
            us.append(np.stack([u1, u2]))
            gs.append(g)
        if with_gradient:
            return np.stack(us), gs
        return np.stack(us)

    def boundary_residual(self, gamma, kinds, angles, m: int, npts: int = 64):
        """Boundary quantity of the TOTAL field (background + scattered) on the circle of particle m,
        evaluated by direct sums: displacement for a rigid particle, traction (normal r-hat) for a
        traction-free one.  Returns (residual, scale) arrays of shape (nrhs, 2, npts); the boundary
        condition of Sec. 2 says the residual vanishes up to truncation error."""
        th = np.linspace(0, 2 * np.pi, npts, endpoint=False)
        R = self.radius[m]
        X = self.centres[m, 0] + R * np.cos(th)
        Y = self.centres[m, 1] + R * np.sin(th)
        us, gs = self.scattered_field(gamma, X, Y, with_gradient=True)
        res = []
        scale = []
        lam, mu = self.L.lam_l, self.L.mu_l
        for r, (kind, ang) in enumerate(zip(kinds, angles)):
            xi, D, _, _ = sommerfeld.plane_wave_incidence(int(kind), float(ang), self.L)
            b1, b2, gb = sommerfeld.downgoing_field(np.array([xi]), np.array([1.0]), self.L,
                                                    np.array([D[0]]), np.array([D[1]]), X, Y)
            if self.bc[m] == 0:
                tot = np.stack([us[r][0] + b1, us[r][1] + b2])
                sc = np.stack([b1, b2])
            else:
                g = [[gs[r][i][j] + gb[i][j] for j in range(2)] for i in range(2)]
                tot = np.stack(traction(g, np.cos(th), np.sin(th), lam, mu))
                sc = np.stack(traction(gb, np.cos(th), np.sin(th), lam, mu))
            res.append(tot)
            scale.append(sc)
        return np.stack(res), np.stack(scale)
