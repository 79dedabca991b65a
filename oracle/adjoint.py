"""Adjoint gradients of a receiver misfit with respect to particle centres, radii and frequency.

Test infrastructure only (see oracle/__init__.py).

Loss: L = 1/2 sum_{r,k,c} |u_{r,k,c} - d_{r,k,c}|^2 with u the scattered displacement at the
receivers (Sec. 5, total-field representation) of the solution of A gamma = b (mul2 with the
layered Schur complement, Sec. 4.2 / 5.2; b = S a0, Sec. 7.3).  Writing w = u - d,

    dL/dtheta = Re[ w^H (dF/dtheta) gamma ] + Re[ lambda^H (db/dtheta - (dA/dtheta) gamma) ],
    A^H lambda = F^H w,

with A = I - S (T + R).  Everything is dense and small: A and the receiver map F are assembled,
and the derivative of each operator applied to gamma is written out from the formulas:
  * Graf entries h_k = H_k(k |v|) e^{ik arg v}:  d/dv_x h_k = (k/2)(h_{k-1} - h_{k+1}),
    d/dv_y h_k = (ik/2)(h_{k-1} + h_{k+1})  (DLMF 10.6);
  * spectral factors e^{s y_l - i xi x_l} (source) and e^{i xi x_m + s y_m} (target): the derivative
    multiplies by (-i xi, s) and (i xi, s);
  * plane-wave right-hand side e^{i xi x_m + s y_m}: (i xi, s);
  * receiver fields: the derivative of a particle's field with respect to its centre is minus its
    gradient with respect to the receiver (second derivatives by the same order shifts);
  * disc scattering matrix S = -M_H^{-1} M_J per mode: dS = -M_H^{-1}(dM_J + dM_H S) with the
    derivative of the mode matrix in R (Bessel derivatives up to third order).
The frequency derivative of A, b and F is taken by central differences of the assembled
operators (every factor depends on omega).
"""
from __future__ import annotations

import copy

import numpy as np

from . import disc, graf, sommerfeld
from .system import Problem
from .waves import Z


# ----------------------------------------------------------------------------- assembled pieces
def field_matrix(P: Problem, receivers):
    """F with u = F gamma: rows (receiver k, component c), columns (m, b, n); one column at a time."""
    N = P.M * 2 * P.nc
    E = np.eye(N, dtype=complex).reshape(P.M, 2, P.nc, N)
    cols = []
    for j in range(N):
        u = P.scattered_field(E[..., j:j + 1], receivers[:, 0], receivers[:, 1])   # (1, 2, R)
        cols.append(u[0].T.ravel())                                              # (R*2,)
    return np.stack(cols, axis=1)


def forward(P: Problem, kinds, angles, receivers):
    b = P.rhs(kinds, angles)
    N = P.M * 2 * P.nc
    gamma = np.linalg.solve(P.assemble(), b.reshape(N, -1)).reshape(b.shape)
    u = np.stack([P.scattered_field(gamma[..., r:r + 1], receivers[:, 0], receivers[:, 1])[0].T
                  for r in range(b.shape[-1])])        # (nrhs, R, 2)
    return gamma, u


def loss(P: Problem, kinds, angles, receivers, d):
    _, u = forward(P, kinds, angles, receivers)
    return 0.5 * float(np.sum(np.abs(u - d) ** 2))


# ----------------------------------------------------------------------------- derivative pieces
def _hseq(k, v, K):
    """h_j = H_j(k|v|) e^{ij arg v} for j in [-K, K]."""
    d = np.hypot(v[0], v[1])
    th = np.arctan2(v[1], v[0])
    j = np.arange(-K, K + 1)
    from scipy import special
    return special.hankel1(j, k * d) * np.exp(1j * j * th)


def _dT(p, k, v, axis):
    """Derivative of the Graf matrix T[i, j] = h_{j-i}(v) with respect to v_x (axis 0) or v_y (1)."""
    K = 2 * p + 1
    h = _hseq(k, v, K)
    i = np.arange(-p, p + 1)[:, None]
    jj = np.arange(-p, p + 1)[None, :]
    kk = jj - i + K
    if axis == 0:
        return 0.5 * k * (h[kk - 1] - h[kk + 1])
    return 0.5j * k * (h[kk - 1] + h[kk + 1])


def dT_gamma(P: Problem, gamma, m: int, axis: int):
    """(d/dc_m T) gamma for the centre coordinate c_m[axis]: target row m and source column m."""
    out = np.zeros_like(gamma)
    for b, k in ((0, P.L.kp_l), (1, P.L.ks_l)):
        for l in range(P.M):
            if l == m:
                continue
            v = P.centres[m] - P.centres[l]
            D = _dT(P.p, k, v, axis)                   # d T^{ml} / d v = d / d c_m
            out[m, b] += D @ gamma[l, b]
            out[l, b] -= _dT(P.p, k, P.centres[l] - P.centres[m], axis) @ gamma[m, b]   # d/dc_m = -d/dv
    return out


def dR_gamma(P: Problem, gamma, m: int, axis: int):
    """(d/dc_m R) gamma: the target factor of row m and the source factor of column m."""
    xi, W, L = P.xi, P.W, P.L
    R = P.reflection_table()
    # target side: rows of particle m with factor (i xi, s_b)
    U_P, U_S = sommerfeld.m2s(xi, L, P.centres, gamma)
    D_P = R[:, 0, 0, None] * U_P + R[:, 0, 1, None] * U_S
    D_S = R[:, 1, 0, None] * U_P + R[:, 1, 1, None] * U_S
    out = np.zeros_like(gamma)
    fac_p = 1j * xi if axis == 0 else sommerfeld.branch_s(xi, L.kp_l)
    fac_s = 1j * xi if axis == 0 else sommerfeld.branch_s(xi, L.ks_l)
    a_m = sommerfeld.s2l(xi, W, L, P.centres[m:m + 1], fac_p[:, None] * D_P, fac_s[:, None] * D_S, P.p)
    out[m] += a_m[0]
    # source side: particle m's own upgoing amplitudes with factor (-i xi, s_b)
    gm = np.zeros_like(gamma)
    gm[m] = gamma[m]
    Um_P, Um_S = sommerfeld.m2s(xi, L, P.centres, gm)
    g_p = -1j * xi if axis == 0 else sommerfeld.branch_s(xi, L.kp_l)
    g_s = -1j * xi if axis == 0 else sommerfeld.branch_s(xi, L.ks_l)
    Um_P = g_p[:, None] * Um_P
    Um_S = g_s[:, None] * Um_S
    D2_P = R[:, 0, 0, None] * Um_P + R[:, 0, 1, None] * Um_S
    D2_S = R[:, 1, 0, None] * Um_P + R[:, 1, 1, None] * Um_S
    out += sommerfeld.s2l(xi, W, L, P.centres, D2_P, D2_S, P.p)
    return out


def db(P: Problem, kinds, angles, m: int, axis: int):
    """d b / d c_m[axis] with b = S a0, a0^m = D_b e^{i xi x_m + s y_m} i^n q^n."""
    a0 = P.incident_local(kinds, angles)          # (M, 2, nc, nrhs)
    fac = np.zeros((2, len(angles)), dtype=complex)
    for r, (kind, ang) in enumerate(zip(kinds, angles)):
        xi, _, _, _ = sommerfeld.plane_wave_incidence(int(kind), float(ang), P.L)
        for b, k in ((0, P.L.kp_l), (1, P.L.ks_l)):
            fac[b, r] = 1j * xi if axis == 0 else sommerfeld.branch_s(xi, k)
    da = np.zeros_like(a0)
    da[m] = a0[m] * fac[:, None, :]
    return P.apply_S(da)


def dF_gamma(P: Problem, gamma, receivers, m: int, axis: int):
    """(d/dc_m F) gamma at the receivers, (nrhs, R, 2)."""
    X = receivers[:, 0] - P.centres[m, 0]
    Y = receivers[:, 1] - P.centres[m, 1]
    nrhs = gamma.shape[3]
    out = np.zeros((nrhs, receivers.shape[0], 2), dtype=complex)
    # direct part: minus the receiver-gradient of particle m's outgoing field
    key = "x" if axis == 0 else "y"
    for r in range(nrhs):
        phi = {kk: np.zeros(X.shape, complex) for kk in ("x", "y", "xx", "xy", "yy")}
        psi = {kk: np.zeros(X.shape, complex) for kk in ("x", "y", "xx", "xy", "yy")}
        for i, n in enumerate(range(-P.p, P.p + 1)):
            for store, k, c in ((phi, P.L.kp_l, gamma[m, 0, i, r]), (psi, P.L.ks_l, gamma[m, 1, i, r])):
                if c == 0:
                    continue
                from .waves import wave_derivs
                dd = wave_derivs("H", n, k, X, Y)
                for kk in store:
                    store[kk] += c * dd[kk]
        # u1 = phi_x - psi_y, u2 = phi_y + psi_x; derivative along the receiver axis
        if axis == 0:
            du1 = phi["xx"] - psi["xy"]
            du2 = phi["xy"] + psi["xx"]
        else:
            du1 = phi["xy"] - psi["yy"]
            du2 = phi["yy"] + psi["xy"]
        out[r, :, 0] -= du1
        out[r, :, 1] -= du2
    # reflected part: particle m's upgoing amplitudes with the source factor (-i xi, s_b)
    xi, W, L = P.xi, P.W, P.L
    gm = np.zeros_like(gamma)
    gm[m] = gamma[m]
    U_P, U_S = sommerfeld.m2s(xi, L, P.centres, gm)
    g_p = -1j * xi if axis == 0 else sommerfeld.branch_s(xi, L.kp_l)
    g_s = -1j * xi if axis == 0 else sommerfeld.branch_s(xi, L.ks_l)
    U_P = g_p[:, None] * U_P
    U_S = g_s[:, None] * U_S
    R = P.reflection_table()
    D_P = R[:, 0, 0, None] * U_P + R[:, 0, 1, None] * U_S
    D_S = R[:, 1, 0, None] * U_P + R[:, 1, 1, None] * U_S
    for r in range(nrhs):
        u1, u2, _ = sommerfeld.downgoing_field(xi, W, L, D_P[:, r], D_S[:, r], receivers[:, 0], receivers[:, 1])
        out[r, :, 0] += u1
        out[r, :, 1] += u2
    return out


def _zd3(kind, n, k, R):
    """Z_n(kR) and its first three R-derivatives (DLMF 10.6.1 applied repeatedly)."""
    z = lambda j: Z(kind, j, k * R)
    return (z(n), 0.5 * k * (z(n - 1) - z(n + 1)),
            0.25 * k ** 2 * (z(n - 2) - 2 * z(n) + z(n + 2)),
            0.125 * k ** 3 * (z(n - 3) - 3 * z(n - 1) + 3 * z(n + 1) - z(n + 3)))


def mode_matrix_dR(kind, n, kp, ks, R, bc, lam, mu):
    """d/dR of disc.mode_matrix."""
    f, f1, f2, f3 = _zd3(kind, n, kp, R)
    g, g1, g2, g3 = _zd3(kind, n, ks, R)
    if bc == 0:
        return np.array([[f2, 1j * n / R ** 2 * g - 1j * n / R * g1],
                         [-1j * n / R ** 2 * f + 1j * n / R * f1, g2]], dtype=complex)
    return np.array([
        [-lam * kp * kp * f1 + 2 * mu * f3, -2 * mu * 1j * n * (g2 / R - 2 * g1 / R ** 2 + 2 * g / R ** 3)],
        [2 * mu * 1j * n * (f2 / R - 2 * f1 / R ** 2 + 2 * f / R ** 3),
         mu * (g3 - g2 / R + g1 / R ** 2 + n * n * g1 / R ** 2 - 2 * n * n * g / R ** 3)]], dtype=complex)


def disc_dS_dR(P: Problem, m: int):
    """(nc, 2, 2) derivative of the disc scattering matrix of particle m with respect to R_m."""
    out = np.empty((P.nc, 2, 2), dtype=complex)
    R = P.radius[m]
    lam, mu = P.L.lam_l, P.L.mu_l
    S = P.disc_S(m)
    for i, n in enumerate(range(-P.p, P.p + 1)):
        MH = disc.mode_matrix("H", n, P.L.kp_l, P.L.ks_l, R, int(P.bc[m]), lam, mu)
        dMH = mode_matrix_dR("H", n, P.L.kp_l, P.L.ks_l, R, int(P.bc[m]), lam, mu)
        dMJ = mode_matrix_dR("J", n, P.L.kp_l, P.L.ks_l, R, int(P.bc[m]), lam, mu)
        out[i] = -np.linalg.solve(MH, dMJ + dMH @ S[i])
    return out


# ----------------------------------------------------------------------------- gradient
def gradient(wl, kinds, angles, receivers, d, h_omega: float = 1e-6):
    """(L, dL/dcentres (M,2), dL/dradii (M,), dL/domega) by the adjoint method."""
    P = Problem(wl)
    N = P.M * 2 * P.nc
    A = P.assemble()
    gamma, u = forward(P, kinds, angles, receivers)
    w = u - d                                                     # (nrhs, R, 2)
    F = field_matrix(P, receivers)                                # (R*2, N)
    nrhs = gamma.shape[3]
    g = np.stack([F.conj().T @ w[r].ravel() for r in range(nrhs)], axis=1)      # (N, nrhs)
    lam = np.linalg.solve(A.conj().T, g).reshape(gamma.shape)
    Lval = 0.5 * float(np.sum(np.abs(w) ** 2))

    def contract(dFg, dbv, dAg):
        t = np.sum(np.conj(w) * dFg).real
        t += np.sum(np.conj(lam) * (dbv - dAg)).real
        return t

    gc = np.zeros((P.M, 2))
    for m in range(P.M):
        for axis in (0, 1):
            dTR = dT_gamma(P, gamma, m, axis) + dR_gamma(P, gamma, m, axis)
            dAg = -P.apply_S(dTR)
            gc[m, axis] = contract(dF_gamma(P, gamma, receivers, m, axis), db(P, kinds, angles, m, axis), dAg)
    # radii: dA/dR_m gamma = -(dS_m/dR)(T+R)gamma restricted to m, db = (dS_m/dR) a0^m
    a_loc = P.translate(gamma) + P.reflect(gamma) + P.incident_local(kinds, angles)
    gr = np.zeros(P.M)
    for m in range(P.M):
        dS = disc_dS_dR(P, m)
        v = np.einsum("nij,jnr->inr", dS, a_loc[m])
        gr[m] = np.sum(np.conj(lam[m]) * v).real
    # frequency: central differences of the assembled operators
    hw = h_omega * wl.omega
    mats = []
    for sgn in (1.0, -1.0):
        wl2 = copy.deepcopy(wl)
        wl2.omega = wl.omega + sgn * hw
        P2 = Problem(wl2)
        mats.append((P2.assemble() @ gamma.reshape(N, -1), P2.rhs(kinds, angles).reshape(N, -1),
                     field_matrix(P2, receivers)))
    dAg = ((mats[0][0] - mats[1][0]) / (2 * hw)).reshape(gamma.shape)
    dbv = ((mats[0][1] - mats[1][1]) / (2 * hw)).reshape(gamma.shape)
    dF = (mats[0][2] - mats[1][2]) / (2 * hw)
    dFg = np.stack([(dF @ gamma[..., r].ravel()).reshape(-1, 2) for r in range(nrhs)])
    gw = contract(dFg, dbv, dAg)
    return Lval, gc, gr, gw
