"""Closed-form scattering matrix of a circular particle, one 2x2 block per mode.

Test infrastructure only (see oracle/__init__.py).

Sec. 4.1 expands the incoming field as sum a_n grad(J_n(kp r)e^{in th}) + b_n grad_perp(J_n(ks r)e^{in th})
and the outgoing field with H_n in place of J_n (scatspan); the scattering matrix maps
(a_n, b_n) to (alpha_n, beta_n) and is diagonal in n for a disc.  In polar components
    grad(f(r) e^{in th})      = ( f'        , (in/r) f ) e^{in th}     (r-hat, theta-hat)
    grad_perp(g(r) e^{in th}) = ( -(in/r) g , g'       ) e^{in th}
so the rigid condition u = 0 on r = R gives the 2x2 mode matrix printed in the
projection formula of Sec. 4.3,
    M_Z = [[kp Z_n'(kp R), -(in/R) Z_n(ks R)], [(in/R) Z_n(kp R), ks Z_n'(ks R)]],
and S_n = -M_H^{-1} M_J.  The traction-free condition uses the traction of Sec. 2
(tracdef) on the normal r-hat:  t_r = lam div u + 2 mu d_r u_r,
t_th = mu (d_r u_th - u_th / r + (1/r) d_th u_r), which for each potential gives
    P:  t_r = -lam kp^2 f + 2 mu f'',          t_th = 2 mu i n (f'/r - f/r^2)
    S:  t_r = -2 mu i n (g'/r - g/r^2),        t_th = mu (g'' - g'/r + n^2 g / r^2)
with f = Z_n(kp r), g = Z_n(ks r).  Z'' = (Z_{n-2} - 2 Z_n + Z_{n+2})/4 (DLMF 10.6.1 applied twice).
"""
from __future__ import annotations

import numpy as np

from .waves import Z


def _zd(kind, n, k, R):
    z = Z(kind, n, k * R)
    z1 = 0.5 * k * (Z(kind, n - 1, k * R) - Z(kind, n + 1, k * R))
    z2 = 0.25 * k * k * (Z(kind, n - 2, k * R) - 2 * Z(kind, n, k * R) + Z(kind, n + 2, k * R))
    return z, z1, z2


def mode_matrix(kind: str, n: int, kp: float, ks: float, R: float, bc: int, lam: float, mu: float):
    """2x2 matrix mapping (P coef, S coef) of mode n to the boundary quantity at r = R:
    displacement (u_r, u_th) for bc=0 (rigid), traction (t_r, t_th) for bc=1 (traction-free)."""
    f, f1, f2 = _zd(kind, n, kp, R)
    g, g1, g2 = _zd(kind, n, ks, R)
    if bc == 0:
        return np.array([[f1, -1j * n / R * g], [1j * n / R * f, g1]], dtype=complex)
    tp_r = -lam * kp * kp * f + 2 * mu * f2
    tp_t = 2 * mu * 1j * n * (f1 / R - f / R ** 2)
    ts_r = -2 * mu * 1j * n * (g1 / R - g / R ** 2)
    ts_t = mu * (g2 - g1 / R + n * n * g / R ** 2)
    return np.array([[tp_r, ts_r], [tp_t, ts_t]], dtype=complex)


def disc_smatrix(p: int, kp: float, ks: float, R: float, bc: int, lam: float, mu: float):
    """(2p+1, 2, 2) complex array: S[n+p] maps (a_n, b_n) to (alpha_n, beta_n)."""
    out = np.empty((2 * p + 1, 2, 2), dtype=complex)
    for i, n in enumerate(range(-p, p + 1)):
        MH = mode_matrix("H", n, kp, ks, R, bc, lam, mu)
        MJ = mode_matrix("J", n, kp, ks, R, bc, lam, mu)
        out[i] = -np.linalg.solve(MH, MJ)
    return out
