"""Cylindrical wave functions, their Cartesian derivatives, and elastic traction.

Test infrastructure only (see oracle/__init__.py).

w_n(x) = Z_n(k r) e^{i n theta} with Z = J (incoming, u_n of Sec. 4.1) or Z = H^(1)
(outgoing, v_n of Sec. 4.1).  Derivatives use the order-shift rules that follow from
DLMF 10.6.1 / 10.6.2:
    d/dx w_n = (k/2)(w_{n-1} - w_{n+1}),      d/dy w_n = (i k/2)(w_{n-1} + w_{n+1}),
and their compositions for second derivatives.  The displacement of a pair of
potentials is u = grad(phi) + grad_perp(psi), grad_perp = (-d/dy, d/dx) (Sec. 2), and
the traction on a unit normal nu is  sigma(u) nu = lam (div u) nu + mu (grad u + grad u^T) nu
(Sec. 2, tracdef).
"""
from __future__ import annotations

import numpy as np
from scipy import special


def Z(kind: str, n, x):
    if kind == "J":
        return special.jv(n, x)
    if kind == "H":
        return special.hankel1(n, x)
    raise ValueError(kind)


def wave_derivs(kind: str, n: int, k: float, X, Y):
    """Value and first/second Cartesian derivatives of Z_n(k r) e^{i n theta} at (X, Y).

    Returns a dict with keys '', 'x', 'y', 'xx', 'xy', 'yy' (arrays shaped like X)."""
    X = np.asarray(X, dtype=float)
    Y = np.asarray(Y, dtype=float)
    r = np.hypot(X, Y)
    th = np.arctan2(Y, X)

    def w(m):
        return Z(kind, m, k * r) * np.exp(1j * m * th)

    wm2, wm1, w0, wp1, wp2 = w(n - 2), w(n - 1), w(n), w(n + 1), w(n + 2)
    return {
        "": w0,
        "x": 0.5 * k * (wm1 - wp1),
        "y": 0.5j * k * (wm1 + wp1),
        "xx": 0.25 * k * k * (wm2 - 2 * w0 + wp2),
        "xy": 0.25j * k * k * (wm2 - wp2),
        "yy": -0.25 * k * k * (wm2 + 2 * w0 + wp2),
    }


def displacement_and_gradient(phi: dict, psi: dict):
    """u = grad phi + grad_perp psi and its Jacobian, from derivative dicts of phi and psi.

    Returns (u1, u2, [[du1/dx, du1/dy], [du2/dx, du2/dy]])."""
    u1 = phi["x"] - psi["y"]
    u2 = phi["y"] + psi["x"]
    g = [[phi["xx"] - psi["xy"], phi["xy"] - psi["yy"]],
         [phi["xy"] + psi["xx"], phi["yy"] + psi["xy"]]]
    return u1, u2, g


def traction(g, nu1, nu2, lam: float, mu: float):
    """sigma(u) nu for the Jacobian g[i][j] = d u_i / d x_j (Sec. 2, tracdef)."""
    div = g[0][0] + g[1][1]
    e11 = g[0][0]
    e22 = g[1][1]
    e12 = 0.5 * (g[0][1] + g[1][0])
    t1 = lam * div * nu1 + 2 * mu * (e11 * nu1 + e12 * nu2)
    t2 = lam * div * nu2 + 2 * mu * (e12 * nu1 + e22 * nu2)
    return t1, t2


def field_of_coeffs(kind: str, coef_p, coef_s, p: int, kp: float, ks: float, X, Y):
    """u and grad u of  sum_n coef_p[n] grad(Z_n(kp r)e^{in th}) + coef_s[n] grad_perp(Z_n(ks r)e^{in th}).

    coef arrays are indexed by n + p, n in [-p, p]; (X, Y) are coordinates relative to the
    expansion centre."""
    X = np.asarray(X, dtype=float)
    acc_phi = {k: np.zeros(X.shape, complex) for k in ("", "x", "y", "xx", "xy", "yy")}
    acc_psi = {k: np.zeros(X.shape, complex) for k in ("", "x", "y", "xx", "xy", "yy")}
    for i, n in enumerate(range(-p, p + 1)):
        if coef_p[i] != 0:
            d = wave_derivs(kind, n, kp, X, Y)
            for key in acc_phi:
                acc_phi[key] += coef_p[i] * d[key]
        if coef_s[i] != 0:
            d = wave_derivs(kind, n, ks, X, Y)
            for key in acc_psi:
                acc_psi[key] += coef_s[i] * d[key]
    return displacement_and_gradient(acc_phi, acc_psi)
