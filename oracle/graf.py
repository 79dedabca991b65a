"""Multipole-to-local translation between two particles (Sec. 4.2, Graf's addition theorem).

Test infrastructure only (see oracle/__init__.py).

Sec. 4.2 writes T^{ml} = diag(a^{ml}, b^{ml}) with
    a_ij = H_{i-j}(kp |x_l - x_m|) e^{-i (i-j)(theta_ml - pi)}
(b with ks).  We read theta_ml as the polar angle of x_m - x_l (reading A1), which turns
the entry into Graf's form (DLMF 10.23.7)
    T[i, j] = H_{j-i}(k d) e^{i (j-i) theta_d},   d e^{i theta_d} = x_m - x_l,
i.e. a^m_i = sum_j T[i, j] alpha^l_j.  The two forms agree because H_{-n} = (-1)^n H_n.
The pin test evaluates the outgoing potential directly and through the local expansion.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def translation_matrix(p: int, k: float, xm, xl, p_out: int | None = None):
    """(2 p_out + 1, 2p+1) matrix T with T[i, j] = H_{j-i}(k d) e^{i (j-i) theta_d}."""
    if p_out is None:
        p_out = p
    dx = xm[0] - xl[0]
    dy = xm[1] - xl[1]
    d = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    i = np.arange(-p_out, p_out + 1)[:, None]
    j = np.arange(-p, p + 1)[None, :]
    nu = j - i
    return special.hankel1(nu, k * d) * np.exp(1j * nu * th)


def translation_all_sources(p: int, k: float, xm, centres):
    """T^{ml} for one target m against every source l: (M, 2p+1, 2p+1); rows l with d = 0 are zero."""
    dx = xm[0] - centres[:, 0]
    dy = xm[1] - centres[:, 1]
    d = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    kk = np.arange(-2 * p, 2 * p + 1)
    h = np.zeros((centres.shape[0], kk.size), dtype=complex)
    nz = d > 0
    h[nz] = special.hankel1(kk[None, :], k * d[nz, None]) * np.exp(1j * kk[None, :] * th[nz, None])
    i = np.arange(-p, p + 1)[:, None]
    j = np.arange(-p, p + 1)[None, :]
    return h[:, (j - i) + 2 * p]
