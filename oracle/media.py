"""Wavenumbers of the two layers (Sec. 2: kp = omega/sqrt(lam+2mu), ks = omega/sqrt(mu), rho=1).

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import math


def wavenumbers(lam: float, mu: float, omega: float):
    """Compressional and shear wavenumbers of one layer with unit density (Sec. 2)."""
    return omega / math.sqrt(lam + 2.0 * mu), omega / math.sqrt(mu)


class Layered:
    """Upper layer (lam, mu, kp, ks) and lower layer (lam', mu', kp', ks') at frequency omega (Sec. 3)."""

    def __init__(self, media, omega: float):
        self.omega = float(omega)
        self.lam_u, self.mu_u = float(media.lam_u), float(media.mu_u)
        self.lam_l, self.mu_l = float(media.lam_l), float(media.mu_l)
        self.kp_u, self.ks_u = wavenumbers(self.lam_u, self.mu_u, omega)
        self.kp_l, self.ks_l = wavenumbers(self.lam_l, self.mu_l, omega)
