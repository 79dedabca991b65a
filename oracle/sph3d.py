"""Vector spherical wave functions of the 3D elastic extension (Sec. 6): spherical harmonics and their
surface gradients (also at complex unit directions, by analytic continuation), the three families
L = grad v^{kp}, M = curl(x v^{ks}), N = curl curl(x v^{ks}) / (i ks), closed-form sphere scattering
matrices (rigid and traction-free), the plane-wave expansion coefficients a, b, c (Sec. 6.3), and the
free-space translation of outgoing expansions into local ones by projection on a sphere.

Test infrastructure only (see oracle/__init__.py).

Conventions (reading A24)
-------------------------
Y_n^m(theta, phi) = N_nm P_n^|m|(cos theta) e^{i m phi},  N_nm = sqrt((2n+1)/(4 pi) (n-|m|)!/(n+|m|)!),
with P_n^|m|(t) = (1 - t^2)^{|m|/2} d^|m| P_n / dt^|m| (no Condon-Shortley sign), so that
Y_n^{-m} = conj(Y_n^m) on real directions, which is what the paper's plane-wave coefficients (written
with Y_n^{-m}(d) where the textbook expansion has conj(Y_n^m(d))) require.  On the unit sphere
sin^|m| theta e^{+-i|m| phi} = (x +- i y)^|m|, so Y_n^m(d) = N_nm Q(d_z) (d_x +- i d_y)^|m| with the
polynomial Q = d^|m| P_n / dt^|m|: a polynomial in the components of d, which continues Y_n^m
analytically to complex d with d.d = 1.  The surface gradient is Grad Y(d) = grad H(d) - n H(d) d for
the solid harmonic H(x) = |x|^n Y(x/|x|), again a polynomial.

Coefficient layout of one sphere with order p (reading A25): [alpha (n = 1..p) | beta (n = 1..p) |
gamma (n = 0..p)], (n, m) at n^2 + n + m (minus 1 for alpha and beta, which start at n = 1): 2 p (p+2)
+ (p+1)^2 values.  alpha multiplies N, beta M (shear, ks), gamma L (compressional, kp).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import spherical_jn, spherical_yn


# ------------------------------------------------------------------ indexing
def nlm(p: int) -> int:
    """Number of (n, m) pairs with 0 <= n <= p."""
    return (p + 1) ** 2


def idx(n: int, m: int) -> int:
    return n * n + n + m


def sizes(p: int):
    """(alpha/beta block length, gamma block length, total) of one sphere."""
    nmn = p * (p + 2)
    return nmn, nlm(p), 2 * nmn + nlm(p)


def orders(p: int):
    """Arrays n, m over the (n, m) pairs 0 <= n <= p in index order."""
    n = np.concatenate([[k] * (2 * k + 1) for k in range(p + 1)]).astype(int)
    m = np.concatenate([np.arange(-k, k + 1) for k in range(p + 1)]).astype(int)
    return n, m


# ------------------------------------------------------------------ spherical harmonics
def _ylm_poly(p: int):
    """Per (n, m): N_nm, |m|, and the power-series coefficients of Q = d^|m| P_n / dt^|m|."""
    out = []
    for n in range(p + 1):
        pn = np.polynomial.legendre.leg2poly([0] * n + [1])          # P_n in powers of t
        for m in range(-n, n + 1):
            am = abs(m)
            q = np.polynomial.polynomial.polyder(pn, am) if am else pn
            norm = math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - am) / math.factorial(n + am))
            out.append((n, m, am, norm, np.asarray(q, dtype=float)))
    return out


def ylm(p: int, d):
    """Y_n^m(d) for every (n, m), n <= p, at unit directions d (..., 3), real or complex with d.d = 1.
    Returns (..., (p+1)^2)."""
    d = np.asarray(d)
    dz = d[..., 2]
    out = np.zeros(d.shape[:-1] + (nlm(p),), dtype=complex)
    for n, m, am, norm, q in _ylm_poly(p):
        w = d[..., 0] + (1j if m >= 0 else -1j) * d[..., 1]
        out[..., idx(n, m)] = norm * np.polynomial.polynomial.polyval(dz, q) * w ** am
    return out


def grad_ylm(p: int, d):
    """Surface gradient Grad Y_n^m(d) = grad H(d) - n H(d) d for every (n, m), n <= p, at unit directions
    d (..., 3), real or complex.  H(x) = N w^|m| sum_j c_j z^j (x.x)^{k_j}, k_j = (n - |m| - j) / 2, w = x +- i y.
    Returns (..., (p+1)^2, 3)."""
    d = np.asarray(d)
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    out = np.zeros(d.shape[:-1] + (nlm(p), 3), dtype=complex)
    zp = [z ** j for j in range(p + 1)]                                  # z^j, j = 0..p
    for n, m, am, norm, q in _ylm_poly(p):
        sg = 1j if m >= 0 else -1j
        w = x + sg * y
        j = np.arange(len(q))
        k = (n - am - j) / 2.0
        s0 = sum(q[i] * zp[i] for i in range(len(q)))
        s1 = sum(q[i] * k[i] * zp[i] for i in range(len(q)))
        s2 = sum(q[i] * j[i] * zp[i - 1] for i in range(1, len(q))) if len(q) > 1 else 0.0 * z
        wm = w ** am
        wm1 = am * w ** (am - 1) if am > 0 else 0.0 * w
        H = norm * wm * s0
        gx = norm * (wm1 * s0 + wm * 2.0 * x * s1)
        gy = norm * (sg * wm1 * s0 + wm * 2.0 * y * s1)
        gz = norm * wm * (s2 + 2.0 * z * s1)
        out[..., idx(n, m), 0] = gx - n * H * x
        out[..., idx(n, m), 1] = gy - n * H * y
        out[..., idx(n, m), 2] = gz - n * H * z
    return out


def neg_m(p: int):
    """Permutation taking the (n, m) index order to (n, -m)."""
    n, m = orders(p)
    return np.array([idx(a, -b) for a, b in zip(n, m)])


# ------------------------------------------------------------------ radial functions
def radial(nmax: int, x, kind: str):
    """z_n(x) and z_n'(x) for n = 0..nmax at real x: kind 'j' (regular) or 'h' (outgoing h^(1))."""
    x = np.asarray(x, dtype=float)
    n = np.arange(nmax + 1)
    xx = x[..., None]
    j = spherical_jn(n, xx)
    jd = spherical_jn(n, xx, derivative=True)
    if kind == "j":
        return j, jd
    y = spherical_yn(n, xx)
    yd = spherical_yn(n, xx, derivative=True)
    return j + 1j * y, jd + 1j * yd


# ------------------------------------------------------------------ vector spherical wave functions
def vswf(p: int, kp: float, ks: float, x, kind: str):
    """The three families at points x (..., 3) relative to the expansion centre (x != 0):
    N_nm, M_nm (n = 1..p, shear) and L_nm (n = 0..p, compressional), as arrays (..., count, 3):
      L = kp z_n'(kp r) Y rhat + z_n(kp r)/r Grad Y
      M = z_n(ks r) Grad Y x rhat                                   (= curl(x z_n Y))
      N = [n(n+1) z_n(ks r)/r Y rhat + (z_n(ks r) + ks r z_n'(ks r))/r Grad Y] / (i ks)
    with z = j (kind 'j') or h^(1) (kind 'h')."""
    x = np.asarray(x, dtype=float)
    r = np.linalg.norm(x, axis=-1)
    rh = x / r[..., None]
    Y = ylm(p, rh)
    G = grad_ylm(p, rh)
    n, _ = orders(p)
    zs, zsd = radial(p, ks * r, kind)
    zp, zpd = radial(p, kp * r, kind)
    zs_n, zsd_n = zs[..., n], zsd[..., n]
    zp_n, zpd_n = zp[..., n], zpd[..., n]
    rr = r[..., None]
    L = (kp * zpd_n * Y)[..., None] * rh[..., None, :] + (zp_n / rr)[..., None] * G
    X = np.cross(G, rh[..., None, :])
    M = zs_n[..., None] * X
    nn1 = n * (n + 1)
    N = ((nn1 * zs_n / rr * Y)[..., None] * rh[..., None, :]
         + ((zs_n + ks * rr * zsd_n) / rr)[..., None] * G) / (1j * ks)
    return N[..., 1:, :], M[..., 1:, :], L


def field(p: int, kp: float, ks: float, x, coeffs, kind: str = "h"):
    """Displacement sum alpha N + beta M + gamma L at points x (..., 3) relative to the centre, for one
    coefficient vector (layout of the module docstring) or a block (total, nrhs).  Returns (..., 3[, nrhs])."""
    nmn, nl, tot = sizes(p)
    c = np.asarray(coeffs)
    N, M, L = vswf(p, kp, ks, x, kind)
    if c.ndim == 1:
        return (np.einsum("...ki,k->...i", N, c[:nmn]) + np.einsum("...ki,k->...i", M, c[nmn:2 * nmn])
                + np.einsum("...ki,k->...i", L, c[2 * nmn:]))
    return _mode_sum(N, c[:nmn]) + _mode_sum(M, c[nmn:2 * nmn]) + _mode_sum(L, c[2 * nmn:])


def _mode_sum(V, c):
    """sum_k V[..., k, i] c[k, r] -> (..., 3, nrhs), as one matrix product."""
    lead = V.shape[:-2]
    Vt = np.moveaxis(V, -2, -1).reshape(-1, V.shape[-2])
    return (Vt @ c).reshape(lead + (V.shape[-1], c.shape[-1]))


# ------------------------------------------------------------------ traction on a sphere
def _traction_coeffs(n: int, kp: float, ks: float, lam: float, mu: float, R: float, kind: str):
    """Traction sigma(u) rhat on the sphere r = R of the (n, m) wave functions, in the components
    (rhat Y, Grad Y, Grad Y x rhat):  N -> (tN_r, tN_g, 0), M -> (0, 0, tM), L -> (tL_r, tL_g, 0).
    From T u = 2 mu (rhat.grad) u + lam rhat div u + mu rhat x curl u with div N = div M = 0,
    curl M = i ks N, curl N = -i ks M, div L = -kp^2 z Y, curl L = 0."""
    zs, zsd = radial(n + 1, ks * R, kind)
    zp, zpd = radial(n + 1, kp * R, kind)
    z, zd = zs[n], zsd[n]
    # second derivatives from the spherical Bessel equation: x^2 z'' = -2 x z' - (x^2 - n(n+1)) z
    xs, xp = ks * R, kp * R
    zdd = (-2.0 * xs * zd - (xs * xs - n * (n + 1)) * z) / (xs * xs)
    q, qd = zp[n], zpd[n]
    qdd = (-2.0 * xp * qd - (xp * xp - n * (n + 1)) * q) / (xp * xp)
    tM = mu * (ks * zd - z / R)
    # N: radial and tangential parts of d/dr N, plus mu rhat x curl N = -i ks mu z Grad Y
    dr_a = n * (n + 1) * (ks * zd / R - z / (R * R))                      # d/dr [n(n+1) z / r]
    dr_b = ks * zd / R - z / (R * R) + ks * ks * zdd                      # d/dr [(z + ks r z') / r]
    tN_r = 2.0 * mu * dr_a / (1j * ks)
    tN_g = 2.0 * mu * dr_b / (1j * ks) - 1j * ks * mu * z
    tL_r = 2.0 * mu * kp * kp * qdd - lam * kp * kp * q
    tL_g = 2.0 * mu * (kp * qd / R - q / (R * R))
    return tN_r, tN_g, tM, tL_r, tL_g


def sphere_smatrix(p: int, kp: float, ks: float, lam: float, mu: float, R: float, bc: int):
    """Closed-form scattering matrix of a sphere of radius R per order n (independent of m): the
    outgoing (alpha, beta, gamma) for an incoming regular (a, b, c), from the boundary condition on
    r = R -- bc 0 rigid (u = 0), bc 1 traction-free (sigma rhat = 0) -- matched in the components
    rhat Y, Grad Y and Grad Y x rhat, which are orthogonal.  Returns list of (S2 [2x2 on (alpha, gamma)
    from (a, c)], s_beta) for n = 1..p and the scalar s0 for n = 0 (gamma_00 = s0 c_00)."""
    out = []
    for n in range(0, p + 1):
        def comps(kind):
            zs, zsd = radial(n, ks * R, kind)
            zp, zpd = radial(n, kp * R, kind)
            if bc == 0:
                Nr = n * (n + 1) * zs[n] / R / (1j * ks)
                Ng = (zs[n] + ks * R * zsd[n]) / R / (1j * ks)
                Mt = zs[n]
                Lr = kp * zpd[n]
                Lg = zp[n] / R
            else:
                Nr, Ng, Mt, Lr, Lg = _traction_coeffs(n, kp, ks, lam, mu, R, kind)
            return Nr, Ng, Mt, Lr, Lg
        Nr_h, Ng_h, Mt_h, Lr_h, Lg_h = comps("h")
        Nr_j, Ng_j, Mt_j, Lr_j, Lg_j = comps("j")
        if n == 0:
            out.append(-Lr_j / Lr_h)
            continue
        A = np.array([[Nr_h, Lr_h], [Ng_h, Lg_h]])
        B = np.array([[Nr_j, Lr_j], [Ng_j, Lg_j]])
        out.append((-np.linalg.solve(A, B), -Mt_j / Mt_h))
    return out


def apply_sphere_S(p: int, Sn, a):
    """Outgoing coefficients S a for one sphere's incoming block a (total[, nrhs])."""
    nmn, nl, tot = sizes(p)
    a = np.asarray(a)
    out = np.zeros_like(a, dtype=complex)
    nvec, mvec = orders(p)
    for k in range(nl):
        n = nvec[k]
        if n == 0:
            out[2 * nmn + k] = Sn[0] * a[2 * nmn + k]
            continue
        S2, sb = Sn[n]
        ka = k - 1
        out[ka] = S2[0, 0] * a[ka] + S2[0, 1] * a[2 * nmn + k]
        out[2 * nmn + k] = S2[1, 0] * a[ka] + S2[1, 1] * a[2 * nmn + k]
        out[nmn + ka] = sb * a[nmn + ka]
    return out


# ------------------------------------------------------------------ plane waves (Sec. 6.3)
def plane_wave_coeffs(p: int, kp: float, d, pol):
    """Regular coefficients (a, b, c) of exp(i ks x.d) (d x pol) x d + exp(i kp x.d) (d.pol) d about the
    origin, as the paper states them (Sec. 6.3):
      a_nm = 4 pi i^n / (n(n+1)) Grad Y_n^{-m}(d) . pol,  b_nm = -4 pi i^n / (n(n+1)) (d x Grad Y_n^{-m}(d)) . pol,
      c_nm = -4 pi i^{n+1} / kp  Y_n^{-m}(d) (d . pol),
    d a unit direction (d.d = 1, complex allowed), pol any vector; both may carry leading batch axes
    (..., 3).  Returns the coefficient vectors (..., total)."""
    d = np.asarray(d, dtype=complex)
    pol = np.asarray(pol, dtype=complex)
    nmn, nl, tot = sizes(p)
    Y = ylm(p, d)[..., neg_m(p)]
    G = grad_ylm(p, d)[..., neg_m(p), :]
    n, _ = orders(p)
    c = np.zeros(d.shape[:-1] + (tot,), dtype=complex)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = 4.0 * np.pi * (1j ** n) / (n * (n + 1))
    ga = np.einsum("...ki,...i->...k", G, pol)
    gb = np.einsum("...ki,...i->...k", np.cross(d[..., None, :], G), pol)
    c[..., :nmn] = (f * ga)[..., 1:]
    c[..., nmn:2 * nmn] = (-f * gb)[..., 1:]
    c[..., 2 * nmn:] = -4.0 * np.pi * (1j ** (n + 1)) / kp * Y * np.sum(d * pol, axis=-1)[..., None]
    return c


# ------------------------------------------------------------------ projection onto regular waves
def sphere_rule(ntheta: int):
    """Gauss-Legendre in cos(theta) x 2 ntheta equispaced phi: unit directions (K, 3) and weights (K,);
    exact for spherical polynomials of degree <= 2 ntheta - 1."""
    t, w = np.polynomial.legendre.leggauss(ntheta)
    nphi = 2 * ntheta
    ph = 2.0 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1.0 - t * t)
    d = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(t, np.ones(nphi))], axis=-1)
    W = np.outer(w, np.full(nphi, 2.0 * np.pi / nphi))
    return d.reshape(-1, 3), W.reshape(-1)


def project_regular(p: int, kp: float, ks: float, rho: float, u, dirs, wts):
    """Regular coefficients (a, b, c), n <= p, of a field given at rho * dirs (K, 3[, nrhs]) on the sphere
    of radius rho: the components u.rhat, u.Grad Y* / (n(n+1)) and u.(Grad Y x rhat)* / (n(n+1)) are
    projected with the rule, and per n the 2 x 2 system of the N and L waves in the rhat Y and Grad Y
    components is solved; b from the third component."""
    nmn, nl, tot = sizes(p)
    u = np.asarray(u)
    vec = u.ndim == 2
    if vec:
        u = u[..., None]
    Y = ylm(p, dirs)
    G = grad_ylm(p, dirs)
    X = np.cross(G, dirs[:, None, :])
    ur = np.einsum("ki,kir->kr", dirs.astype(complex), u)
    n, _ = orders(p)
    nn1 = np.where(n > 0, n * (n + 1), 1)
    f = (Y.conj() * wts[:, None]).T @ ur                                        # sum_k w_k Y*_kj ur_kr
    g = np.tensordot(G.conj() * wts[:, None, None], u, axes=([0, 2], [0, 1])) / nn1[:, None]
    h = np.tensordot(X.conj() * wts[:, None, None], u, axes=([0, 2], [0, 1])) / nn1[:, None]
    zs, zsd = radial(p, ks * rho, "j")
    zp, zpd = radial(p, kp * rho, "j")
    out = np.zeros((tot, u.shape[-1]), dtype=complex)
    for k in range(nl):
        nk = n[k]
        if nk == 0:
            out[2 * nmn + k] = f[k] / (kp * zpd[0])
            continue
        A = np.array([[nk * (nk + 1) * zs[nk] / rho / (1j * ks), kp * zpd[nk]],
                      [(zs[nk] + ks * rho * zsd[nk]) / rho / (1j * ks), zp[nk] / rho]])
        sol = np.linalg.solve(A, np.stack([f[k], g[k]]))
        out[k - 1] = sol[0]
        out[2 * nmn + k] = sol[1]
        out[nmn + k - 1] = h[k] / zs[nk]
    return out if not vec else out[:, 0]


def translate(p: int, kp: float, ks: float, src_centres, src_coeffs, tgt_centre, rho: float, ntheta: int = 40):
    """Local (regular) coefficients about tgt_centre of the outgoing fields of the given sources
    (centres (L, 3), coefficient blocks (L, total[, nrhs])): the summed field evaluated on the sphere of
    radius rho about the target and projected (project_regular).  rho must be below the distance to
    every source; ntheta sets the rule (exact to degree 2 ntheta - 1).  The field on the sphere holds
    every degree, decaying like (rho/d)^n for a source at distance d: degrees beyond the rule alias into
    the projected ones, so at rho/d = 1/2 the rule needs 2 ntheta - 1 - p >~ 70 (ntheta = 40 gives 1e-13
    at p <= 8; 24 nodes leave 1e-7 at p = 4 and 4e-4 at p = 8)."""
    dirs, wts = sphere_rule(ntheta)
    pts = np.asarray(tgt_centre)[None, :] + rho * dirs
    u = 0.0
    for c, g in zip(np.asarray(src_centres), np.asarray(src_coeffs)):
        u = u + field(p, kp, ks, pts - c[None, :], g, "h")
    return project_regular(p, kp, ks, rho, u, dirs, wts)
