// 3D extension (Sec. 6): spheres below the interface of two welded elastic half-spaces, vector
// spherical wave expansions, 2D Sommerfeld integrals in polar form.  FP64 throughout.
//
// One application of  y = x - S (T + R) x  (ms3_b300.h) runs as
//   k3_cart       each sphere's shear field as three Cartesian scalar outgoing expansions (degree <= p+1)
//   k3_translate  every sphere's Cartesian shear expansions and compressional potential translated to
//                 regular expansions about every other sphere by the scalar addition theorem, on the fly
//   k3_uncart     regular Cartesian shear expansions back to the coefficients a (N) and b (M); the
//                 compressional potential's coefficients are c directly (L = grad v)
//   k3_m2s        upgoing P, SV, SH amplitudes at every Sommerfeld node (block B, Sec. 6.2)
//   k3_reflect    the 3 x 3 reflection at z = 0 per node, quadrature weight folded in
//   k3_s2l        regular expansions of the downgoing waves about every sphere (block C, Sec. 6.3)
//   k3_sapply     the sphere matrices and the combine y = x - S a
//
// Translation (block D).  With x = x' + d, d = c_m - c_l, |x'| < |d|, the scalar addition theorem
//     h_n(k |x|) Y_n^m(x^) = sum_{nu, mu} A^{n m}_{nu mu}(d) j_nu(k |x'|) Y_nu^mu(x'^),
//     A^{n m}_{nu mu} = 4 pi sum_q i^{nu - n + q} h_q(k |d|) Y_q^{m - mu}(d^) G(n, m; nu, mu; q),
//     G = int Y_n^m conj(Y_nu^mu) conj(Y_q^{m - mu}) dOmega   (Gaunt; q = |n - nu|, |n - nu| + 2, ..., n + nu),
// translates the compressional potential sum gamma v^{kp} (L = grad v, so its regular coefficients are c).
// The shear field is not a scalar potential; its three Cartesian components are scalar outgoing waves:
//     N_nm = [(n+1) z_{n-1} V-_nm + n z_{n+1} V+_nm] / (i (2n+1)),   M_nm = z_n X_nm,
//     V-_nm = n Y rhat + Grad Y (components of degree n-1), V+_nm = (n+1) Y rhat - Grad Y (degree n+1),
//     X_nm = Grad Y x rhat (degree n),
// (z_n(kr)/(kr) and z_n' by the three-term relations), so each component is translated as a scalar and
// the regular coefficients come back by orthogonality of V-, V+ and X on the sphere:
//     a_Jm = i <V-_Jm, U_{J-1}> / (J (J+1)),   b_Jm = <X_Jm, U_J> / (J (J+1)),
// U_nu the degree-nu part of the regular Cartesian expansion.  The Gaunt coefficients and the Cartesian
// maps are computed at setup by exact Gauss quadrature on the sphere.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <functional>
#include <new>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "ms3_b300.h"

typedef std::complex<double> cd;

namespace {

constexpr int P3MAX = 10;               // 4 (p+1)^2 translation threads per CTA <= 512
constexpr int RC = 16;                 // right-hand sides per translation / m2s chunk

inline int idx(int n, int m) { return n * n + n + m; }
inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ host: spherical functions
// Q[n][m] = d^m P_n / dt^m (0 <= m <= n <= P) at complex t by the recurrence in n at fixed m:
// Q_m^m = (2m-1)!!, Q_{m+1}^m = (2m+1) t Q_m^m, (n-m+1) Q_{n+1}^m = (2n+1) t Q_n^m - (n+m) Q_{n-1}^m.
std::vector<cd> qtab(int P, cd t) {
    std::vector<cd> Q((size_t)(P + 2) * (P + 2), cd(0));
    auto at = [&](int n, int m) -> cd& { return Q[(size_t)n * (P + 2) + m]; };
    double df = 1.0;
    for (int m = 0; m <= P; ++m) {
        if (m > 0) df *= (2.0 * m - 1.0);
        at(m, m) = df;
        if (m + 1 <= P) at(m + 1, m) = (2.0 * m + 1.0) * t * df;
        for (int n = m + 1; n < P; ++n) at(n + 1, m) = ((2.0 * n + 1.0) * t * at(n, m) - (double)(n + m) * at(n - 1, m)) / (double)(n - m + 1);
    }
    return Q;
}

double ynorm(int n, int am) {
    double r = (2.0 * n + 1.0) / (4.0 * M_PI);
    for (int k = n - am + 1; k <= n + am; ++k) r /= k;
    return sqrt(r);
}

// Y_n^m(d) for n <= P at a unit direction d (d.d = 1, complex allowed): N Q_n^|m|(d_z) (d_x +- i d_y)^|m|
void ylm_c(int P, const cd d[3], std::vector<cd>& Y) {
    Y.assign((size_t)(P + 1) * (P + 1), cd(0));
    const std::vector<cd> Q = qtab(P + 1, d[2]);
    for (int n = 0; n <= P; ++n)
        for (int m = -n; m <= n; ++m) {
            const int am = std::abs(m);
            const cd w = d[0] + (m >= 0 ? cd(0, 1) : cd(0, -1)) * d[1];
            Y[idx(n, m)] = ynorm(n, am) * Q[(size_t)n * (P + 3) + am] * std::pow(w, am);
        }
}

// Surface gradient Grad Y = grad H - n H d of the solid harmonic H = N w^|m| r^{n-|m|} Q(z/r), at r = 1:
//   Grad Y = N [ |m| w^{|m|-1} Q grad w - |m| w^|m| Q d + w^|m| Q_n^{|m|+1} (e_z - d_z d) ],  grad w = (1, +-i, 0)
void grad_ylm_c(int P, const cd d[3], std::vector<cd>& G) {
    G.assign((size_t)(P + 1) * (P + 1) * 3, cd(0));
    const std::vector<cd> Q = qtab(P + 1, d[2]);
    auto q = [&](int n, int m) -> cd { return m > n ? cd(0) : Q[(size_t)n * (P + 3) + m]; };
    for (int n = 0; n <= P; ++n)
        for (int m = -n; m <= n; ++m) {
            const int am = std::abs(m);
            const cd sg = m >= 0 ? cd(0, 1) : cd(0, -1);
            const cd w = d[0] + sg * d[1];
            const double N = ynorm(n, am);
            const cd wm = std::pow(w, am);
            const cd wm1 = am > 0 ? (double)am * std::pow(w, am - 1) : cd(0);
            const cd Qn = q(n, am), Qd = q(n, am + 1);
            const cd gw[3] = {cd(1), sg, cd(0)};
            const cd ez[3] = {cd(0), cd(0), cd(1)};
            for (int i = 0; i < 3; ++i)
                G[(size_t)idx(n, m) * 3 + i] = N * (wm1 * Qn * gw[i] - (double)am * wm * Qn * d[i] + wm * Qd * (ez[i] - d[2] * d[i]));
        }
}

cd dot3(const cd a[3], const cd b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
void cross3(const cd a[3], const cd b[3], cd out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

// spherical Bessel and Hankel values z_n, z_n' at real x, n = 0..N
void sph_jh(int N, double x, std::vector<cd>& j, std::vector<cd>& jd, std::vector<cd>& h, std::vector<cd>& hd) {
    j.resize(N + 2); jd.resize(N + 1); h.resize(N + 2); hd.resize(N + 1);
    for (int n = 0; n <= N + 1; ++n) {
        const double jn = std::sph_bessel((unsigned)n, x), yn = std::sph_neumann((unsigned)n, x);
        j[n] = jn;
        h[n] = cd(jn, yn);
    }
    for (int n = 0; n <= N; ++n) {
        // z_n' = n z_n / x - z_{n+1}
        jd[n] = (double)n * j[n] / x - j[n + 1];
        hd[n] = (double)n * h[n] / x - h[n + 1];
    }
}

// Rigid (bc 0) or traction-free (bc 1) sphere: per n the 2 x 2 map (a, c) -> (alpha, gamma) and the
// scalar b -> beta, from the boundary condition in the orthogonal components (rhat Y, Grad Y, Grad Y x rhat).
void sphere_s(int p, double kp, double ks, double lam, double mu, double R, int bc, cd* out /* [p+1][5] */) {
    std::vector<cd> js, jsd, hs, hsd, jp, jpd, hp, hpd;
    sph_jh(p, ks * R, js, jsd, hs, hsd);
    sph_jh(p, kp * R, jp, jpd, hp, hpd);
    const cd I(0, 1);
    for (int n = 0; n <= p; ++n) {
        cd comp[2][5];     // [j or h][Nr, Ng, Mt, Lr, Lg]
        for (int kind = 0; kind < 2; ++kind) {
            const cd z = kind ? hs[n] : js[n], zd = kind ? hsd[n] : jsd[n];
            const cd qv = kind ? hp[n] : jp[n], qd = kind ? hpd[n] : jpd[n];
            if (bc == 0) {
                comp[kind][0] = (double)(n * (n + 1)) * z / R / (I * ks);
                comp[kind][1] = (z + ks * R * zd) / R / (I * ks);
                comp[kind][2] = z;
                comp[kind][3] = kp * qd;
                comp[kind][4] = qv / R;
            } else {
                // traction sigma(u) rhat = 2 mu d_r u + lam rhat div u + mu rhat x curl u, with
                // x^2 z'' = -2 x z' - (x^2 - n(n+1)) z for the second derivatives
                const double xs = ks * R, xp = kp * R;
                const cd zdd = (-2.0 * xs * zd - (xs * xs - n * (n + 1.0)) * z) / (xs * xs);
                const cd qdd = (-2.0 * xp * qd - (xp * xp - n * (n + 1.0)) * qv) / (xp * xp);
                const cd dra = (double)(n * (n + 1)) * (ks * zd / R - z / (R * R));
                const cd drb = ks * zd / R - z / (R * R) + ks * ks * zdd;
                comp[kind][0] = 2.0 * mu * dra / (I * ks);
                comp[kind][1] = 2.0 * mu * drb / (I * ks) - I * ks * mu * z;
                comp[kind][2] = mu * (ks * zd - z / R);
                comp[kind][3] = 2.0 * mu * kp * kp * qdd - lam * kp * kp * qv;
                comp[kind][4] = 2.0 * mu * (kp * qd / R - qv / (R * R));
            }
        }
        cd* o = out + (size_t)n * 5;
        for (int k = 0; k < 5; ++k) o[k] = 0;
        if (n == 0) {
            o[0] = -comp[0][3] / comp[1][3];
            continue;
        }
        // S2 = -A^{-1} B, A = [[Nr_h, Lr_h], [Ng_h, Lg_h]], B = [[Nr_j, Lr_j], [Ng_j, Lg_j]]
        const cd a11 = comp[1][0], a12 = comp[1][3], a21 = comp[1][1], a22 = comp[1][4];
        const cd det = a11 * a22 - a12 * a21;
        const cd b11 = comp[0][0], b12 = comp[0][3], b21 = comp[0][1], b22 = comp[0][4];
        o[0] = -(a22 * b11 - a12 * b21) / det;
        o[1] = -(a22 * b12 - a12 * b22) / det;
        o[2] = -(-a21 * b11 + a11 * b21) / det;
        o[3] = -(-a21 * b12 + a11 * b22) / det;
        o[4] = -comp[0][2] / comp[1][2];
    }
}

// small dense complex solve (Gaussian elimination with partial pivoting), A n x n row-major, B n x k
bool solve_small(std::vector<cd> A, int n, std::vector<cd>& B, int k) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(A[(size_t)r * n + c]) > std::abs(A[(size_t)piv * n + c])) piv = r;
        if (std::abs(A[(size_t)piv * n + c]) == 0.0) return false;
        if (piv != c) {
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)c * n + j], A[(size_t)piv * n + j]);
            for (int j = 0; j < k; ++j) std::swap(B[(size_t)c * k + j], B[(size_t)piv * k + j]);
        }
        for (int r = c + 1; r < n; ++r) {
            const cd f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
            for (int j = c; j < n; ++j) A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
            for (int j = 0; j < k; ++j) B[(size_t)r * k + j] -= f * B[(size_t)c * k + j];
        }
    }
    for (int c = n - 1; c >= 0; --c)
        for (int j = 0; j < k; ++j) {
            cd v = B[(size_t)c * k + j];
            for (int r = c + 1; r < n; ++r) v -= A[(size_t)c * n + r] * B[(size_t)r * k + j];
            B[(size_t)c * k + j] = v / A[(size_t)c * n + c];
        }
    return true;
}

struct Layer {
    double lam, mu, kp, ks;
};

// k_z = sqrt(k^2 - lam^2) on the branch Im k_z >= 0 (k_z >= 0 when real): the principal root, with
// the sign fixed explicitly because a real lam gives the argument a signed zero imaginary part
cd kz_of(double k, cd lam) {
    cd z = std::sqrt(cd(k * k) - lam * lam);
    if (z.imag() < 0.0 || (z.imag() == 0.0 && z.real() < 0.0)) z = -z;
    return z;
}

// plane wave basis at horizontal wavenumber lam (complex) and azimuth th in a layer: direction, SV, SH
void pw_basis(double k, cd lam, double th, bool up, cd e[3], cd v[3], cd h[3]) {
    const cd kz = kz_of(k, lam);
    const double c = cos(th), s = sin(th);
    e[0] = lam * c / k; e[1] = lam * s / k; e[2] = (up ? kz : -kz) / k;
    h[0] = -s; h[1] = c; h[2] = 0.0;
    cross3(h, e, v);
}

// traction sigma e_z of A e^{i kvec.x}: i [lam (k.A) e_z + mu (k A_z + A k_z)]
void traction(const cd kv[3], const cd A[3], double lam, double mu, cd t[3]) {
    const cd kA = dot3(kv, A), I(0, 1);
    for (int i = 0; i < 3; ++i) t[i] = I * (mu * (kv[i] * A[2] + A[i] * kv[2]));
    t[2] += I * lam * kA;
}

// displacement and traction columns of the three waves (P, SV, SH) of a layer, up or down
void wave_cols(const Layer& L, cd lam, double th, bool up, cd U[3][3], cd Tr[3][3]) {
    cd eP[3], vP[3], hP[3], eS[3], vS[3], hS[3];
    pw_basis(L.kp, lam, th, up, eP, vP, hP);
    pw_basis(L.ks, lam, th, up, eS, vS, hS);
    const cd* pol[3] = {eP, vS, hS};
    const cd* dir[3] = {eP, eS, eS};
    const double kk[3] = {L.kp, L.ks, L.ks};
    for (int w = 0; w < 3; ++w) {
        cd kv[3];
        for (int i = 0; i < 3; ++i) {
            kv[i] = kk[w] * dir[w][i];
            U[w][i] = pol[w][i];
        }
        traction(kv, pol[w], L.lam, L.mu, Tr[w]);
    }
}

// interface system at one node: unknowns (lower down P, SV, SH; upper up P, SV, SH), continuity of
// displacement and traction at z = 0; right-hand columns given as (displacement, traction) pairs
bool interface_solve(const Layer& lo, const Layer& up, cd lam, double th, std::vector<cd>& rhs, int k) {
    cd Ud[3][3], Td[3][3], Uu[3][3], Tu[3][3];
    wave_cols(lo, lam, th, false, Ud, Td);
    wave_cols(up, lam, th, true, Uu, Tu);
    std::vector<cd> A(36);
    for (int w = 0; w < 3; ++w)
        for (int i = 0; i < 3; ++i) {
            A[(size_t)i * 6 + w] = Ud[w][i];
            A[(size_t)(3 + i) * 6 + w] = Td[w][i];
            A[(size_t)i * 6 + 3 + w] = -Uu[w][i];
            A[(size_t)(3 + i) * 6 + 3 + w] = -Tu[w][i];
        }
    return solve_small(A, 6, rhs, k);
}

// Regular coefficients (a, b, c) of e^{i k_s x.d} pol (pol . d = 0) or e^{i k_p x.d} d (Sec. 6.3):
//   a_nm = 4 pi i^n / (n(n+1)) Grad Y_n^{-m}(d) . pol,  b_nm = -4 pi i^n / (n(n+1)) (d x Grad Y_n^{-m}(d)) . pol,
//   c_nm = -4 pi i^{n+1} / kp Y_n^{-m}(d) (d . pol)
void plane_coeffs(int p, double kp, const cd d[3], const cd pol[3], cd* out) {
    std::vector<cd> Y, G;
    ylm_c(p, d, Y);
    grad_ylm_c(p, d, G);
    const int nmn = p * (p + 2);
    const cd I(0, 1);
    const cd dp = dot3(d, pol);
    for (int n = 0; n <= p; ++n) {
        const cd in = std::pow(I, n);
        for (int m = -n; m <= n; ++m) {
            const int k = idx(n, -m);
            const cd* g = &G[(size_t)k * 3];
            out[2 * nmn + idx(n, m)] = -4.0 * M_PI * in * I / kp * Y[k] * dp;
            if (n == 0) continue;
            cd dxg[3];
            cross3(d, g, dxg);
            const double f = 4.0 * M_PI / (n * (n + 1.0));
            out[idx(n, m) - 1] = f * in * dot3(g, pol);
            out[nmn + idx(n, m) - 1] = -f * in * dot3(dxg, pol);
        }
    }
}

// Gaunt table: Gt[k'][t][nu mu] = 4 pi i^{nu - n' + q} 2 pi N N N int P P P dt, q = |n' - nu| + 2t (exact
// Gauss-Legendre in cos(theta); the phi integral is 2 pi)
std::vector<cd> build_gaunt(int p) {
    const int K2 = (p + 2) * (p + 2), nl = (p + 1) * (p + 1);
    std::vector<cd> Gt((size_t)K2 * (p + 1) * nl, cd(0));
    {
        const int NG = 2 * p + 6;
        std::vector<double> gx(NG), gw(NG);
        // Gauss-Legendre nodes by Newton on P_NG
        for (int i = 0; i < NG; ++i) {
            double x = cos(M_PI * (i + 0.75) / (NG + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1, p1 = x;
                for (int k = 2; k <= NG; ++k) { const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
                const double dp = NG * (x * p1 - p0) / (x * x - 1);
                const double dx = p1 / dp;
                x -= dx;
                if (fabs(dx) < 1e-16) break;
            }
            double p0 = 1, p1 = x;
            for (int k = 2; k <= NG; ++k) { const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            const double dp = NG * (x * p1 - p0) / (x * x - 1);
            gx[i] = x;
            gw[i] = 2.0 / ((1 - x * x) * dp * dp);
        }
        const int PQ = 2 * p + 2;
        // Ferrers P_n^k(t) = (1 - t^2)^{k/2} Q_n^k(t) at the nodes, n <= PQ
        std::vector<double> F((size_t)NG * (PQ + 1) * (PQ + 1), 0.0);
        for (int i = 0; i < NG; ++i) {
            const std::vector<cd> Q = qtab(PQ, cd(gx[i]));
            const double s = sqrt(1 - gx[i] * gx[i]);
            for (int n = 0; n <= PQ; ++n)
                for (int k = 0; k <= n; ++k)
                    F[((size_t)i * (PQ + 1) + n) * (PQ + 1) + k] = Q[(size_t)n * (PQ + 2) + k].real() * pow(s, k);
        }
        const cd I(0, 1);
        for (int n1 = 0; n1 <= p + 1; ++n1)
            for (int m1 = -n1; m1 <= n1; ++m1)
                for (int nu = 0; nu <= p; ++nu)
                    for (int mu = -nu; mu <= nu; ++mu)
                        for (int t = 0; t <= std::min(n1, nu); ++t) {
                            const int q = std::abs(n1 - nu) + 2 * t, dm = m1 - mu;
                            if (std::abs(dm) > q) continue;
                            double s = 0;
                            for (int i = 0; i < NG; ++i)
                                s += gw[i] * F[((size_t)i * (PQ + 1) + n1) * (PQ + 1) + std::abs(m1)] *
                                     F[((size_t)i * (PQ + 1) + nu) * (PQ + 1) + std::abs(mu)] *
                                     F[((size_t)i * (PQ + 1) + q) * (PQ + 1) + std::abs(dm)];
                            const double G = 2.0 * M_PI * ynorm(n1, std::abs(m1)) * ynorm(nu, std::abs(mu)) * ynorm(q, std::abs(dm)) * s;
                            Gt[((size_t)idx(n1, m1) * (p + 1) + t) * nl + idx(nu, mu)] = 4.0 * M_PI * std::pow(I, nu - n1 + q) * G;
                        }
    }
    return Gt;
}

// Sparse Cartesian maps (<= 9 terms per row) by exact quadrature on the unit sphere (real directions):
// forward, the outgoing Cartesian expansions W[c][(n', m')] of the shear coefficients; back, a and b from
// the regular Cartesian expansions.  Returns false if a row needs more than 9 terms.
bool build_cart_maps(int p, std::vector<int>& midx, std::vector<cd>& mcoef, std::vector<int>& uidx,
                     std::vector<cd>& ucoef) {
    const int K2 = (p + 2) * (p + 2), nl = (p + 1) * (p + 1), nmn = p * (p + 2);
    midx.assign((size_t)3 * K2 * 9, -1);
    uidx.assign((size_t)2 * nmn * 9, -1);
    mcoef.assign((size_t)3 * K2 * 9, cd(0));
    ucoef.assign((size_t)2 * nmn * 9, cd(0));
    bool map_overflow = false;
    {
        const int NT = p + 5, NP = 2 * p + 10, P1 = p + 1;
        std::vector<double> tx(NT), tw(NT);
        for (int i = 0; i < NT; ++i) {
            double x = cos(M_PI * (i + 0.75) / (NT + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1, p1 = x;
                for (int k = 2; k <= NT; ++k) { const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
                const double dp = NT * (x * p1 - p0) / (x * x - 1);
                const double dx = p1 / dp;
                x -= dx;
                if (fabs(dx) < 1e-16) break;
            }
            double p0 = 1, p1 = x;
            for (int k = 2; k <= NT; ++k) { const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            const double dp = NT * (x * p1 - p0) / (x * x - 1);
            tx[i] = x;
            tw[i] = 2.0 / ((1 - x * x) * dp * dp);
        }
        const int NY = (P1 + 1) * (P1 + 1);
        // C[kind][c][(n, m)][(n2, m2)] accumulated densely over (n, m) <= P1 and (n2, m2) <= P1
        std::vector<cd> Cm((size_t)3 * NY * NY, cd(0)), Cp((size_t)3 * NY * NY, cd(0)), Cx((size_t)3 * NY * NY, cd(0));
        std::vector<cd> Y, G;
        for (int i = 0; i < NT; ++i)
            for (int j = 0; j < NP; ++j) {
                const double ph = 2.0 * M_PI * j / NP, st = sqrt(1 - tx[i] * tx[i]);
                const cd d[3] = {st * cos(ph), st * sin(ph), tx[i]};
                const double wq = tw[i] * 2.0 * M_PI / NP;
                ylm_c(P1, d, Y);
                grad_ylm_c(P1, d, G);
                for (int k = 0; k < NY; ++k) {
                    const int n = (int)sqrt((double)k + 0.5);
                    const cd* gk = &G[(size_t)k * 3];
                    cd X[3];
                    cross3(gk, d, X);
                    for (int c = 0; c < 3; ++c) {
                        const cd vm = (double)n * Y[k] * d[c] + gk[c];
                        const cd vp = (double)(n + 1) * Y[k] * d[c] - gk[c];
                        for (int k2 = 0; k2 < NY; ++k2) {
                            const cd yc = std::conj(Y[k2]) * wq;
                            Cm[((size_t)c * NY + k) * NY + k2] += vm * yc;
                            Cp[((size_t)c * NY + k) * NY + k2] += vp * yc;
                            Cx[((size_t)c * NY + k) * NY + k2] += X[c] * yc;
                        }
                    }
                }
            }
        const cd I(0, 1);
        auto C = [&](std::vector<cd>& A, int c, int k, int k2) -> cd { return A[((size_t)c * NY + k) * NY + k2]; };
        // forward: W[c][(n', m')] from alpha_{n'+1, m} (V-), alpha_{n'-1, m} (V+), beta_{n', m} (X)
        for (int c = 0; c < 3; ++c)
            for (int n1 = 0; n1 <= p + 1; ++n1)
                for (int m1 = -n1; m1 <= n1; ++m1) {
                    const int row = c * K2 + idx(n1, m1);
                    int cnt = 0;
                    auto add = [&](int src, cd coef) {
                        if (std::abs(coef) < 1e-13) return;
                        if (cnt >= 9) { map_overflow = true; return; }
                        midx[(size_t)row * 9 + cnt] = src;
                        mcoef[(size_t)row * 9 + cnt] = coef;
                        ++cnt;
                    };
                    const int n = n1 + 1;
                    if (n <= p)
                        for (int m = -n; m <= n; ++m)
                            add(idx(n, m) - 1, (double)(n + 1) / (I * (2.0 * n + 1)) * C(Cm, c, idx(n, m), idx(n1, m1)));
                    const int nb = n1 - 1;
                    if (nb >= 1 && nb <= p)
                        for (int m = -nb; m <= nb; ++m)
                            add(idx(nb, m) - 1, (double)nb / (I * (2.0 * nb + 1)) * C(Cp, c, idx(nb, m), idx(n1, m1)));
                    if (n1 >= 1 && n1 <= p)
                        for (int m = -n1; m <= n1; ++m) add(nmn + idx(n1, m) - 1, C(Cx, c, idx(n1, m), idx(n1, m1)));
                }
        // back: a_Jm = i/(J(J+1)) sum conj(C-(J, m -> J-1, mu)) R_c(J-1, mu); b_Jm = 1/(J(J+1)) sum conj(CX) R_c(J, mu)
        for (int J = 1; J <= p; ++J)
            for (int m = -J; m <= J; ++m)
                for (int which = 0; which < 2; ++which) {
                    const int row = which * nmn + idx(J, m) - 1;
                    int cnt = 0;
                    const int nd = which == 0 ? J - 1 : J;
                    for (int c = 0; c < 3; ++c)
                        for (int mu = -nd; mu <= nd; ++mu) {
                            const cd cc = which == 0 ? std::conj(C(Cm, c, idx(J, m), idx(nd, mu))) * I / (J * (J + 1.0))
                                                     : std::conj(C(Cx, c, idx(J, m), idx(nd, mu))) / (J * (J + 1.0));
                            if (std::abs(cc) < 1e-13) continue;
                            if (cnt >= 9) { map_overflow = true; continue; }
                            uidx[(size_t)row * 9 + cnt] = c * nl + idx(nd, mu);
                            ucoef[(size_t)row * 9 + cnt] = cc;
                            ++cnt;
                        }
                }
    }
    return !map_overflow;
}

// ------------------------------------------------------------------ device kernels (T = double or float)
__constant__ int c_deg[(P3MAX + 2) * (P3MAX + 2)];
__constant__ int c_ord[(P3MAX + 2) * (P3MAX + 2)];
__constant__ double c_ynorm[(2 * P3MAX + 2) * (2 * P3MAX + 2)];     // N_qk, k >= 0, at [q * (2P+2) + k]

__device__ __forceinline__ int didx(int n, int m) { return n * n + n + m; }
__device__ __forceinline__ void sc(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void sc(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ float ex(float x) { return expf(x); }

// y = (identity ? x : 0) - S a  (identity) or S a (apply only), per sphere and order
template <typename T>
__global__ void k3_sapply(const typename CT<T>::c* __restrict__ x, const typename CT<T>::c* __restrict__ a,
                          typename CT<T>::c* __restrict__ y, const typename CT<T>::c* __restrict__ Sd, int M, int p,
                          int nrhs, int identity, int apply_s) {
    typedef typename CT<T>::c C;
    const int nmn = p * (p + 2), nl = (p + 1) * (p + 1), T3 = 2 * nmn + nl;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * T3 * nrhs) return;
    const int r = (int)(i % nrhs);
    const long long mk = i / nrhs;
    const int m = (int)(mk / T3), k = (int)(mk % T3);
    const C* A = a + (size_t)m * T3 * nrhs;
    C v;
    if (!apply_s) {
        v = A[(size_t)k * nrhs + r];
    } else {
        int blk, kk;
        if (k < nmn) { blk = 0; kk = k + 1; }
        else if (k < 2 * nmn) { blk = 1; kk = k - nmn + 1; }
        else { blk = 2; kk = k - 2 * nmn; }
        const int n = (int)sqrtf((float)kk + 0.5f);
        const C* S = Sd + ((size_t)m * (p + 1) + n) * 5;
        if (blk == 2 && n == 0) {
            v = cmul(S[0], A[(size_t)k * nrhs + r]);
        } else if (blk == 1) {
            v = cmul(S[4], A[(size_t)k * nrhs + r]);
        } else {
            const C aa = A[(size_t)(kk - 1) * nrhs + r];                // alpha-block entry of (n, m)
            const C ac = A[(size_t)(2 * nmn + kk) * nrhs + r];         // gamma-block entry
            v = blk == 0 ? cadd(cmul(S[0], aa), cmul(S[1], ac)) : cadd(cmul(S[2], aa), cmul(S[3], ac));
        }
    }
    y[i] = identity ? csub(x[i], v) : v;
}

// Cartesian outgoing expansions of each sphere's shear field: W[l][c][k'][r] = sum of <= 9 terms
template <typename T>
__global__ void k3_cart(const typename CT<T>::c* __restrict__ x, typename CT<T>::c* __restrict__ W,
                        const int* __restrict__ midx, const typename CT<T>::c* __restrict__ mcoef, int M, int p,
                        int nrhs) {
    typedef typename CT<T>::c C;
    const int nmn = p * (p + 2), nl = (p + 1) * (p + 1), T3 = 2 * nmn + nl, K2 = (p + 2) * (p + 2);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * 3 * K2 * nrhs) return;
    const int r = (int)(i % nrhs);
    const long long row = i / nrhs;
    const int l = (int)(row / (3 * K2)), ck = (int)(row % (3 * K2));
    C acc = mk((T)0, (T)0);
    for (int t = 0; t < 9; ++t) {
        const int s = midx[ck * 9 + t];
        if (s < 0) break;
        cfma(acc, mcoef[ck * 9 + t], x[((size_t)l * T3 + s) * nrhs + r]);
    }
    W[i] = acc;
}

// h_q(x), q = 0..Q, real x > 0: h_0 = -i e^{ix}/x, h_1 = -e^{ix}(x + i)/x^2, upward recurrence
template <typename T>
__device__ void sph_hankel_seq(int Q, T x, typename CT<T>::c* h) {
    T s, c;
    sc(x, &s, &c);
    h[0] = mk(s / x, -c / x);
    if (Q >= 1) h[1] = mk(-(c * x - s) / (x * x), -(s * x + c) / (x * x));
    for (int q = 1; q < Q; ++q) {
        const T f = (T)(2 * q + 1) / x;
        h[q + 1] = mk(f * h[q].x - h[q - 1].x, f * h[q].y - h[q - 1].y);
    }
}

// Translation of every other sphere's expansions into sphere m's regular ones (one CTA per target and
// right-hand-side chunk; thread (c, nu mu) for the three Cartesian shear components, thread (nu mu)
// for the compressional potential).  Gt[k'][t][nu mu] = 4 pi i^{nu - n' + q} G(n', m'; nu, mu; q),
// q = |n' - nu| + 2t.  Shared: the source's Cartesian expansions and potential for the chunk, and
// H_q^k = h_q(k |d|) Y_q^k(d^) for both wavenumbers.
template <typename T>
__global__ void __launch_bounds__(512) k3_translate(const typename CT<T>::c* __restrict__ W,
                                                    const typename CT<T>::c* __restrict__ x, const T* __restrict__ cen,
                                                    const typename CT<T>::c* __restrict__ Gt,
                                                    typename CT<T>::c* __restrict__ Rr, typename CT<T>::c* __restrict__ Cr,
                                                    T kp, T ks, int M, int p, int nrhs) {
    typedef typename CT<T>::c C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* sm = reinterpret_cast<C*>(sm_raw);
    const int nmn = p * (p + 2), nl = (p + 1) * (p + 1), T3 = 2 * nmn + nl, K2 = (p + 2) * (p + 2);
    const int P2 = 2 * p + 1, QN = (P2 + 1) * (P2 + 1), TT = p + 1;
    C* Ws = sm;                           // [3][K2][RC]
    C* Gs = Ws + 3 * K2 * RC;             // [nl][RC]
    C* Hs = Gs + nl * RC;                 // [QN]
    C* Hp = Hs + QN;                      // [QN]
    C* hs = Hp + QN;                      // [P2 + 1]
    C* hp = hs + P2 + 1;                  // [P2 + 1]
    __shared__ T dsh[4];
    const int m = blockIdx.x, r0 = blockIdx.y * RC;
    const int nr = min(RC, nrhs - r0);
    const int tid = threadIdx.x;
    const bool sth = tid < 3 * nl, pth = tid >= 3 * nl && tid < 4 * nl;
    const int comp = sth ? tid / nl : 0;
    const int vm = sth ? tid % nl : tid - 3 * nl;
    const int nu = (sth || pth) ? c_deg[vm] : 0, mu = (sth || pth) ? c_ord[vm] : 0;
    C acc[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) acc[r] = mk((T)0, (T)0);
    for (int l = 0; l < M; ++l) {
        if (l == m) continue;
        if (tid == 0) {
            const T dx = cen[3 * m] - cen[3 * l], dy = cen[3 * m + 1] - cen[3 * l + 1], dz = cen[3 * m + 2] - cen[3 * l + 2];
            const T dd = sqrt(dx * dx + dy * dy + dz * dz);
            dsh[0] = dx / dd; dsh[1] = dy / dd; dsh[2] = dz / dd; dsh[3] = dd;
            sph_hankel_seq<T>(P2, ks * dd, hs);
            sph_hankel_seq<T>(P2, kp * dd, hp);
        }
        for (int e = tid; e < 3 * K2 * RC; e += blockDim.x) {
            const int r = e % RC, ck = e / RC;
            Ws[e] = r < nr ? W[(((size_t)l * 3 * K2) + ck) * nrhs + r0 + r] : mk((T)0, (T)0);
        }
        for (int e = tid; e < nl * RC; e += blockDim.x) {
            const int r = e % RC, k = e / RC;
            Gs[e] = r < nr ? x[((size_t)l * T3 + 2 * nmn + k) * nrhs + r0 + r] : mk((T)0, (T)0);
        }
        __syncthreads();
        if (tid <= P2) {
            // Y_q^k(d^), k = tid >= 0, q = k..P2: N Q_q^k(t) w^k, w = d_x + i d_y; Y_q^{-k} = conj(Y_q^k)
            const int k = tid;
            const T t = dsh[2];
            C wk = mk((T)1, (T)0);
            const C w = mk(dsh[0], dsh[1]);
            for (int i = 0; i < k; ++i) wk = cmul(wk, w);
            T df = 1;
            for (int i = 1; i <= k; ++i) df *= (T)(2 * i - 1);
            T qm1 = 0, q0 = df;                 // Q_{k-1}^k = 0, Q_k^k
            for (int q = k; q <= P2; ++q) {
                const T y = (T)c_ynorm[q * (2 * P3MAX + 2) + k] * q0;
                const C Y = mk(y * wk.x, y * wk.y);
                const C Yc = cconj(Y);
                Hs[didx(q, k)] = cmul(hs[q], Y);
                Hp[didx(q, k)] = cmul(hp[q], Y);
                if (k > 0) {
                    Hs[didx(q, -k)] = cmul(hs[q], Yc);
                    Hp[didx(q, -k)] = cmul(hp[q], Yc);
                }
                const T qn = ((T)(2 * q + 1) * t * q0 - (T)(q + k) * qm1) / (T)(q - k + 1);
                qm1 = q0;
                q0 = qn;
            }
        }
        __syncthreads();
        if (sth || pth) {
            const C* Hq = sth ? Hs : Hp;
            const int nk = sth ? K2 : nl;
            const C* src = sth ? Ws + (size_t)comp * K2 * RC : Gs;
            for (int kk = 0; kk < nk; ++kk) {
                const int n1 = c_deg[kk], m1 = c_ord[kk];
                const int dm = m1 - mu;
                C A = mk((T)0, (T)0);
                const int tmax = min(n1, nu);
                for (int t = 0; t <= tmax; ++t) {
                    const int q = abs(n1 - nu) + 2 * t;
                    if (abs(dm) > q) continue;
                    cfma(A, Gt[((size_t)kk * TT + t) * nl + vm], Hq[didx(q, dm)]);
                }
                const C* s = src + (size_t)kk * RC;
#pragma unroll
                for (int r = 0; r < RC; ++r) cfma(acc[r], A, s[r]);
            }
        }
        __syncthreads();
    }
    if (sth) {
#pragma unroll
        for (int r = 0; r < RC; ++r)
            if (r < nr) Rr[(((size_t)m * 3 + comp) * nl + vm) * nrhs + r0 + r] = acc[r];
    } else if (pth) {
#pragma unroll
        for (int r = 0; r < RC; ++r)
            if (r < nr) Cr[((size_t)m * nl + vm) * nrhs + r0 + r] = acc[r];
    }
}

// a (+)= the translated coefficients: a_Jm and b_Jm from the regular Cartesian shear expansions (<= 9
// terms each), c from the translated potential
template <typename T>
__global__ void k3_uncart(const typename CT<T>::c* __restrict__ Rr, const typename CT<T>::c* __restrict__ Cr,
                          typename CT<T>::c* __restrict__ a, const int* __restrict__ uidx,
                          const typename CT<T>::c* __restrict__ ucoef, int M, int p, int nrhs, int accumulate) {
    typedef typename CT<T>::c C;
    const int nmn = p * (p + 2), nl = (p + 1) * (p + 1), T3 = 2 * nmn + nl;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * T3 * nrhs) return;
    const int r = (int)(i % nrhs);
    const long long mk_ = i / nrhs;
    const int m = (int)(mk_ / T3), k = (int)(mk_ % T3);
    C v = mk((T)0, (T)0);
    if (k < 2 * nmn) {
        for (int t = 0; t < 9; ++t) {
            const int s = uidx[k * 9 + t];                   // (c, nu mu) as c * nl + nu mu
            if (s < 0) break;
            cfma(v, ucoef[k * 9 + t], Rr[((size_t)m * 3 * nl + s) * nrhs + r]);
        }
    } else {
        v = Cr[((size_t)m * nl + (k - 2 * nmn)) * nrhs + r];
    }
    a[i] = accumulate ? cadd(a[i], v) : v;
}

// Block B: U[q][w][r] = sum_l e^{-i (k_x x_l + k_y y_l) - i k_z^w z_l} sum_k Tw[q][k] x_l[k][r],
// w = P (gamma block), SV, SH (alpha then beta).  One CTA per node; thread (w, r, l-slice).
constexpr int M2S_LS = 5;
template <typename T>
__global__ void __launch_bounds__(3 * RC * M2S_LS) k3_m2s(const typename CT<T>::c* __restrict__ x,
                                                          const typename CT<T>::c* __restrict__ TP,
                                                          const typename CT<T>::c* __restrict__ TV,
                                                          const typename CT<T>::c* __restrict__ TH,
                                                          const typename CT<T>::c* __restrict__ node,
                                                          const T* __restrict__ cen, typename CT<T>::c* __restrict__ U,
                                                          int M, int p, int nrhs, int r0) {
    typedef typename CT<T>::c C;
    __shared__ C red[3 * RC * M2S_LS];
    const int nmn = p * (p + 2), nl = (p + 1) * (p + 1), T3 = 2 * nmn + nl;
    const int q = blockIdx.x, tid = threadIdx.x;
    const int w = tid / (RC * M2S_LS), rem = tid % (RC * M2S_LS), r = rem % RC, ls = rem / RC;
    // node: (k_x, k_y, k_z^P, k_z^S)
    const C kx = node[(size_t)q * 4], ky = node[(size_t)q * 4 + 1];
    const C kz = node[(size_t)q * 4 + (w == 0 ? 2 : 3)];
    const C* Tw = w == 0 ? TP + (size_t)q * nl : (w == 1 ? TV : TH) + (size_t)q * 2 * nmn;
    const int off = w == 0 ? 2 * nmn : 0, len = w == 0 ? nl : 2 * nmn;
    C acc = mk((T)0, (T)0);
    if (r0 + r < nrhs) {
        for (int l = ls; l < M; l += M2S_LS) {
            const T X = cen[3 * l], Y = cen[3 * l + 1], Z = cen[3 * l + 2];
            // phase = exp(-i (kx X + ky Y + kz Z))
            const T re = kx.x * X + ky.x * Y + kz.x * Z, im = kx.y * X + ky.y * Y + kz.y * Z;
            T s, c;
            sc(-re, &s, &c);
            const T mag = ex(im);
            const C ph = mk(mag * c, mag * s);
            const C* xl = x + ((size_t)l * T3 + off) * nrhs + r0 + r;
            C d = mk((T)0, (T)0);
            for (int k = 0; k < len; ++k) cfma(d, Tw[k], xl[(size_t)k * nrhs]);
            cfma(acc, ph, d);
        }
    }
    red[tid] = acc;
    __syncthreads();
    if (ls == 0 && r0 + r < nrhs) {
        C s = acc;
        for (int j = 1; j < M2S_LS; ++j) s = cadd(s, red[tid + j * RC]);
        U[((size_t)q * 3 + w) * nrhs + r0 + r] = s;
    }
}

// D[q][w][r] = sum_v RW[q][w][v] U[q][v][r]
template <typename T>
__global__ void k3_reflect(const typename CT<T>::c* __restrict__ U, const typename CT<T>::c* __restrict__ RW,
                           typename CT<T>::c* __restrict__ D, int NS, int nrhs) {
    typedef typename CT<T>::c C;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)NS * 3 * nrhs) return;
    const int r = (int)(i % nrhs);
    const long long qw = i / nrhs;
    const int q = (int)(qw / 3), w = (int)(qw % 3);
    C v = mk((T)0, (T)0);
    for (int u = 0; u < 3; ++u) cfma(v, RW[(size_t)q * 9 + w * 3 + u], U[((size_t)q * 3 + u) * nrhs + r]);
    D[i] = v;
}

// Block C: a[m][k][r] += sum_q [e^{i(k_x x_m + k_y y_m) - i k_z^P z_m} CP[q][k] D[q][P][r]
//                               + e^{... - i k_z^S z_m} (CV[q][k] D[q][SV][r] + CH[q][k] D[q][SH][r])]
// One CTA per sphere, right-hand-side chunk and slice of 288 coefficients; nodes staged in chunks.
constexpr int S2L_QC = 32;
constexpr int S2L_KSPAN = 288;            // coefficients per CTA (grid z covers T in slices)
template <typename T>
__global__ void __launch_bounds__(256) k3_s2l(const typename CT<T>::c* __restrict__ D, const typename CT<T>::c* __restrict__ CP,
                                              const typename CT<T>::c* __restrict__ CV,
                                              const typename CT<T>::c* __restrict__ CH,
                                              const typename CT<T>::c* __restrict__ node, const T* __restrict__ cen,
                                              typename CT<T>::c* __restrict__ a, int NS, int p, int nrhs) {
    typedef typename CT<T>::c C;
    __shared__ C Ds[S2L_QC][3][RC];
    __shared__ C ph[S2L_QC][2];
    const int nmn = p * (p + 2), nl = (p + 1) * (p + 1), T3 = 2 * nmn + nl;
    const int m = blockIdx.x, r0 = blockIdx.y * RC, tid = threadIdx.x;
    const int r = tid % RC, kg = tid / RC + S2L_KSPAN * blockIdx.z;   // 16 groups of k per z-slice
    constexpr int KPT = S2L_KSPAN / 16;                               // k values per thread
    C acc[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) acc[j] = mk((T)0, (T)0);
    const T X = cen[3 * m], Y = cen[3 * m + 1], Z = cen[3 * m + 2];
    for (int q0 = 0; q0 < NS; q0 += S2L_QC) {
        const int nq = min(S2L_QC, NS - q0);
        for (int e = tid; e < S2L_QC * 3 * RC; e += blockDim.x) {
            const int rr = e % RC, w = (e / RC) % 3, qq = e / (3 * RC);
            Ds[qq][w][rr] = (qq < nq && r0 + rr < nrhs) ? D[((size_t)(q0 + qq) * 3 + w) * nrhs + r0 + rr] : mk((T)0, (T)0);
        }
        if (tid < 2 * S2L_QC) {
            const int qq = tid / 2, wv = tid % 2;
            C v = mk((T)0, (T)0);
            if (qq < nq) {
                const size_t q = q0 + qq;
                const C kx = node[q * 4], ky = node[q * 4 + 1], kz = node[q * 4 + 2 + wv];
                // exp(i (kx X + ky Y - kz Z))
                const T re = kx.x * X + ky.x * Y - kz.x * Z, im = kx.y * X + ky.y * Y - kz.y * Z;
                T s, c;
                sc(re, &s, &c);
                const T mag = ex(-im);
                v = mk(mag * c, mag * s);
            }
            ph[qq][wv] = v;
        }
        __syncthreads();
        for (int qq = 0; qq < nq; ++qq) {
            const size_t q = q0 + qq;
            const C dp = cmul(ph[qq][0], Ds[qq][0][r]);
            const C dv = cmul(ph[qq][1], Ds[qq][1][r]);
            const C dh = cmul(ph[qq][1], Ds[qq][2][r]);
#pragma unroll
            for (int j = 0; j < KPT; ++j) {
                const int k = kg + 16 * j;
                if (k < T3 && k < S2L_KSPAN * (blockIdx.z + 1)) {
                    cfma(acc[j], CP[q * T3 + k], dp);
                    cfma(acc[j], CV[q * T3 + k], dv);
                    cfma(acc[j], CH[q * T3 + k], dh);
                }
            }
        }
        __syncthreads();
    }
    if (r0 + r < nrhs)
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const int k = kg + 16 * j;
            if (k < T3 && k < S2L_KSPAN * (blockIdx.z + 1)) {
                C* o = a + ((size_t)m * T3 + k) * nrhs + r0 + r;
                *o = cadd(*o, acc[j]);
            }
        }
}

// FP64 <-> FP32 blocks and y = b - y (FP64), column squared norms
__global__ void k3_to_f32(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void k3_add_f32(double2* __restrict__ x, const float2* __restrict__ d, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) x[i] = make_double2(x[i].x + (double)d[i].x, x[i].y + (double)d[i].y);
}
__global__ void k3_from_f32(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_double2((double)a[i].x, (double)a[i].y);
}
__global__ void k3_residual(const double2* __restrict__ b, double2* __restrict__ y, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = csub(b[i], y[i]);
}
__global__ void k3_colnorm2(const double2* __restrict__ v, double* __restrict__ out, long long rows, int nrhs) {
    __shared__ double part[256];
    const int r = blockIdx.y;
    double s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows; i += (long long)gridDim.x * blockDim.x)
        s += cabs2(v[i * nrhs + r]);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&out[r], part[0]);
}

}  // namespace

// ------------------------------------------------------------------ handle
// device tables of one precision
template <typename T>
struct Tab3 {
    typedef typename CT<T>::c C;
    T* cen = nullptr;                       // [M][3]
    C* Sd = nullptr;                        // [M][p+1][5]
    C* Gt = nullptr;                        // [K2][p+1][nl]
    C* mcoef = nullptr;                     // [3 K2][9]
    C* ucoef = nullptr;                     // [2 nmn][9]
    C *TP = nullptr, *TV = nullptr, *TH = nullptr;     // [NS][nl], [NS][2 nmn] x 2
    C *CP = nullptr, *CV = nullptr, *CH = nullptr;     // [NS][T] x 3
    C* node = nullptr;                      // [NS][4]: k_x, k_y, k_z^P, k_z^S (lower layer)
    C* RW = nullptr;                        // [NS][3][3] reflection times weight
    void release() {
        cudaFree(cen); cudaFree(Sd); cudaFree(Gt); cudaFree(mcoef); cudaFree(ucoef); cudaFree(TP); cudaFree(TV);
        cudaFree(TH); cudaFree(CP); cudaFree(CV); cudaFree(CH); cudaFree(node); cudaFree(RW);
        *this = Tab3{};
    }
};

struct ms3_handle {
    int M = 0, p = 0, T = 0, NS = 0, K2 = 0, nl = 0, nmn = 0;
    double omega = 0;
    Layer lo{}, up{};
    ms3_options opt{};
    std::vector<double> h_cen, h_rad;
    std::vector<int> h_bc;
    ms_handle* herr = nullptr;              // status plumbing shared with the 2D solver's Krylov code
    int* midx = nullptr;                    // [3 K2][9]
    int* uidx = nullptr;                    // [2 nmn][9]
    Tab3<double> t64;
    Tab3<float> t32;
    // workspace (sized in complex doubles, reused for FP32; grown to the largest nrhs seen)
    int ws_nrhs = 0;
    void *W = nullptr, *Rr = nullptr, *Cr = nullptr, *U = nullptr, *Dd = nullptr, *wa = nullptr, *wx = nullptr,
         *wy = nullptr;
    template <typename T> Tab3<T>& tab();
};
template <> Tab3<double>& ms3_handle::tab<double>() { return t64; }
template <> Tab3<float>& ms3_handle::tab<float>() { return t32; }

namespace {

void free_ws(ms3_handle* h) {
    cudaFree(h->W); cudaFree(h->Rr); cudaFree(h->Cr); cudaFree(h->U); cudaFree(h->Dd); cudaFree(h->wa); cudaFree(h->wx);
    cudaFree(h->wy);
    h->W = h->Rr = h->Cr = h->U = h->Dd = h->wa = h->wx = h->wy = nullptr;
    h->ws_nrhs = 0;
}

void free_all(ms3_handle* h) {
    h->t64.release();
    h->t32.release();
    cudaFree(h->midx); cudaFree(h->uidx);
    h->midx = h->uidx = nullptr;
    free_ws(h);
}

template <typename X>
int upload(ms3_handle* h, X** dst, const std::vector<X>& v) {
    *dst = nullptr;
    if (v.empty()) return MS_OK;
    if (cudaMalloc((void**)dst, v.size() * sizeof(X)) != cudaSuccess) return MS_ERR_ALLOC;
    return ms_check(h->herr, cudaMemcpy(*dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice));
}

template <typename T>
std::vector<typename CT<T>::c> to_dev(const std::vector<cd>& v) {
    std::vector<typename CT<T>::c> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = to_c<T>(make_double2(v[i].real(), v[i].imag()));
    return o;
}

template <typename T>
int upload_tables(ms3_handle* h, const std::vector<cd>& S, const std::vector<cd>& Gt, const std::vector<cd>& mcoef,
                  const std::vector<cd>& ucoef, const std::vector<cd>& TP, const std::vector<cd>& TV,
                  const std::vector<cd>& TH, const std::vector<cd>& CPv, const std::vector<cd>& CVv,
                  const std::vector<cd>& CHv, const std::vector<cd>& node, const std::vector<cd>& RW) {
    Tab3<T>& t = h->tab<T>();
    std::vector<T> cen(h->h_cen.begin(), h->h_cen.end());
    int rc;
    if ((rc = upload(h, &t.cen, cen)) || (rc = upload(h, &t.Sd, to_dev<T>(S))) || (rc = upload(h, &t.Gt, to_dev<T>(Gt))) ||
        (rc = upload(h, &t.mcoef, to_dev<T>(mcoef))) || (rc = upload(h, &t.ucoef, to_dev<T>(ucoef))) ||
        (rc = upload(h, &t.TP, to_dev<T>(TP))) || (rc = upload(h, &t.TV, to_dev<T>(TV))) ||
        (rc = upload(h, &t.TH, to_dev<T>(TH))) || (rc = upload(h, &t.CP, to_dev<T>(CPv))) ||
        (rc = upload(h, &t.CV, to_dev<T>(CVv))) || (rc = upload(h, &t.CH, to_dev<T>(CHv))) ||
        (rc = upload(h, &t.node, to_dev<T>(node))) || (rc = upload(h, &t.RW, to_dev<T>(RW))))
        return rc;
    return MS_OK;
}

int workspace(ms3_handle* h, int nrhs) {
    if (nrhs <= h->ws_nrhs) return MS_OK;
    free_ws(h);
    const size_t M = h->M, e = sizeof(double2);
    if (cudaMalloc(&h->W, M * 3 * h->K2 * nrhs * e) != cudaSuccess ||
        cudaMalloc(&h->Rr, M * 3 * h->nl * nrhs * e) != cudaSuccess ||
        cudaMalloc(&h->Cr, M * h->nl * nrhs * e) != cudaSuccess ||
        cudaMalloc(&h->U, (size_t)h->NS * 3 * nrhs * e) != cudaSuccess ||
        cudaMalloc(&h->Dd, (size_t)h->NS * 3 * nrhs * e) != cudaSuccess ||
        cudaMalloc(&h->wa, M * h->T * nrhs * e) != cudaSuccess || cudaMalloc(&h->wx, M * h->T * nrhs * e) != cudaSuccess ||
        cudaMalloc(&h->wy, M * h->T * nrhs * e) != cudaSuccess) {
        cudaGetLastError();
        free_ws(h);
        return MS_ERR_ALLOC;
    }
    h->ws_nrhs = nrhs;
    return MS_OK;
}

template <typename T>
size_t translate_smem(int p) {
    return (size_t)(3 * (p + 2) * (p + 2) * RC + (p + 1) * (p + 1) * RC + 2 * (2 * p + 2) * (2 * p + 2) + 2 * (2 * p + 2)) *
           sizeof(typename CT<T>::c);
}

// incoming coefficients of the selected parts into h->wa (precision T)
template <typename T>
int incoming(ms3_handle* h, const typename CT<T>::c* x, int nrhs, int parts, cudaStream_t st) {
    typedef typename CT<T>::c C;
    const Tab3<T>& t = h->tab<T>();
    const int M = h->M, p = h->p, T3 = h->T;
    C* wa = (C*)h->wa;
    const long long n = (long long)M * T3 * nrhs;
    int rc;
    if ((rc = ms_check(h->herr, cudaMemsetAsync(wa, 0, n * sizeof(C), st)))) return rc;
    if ((parts & MS3_PART_T) && M > 1) {
        k3_cart<T><<<nblk((long long)M * 3 * h->K2 * nrhs, 256), 256, 0, st>>>(x, (C*)h->W, h->midx, t.mcoef, M, p, nrhs);
        const int threads = ((4 * h->nl + 31) / 32) * 32;
        k3_translate<T><<<dim3(M, nblk(nrhs, RC)), threads, translate_smem<T>(p), st>>>(
            (const C*)h->W, x, t.cen, t.Gt, (C*)h->Rr, (C*)h->Cr, (T)h->lo.kp, (T)h->lo.ks, M, p, nrhs);
        k3_uncart<T><<<nblk(n, 256), 256, 0, st>>>((const C*)h->Rr, (const C*)h->Cr, wa, h->uidx, t.ucoef, M, p, nrhs, 1);
        if ((rc = ms_check(h->herr, cudaGetLastError()))) return rc;
    }
    if (parts & MS3_PART_R) {
        for (int r0 = 0; r0 < nrhs; r0 += RC)
            k3_m2s<T><<<h->NS, 3 * RC * M2S_LS, 0, st>>>(x, t.TP, t.TV, t.TH, t.node, t.cen, (C*)h->U, M, p, nrhs, r0);
        k3_reflect<T><<<nblk((long long)h->NS * 3 * nrhs, 256), 256, 0, st>>>((const C*)h->U, t.RW, (C*)h->Dd, h->NS, nrhs);
        k3_s2l<T><<<dim3(M, nblk(nrhs, RC), nblk(T3, S2L_KSPAN)), 256, 0, st>>>((const C*)h->Dd, t.CP, t.CV, t.CH, t.node,
                                                                                 t.cen, wa, h->NS, p, nrhs);
        if ((rc = ms_check(h->herr, cudaGetLastError()))) return rc;
    }
    return MS_OK;
}

// y = x - S (parts) x (with MS3_PART_S) or (parts) x, x and y of precision T, y != x, neither a workspace
template <typename T>
int op3(ms3_handle* h, const typename CT<T>::c* x, typename CT<T>::c* y, int nrhs, int parts, cudaStream_t st) {
    typedef typename CT<T>::c C;
    int rc;
    if ((rc = workspace(h, nrhs))) return rc;
    if ((rc = incoming<T>(h, x, nrhs, parts, st))) return rc;
    const long long n = (long long)h->M * h->T * nrhs;
    const bool s = (parts & MS3_PART_S) != 0;
    k3_sapply<T><<<nblk(n, 256), 256, 0, st>>>(x, (const C*)h->wa, y, h->tab<T>().Sd, h->M, h->p, nrhs, s ? 1 : 0,
                                                s ? 1 : 0);
    return ms_check(h->herr, cudaGetLastError());
}

int check_3d_args(const ms3_handle* h, const void* x, const void* y, int nrhs, int prec) {
    if (!h || !x || !y || nrhs < 1 || nrhs > 64 || x == y) return MS_ERR_ARG;
    if (prec != MS_PREC_FP64 && prec != MS_PREC_FP32) return MS_ERR_ARG;
    return MS_OK;
}

// max over columns of ||v_c|| / ||b_c|| (FP64 blocks of rows x nrhs), norms of b in bn
int rel_norms(ms3_handle* h, const double2* v, long long rows, int nrhs, std::vector<double>& out, cudaStream_t st) {
    double* d = nullptr;
    if (cudaMalloc(&d, nrhs * sizeof(double)) != cudaSuccess) return MS_ERR_ALLOC;
    int rc = ms_check(h->herr, cudaMemsetAsync(d, 0, nrhs * sizeof(double), st));
    if (!rc) {
        k3_colnorm2<<<dim3(std::min<long long>(1184, (rows + 255) / 256), nrhs), 256, 0, st>>>(v, d, rows, nrhs);
        rc = ms_check(h->herr, cudaGetLastError());
    }
    out.assign(nrhs, 0.0);
    if (!rc) rc = ms_check(h->herr, cudaMemcpyAsync(out.data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = ms_check(h->herr, cudaStreamSynchronize(st));
    cudaFree(d);
    for (double& x : out) x = sqrt(x);
    return rc;
}

}  // namespace

template <typename T>
int ms_block_solve(ms_handle* herr, long long N, int nrhs, int restart,
                   const std::function<int(const typename CT<T>::c*, typename CT<T>::c*)>& op,
                   const typename CT<T>::c* b, typename CT<T>::c* x, double tol, int max_iters, int& iters, int& matvecs,
                   std::vector<double>& relres, cudaStream_t st);

extern "C" void ms3_default_options(ms3_options* o) {
    if (!o) return;
    o->n_r = 128;
    o->n_theta = 64;
    o->n_panels = 4;
    o->t_max = 10.0;
    o->alpha = 1.0;
    o->beta = 1.0;
    o->restart = 60;
    o->max_iters = 1000;
}

constexpr long long MS3_MAX_NODES = 1LL << 18;   // Sommerfeld nodes n_r n_theta (the tables hold 3 T per node)

// The body of ms3_setup; `made` receives the handle as soon as it exists, so that the C entry point can
// release it if a host allocation throws.
static int ms3_setup_impl(const ms3_geometry* g, const ms_media* md, double omega, int32_t p, const ms3_options* o,
                   ms3_handle** out, ms3_handle*& made) {
    if (!out) return MS_ERR_ARG;
    *out = nullptr;
    if (!g || !md || !g->centres || !g->radius || !g->bc || g->M < 1 || !(omega > 0) || !std::isfinite(omega) ||
        p < 1 || p > P3MAX)
        return MS_ERR_ARG;
    if (!(md->mu_u > 0) || !(md->mu_l > 0) || !(md->lam_u + md->mu_u > 0) || !(md->lam_l + md->mu_l > 0)) return MS_ERR_ARG;
    ms3_options opt;
    ms3_default_options(&opt);
    if (o) opt = *o;
    if (opt.n_r < 1 || opt.n_theta < 1 || opt.n_panels < 1 || opt.n_r % opt.n_panels || !(opt.t_max > 0) ||
        !(opt.alpha >= 0) || !(opt.beta > 0) || !std::isfinite(opt.t_max) || !std::isfinite(opt.alpha) ||
        !std::isfinite(opt.beta) || opt.restart < 1 || opt.max_iters < 1 ||
        (long long)opt.n_r * opt.n_theta > MS3_MAX_NODES)
        return MS_ERR_ARG;
    const int M = g->M;
    for (int m = 0; m < M; ++m) {
        if (!(g->radius[m] > 0) || !std::isfinite(g->radius[m]) || (g->bc[m] != 0 && g->bc[m] != 1)) return MS_ERR_ARG;
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(g->centres[3 * m + i])) return MS_ERR_ARG;
        if (g->centres[3 * m + 2] + 1.1 * g->radius[m] > 0.0) return MS_ERR_NOT_BURIED;
    }
    for (int m = 0; m < M; ++m)
        for (int l = m + 1; l < M; ++l) {
            double d2 = 0;
            for (int i = 0; i < 3; ++i) d2 += (g->centres[3 * m + i] - g->centres[3 * l + i]) * (g->centres[3 * m + i] - g->centres[3 * l + i]);
            if (sqrt(d2) < 1.1 * (g->radius[m] + g->radius[l])) return MS_ERR_OVERLAP;
        }
    ms3_handle* h = new ms3_handle;
    made = h;
    h->herr = new ms_handle;
    h->M = M;
    h->p = p;
    h->nmn = p * (p + 2);
    h->nl = (p + 1) * (p + 1);
    h->T = 2 * h->nmn + h->nl;
    h->K2 = (p + 2) * (p + 2);
    h->omega = omega;
    h->opt = opt;
    h->lo = Layer{md->lam_l, md->mu_l, omega / sqrt(md->lam_l + 2 * md->mu_l), omega / sqrt(md->mu_l)};
    h->up = Layer{md->lam_u, md->mu_u, omega / sqrt(md->lam_u + 2 * md->mu_u), omega / sqrt(md->mu_u)};
    h->h_cen.assign(g->centres, g->centres + 3 * M);
    h->h_rad.assign(g->radius, g->radius + M);
    h->h_bc.assign(g->bc, g->bc + M);
    const int nmn = h->nmn, nl = h->nl, T = h->T, K2 = h->K2;
    int rc = MS_OK;
    auto fail = [&](int code) {
        free_all(h);
        delete h->herr;
        delete h;
        made = nullptr;
        return code;
    };
    // sphere matrices
    std::vector<cd> S((size_t)M * (p + 1) * 5);
    for (int m = 0; m < M; ++m)
        sphere_s(p, h->lo.kp, h->lo.ks, h->lo.lam, h->lo.mu, g->radius[m], g->bc[m], &S[(size_t)m * (p + 1) * 5]);
    // index tables in constant memory
    {
        std::vector<int> deg((P3MAX + 2) * (P3MAX + 2), 0), ord((P3MAX + 2) * (P3MAX + 2), 0);
        for (int n = 0; n <= P3MAX + 1; ++n)
            for (int m = -n; m <= n; ++m) { deg[idx(n, m)] = n; ord[idx(n, m)] = m; }
        std::vector<double> yn((2 * P3MAX + 2) * (2 * P3MAX + 2), 0.0);
        for (int q = 0; q <= 2 * P3MAX + 1; ++q)
            for (int k = 0; k <= q; ++k) yn[q * (2 * P3MAX + 2) + k] = ynorm(q, k);
        if (cudaMemcpyToSymbol(c_deg, deg.data(), deg.size() * sizeof(int)) != cudaSuccess ||
            cudaMemcpyToSymbol(c_ord, ord.data(), ord.size() * sizeof(int)) != cudaSuccess ||
            cudaMemcpyToSymbol(c_ynorm, yn.data(), yn.size() * sizeof(double)) != cudaSuccess)
            return fail(MS_ERR_CUDA);
    }
    const std::vector<cd> Gt = build_gaunt(p);
    std::vector<int> midx, uidx;
    std::vector<cd> mcoef, ucoef;
    if (!build_cart_maps(p, midx, mcoef, uidx, ucoef)) return fail(MS_ERR_UNSUPPORTED);
    // Sommerfeld nodes, blocks B and C, reflection
    const int NS = opt.n_r * opt.n_theta;
    h->NS = NS;
    std::vector<cd> TP((size_t)NS * nl), TV((size_t)NS * 2 * nmn), TH((size_t)NS * 2 * nmn);
    std::vector<cd> CPv((size_t)NS * T), CVv((size_t)NS * T), CHv((size_t)NS * T), node((size_t)NS * 4), RW((size_t)NS * 9);
    {
        const int per = opt.n_r / opt.n_panels;
        std::vector<double> gx(per), gw(per);
        for (int i = 0; i < per; ++i) {
            double x = cos(M_PI * (i + 0.75) / (per + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1, p1 = x;
                for (int k = 2; k <= per; ++k) { const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
                const double dp = per == 1 ? 1.0 : per * (x * p1 - p0) / (x * x - 1);
                const double dx = per == 1 ? x : p1 / dp;
                x -= dx;
                if (fabs(dx) < 1e-16) break;
            }
            double p0 = 1, p1 = x;
            for (int k = 2; k <= per; ++k) { const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            const double dp = per == 1 ? 1.0 : per * (x * p1 - p0) / (x * x - 1);
            gx[i] = x;
            gw[i] = 2.0 / ((1 - x * x) * dp * dp);
        }
        const cd I(0, 1);
        std::vector<cd> Y, G;
        for (int ir = 0; ir < opt.n_r; ++ir) {
            const int pan = ir / per, k = ir % per;
            const double a = pan * opt.t_max / opt.n_panels, b = (pan + 1) * opt.t_max / opt.n_panels;
            const double t = 0.5 * (b - a) * gx[k] + 0.5 * (a + b), wt = 0.5 * (b - a) * gw[k];
            const cd lam = cd(t, -opt.alpha * tanh(opt.beta * t));
            const cd dlam = cd(1.0, -opt.alpha * opt.beta / (cosh(opt.beta * t) * cosh(opt.beta * t)));
            for (int it = 0; it < opt.n_theta; ++it) {
                const size_t q = (size_t)ir * opt.n_theta + it;
                const double th = 2.0 * M_PI * it / opt.n_theta;
                const cd W = wt * lam * dlam * (2.0 * M_PI / opt.n_theta);
                const cd kzp = kz_of(h->lo.kp, lam), kzs = kz_of(h->lo.ks, lam);
                node[q * 4] = lam * cos(th);
                node[q * 4 + 1] = lam * sin(th);
                node[q * 4 + 2] = kzp;
                node[q * 4 + 3] = kzs;
                cd eP[3], vP[3], hP[3], eS[3], vS[3], hS[3];
                // block B (upgoing)
                pw_basis(h->lo.kp, lam, th, true, eP, vP, hP);
                pw_basis(h->lo.ks, lam, th, true, eS, vS, hS);
                ylm_c(p, eP, Y);
                for (int n = 0; n <= p; ++n)
                    for (int m = -n; m <= n; ++m)
                        TP[q * nl + idx(n, m)] = std::pow(-I, n - 1) * Y[idx(n, m)] / (2.0 * M_PI * kzp);
                grad_ylm_c(p, eS, G);
                for (int n = 1; n <= p; ++n)
                    for (int m = -n; m <= n; ++m) {
                        const cd f = std::pow(-I, n) / (2.0 * M_PI * h->lo.ks * kzs);
                        const cd* gk = &G[(size_t)idx(n, m) * 3];
                        cd gx3[3];
                        cross3(gk, eS, gx3);
                        const int k1 = idx(n, m) - 1;
                        TV[q * 2 * nmn + k1] = f * dot3(gk, vS);
                        TV[q * 2 * nmn + nmn + k1] = f * dot3(gx3, vS);
                        TH[q * 2 * nmn + k1] = f * dot3(gk, hS);
                        TH[q * 2 * nmn + nmn + k1] = f * dot3(gx3, hS);
                    }
                // block C (downgoing)
                pw_basis(h->lo.kp, lam, th, false, eP, vP, hP);
                pw_basis(h->lo.ks, lam, th, false, eS, vS, hS);
                plane_coeffs(p, h->lo.kp, eP, eP, &CPv[q * T]);
                plane_coeffs(p, h->lo.kp, eS, vS, &CVv[q * T]);
                plane_coeffs(p, h->lo.kp, eS, hS, &CHv[q * T]);
                // reflection: unit upgoing lower P, SV, SH -> downgoing lower amplitudes
                cd Ul[3][3], Tl[3][3];
                wave_cols(h->lo, lam, th, true, Ul, Tl);
                std::vector<cd> rhs(18);
                for (int w = 0; w < 3; ++w)
                    for (int i = 0; i < 3; ++i) {
                        rhs[(size_t)i * 3 + w] = -Ul[w][i];
                        rhs[(size_t)(3 + i) * 3 + w] = -Tl[w][i];
                    }
                if (!interface_solve(h->lo, h->up, lam, th, rhs, 3)) return fail(MS_ERR_ARG);
                for (int i = 0; i < 3; ++i)
                    for (int w = 0; w < 3; ++w) RW[q * 9 + i * 3 + w] = W * rhs[(size_t)i * 3 + w];
            }
        }
    }
    if ((rc = upload(h, &h->midx, midx)) || (rc = upload(h, &h->uidx, uidx)) ||
        (rc = upload_tables<double>(h, S, Gt, mcoef, ucoef, TP, TV, TH, CPv, CVv, CHv, node, RW)) ||
        (rc = upload_tables<float>(h, S, Gt, mcoef, ucoef, TP, TV, TH, CPv, CVv, CHv, node, RW)))
        return fail(rc);
    if (cudaFuncSetAttribute(k3_translate<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)translate_smem<double>(p)) != cudaSuccess ||
        cudaFuncSetAttribute(k3_translate<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)translate_smem<float>(p)) != cudaSuccess)
        return fail(MS_ERR_CUDA);
    *out = h;
    return MS_OK;
}

extern "C" int ms3_setup(const ms3_geometry* g, const ms_media* md, double omega, int32_t p, const ms3_options* o,
                         ms3_handle** out) {
    ms3_handle* made = nullptr;
    try {
        return ms3_setup_impl(g, md, omega, p, o, out, made);
    } catch (const std::bad_alloc&) {
        if (made) {
            free_all(made);
            delete made->herr;
            delete made;
        }
        if (out) *out = nullptr;
        return MS_ERR_ALLOC;
    }
}

extern "C" int ms3_operator(ms3_handle* h, const void* x, void* y, int32_t nrhs, int32_t parts, int32_t prec,
                            void* stream) {
    if (int rc = check_3d_args(h, x, y, nrhs, prec)) return rc;
    if (parts < 0 || parts > 7) return MS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == MS_PREC_FP64) return op3<double>(h, (const double2*)x, (double2*)y, nrhs, parts, st);
    // FP32 operator on FP64 blocks: staged through the FP32 workspace
    int rc;
    if ((rc = workspace(h, nrhs))) return rc;
    const long long n = (long long)h->M * h->T * nrhs;
    k3_to_f32<<<nblk(n, 256), 256, 0, st>>>((const double2*)x, (float2*)h->wx, n);
    if ((rc = op3<float>(h, (const float2*)h->wx, (float2*)h->wy, nrhs, parts, st))) return rc;
    k3_from_f32<<<nblk(n, 256), 256, 0, st>>>((const float2*)h->wy, (double2*)y, n);
    return ms_check(h->herr, cudaGetLastError());
}

extern "C" int ms3_apply(ms3_handle* h, const void* x, void* y, int32_t nrhs, int32_t prec, void* stream) {
    return ms3_operator(h, x, y, nrhs, MS3_PART_T | MS3_PART_R | MS3_PART_S, prec, stream);
}

extern "C" int ms3_rhs(ms3_handle* h, const ms3_incidence* inc, void* b, void* stream) {
    if (!h || !inc || !b || inc->nrhs < 1 || inc->nrhs > 64 || !inc->kind || !inc->theta || !inc->phi) return MS_ERR_ARG;
    const int nrhs = inc->nrhs, M = h->M, p = h->p, T = h->T;
    for (int r = 0; r < nrhs; ++r)
        if ((inc->kind[r] < 0 || inc->kind[r] > 2) || !(inc->theta[r] >= 0 && inc->theta[r] < 0.5 * M_PI) ||
            !std::isfinite(inc->phi[r]))
            return MS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = workspace(h, nrhs))) return rc;
    std::vector<double2> a((size_t)M * T * nrhs);
    std::vector<cd> CP(T), CV(T), CH(T);
    for (int r = 0; r < nrhs; ++r) {
        const int kind = inc->kind[r];
        const double kin = kind == 0 ? h->up.kp : h->up.ks;
        const cd lam = kin * sin(inc->theta[r]);
        const double th = inc->phi[r];
        // incident downgoing upper wave (displacement, traction) as the right-hand side
        cd Uu[3][3], Tu[3][3];
        wave_cols(h->up, lam, th, false, Uu, Tu);
        std::vector<cd> rhs(6);
        for (int i = 0; i < 3; ++i) {
            rhs[i] = Uu[kind][i];
            rhs[3 + i] = Tu[kind][i];
        }
        if (!interface_solve(h->lo, h->up, lam, th, rhs, 1)) return MS_ERR_ARG;
        cd eP[3], vP[3], hP[3], eS[3], vS[3], hS[3];
        pw_basis(h->lo.kp, lam, th, false, eP, vP, hP);
        pw_basis(h->lo.ks, lam, th, false, eS, vS, hS);
        plane_coeffs(p, h->lo.kp, eP, eP, CP.data());
        plane_coeffs(p, h->lo.kp, eS, vS, CV.data());
        plane_coeffs(p, h->lo.kp, eS, hS, CH.data());
        for (int m = 0; m < M; ++m) {
            const double* c = &h->h_cen[3 * m];
            const cd I(0, 1);
            const cd fp = rhs[0] * std::exp(I * h->lo.kp * (eP[0] * c[0] + eP[1] * c[1] + eP[2] * c[2]));
            const cd fs = std::exp(I * h->lo.ks * (eS[0] * c[0] + eS[1] * c[1] + eS[2] * c[2]));
            for (int k = 0; k < T; ++k) {
                const cd v = fp * CP[k] + fs * (rhs[1] * CV[k] + rhs[2] * CH[k]);
                a[((size_t)m * T + k) * nrhs + r] = make_double2(v.real(), v.imag());
            }
        }
    }
    if ((rc = ms_check(h->herr, cudaMemcpyAsync(h->wa, a.data(), a.size() * sizeof(double2), cudaMemcpyHostToDevice, st))))
        return rc;
    const long long n = (long long)M * T * nrhs;
    k3_sapply<double><<<nblk(n, 256), 256, 0, st>>>(nullptr, (const double2*)h->wa, (double2*)b, h->t64.Sd, M, p, nrhs, 0, 1);
    if ((rc = ms_check(h->herr, cudaGetLastError()))) return rc;
    return ms_check(h->herr, cudaStreamSynchronize(st));     // a is pageable host memory
}

// FP64: block GMRES on the FP64 operator.  FP32: iterative refinement -- the FP64 residual r = b - A x,
// an FP32 block GMRES solve of A d = r to 1e-3 relative (FP32 operator and basis), x += d -- until every
// column's FP64 relative residual is <= tol or the iteration cap is spent.
extern "C" int ms3_solve(ms3_handle* h, const ms3_incidence* inc, double tol, int32_t prec, void* tau,
                         ms_solve_info* info, void* stream) {
    if (!h || !inc || !tau || !(tol > 0) || (prec != MS_PREC_FP64 && prec != MS_PREC_FP32)) return MS_ERR_ARG;
    const int nrhs = inc->nrhs;
    if (nrhs < 1 || nrhs > 64) return MS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    const long long rows = (long long)h->M * h->T;
    const size_t n = (size_t)rows * nrhs;
    double2 *b = nullptr, *tmp = nullptr, *r = nullptr;
    float2 *r32 = nullptr, *d32 = nullptr, *tmp32 = nullptr;
    int rc = MS_OK;
    if (cudaMalloc(&b, n * sizeof(double2)) != cudaSuccess || cudaMalloc(&tmp, n * sizeof(double2)) != cudaSuccess)
        rc = MS_ERR_ALLOC;
    if (!rc) rc = ms3_rhs(h, inc, b, stream);
    int iters = 0, matvecs = 0, refinements = 0;
    std::vector<double> relres(nrhs, 1.0);
    if (!rc) rc = ms_check(h->herr, cudaMemsetAsync(tau, 0, n * sizeof(double2), st));
    if (!rc && prec == MS_PREC_FP64) {
        std::function<int(const double2*, double2*)> op = [&](const double2* in, double2* out) -> int {
            if (in == out) {
                if (int e = ms_check(h->herr, cudaMemcpyAsync(tmp, in, n * sizeof(double2), cudaMemcpyDeviceToDevice, st))) return e;
                in = tmp;
            }
            return op3<double>(h, in, out, nrhs, MS3_PART_T | MS3_PART_R | MS3_PART_S, st);
        };
        rc = ms_block_solve<double>(h->herr, rows, nrhs, h->opt.restart, op, b, (double2*)tau, tol, h->opt.max_iters,
                                    iters, matvecs, relres, st);
    } else if (!rc) {
        if (cudaMalloc(&r, n * sizeof(double2)) != cudaSuccess || cudaMalloc(&r32, n * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&d32, n * sizeof(float2)) != cudaSuccess || cudaMalloc(&tmp32, n * sizeof(float2)) != cudaSuccess)
            rc = MS_ERR_ALLOC;
        std::vector<double> bn, rn;
        if (!rc) rc = rel_norms(h, b, rows, nrhs, bn, st);
        std::function<int(const float2*, float2*)> op32 = [&](const float2* in, float2* out) -> int {
            if (in == out) {
                if (int e = ms_check(h->herr, cudaMemcpyAsync(tmp32, in, n * sizeof(float2), cudaMemcpyDeviceToDevice, st))) return e;
                in = tmp32;
            }
            return op3<float>(h, in, out, nrhs, MS3_PART_T | MS3_PART_R | MS3_PART_S, st);
        };
        while (!rc) {
            // r = b - A x in FP64
            if ((rc = op3<double>(h, (const double2*)tau, r, nrhs, MS3_PART_T | MS3_PART_R | MS3_PART_S, st))) break;
            ++matvecs;
            k3_residual<<<nblk((long long)n, 256), 256, 0, st>>>(b, r, (long long)n);
            if ((rc = rel_norms(h, r, rows, nrhs, rn, st))) break;
            bool all = true;
            for (int c = 0; c < nrhs; ++c) {
                relres[c] = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
                if (!std::isfinite(relres[c])) rc = MS_ERR_NONFINITE;
                all = all && relres[c] <= tol;
            }
            if (rc || all || iters >= h->opt.max_iters) break;
            k3_to_f32<<<nblk((long long)n, 256), 256, 0, st>>>(r, r32, (long long)n);
            if ((rc = ms_check(h->herr, cudaMemsetAsync(d32, 0, n * sizeof(float2), st)))) break;
            int it = 0, mv = 0;
            std::vector<double> inner;
            rc = ms_block_solve<float>(h->herr, rows, nrhs, h->opt.restart, op32, r32, d32, 1e-3, h->opt.max_iters - iters,
                                       it, mv, inner, st);
            if (rc) break;
            iters += it;
            matvecs += mv;
            ++refinements;
            k3_add_f32<<<nblk((long long)n, 256), 256, 0, st>>>((double2*)tau, d32, (long long)n);
            if ((rc = ms_check(h->herr, cudaGetLastError()))) break;
            if (it == 0) break;                          // no progress possible
        }
    }
    cudaFree(b); cudaFree(tmp); cudaFree(r); cudaFree(r32); cudaFree(d32); cudaFree(tmp32);
    double worst = 0;
    for (double v : relres) worst = std::max(worst, v);
    if (info) {
        info->iterations = iters;
        info->refinements = refinements;
        info->matvecs = matvecs;
        info->max_rel_residual = worst;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (rc) return rc;
    return worst <= tol ? MS_OK : MS_NOT_CONVERGED;
}

extern "C" int ms3_info(const ms3_handle* h, int32_t* M, int32_t* p, int32_t* T, int32_t* n_nodes) {
    if (!h) return MS_ERR_ARG;
    if (M) *M = h->M;
    if (p) *p = h->p;
    if (T) *T = h->T;
    if (n_nodes) *n_nodes = h->NS;
    return MS_OK;
}

extern "C" void ms3_destroy(ms3_handle* h) {
    if (!h) return;
    free_all(h);
    delete h->herr;
    delete h;
}
