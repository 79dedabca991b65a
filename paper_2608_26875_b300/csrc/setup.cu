// Handle construction: validation, wavenumbers, scale exponents, scattering matrices,
// Sommerfeld contour and reflection table, near-field pair list, device upload.
// All set-up arithmetic is FP64 on the host and runs once per geometry and frequency.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <new>
#include <vector>

#include "common.cuh"
#include "handle.h"

typedef std::complex<double> cd;

// ------------------------------------------------------------------ small host utilities
static double bess(int kind, int n, double x) {  // kind 0: J_n, 1: Y_n, any integer n
    int a = n < 0 ? -n : n;
    double v = kind == 0 ? jn(a, x) : yn(a, x);
    return (n < 0 && (a & 1)) ? -v : v;
}
static cd zfun(int kind, int n, double x) {  // kind 0: J, 1: H^(1)
    return kind == 0 ? cd(bess(0, n, x), 0.0) : cd(bess(0, n, x), bess(1, n, x));
}

// Gaussian elimination with partial pivoting on an n x n complex system (n <= 4), in place.
static bool solve_small(int n, cd* A, cd* b, int nb) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(A[r * n + c]) > std::abs(A[piv * n + c])) piv = r;
        if (std::abs(A[piv * n + c]) == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            for (int k = 0; k < nb; ++k) std::swap(b[c * nb + k], b[piv * nb + k]);
        }
        for (int r = c + 1; r < n; ++r) {
            cd f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            for (int k = 0; k < nb; ++k) b[r * nb + k] -= f * b[c * nb + k];
        }
    }
    for (int c = n - 1; c >= 0; --c)
        for (int k = 0; k < nb; ++k) {
            cd s = b[c * nb + k];
            for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * b[j * nb + k];
            b[c * nb + k] = s / A[c * n + c];
        }
    return true;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        // derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// s = sqrt(xi^2 - k^2) with Re s >= 0, as -i sqrt(k^2 - xi^2) (principal root).
static cd branch(cd xi, double k) { return cd(0, -1) * std::sqrt(cd(k * k, 0) - xi * xi); }

// Displacement and traction T_y of grad(e^{i xi x + d y}) (P) or grad_perp(.) (S) at y = 0 (Sec. 3).
static void wave_col(int S, cd xi, cd d, double lam, double mu, cd* col) {
    cd I(0, 1);
    cd u1 = S ? -d : I * xi;
    cd u2 = S ? I * xi : d;
    col[0] = u1;
    col[1] = u2;
    col[2] = mu * (d * u1 + I * xi * u2);
    col[3] = (lam + 2 * mu) * d * u2 + lam * I * xi * u1;
}

// Welded interface (Sec. 3): continuity of displacement and traction across y = 0 for the four
// plane waves at horizontal wavenumber xi.  Inputs: upgoing lower amplitudes U and downgoing
// upper amplitudes I; outputs: downgoing lower D and upgoing upper E amplitudes.
static bool interface_solve(const ms_handle* h, cd xi, const cd U[2], const cd In[2], cd D[2], cd E[2]) {
    cd spl = branch(xi, h->kp_l), ssl = branch(xi, h->ks_l);
    cd spu = branch(xi, h->kp_u), ssu = branch(xi, h->ks_u);
    cd A[16], rhs[4], c[4];
    cd cols[4][4];
    wave_col(0, xi, spl, h->lam_l, h->mu_l, cols[0]);
    wave_col(1, xi, ssl, h->lam_l, h->mu_l, cols[1]);
    wave_col(0, xi, -spu, h->lam_u, h->mu_u, cols[2]);
    wave_col(1, xi, -ssu, h->lam_u, h->mu_u, cols[3]);
    for (int r = 0; r < 4; ++r) {
        A[r * 4 + 0] = cols[0][r];
        A[r * 4 + 1] = cols[1][r];
        A[r * 4 + 2] = -cols[2][r];
        A[r * 4 + 3] = -cols[3][r];
        rhs[r] = 0;
    }
    wave_col(0, xi, -spl, h->lam_l, h->mu_l, c);
    for (int r = 0; r < 4; ++r) rhs[r] -= U[0] * c[r];
    wave_col(1, xi, -ssl, h->lam_l, h->mu_l, c);
    for (int r = 0; r < 4; ++r) rhs[r] -= U[1] * c[r];
    wave_col(0, xi, spu, h->lam_u, h->mu_u, c);
    for (int r = 0; r < 4; ++r) rhs[r] += In[0] * c[r];
    wave_col(1, xi, ssu, h->lam_u, h->mu_u, c);
    for (int r = 0; r < 4; ++r) rhs[r] += In[1] * c[r];
    if (!solve_small(4, A, rhs, 1)) return false;
    D[0] = rhs[0]; D[1] = rhs[1]; E[0] = rhs[2]; E[1] = rhs[3];
    return true;
}

// Transmitted (lower, downgoing) amplitudes of a plane wave incident from the upper layer along
// (cos t, -sin t) (Sec. 7.3): P-wave = grad(e^{i kp d.x})/(i kp), S-wave = grad_perp(e^{i ks d.x})/(i ks).
bool ms_plane_wave_transmission(const ms_handle* h, int kind, double angle, double* xi_out, cd D[2]) {
    double k = kind == 0 ? h->kp_u : h->ks_u;
    cd xi(k * cos(angle), 0.0);
    cd U[2] = {0.0, 0.0};
    cd In[2] = {0.0, 0.0};
    In[kind == 0 ? 0 : 1] = cd(1.0, 0.0) / cd(0.0, k);
    cd E[2];
    *xi_out = xi.real();
    return interface_solve(h, xi, U, In, D, E);
}

// Transmitted (lower, downgoing) amplitudes D at the node xi of the field of a unit point force q at z
// in the upper layer (Sec. 7.2 point-source incidence).  Below the source its downgoing spectrum in the
// basis grad(e^{i xi x + s_p y}), grad_perp(e^{i xi x + s_s y}) (upper wavenumbers) is, from som1 with
// d/dx -> i xi, d/dy -> s applied to Phi = -(i/(4 w^2)) [grad (q.grad) H_0(kp r) + grad_perp (q.grad_perp) H_0(ks r)],
//   I_P = -(i xi q_1 + s_p q_2) e^{-i xi z_1 - s_p z_2} / (4 pi w^2 s_p),
//   I_S = -(i xi q_2 - s_s q_1) e^{-i xi z_1 - s_s z_2} / (4 pi w^2 s_s);
// the welded interface then gives D.
bool ms_point_force_transmission(const ms_handle* h, cd xi, const double z[2], const double q[2], cd D[2]) {
    const cd I(0, 1);
    const cd sp = branch(xi, h->kp_u), ss = branch(xi, h->ks_u);
    const double f = 1.0 / (4.0 * M_PI * h->omega * h->omega);
    cd In[2];
    In[0] = -(I * xi * q[0] + sp * q[1]) * std::exp(-I * xi * z[0] - sp * z[1]) * f / sp;
    In[1] = -(I * xi * q[1] - ss * q[0]) * std::exp(-I * xi * z[0] - ss * z[1]) * f / ss;
    const cd U[2] = {0.0, 0.0};
    cd E[2];
    return interface_solve(h, xi, U, In, D, E);
}

// Disc mode matrix (Sec. 4.1; projection-formula matrix of Sec. 4.3 for rigid particles):
// boundary displacement (rigid) or traction (traction-free) of (P coef, S coef) of mode n at r = R.
static void disc_mode(int kind, int n, double kp, double ks, double R, int bc, double lam, double mu, cd M[4]) {
    cd I(0, 1);
    cd f = zfun(kind, n, kp * R), g = zfun(kind, n, ks * R);
    cd f1 = 0.5 * kp * (zfun(kind, n - 1, kp * R) - zfun(kind, n + 1, kp * R));
    cd g1 = 0.5 * ks * (zfun(kind, n - 1, ks * R) - zfun(kind, n + 1, ks * R));
    if (bc == 0) {
        M[0] = f1;
        M[1] = -I * (double)n / R * g;
        M[2] = I * (double)n / R * f;
        M[3] = g1;
        return;
    }
    cd f2 = 0.25 * kp * kp * (zfun(kind, n - 2, kp * R) - 2.0 * f + zfun(kind, n + 2, kp * R));
    cd g2 = 0.25 * ks * ks * (zfun(kind, n - 2, ks * R) - 2.0 * g + zfun(kind, n + 2, ks * R));
    double nn = (double)n;
    M[0] = -lam * kp * kp * f + 2.0 * mu * f2;                 // t_r from P
    M[1] = -2.0 * mu * I * nn * (g1 / R - g / (R * R));        // t_r from S
    M[2] = 2.0 * mu * I * nn * (f1 / R - f / (R * R));         // t_theta from P
    M[3] = mu * (g2 - g1 / R + nn * nn * g / (R * R));         // t_theta from S
}

// d/dR of disc_mode: derivatives of Z_n(kR) up to third order (DLMF 10.6.1 applied repeatedly).
static void disc_mode_dR(int kind, int n, double kp, double ks, double R, int bc, double lam, double mu, cd M[4]) {
    cd I(0, 1);
    auto zd = [&](double k, cd* z) {   // z[0..3] = Z, dZ/dR, d2Z/dR2, d3Z/dR3 of Z_n(kR)
        cd a = zfun(kind, n - 3, k * R), b = zfun(kind, n - 2, k * R), c = zfun(kind, n - 1, k * R),
           d = zfun(kind, n, k * R), e = zfun(kind, n + 1, k * R), f = zfun(kind, n + 2, k * R),
           g = zfun(kind, n + 3, k * R);
        z[0] = d;
        z[1] = 0.5 * k * (c - e);
        z[2] = 0.25 * k * k * (b - 2.0 * d + f);
        z[3] = 0.125 * k * k * k * (a - 3.0 * c + 3.0 * e - g);
    };
    cd f[4], g[4];
    zd(kp, f);
    zd(ks, g);
    double nn = (double)n, R2 = R * R, R3 = R2 * R;
    if (bc == 0) {
        M[0] = f[2];
        M[1] = I * nn / R2 * g[0] - I * nn / R * g[1];
        M[2] = -I * nn / R2 * f[0] + I * nn / R * f[1];
        M[3] = g[2];
        return;
    }
    M[0] = -lam * kp * kp * f[1] + 2.0 * mu * f[3];
    M[1] = -2.0 * mu * I * nn * (g[2] / R - 2.0 * g[1] / R2 + 2.0 * g[0] / R3);
    M[2] = 2.0 * mu * I * nn * (f[2] / R - 2.0 * f[1] / R2 + 2.0 * f[0] / R3);
    M[3] = mu * (g[3] - g[2] / R + g[1] / R2 + nn * nn * g[1] / R2 - 2.0 * nn * nn * g[0] / R3);
}

// ------------------------------------------------------------------ device upload helper
template <typename X>
static int upload(ms_handle* h, X** dst, const X* src, size_t n) {
    if (n == 0) return MS_OK;
    if (cudaMalloc((void**)dst, n * sizeof(X)) != cudaSuccess) return MS_ERR_ALLOC;
    return ms_check(h, cudaMemcpy(*dst, src, n * sizeof(X), cudaMemcpyHostToDevice));
}

static double2 d2(cd v) { return make_double2(v.real(), v.imag()); }

extern "C" void ms_default_options(ms_options* o) {
    if (!o) return;
    o->n_panels = 32;
    o->nodes_per_panel = 16;
    o->t_max = 20.0;
    o->restart = 50;
    o->max_iters = 2000;
    o->check_geometry = 1;
    o->use_fmm = 1;
    o->leaf_target = 10;
    o->depth = 0.5;
    o->grade = 0;
    o->tensor_cores = 1;
    o->inner_tol = 0.0;
    o->block_krylov = 1;
    o->cuda_graph = 1;
    o->tc_wait_test = 0;
    o->store_near = 0;
    o->precond_group = 0;
}

// Panel edges of the Sommerfeld rule on [-t_max, t_max]: n uniform panels (edge k at
// -t_max + k (2 t_max / n)); with grade > 0 also every branch point c in {+-kp, +-ks} of both
// layers and c +- depth 2^j, j < grade, inside the interval.  Sorted; an edge closer than 1e-9 to
// the previous kept edge is dropped.
static std::vector<double> contour_edges(const ms_handle* h, const ms_options& o) {
    std::vector<double> e;
    for (int k = 0; k <= o.n_panels; ++k) e.push_back(-o.t_max + k * (2.0 * o.t_max / o.n_panels));
    if (o.grade > 0) {
        const double bp[4] = {h->kp_u, h->ks_u, h->kp_l, h->ks_l};
        for (double kb : bp)
            for (int sg = -1; sg <= 1; sg += 2) {
                double c = sg * kb;
                std::vector<double> add = {c};
                for (int j = 0; j < o.grade; ++j) {
                    add.push_back(c - o.depth * std::ldexp(1.0, j));
                    add.push_back(c + o.depth * std::ldexp(1.0, j));
                }
                for (double v : add)
                    if (v > -o.t_max && v < o.t_max) e.push_back(v);
            }
    }
    std::sort(e.begin(), e.end());
    std::vector<double> out;
    for (double v : e)
        if (out.empty() || v - out.back() > 1e-9) out.push_back(v);
    return out;
}

constexpr long long MS_MAX_NODES = 1LL << 20;   // Sommerfeld nodes n_panels x nodes_per_panel

// The body of ms_setup; `made` receives the handle as soon as it exists, so that the C entry point can
// release it if a host allocation throws.
static int ms_setup_impl(const ms_geometry* g, const ms_media* md, double omega, int32_t p,
                         const ms_options* o, ms_handle** out, ms_handle*& made) {
    if (!out) return MS_ERR_ARG;
    *out = nullptr;
    if (!g || !md || !g->centres || !g->radius || !g->bc || g->M < 1 || !(omega > 0) || !std::isfinite(omega) || p < 0 ||
        p > 30)
        return MS_ERR_ARG;
    if (!(md->mu_u > 0) || !(md->mu_l > 0) || !(md->lam_u + md->mu_u > 0) || !(md->lam_l + md->mu_l > 0))
        return MS_ERR_ARG;
    ms_options opt;
    ms_default_options(&opt);
    if (o) opt = *o;
    if (opt.n_panels < 1 || opt.nodes_per_panel < 1 || !(opt.t_max > 0) || !std::isfinite(opt.t_max) ||
        (long long)opt.n_panels * opt.nodes_per_panel > MS_MAX_NODES || opt.restart < 1 || opt.max_iters < 1 ||
        opt.leaf_target < 1 || !(opt.depth > 0) || opt.grade < 0 || opt.grade > 30 ||
        (opt.tensor_cores != 0 && opt.tensor_cores != 1) || !(opt.inner_tol >= 0.0 && opt.inner_tol < 1.0) ||
        opt.tc_wait_test < 0 || opt.tc_wait_test > 1000000 || (opt.block_krylov != 0 && opt.block_krylov != 1) ||
        (opt.cuda_graph != 0 && opt.cuda_graph != 1) || opt.store_near < 0 || opt.store_near > 1024 ||
        opt.precond_group < 0 || opt.precond_group > 64)
        return MS_ERR_ARG;
    const int M = g->M, nc = 2 * p + 1;
    for (int m = 0; m < M; ++m) {
        if (!(g->radius[m] > 0) || !std::isfinite(g->radius[m]) || !std::isfinite(g->centres[2 * m]) ||
            !std::isfinite(g->centres[2 * m + 1]))
            return MS_ERR_ARG;
        if (g->bc[m] != 0 && g->bc[m] != 1) return MS_ERR_ARG;
        if (g->proto && (g->proto[m] >= g->n_proto || g->proto[m] < -1)) return MS_ERR_ARG;
    }
    if (g->n_proto > 0 && !g->proto_S) return MS_ERR_ARG;
    if (opt.check_geometry) {
        for (int m = 0; m < M; ++m)
            if (g->centres[2 * m + 1] + 1.1 * g->radius[m] > 0.0) return MS_ERR_NOT_BURIED;
        // separation rule |x_l - x_m| >= 1.1 (R_l + R_m) (Sec. 2), checked on a uniform grid
        double rmax = 0, xmin = 1e300, ymin = 1e300;
        for (int m = 0; m < M; ++m) {
            rmax = std::max(rmax, g->radius[m]);
            xmin = std::min(xmin, g->centres[2 * m]);
            ymin = std::min(ymin, g->centres[2 * m + 1]);
        }
        double cell = 2.2 * rmax;
        std::vector<std::pair<long long, int>> keys(M);
        auto key = [&](long long ix, long long iy) { return ix * 2000003LL + iy; };
        for (int m = 0; m < M; ++m) {
            long long ix = (long long)((g->centres[2 * m] - xmin) / cell);
            long long iy = (long long)((g->centres[2 * m + 1] - ymin) / cell);
            keys[m] = {key(ix, iy), m};
        }
        std::sort(keys.begin(), keys.end());
        for (int m = 0; m < M; ++m) {
            long long ix = (long long)((g->centres[2 * m] - xmin) / cell);
            long long iy = (long long)((g->centres[2 * m + 1] - ymin) / cell);
            for (long long dx = -1; dx <= 1; ++dx)
                for (long long dy = -1; dy <= 1; ++dy) {
                    long long kk = key(ix + dx, iy + dy);
                    auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(kk, -1));
                    for (; it != keys.end() && it->first == kk; ++it) {
                        int l = it->second;
                        if (l == m) continue;
                        double ddx = g->centres[2 * m] - g->centres[2 * l];
                        double ddy = g->centres[2 * m + 1] - g->centres[2 * l + 1];
                        double lim = 1.1 * (g->radius[m] + g->radius[l]);
                        if (ddx * ddx + ddy * ddy < lim * lim) return MS_ERR_OVERLAP;
                    }
                }
        }
    }

    ms_handle* h = new ms_handle();
    made = h;
    h->M = M;
    h->p = p;
    h->nc = nc;
    h->NS = 0;   // set from the contour edges below
    h->omega = omega;
    h->lam_u = md->lam_u; h->mu_u = md->mu_u; h->lam_l = md->lam_l; h->mu_l = md->mu_l;
    h->kp_u = omega / sqrt(md->lam_u + 2 * md->mu_u);
    h->ks_u = omega / sqrt(md->mu_u);
    h->kp_l = omega / sqrt(md->lam_l + 2 * md->mu_l);
    h->ks_l = omega / sqrt(md->mu_l);
    h->opt = opt;
    h->n_proto = g->n_proto;
    h->h_centres.assign(g->centres, g->centres + 2 * M);
    h->h_radius.assign(g->radius, g->radius + M);
    h->h_bc.assign(g->bc, g->bc + M);
    if (g->proto) h->h_proto.assign(g->proto, g->proto + M);
    if (g->rotation) h->h_rot.assign(g->rotation, g->rotation + M);
    if (g->n_proto > 0) h->h_protoS.assign(g->proto_S, g->proto_S + (size_t)g->n_proto * 2 * (2 * nc) * (2 * nc));
    h->media = *md;
    int rc = MS_OK;

    // scale exponents a = round(log2((k R / 2)^|n| / |n|!))
    std::vector<int> expo((size_t)M * 2 * nc);
    for (int m = 0; m < M; ++m)
        for (int b = 0; b < 2; ++b) {
            double k = b ? h->ks_l : h->kp_l;
            for (int i = 0; i < nc; ++i) {
                int n = abs(i - p);
                double l2 = n * log2(k * g->radius[m] / 2.0) - lgamma(n + 1.0) / log(2.0);
                int a = (int)lround(l2);
                if (a < -900) a = -900;
                if (a > 900) a = 900;
                expo[((size_t)m * 2 + b) * nc + i] = a;
            }
        }
    h->h_expo = expo;

    // scattering matrices: discs closed form, scaled S~ = D^-1 S D^-1
    std::vector<double2> sdisc((size_t)M * nc * 4);
    std::vector<double2> dsdr((size_t)M * nc * 4);   // unscaled dS/dR (zero for prototypes)
    std::vector<float2> sdisc_f((size_t)M * nc * 4);
    std::vector<int> proto(M, -1);
    std::vector<double> rot(M, 0.0);
    for (int m = 0; m < M; ++m) {
        if (g->proto && g->proto[m] >= 0) {
            proto[m] = g->proto[m];
            h->any_proto = true;
        }
        if (g->rotation) rot[m] = g->rotation[m];
    }
    for (int m = 0; m < M; ++m) {
        for (int i = 0; i < nc; ++i) {
            cd S[4] = {0.0, 0.0, 0.0, 0.0};
            if (proto[m] < 0) {
                int n = i - p;
                cd MH[4], MJ[4];
                disc_mode(1, n, h->kp_l, h->ks_l, g->radius[m], g->bc[m], h->lam_l, h->mu_l, MH);
                disc_mode(0, n, h->kp_l, h->ks_l, g->radius[m], g->bc[m], h->lam_l, h->mu_l, MJ);
                cd MHc[4] = {MH[0], MH[1], MH[2], MH[3]};
                cd B[4] = {-MJ[0], -MJ[1], -MJ[2], -MJ[3]};
                if (!solve_small(2, MH, B, 2)) { ms_destroy(h); return MS_ERR_ARG; }
                for (int k = 0; k < 4; ++k) S[k] = B[k];
                // dS = -M_H^{-1} (dM_J + dM_H S)
                cd dMH[4], dMJ[4];
                disc_mode_dR(1, n, h->kp_l, h->ks_l, g->radius[m], g->bc[m], h->lam_l, h->mu_l, dMH);
                disc_mode_dR(0, n, h->kp_l, h->ks_l, g->radius[m], g->bc[m], h->lam_l, h->mu_l, dMJ);
                cd rhs[4];
                for (int r = 0; r < 2; ++r)
                    for (int c = 0; c < 2; ++c)
                        rhs[r * 2 + c] = -(dMJ[r * 2 + c] + dMH[r * 2 + 0] * S[0 * 2 + c] + dMH[r * 2 + 1] * S[1 * 2 + c]);
                if (!solve_small(2, MHc, rhs, 2)) { ms_destroy(h); return MS_ERR_ARG; }
                for (int k = 0; k < 4; ++k) dsdr[((size_t)m * nc + i) * 4 + k] = d2(rhs[k]);
            }
            int ap = expo[((size_t)m * 2 + 0) * nc + i], as = expo[((size_t)m * 2 + 1) * nc + i];
            int ea[2] = {ap, as};
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) {
                    cd v = S[r * 2 + c] * pow2d(-ea[r] - ea[c]);
                    sdisc[((size_t)m * nc + i) * 4 + r * 2 + c] = d2(v);
                    sdisc_f[((size_t)m * nc + i) * 4 + r * 2 + c] = make_float2((float)v.real(), (float)v.imag());
                }
        }
    }

    // contour (Sec. 5.1), per-node factors and reflection table
    std::vector<double> gx, gw;
    gauss_legendre(opt.nodes_per_panel, gx, gw);
    const std::vector<double> edges = contour_edges(h, opt);
    const int npan = (int)edges.size() - 1;
    h->NS = npan * opt.nodes_per_panel;
    const int NS = h->NS;
    std::vector<double2> node(NS), wq(NS), sq(NS * 2), qq(NS * 2), refl(NS * 4), trans(NS * 4), squ(NS * 2);
    std::vector<double2> qpm((size_t)2 * NS * nc), qps((size_t)2 * NS * nc);
    for (int pnl = 0; pnl < npan; ++pnl) {
        double a = edges[pnl], width = edges[pnl + 1] - edges[pnl];
        for (int j = 0; j < opt.nodes_per_panel; ++j) {
            int q = pnl * opt.nodes_per_panel + j;
            double t = a + 0.5 * width * (gx[j] + 1.0);
            double w = 0.5 * width * gw[j];
            double th = tanh(t);
            cd xi(t, -opt.depth * th);
            cd dxi(1.0, -opt.depth * (1.0 - th * th));
            node[q] = d2(xi);
            wq[q] = d2(w * dxi);
            cd U[2], D[2], E[2], In[2] = {0.0, 0.0};
            cd R[4], Tu[4];
            for (int c = 0; c < 2; ++c) {
                U[0] = c == 0 ? 1.0 : 0.0;
                U[1] = c == 1 ? 1.0 : 0.0;
                if (!interface_solve(h, xi, U, In, D, E)) { ms_destroy(h); return MS_ERR_ARG; }
                R[0 * 2 + c] = D[0];
                R[1 * 2 + c] = D[1];
                Tu[0 * 2 + c] = E[0];
                Tu[1 * 2 + c] = E[1];
            }
            for (int k = 0; k < 4; ++k) refl[(size_t)q * 4 + k] = d2(R[k]);
            for (int k = 0; k < 4; ++k) trans[(size_t)q * 4 + k] = d2(Tu[k]);
            squ[q * 2 + 0] = d2(branch(xi, h->kp_u));
            squ[q * 2 + 1] = d2(branch(xi, h->ks_u));
            for (int b = 0; b < 2; ++b) {
                double k = b ? h->ks_l : h->kp_l;
                cd s = branch(xi, k);
                cd qv = (xi - s) / k;
                sq[q * 2 + b] = d2(s);
                qq[q * 2 + b] = d2(qv);
                // (-i)^n q^n / (i pi s) and i^n q^n W_q for n in [-p, p]
                cd base_m = cd(1.0, 0.0) / (cd(0.0, M_PI) * s);
                cd base_s = w * dxi;
                for (int i = 0; i < nc; ++i) {
                    int n = i - p;
                    cd qn = std::pow(qv, n);
                    cd in = std::pow(cd(0, 1), n);
                    cd mi = std::pow(cd(0, -1), n);
                    qpm[((size_t)b * NS + q) * nc + i] = d2(mi * qn * base_m);
                    qps[((size_t)b * NS + q) * nc + i] = d2(in * qn * base_s);
                }
            }
        }
    }

    std::vector<double2> cen(M);
    for (int m = 0; m < M; ++m) cen[m] = make_double2(g->centres[2 * m], g->centres[2 * m + 1]);
    if ((rc = upload(h, &h->d.centre, cen.data(), M)) ||
        (rc = upload(h, &h->d.expo, expo.data(), expo.size())) ||
        (rc = upload(h, &h->d.sdisc, sdisc.data(), sdisc.size())) ||
        (rc = upload(h, &h->d.sdisc_f, sdisc_f.data(), sdisc_f.size())) ||
        (rc = upload(h, &h->d.dsdr, dsdr.data(), dsdr.size())) ||
        (rc = upload(h, &h->d.proto, proto.data(), proto.size())) ||
        (rc = upload(h, &h->d.rot, rot.data(), rot.size())) ||
        (rc = upload(h, &h->d.node, node.data(), node.size())) ||
        (rc = upload(h, &h->d.wq, wq.data(), wq.size())) ||
        (rc = upload(h, &h->d.sq, sq.data(), sq.size())) ||
        (rc = upload(h, &h->d.qq, qq.data(), qq.size())) ||
        (rc = upload(h, &h->d.refl, refl.data(), refl.size())) ||
        (rc = upload(h, &h->d.trans, trans.data(), trans.size())) ||
        (rc = upload(h, &h->d.squ, squ.data(), squ.size())) ||
        (rc = upload(h, &h->d.qpow_m2s, qpm.data(), qpm.size())) ||
        (rc = upload(h, &h->d.qpow_s2l, qps.data(), qps.size()))) {
        ms_destroy(h);
        return rc;
    }
    {
        std::vector<float2> mm(qpm.size()), ms2(qps.size());
        std::vector<int> em(qpm.size()), es(qps.size());
        for (size_t k = 0; k < qpm.size(); ++k) split_exp(qpm[k], mm[k], em[k]);
        for (size_t k = 0; k < qps.size(); ++k) split_exp(qps[k], ms2[k], es[k]);
        if ((rc = upload(h, &h->d.qpm_m, mm.data(), mm.size())) || (rc = upload(h, &h->d.qpm_e, em.data(), em.size())) ||
            (rc = upload(h, &h->d.qps_m, ms2.data(), ms2.size())) || (rc = upload(h, &h->d.qps_e, es.data(), es.size()))) {
            ms_destroy(h);
            return rc;
        }
    }
    {
        std::vector<int> z(std::max((size_t)M * 2 * nc, (size_t)4096), 0);
        if ((rc = upload(h, &h->d.zexp, z.data(), z.size()))) { ms_destroy(h); return rc; }
    }
    if ((rc = ms_sapply_setup(h))) {
        ms_destroy(h);
        return rc;
    }
    if ((rc = ms_build_translations(h, opt.use_fmm, opt.leaf_target))) {
        ms_destroy(h);
        return rc;
    }
    if (opt.tensor_cores && ((rc = ms_spectral_tc_setup(h)) || (rc = ms_near_store_build(h)))) {
        ms_destroy(h);
        return rc;
    }
    if ((rc = ms_precond_build(h))) {
        ms_destroy(h);
        return rc;
    }
    *out = h;
    return MS_OK;
}

extern "C" int ms_setup(const ms_geometry* g, const ms_media* md, double omega, int32_t p,
                        const ms_options* o, ms_handle** out) {
    ms_handle* made = nullptr;
    try {
        const int rc = ms_setup_impl(g, md, omega, p, o, out, made);
        return rc;
    } catch (const std::bad_alloc&) {
        if (made) ms_destroy(made);
        if (out) *out = nullptr;
        return MS_ERR_ALLOC;
    }
}
