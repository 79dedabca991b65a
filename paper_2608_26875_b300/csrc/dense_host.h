// Small dense host algebra shared by the solvers (FP64, std::complex): the one-sided Jacobi SVD of the
// deflation and of the time-reversal matrix, and the factors, block Householder QR and triangular solve of
// block GMRES.  Host code only, so that it also builds and is tested without a GPU.
#pragma once

#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

namespace dense {

typedef std::complex<double> cd;

// One-sided Jacobi on the columns of A (n x n, column-major): A V = U Sigma.  Returns the squared
// column norms (eigenvalues of A^H A) and V (column-major).
inline void jacobi_svd(std::vector<cd>& A, int n, std::vector<double>& ev, std::vector<cd>& V) {
    V.assign((size_t)n * n, cd(0));
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                cd* ap = &A[(size_t)p * n];
                cd* aq = &A[(size_t)q * n];
                double alpha = 0, beta = 0;
                cd gamma = 0;
                for (int i = 0; i < n; ++i) {
                    alpha += std::norm(ap[i]);
                    beta += std::norm(aq[i]);
                    gamma += std::conj(ap[i]) * aq[i];
                }
                const double g = std::abs(gamma);
                if (g == 0 || g <= 1e-15 * sqrt(alpha * beta)) continue;
                off = std::max(off, g / sqrt(alpha * beta));
                // rotate (a_p, e a_q), e = conj(gamma)/|gamma|, which makes the inner product real
                const cd e = std::conj(gamma) / g;
                const double zeta = (beta - alpha) / (2 * g);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1 + zeta * zeta));
                const double c = 1 / sqrt(1 + t * t), s = c * t;
                for (int i = 0; i < n; ++i) {
                    const cd x = ap[i], y = e * aq[i];
                    ap[i] = c * x - s * y;
                    aq[i] = s * x + c * y;
                }
                cd* vp = &V[(size_t)p * n];
                cd* vq = &V[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    const cd x = vp[i], y = e * vq[i];
                    vp[i] = c * x - s * y;
                    vq[i] = s * x + c * y;
                }
            }
        if (off <= 1e-15) break;
    }
    ev.resize(n);
    for (int p = 0; p < n; ++p) {
        double a = 0;
        for (int i = 0; i < n; ++i) a += std::norm(A[(size_t)p * n + i]);
        ev[p] = a;
    }
}

// ------------------------------------------------------------------ block GMRES: factors and least squares
// Upper-triangular R with G = R^H R (G Hermitian positive definite, s x s row-major); a diagonal
// shift of shift * max diag(G) keeps the factorisation defined for (nearly) dependent blocks.
inline bool chol_upper(const std::vector<cd>& G, int s, double shift, std::vector<cd>& R) {
    double dmax = 0;
    for (int i = 0; i < s; ++i) dmax = std::max(dmax, G[i * s + i].real());
    const double add = shift * dmax + 1e-300;
    R.assign((size_t)s * s, cd(0));
    for (int i = 0; i < s; ++i) {
        cd d = G[i * s + i] + add;
        for (int k = 0; k < i; ++k) d -= std::conj(R[k * s + i]) * R[k * s + i];
        if (!(d.real() > 0)) return false;
        const double rii = sqrt(d.real());
        R[i * s + i] = rii;
        for (int j = i + 1; j < s; ++j) {
            cd v = G[i * s + j];
            for (int k = 0; k < i; ++k) v -= std::conj(R[k * s + i]) * R[k * s + j];
            R[i * s + j] = v / rii;
        }
    }
    return true;
}

// inverse of an upper-triangular s x s matrix (row-major)
inline void tri_inv_upper(const std::vector<cd>& R, int s, std::vector<cd>& Ri) {
    Ri.assign((size_t)s * s, cd(0));
    for (int j = 0; j < s; ++j) {
        Ri[j * s + j] = 1.0 / R[j * s + j];
        for (int i = j - 1; i >= 0; --i) {
            cd v = 0;
            for (int k = i + 1; k <= j; ++k) v += R[i * s + k] * Ri[k * s + j];
            Ri[i * s + j] = -v / R[i * s + i];
        }
    }
}

// C = A B (s x s, row-major)
inline std::vector<cd> matmul(const std::vector<cd>& A, const std::vector<cd>& B, int s) {
    std::vector<cd> C((size_t)s * s, cd(0));
    for (int i = 0; i < s; ++i)
        for (int k = 0; k < s; ++k) {
            const cd a = A[i * s + k];
            if (a == 0.0) continue;
            for (int j = 0; j < s; ++j) C[i * s + j] += a * B[k * s + j];
        }
    return C;
}

// Householder reflectors of one block step: acting on rows [j s, (j+2) s) of the block Hessenberg
// matrix; reflector k has vector v_k (2s entries, zero above k) and factor tau_k: (I - tau v v^H).
struct StepQR {
    std::vector<cd> v;      // [s][2s]
    std::vector<double> tau;
};

// Householder QR in place of the 2s x s panel P (row stride s): on return its upper s x s block is R
// (up to rounding, zeros below), and q holds the s reflectors, reflector k zeroing column k below row k
// (a zero column gets tau_k = 0, the identity).
inline void step_qr(cd* P, int s, StepQR& q) {
    q.v.assign((size_t)s * 2 * s, cd(0));
    q.tau.assign(s, 0.0);
    for (int k = 0; k < s; ++k) {
        double nx = 0;
        for (int i = k; i < 2 * s; ++i) nx += std::norm(P[(size_t)i * s + k]);
        nx = sqrt(nx);
        cd* v = &q.v[(size_t)k * 2 * s];
        if (nx == 0) continue;
        const cd x0 = P[(size_t)k * s + k];
        const cd alpha = -(std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0)) * nx;
        for (int i = k; i < 2 * s; ++i) v[i] = P[(size_t)i * s + k];
        v[k] -= alpha;
        double vn = 0;
        for (int i = k; i < 2 * s; ++i) vn += std::norm(v[i]);
        if (vn == 0) continue;
        q.tau[k] = 2.0 / vn;
        for (int c = k; c < s; ++c) {
            cd d = 0;
            for (int i = k; i < 2 * s; ++i) d += std::conj(v[i]) * P[(size_t)i * s + c];
            d *= q.tau[k];
            for (int i = k; i < 2 * s; ++i) P[(size_t)i * s + c] -= v[i] * d;
        }
    }
}

// Steps i0 .. i1-1 of qr, in order, on all s columns of the block column H (row-major, row stride s):
// step i acts on rows [i s, (i+2) s), and each of its reflectors k in order maps a column y (those 2s
// rows) to y - tau_k v_k (v_k^H y).  The columns are processed in chunks of 8 adjacent ones (one chunk
// per thread), so that the rows are read contiguously and no two threads write the same cache line.
inline void apply_steps(const std::vector<StepQR>& qr, int i0, int i1, int s, cd* H) {
    constexpr int CH = 8;
    const int nch = (s + CH - 1) / CH;
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < nch; ++ch) {
        const int c0 = ch * CH, w = std::min(CH, s - c0);
        for (int i = i0; i < i1; ++i) {
            cd* Y = H + (size_t)i * s * s + c0;
            const StepQR& q = qr[i];
            for (int k = 0; k < s; ++k) {
                const cd* v = &q.v[(size_t)k * 2 * s];
                cd d[CH];
                for (int c = 0; c < w; ++c) d[c] = 0;
                for (int r = k; r < 2 * s; ++r) {
                    const cd vr = std::conj(v[r]);
                    const cd* y = Y + (size_t)r * s;
                    for (int c = 0; c < w; ++c) d[c] += vr * y[c];
                }
                for (int c = 0; c < w; ++c) d[c] *= q.tau[k];
                for (int r = k; r < 2 * s; ++r) {
                    const cd vr = v[r];
                    cd* y = Y + (size_t)r * s;
                    for (int c = 0; c < w; ++c) y[c] -= vr * d[c];
                }
            }
        }
    }
}

// Y (j s x s, row-major: Y[row * s + c]) with R Y = g[0 : j s] for the block upper-triangular R whose
// block column jj is Rcol[jj] ((jj + 1) s x s, row-major), g[row * s + c] the transformed right-hand
// side.  Truncated: a diagonal entry at or below floor_rel times the largest is a direction the basis
// cannot resolve (deflated or stagnant), and its component is left at zero.  The columns go in chunks
// of 8 adjacent ones (one chunk per thread), each column with the operations of a plain per-column
// back substitution in the same order.
inline void block_back_substitute(const std::vector<std::vector<cd>>& Rcol, const std::vector<cd>& g, int s, int j,
                                  double floor_rel, std::vector<cd>& Y) {
    constexpr int CH = 8;
    const int nbj = j * s;
    Y.assign((size_t)nbj * s, cd(0));
    double dmax = 0;
    for (int row = 0; row < nbj; ++row) dmax = std::max(dmax, std::abs(Rcol[row / s][(size_t)row * s + (row % s)]));
    const double dfloor = floor_rel * dmax;
    const int nch = (s + CH - 1) / CH;
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < nch; ++ch) {
        const int c0 = ch * CH, w = std::min(CH, s - c0);
        for (int row = nbj - 1; row >= 0; --row) {
            cd v[CH];
            for (int c = 0; c < w; ++c) v[c] = g[(size_t)row * s + c0 + c];
            // entries of row `row` in block columns jj >= its own block
            const int jb = row / s;
            for (int jj = jb; jj < j; ++jj) {
                const cd* Rr = &Rcol[jj][(size_t)row * s];
                for (int cc = 0; cc < s; ++cc) {
                    const int col = jj * s + cc;
                    if (col <= row) continue;
                    const cd r = Rr[cc];
                    const cd* y = &Y[(size_t)col * s + c0];
                    for (int c = 0; c < w; ++c) v[c] -= r * y[c];
                }
            }
            const cd d = Rcol[jb][(size_t)row * s + (row - jb * s)];
            for (int c = 0; c < w; ++c) Y[(size_t)row * s + c0 + c] = std::abs(d) > dfloor ? v[c] / d : cd(0);
        }
    }
}

}  // namespace dense
