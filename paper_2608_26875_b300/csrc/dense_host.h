// Small dense host algebra shared by the solvers (FP64, std::complex).
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

}  // namespace dense
