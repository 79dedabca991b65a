// FP64 Bessel / Hankel sequences at real argument for the Graf translation (Sec. 4.2)
// and the receiver-field sums (Sec. 5).
//
// Y_0, Y_1, J_0, J_1 come from CUDA's own y0/y1/j0/j1.  Higher orders follow the
// three-term recurrence Z_{k+1} = (2k/x) Z_k - Z_{k-1} (DLMF 10.6.1):
//   * Y_k: upward, which is the stable direction for Y at every k;
//   * J_k: upward when x > N (stable while k < x); otherwise Miller's downward recurrence
//     (DLMF 3.6(vi)) from an even start order N + 16 + ceil(x) + floor(sqrt(40 N)), with
//     rescaling against overflow, normalised by whichever of J_0, J_1 is larger in
//     magnitude.  Checked against scipy to <= 3e-12 of max_k |J_k| for N <= 82, 0.05 <= x.
#pragma once

#include "common.cuh"

#define MS_PMAX 30                    // largest supported expansion order p
#define MS_KMAX (2 * MS_PMAX + 2)     // largest Hankel order a kernel asks for

// J[k], Y[k] for k = 0..N (N <= MS_KMAX), x > 0.  J and Y may live in any address space.
__device__ inline void bessel_jy_seq(int N, double x, double* J, double* Y) {
    Y[0] = y0(x);
    if (N >= 1) Y[1] = y1(x);
    for (int k = 1; k < N; ++k) Y[k + 1] = (2.0 * k / x) * Y[k] - Y[k - 1];
    if (x > (double)N) {
        J[0] = j0(x);
        if (N >= 1) J[1] = j1(x);
        for (int k = 1; k < N; ++k) J[k + 1] = (2.0 * k / x) * J[k] - J[k - 1];
        return;
    }
    int ns = N + 16 + (int)ceil(x) + (int)sqrt(40.0 * N);
    ns += ns & 1;
    double jp1 = 0.0, j = 1e-300;
    double j0s = 0.0, j1s = 0.0;
    for (int k = ns; k >= 1; --k) {
        double jm1 = (2.0 * k / x) * j - jp1;
        jp1 = j;
        j = jm1;
        if (k - 1 <= N) J[k - 1] = jm1;
        if (fabs(j) > 1e250) {
            j *= 1e-250;
            jp1 *= 1e-250;
            for (int i = k - 1; i <= N; ++i)
                if (i >= 0) J[i] *= 1e-250;
        }
    }
    j0s = J[0];
    j1s = (N >= 1) ? J[1] : jp1;
    double c = (fabs(j0s) > fabs(j1s)) ? j0(x) / j0s : j1(x) / j1s;
    for (int k = 0; k <= N; ++k) J[k] *= c;
}

// h[k + K] = H_k(kx) e^{i k theta} for k in [-K, K], with (cos theta, sin theta) = (ux, uy).
// Scratch J, Y of length K + 1 are supplied by the caller.
__device__ inline void hankel_phase_seq(int K, double x, double ux, double uy, double2* h, double* J,
                                        double* Y) {
    bessel_jy_seq(K, x, J, Y);
    double2 e = make_double2(1.0, 0.0);
    double2 u = make_double2(ux, uy);
    for (int k = 0; k <= K; ++k) {
        double2 H = make_double2(J[k], Y[k]);
        double2 v = cmul(H, e);
        h[K + k] = v;
        if (k > 0) {
            // H_{-k} e^{-ik th} = (-1)^k H_k conj(e^{ik th})
            double2 w = cmul(H, cconj(e));
            if (k & 1) w = make_double2(-w.x, -w.y);
            h[K - k] = w;
        }
        e = cmul(e, u);
    }
}
