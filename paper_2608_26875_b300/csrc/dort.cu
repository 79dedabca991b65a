// Time-reversal matrix of a mirror in the upper layer (Sec. 7.5, the DORT method): point forces at the
// mirror's n points, x and y polarised, are the 2n incident fields (point-source incidence, Sec. 7.2);
// one batched solve gives the 2n scattered fields, whose values at the mirror points in the upper
// layer form the response matrix
//     F[(i, c), (j, d)] = component c at mirror point i of the field scattered under the force e_d at point j,
// and T = conj(F)^T F.  Eigenvalues and eigenvectors of T come from one-sided Jacobi on F: the columns
// of F are orthogonalised by plane rotations, so T's eigenvalues are the squared column norms and its
// eigenvectors the accumulated rotations (the densities that focus on single particles).
#include <math.h>

#include <algorithm>
#include <complex>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "dense_host.h"
#include "handle.h"

typedef std::complex<double> cd;


extern "C" int ms_time_reversal(ms_handle* h, const double* trm, int32_t n, double tol, int32_t prec, double* F,
                                double* eig, double* vec, ms_solve_info* info, void* stream) {
    if (!h || !trm || n < 1 || !(tol > 0) || (!F && !eig && !vec)) return MS_ERR_ARG;
    if (2 * n > 64) return MS_ERR_UNSUPPORTED;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(trm[2 * i]) || !(trm[2 * i + 1] > 0)) return MS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int nr = 2 * n;
    std::vector<double> src((size_t)2 * nr), force((size_t)2 * nr, 0.0);
    for (int j = 0; j < n; ++j)
        for (int d = 0; d < 2; ++d) {
            src[2 * (2 * j + d)] = trm[2 * j];
            src[2 * (2 * j + d) + 1] = trm[2 * j + 1];
            force[2 * (2 * j + d) + d] = 1.0;
        }
    const size_t nvec = (size_t)h->M * 2 * h->nc * nr;
    double2 *b = nullptr, *g = nullptr, *u = nullptr;
    double* rx = nullptr;
    int rc;
    if ((rc = ms_check(h, cudaMalloc(&b, nvec * sizeof(double2)))) ||
        (rc = ms_check(h, cudaMalloc(&g, nvec * sizeof(double2)))) ||
        (rc = ms_check(h, cudaMalloc(&u, (size_t)nr * n * 2 * sizeof(double2)))) ||
        (rc = ms_check(h, cudaMalloc(&rx, (size_t)n * 2 * sizeof(double))))) {
        cudaFree(b); cudaFree(g); cudaFree(u); cudaFree(rx);
        return rc;
    }
    std::vector<double2> uh((size_t)nr * n * 2);
    rc = ms_rhs_point(h, src.data(), force.data(), nr, b, stream);
    int solve_rc = MS_OK;
    if (!rc) {
        solve_rc = ms_solve_rhs(h, b, nr, tol, prec, g, 0, info, stream);
        if (solve_rc < 0) rc = solve_rc;
    }
    if (!rc) rc = ms_check(h, cudaMemcpyAsync(rx, trm, (size_t)n * 2 * sizeof(double), cudaMemcpyHostToDevice, st));
    if (!rc) rc = ms_fields_upper_impl(h, g, nr, rx, n, u, st);
    if (!rc) rc = ms_check(h, cudaMemcpyAsync(uh.data(), u, uh.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = ms_check(h, cudaStreamSynchronize(st));
    cudaFree(b); cudaFree(g); cudaFree(u); cudaFree(rx);
    if (rc) return rc;
    // F row (i, c) = 2i + c, column (j, d) = 2j + d: u[(2j + d)][i][c]
    std::vector<cd> Fc((size_t)nr * nr);                 // column-major
    for (int col = 0; col < nr; ++col)
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 2; ++c) {
                const double2 v = uh[((size_t)col * n + i) * 2 + c];
                Fc[(size_t)col * nr + 2 * i + c] = cd(v.x, v.y);
            }
    if (F)
        for (int row = 0; row < nr; ++row)
            for (int col = 0; col < nr; ++col) {
                F[2 * ((size_t)row * nr + col)] = Fc[(size_t)col * nr + row].real();
                F[2 * ((size_t)row * nr + col) + 1] = Fc[(size_t)col * nr + row].imag();
            }
    if (eig || vec) {
        std::vector<double> ev;
        std::vector<cd> V;
        dense::jacobi_svd(Fc, nr, ev, V);
        std::vector<int> order(nr);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int a, int c) { return ev[a] > ev[c]; });
        for (int k = 0; k < nr; ++k) {
            if (eig) eig[k] = ev[order[k]];
            if (vec)
                for (int i = 0; i < nr; ++i) {
                    vec[2 * ((size_t)i * nr + k)] = V[(size_t)order[k] * nr + i].real();
                    vec[2 * ((size_t)i * nr + k) + 1] = V[(size_t)order[k] * nr + i].imag();
                }
        }
    }
    return solve_rc;
}
