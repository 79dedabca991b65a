// Command-line harness for the host dense algebra of the solvers (paper_2608_26875_b300/csrc/dense_host.h),
// built and driven by tests/test_host_dense.py without a GPU.
//
//   host_dense_check <mode> <in> <out>
//
// <in> and <out> are flat little-endian files: int32 sizes first, then complex128 (or float64) arrays
// in the order listed per mode below.
//   chol    in: s, G[s][s]                     out: ok (int32), R[s][s]
//   triinv  in: s, R[s][s]                     out: Ri[s][s]
//   jacobi  in: n, A (n x n column-major)      out: ev[n] (float64), V (column-major), A after rotation
//   lsq     in: s, m, H[(m+1)s][m s], S0[s][s], floor_rel (float64)
//           out: Y[m s][s], residual estimate per column after the last step (float64[s])
//   The lsq mode runs the block GMRES least-squares sequence: per block column j, the earlier steps'
//   reflectors on the new column, the step's Householder QR of its 2s x s panel, the step applied to
//   the transformed right-hand side g = [S0; 0], and at the end the truncated block back substitution.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dense_host.h"

using dense::cd;

namespace {

struct Reader {
    FILE* f;
    int32_t i32() {
        int32_t v = 0;
        if (fread(&v, sizeof v, 1, f) != 1) throw 1;
        return v;
    }
    double f64() {
        double v = 0;
        if (fread(&v, sizeof v, 1, f) != 1) throw 1;
        return v;
    }
    std::vector<cd> c128(size_t n) {
        std::vector<cd> v(n);
        if (n && fread(v.data(), sizeof(cd), n, f) != n) throw 1;
        return v;
    }
};

void put(FILE* f, const void* p, size_t bytes) {
    if (bytes && fwrite(p, 1, bytes, f) != bytes) throw 2;
}

}  // namespace

int main(int argc, char** argv) {
    if (argc != 4) return 2;
    const std::string mode = argv[1];
    FILE* fi = fopen(argv[2], "rb");
    FILE* fo = fopen(argv[3], "wb");
    if (!fi || !fo) return 3;
    Reader in{fi};
    try {
        if (mode == "chol") {
            const int s = in.i32();
            const std::vector<cd> G = in.c128((size_t)s * s);
            std::vector<cd> R;
            const int32_t ok = dense::chol_upper(G, s, 0.0, R) ? 1 : 0;
            R.resize((size_t)s * s);
            put(fo, &ok, sizeof ok);
            put(fo, R.data(), R.size() * sizeof(cd));
        } else if (mode == "triinv") {
            const int s = in.i32();
            const std::vector<cd> R = in.c128((size_t)s * s);
            std::vector<cd> Ri;
            dense::tri_inv_upper(R, s, Ri);
            put(fo, Ri.data(), Ri.size() * sizeof(cd));
        } else if (mode == "jacobi") {
            const int n = in.i32();
            std::vector<cd> A = in.c128((size_t)n * n), V;
            std::vector<double> ev;
            dense::jacobi_svd(A, n, ev, V);
            put(fo, ev.data(), ev.size() * sizeof(double));
            put(fo, V.data(), V.size() * sizeof(cd));
            put(fo, A.data(), A.size() * sizeof(cd));
        } else if (mode == "lsq") {
            const int s = in.i32(), m = in.i32();
            const int rows = (m + 1) * s, cols = m * s;
            const std::vector<cd> H = in.c128((size_t)rows * cols);
            const std::vector<cd> S0 = in.c128((size_t)s * s);
            const double floor_rel = in.f64();
            std::vector<cd> g((size_t)rows * s, cd(0));
            for (size_t i = 0; i < S0.size(); ++i) g[i] = S0[i];
            std::vector<std::vector<cd>> Rcol;
            std::vector<dense::StepQR> qr;
            std::vector<double> res(s, 0.0);
            for (int j = 0; j < m; ++j) {
                const int nb = (j + 1) * s;
                std::vector<cd> hcol((size_t)(nb + s) * s);
                for (int r = 0; r < nb + s; ++r)
                    for (int c = 0; c < s; ++c) hcol[(size_t)r * s + c] = H[(size_t)r * cols + j * s + c];
                dense::apply_steps(qr, 0, j, s, hcol.data());
                dense::StepQR q;
                dense::step_qr(&hcol[(size_t)(j * s) * s], s, q);
                qr.push_back(std::move(q));
                dense::apply_steps(qr, j, j + 1, s, g.data());
                Rcol.emplace_back(hcol.begin(), hcol.begin() + (size_t)nb * s);
                for (int c = 0; c < s; ++c) {
                    double r2 = 0;
                    for (int i = 0; i < s; ++i) r2 += std::norm(g[(size_t)(nb + i) * s + c]);
                    res[c] = sqrt(r2);
                }
            }
            std::vector<cd> Y;
            dense::block_back_substitute(Rcol, g, s, m, floor_rel, Y);
            put(fo, Y.data(), Y.size() * sizeof(cd));
            put(fo, res.data(), res.size() * sizeof(double));
        } else {
            return 4;
        }
    } catch (int e) {
        return 10 + e;
    }
    fclose(fi);
    fclose(fo);
    return 0;
}
