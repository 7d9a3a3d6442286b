// Builds and packs the library's hierarchical boundary matrix for a surface read
// from a binary file, then applies it to B vectors through the packed layout with
// a plain reference product written here (t = V x_sigma for every low-rank leaf;
// then every row owner sums its entries in the listed order -- dense rows times
// x_sigma, or rows of U times t -- and writes its rows) and writes the leaf table
// and y.
//   input : int32 N, nb, F, n_min, threads, B; double eta, eps; double xyz[N*3];
//           int32 bidx[nb]; int32 tris[F*3]; double x[nb*B] (position-major)
//   output: "error <message>\n", or "ok" then int32 n_leaves; per leaf int32 row_begin, m,
//           col_begin, n, kind, rank; int32 n_idx, idx[n_idx] (all clusters' positions);
//           double y[nb*B]
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "lbm_host.h"

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* in = fopen(argv[1], "rb");
    if (!in) return 3;
    int32_t hdr[6];
    double par[2];
    if (fread(hdr, 4, 6, in) != 6 || fread(par, 8, 2, in) != 2) return 4;
    const int N = hdr[0], nb = hdr[1], F = hdr[2], n_min = hdr[3], threads = hdr[4], B = hdr[5];
    std::vector<double> xyz(3 * (size_t)N), x((size_t)nb * B);
    std::vector<int32_t> bidx((size_t)nb), tris(3 * (size_t)F);
    if (fread(xyz.data(), 8, xyz.size(), in) != xyz.size()) return 5;
    if (fread(bidx.data(), 4, bidx.size(), in) != bidx.size()) return 6;
    if (fread(tris.data(), 4, tris.size(), in) != tris.size()) return 7;
    if (fread(x.data(), 8, x.size(), in) != x.size()) return 8;
    fclose(in);
    lbm::HMatrixHost H;
    lbm::HPacked P;
    std::string why = lbm::host_hmatrix_build(N, xyz.data(), nb, bidx.data(), F, tris.data(), par[0], n_min, par[1],
                                              threads, H);
    if (why.empty()) why = lbm::host_hmatrix_pack(H, nb, P);
    FILE* out = fopen(argv[2], "wb");
    if (!out) return 9;
    if (!why.empty()) {
        fprintf(out, "error %s\n", why.c_str());
        fclose(out);
        return 0;
    }
    // pass 1: t = V x_sigma of every low-rank leaf
    std::vector<double> t(P.n_t * (size_t)B, 0.0), y((size_t)nb * B, 0.0);
    for (const auto& e : P.leaves) {
        if (!e.kind) continue;
        const float* V = P.values.data() + e.val;
        const int* Cc = P.idx.data() + e.col_begin;
        for (int l = 0; l < e.rank; ++l)
            for (int c = 0; c < B; ++c) {
                double s = 0.0;
                for (int b = 0; b < e.n; ++b) s += (double)V[(size_t)l * e.n + b] * x[(size_t)Cc[b] * B + c];
                t[(e.t_off + l) * B + c] = s;
            }
    }
    // pass 2: every row owner sums its entries in order and writes its rows once
    for (size_t o = 0; o + 1 < P.owner_ptr.size(); ++o) {
        const int* own = P.idx.data() + P.owner_begin[o];
        const int rows = P.owner_size[o];
        std::vector<double> acc((size_t)rows * B, 0.0);
        for (size_t q = P.owner_ptr[o]; q < P.owner_ptr[o + 1]; ++q) {
            const auto& en = P.entries[q];
            const auto& e = P.leaves[en.leaf];
            const int* rm = P.row_map.data() + en.rows;
            const float* v = P.values.data() + e.val;
            const int* Cc = P.idx.data() + e.col_begin;
            for (int a = 0; a < rows; ++a)
                for (int c = 0; c < B; ++c) {
                    double s = 0.0;
                    if (!e.kind) {
                        for (int b = 0; b < e.n; ++b) s += (double)v[(size_t)rm[a] * e.n + b] * x[(size_t)Cc[b] * B + c];
                    } else {
                        const float* U = v + (size_t)e.rank * e.n;
                        for (int l = 0; l < e.rank; ++l) s += (double)U[(size_t)rm[a] * e.rank + l] * t[(e.t_off + l) * B + c];
                    }
                    acc[(size_t)a * B + c] += s;
                }
        }
        for (int a = 0; a < rows; ++a)
            for (int c = 0; c < B; ++c) y[(size_t)own[a] * B + c] = acc[(size_t)a * B + c];
    }
    fwrite("ok", 1, 2, out);
    const int32_t nl = (int32_t)P.leaves.size();
    fwrite(&nl, 4, 1, out);
    for (const auto& e : P.leaves) {
        const int32_t d[6] = {e.row_begin, e.m, e.col_begin, e.n, e.kind, e.rank};
        fwrite(d, 4, 6, out);
    }
    const int32_t ni = (int32_t)P.idx.size();
    fwrite(&ni, 4, 1, out);
    fwrite(P.idx.data(), 4, P.idx.size(), out);
    fwrite(y.data(), 8, y.size(), out);
    fclose(out);
    return 0;
}
