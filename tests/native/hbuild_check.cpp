// Runs the library's host construction of the hierarchical boundary matrix on a
// surface read from a binary file and writes the leaves and their values.
//   input : int32 N, nb, F, n_min, threads; double eta, eps; double xyz[N*3]; int32 bidx[nb]; int32 tris[F*3]
//   output: "error <message>\n", or "ok" then int32 n_leaves, fallbacks and, per leaf
//           (depth-first): int32 m, n, kind, rank, the m row and n column positions,
//           then the leaf's values (m*n dense, or m*k + k*n factors) as doubles
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "lbm_host.h"

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* in = fopen(argv[1], "rb");
    if (!in) return 3;
    int32_t hdr[5];
    double par[2];
    if (fread(hdr, 4, 5, in) != 5 || fread(par, 8, 2, in) != 2) return 4;
    const int N = hdr[0], nb = hdr[1], F = hdr[2], n_min = hdr[3], threads = hdr[4];
    std::vector<double> xyz(3 * (size_t)N);
    std::vector<int32_t> bidx((size_t)nb), tris(3 * (size_t)F);
    if (fread(xyz.data(), 8, xyz.size(), in) != xyz.size()) return 5;
    if (fread(bidx.data(), 4, bidx.size(), in) != bidx.size()) return 6;
    if (fread(tris.data(), 4, tris.size(), in) != tris.size()) return 7;
    fclose(in);
    lbm::HMatrixHost H;
    const std::string why =
        lbm::host_hmatrix_build(N, xyz.data(), nb, bidx.data(), F, tris.data(), par[0], n_min, par[1], threads, H);
    FILE* out = fopen(argv[2], "wb");
    if (!out) return 8;
    if (!why.empty()) {
        fprintf(out, "error %s\n", why.c_str());
        fclose(out);
        return 0;
    }
    fwrite("ok", 1, 2, out);
    const int32_t head[2] = {(int32_t)H.P.leaves.size(), H.fallbacks};
    fwrite(head, 4, 2, out);
    for (size_t l = 0; l < H.P.leaves.size(); ++l) {
        const auto& ct = H.P.clusters[H.P.leaves[l].row];
        const auto& cs = H.P.clusters[H.P.leaves[l].col];
        const int32_t d[4] = {ct.size, cs.size, H.kind[l], H.rank[l]};
        fwrite(d, 4, 4, out);
        fwrite(H.P.idx.data() + ct.begin, 4, (size_t)ct.size, out);
        fwrite(H.P.idx.data() + cs.begin, 4, (size_t)cs.size, out);
        const size_t cnt = H.kind[l] ? (size_t)H.rank[l] * (ct.size + cs.size) : (size_t)ct.size * cs.size;
        fwrite(H.data.data() + H.off[l], 8, cnt, out);
    }
    fclose(out);
    return 0;
}
