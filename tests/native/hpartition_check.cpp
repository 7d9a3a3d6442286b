// Runs the library's host set-up of the hierarchical boundary matrix (support
// boxes, cluster tree, block-tree leaves) on a surface read from a binary file
// and writes what it built, for comparison with the CPU oracle.
//   input : int32 N, nb, F, n_min; double eta; double xyz[N*3]; int32 bidx[nb]; int32 tris[F*3]
//   output: "error <message>\n", or "ok" then double lo[nb*3], hi[nb*3]; int32 n_clusters and, per
//           cluster (breadth-first), int32 size, positions; int32 n_leaves and, per leaf
//           (depth-first), int32 row cluster, column cluster, low_rank
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "lbm_host.h"

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* in = fopen(argv[1], "rb");
    if (!in) return 3;
    int32_t hdr[4];
    double eta = 0.0;
    if (fread(hdr, 4, 4, in) != 4 || fread(&eta, 8, 1, in) != 1) return 4;
    const int N = hdr[0], nb = hdr[1], F = hdr[2], n_min = hdr[3];
    std::vector<double> xyz(3 * (size_t)N);
    std::vector<int32_t> bidx((size_t)nb), tris(3 * (size_t)F);
    if (fread(xyz.data(), 8, xyz.size(), in) != xyz.size()) return 5;
    if (fread(bidx.data(), 4, bidx.size(), in) != bidx.size()) return 6;
    if (fread(tris.data(), 4, tris.size(), in) != tris.size()) return 7;
    fclose(in);
    std::vector<double> lo(3 * (size_t)nb), hi(3 * (size_t)nb), pts(3 * (size_t)nb);
    lbm::host_support_boxes(N, xyz.data(), nb, bidx.data(), F, tris.data(), lo.data(), hi.data());
    for (int j = 0; j < nb; ++j)
        for (int d = 0; d < 3; ++d) pts[3 * j + d] = xyz[3 * (size_t)bidx[j] + d];
    lbm::HPartition P;
    const std::string why = lbm::host_hmatrix_partition(nb, pts.data(), lo.data(), hi.data(), eta, n_min, P);
    FILE* out = fopen(argv[2], "wb");
    if (!out) return 8;
    if (!why.empty()) {
        fprintf(out, "error %s\n", why.c_str());
        fclose(out);
        return 0;
    }
    fwrite("ok", 1, 2, out);
    fwrite(lo.data(), 8, lo.size(), out);
    fwrite(hi.data(), 8, hi.size(), out);
    const int32_t nc = (int32_t)P.clusters.size();
    fwrite(&nc, 4, 1, out);
    for (const auto& c : P.clusters) {
        fwrite(&c.size, 4, 1, out);
        fwrite(P.idx.data() + c.begin, 4, (size_t)c.size, out);
    }
    const int32_t nl = (int32_t)P.leaves.size();
    fwrite(&nl, 4, 1, out);
    for (const auto& L : P.leaves) {
        const int32_t v[3] = {L.row, L.col, L.low_rank};
        fwrite(v, 4, 3, out);
    }
    fclose(out);
    return 0;
}
