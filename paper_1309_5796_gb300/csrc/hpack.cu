// Packing of a built hierarchical boundary matrix (csrc/hbuild.cu) into the
// flat FP32 layout a device product reads, y = B_H x for B instances at once:
//   * leaves in the order (kind, rows, columns, block-tree position): dense leaves
//     first, then low-rank ones, each group by size, so that a launch can give
//     leaves of one shape to one kind of thread group;
//   * values in FP32: a dense leaf's m x n entries (row-major); a low-rank leaf's
//     V (k x n, row-major) followed by U (m x k, row-major), in the order the
//     product uses them (t = V x_sigma, then y_tau += U t);
//   * every leaf writes its m rows of the product to its own output slots (no two
//     leaves share a slot), and a second pass adds, for every boundary position,
//     the slots of the leaves whose row cluster holds it, in block-tree order:
//     the sum's order is fixed by the block tree, whatever order the leaves run in.
// Host code only; no kernel lives here.
#include <algorithm>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "lbm_host.h"

namespace lbm {

std::string host_hmatrix_pack(const HMatrixHost& H, int nb, HPacked& P) {
    const size_t L = H.P.leaves.size();
    if (H.kind.size() != L || H.rank.size() != L || H.off.size() != L) return "inconsistent operator";
    P = HPacked{};
    P.nb = nb;
    std::vector<size_t> order(L);
    std::iota(order.begin(), order.end(), 0);
    auto shape = [&](size_t l) {
        const HLeaf& lf = H.P.leaves[l];
        return std::make_tuple(H.kind[l], H.P.clusters[lf.row].size, H.P.clusters[lf.col].size);
    };
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return shape(a) < shape(b); });
    P.leaves.resize(L);
    size_t vals = 0, slots = 0;
    std::vector<size_t> slot_of(L);                  // first output slot of each leaf (block-tree index)
    for (size_t q = 0; q < L; ++q) {
        const size_t l = order[q];
        const HLeaf& lf = H.P.leaves[l];
        const HCluster& ct = H.P.clusters[lf.row];
        const HCluster& cs = H.P.clusters[lf.col];
        HPackedLeaf& e = P.leaves[q];
        e.row_begin = ct.begin;
        e.m = ct.size;
        e.col_begin = cs.begin;
        e.n = cs.size;
        e.kind = H.kind[l];
        e.rank = H.rank[l];
        e.val = vals;
        e.slot = slots;
        slot_of[l] = slots;
        vals += e.kind ? (size_t)e.rank * (e.m + e.n) : (size_t)e.m * e.n;
        slots += e.m;
    }
    P.idx = H.P.idx;
    P.values.resize(vals);
    for (size_t q = 0; q < L; ++q) {
        const size_t l = order[q];
        const HPackedLeaf& e = P.leaves[q];
        const double* src = H.data.data() + H.off[l];
        float* dst = P.values.data() + e.val;
        if (!e.kind) {
            for (size_t i = 0; i < (size_t)e.m * e.n; ++i) dst[i] = (float)src[i];
        } else {
            const size_t nu = (size_t)e.m * e.rank, nv = (size_t)e.rank * e.n;
            for (size_t i = 0; i < nv; ++i) dst[i] = (float)src[nu + i];        // V first
            for (size_t i = 0; i < nu; ++i) dst[nv + i] = (float)src[i];        // then U
        }
    }
    P.n_slots = slots;
    // boundary position -> its slots, in block-tree order of the leaves
    std::vector<std::vector<size_t>> per(nb);
    for (size_t l = 0; l < L; ++l) {
        const HCluster& ct = H.P.clusters[H.P.leaves[l].row];
        for (int a = 0; a < ct.size; ++a) {
            const int p = H.P.idx[ct.begin + a];
            if (p < 0 || p >= nb) return "position out of range";
            per[p].push_back(slot_of[l] + a);
        }
    }
    P.row_ptr.assign(nb + 1, 0);
    for (int p = 0; p < nb; ++p) P.row_ptr[p + 1] = P.row_ptr[p] + per[p].size();
    P.row_slots.resize(P.row_ptr[nb]);
    for (int p = 0; p < nb; ++p) std::copy(per[p].begin(), per[p].end(), P.row_slots.begin() + P.row_ptr[p]);
    return {};
}

}  // namespace lbm
