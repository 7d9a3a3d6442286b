// Packing of a built hierarchical boundary matrix (csrc/hbuild.cu) into the
// flat FP32 layout a device product reads, y = B_H x for B instances at once,
// in two passes:
//   1. t_l = V_l x_sigma(l) for every low-rank leaf l (k_l x B values: small);
//   2. every leaf of the cluster tree (a "row owner": at most n_min positions,
//      together they partition the positions) forms its rows of y as the sum,
//      in block-tree order, of the contributions of all block-tree leaves whose
//      row cluster contains it -- rows of a dense leaf times x_sigma, or rows of
//      U_l times t_l -- and writes them once.  No two owners share a position,
//      so the result needs no atomics and its summation order is fixed.
// Layout: the leaves in the order (kind, rows, columns, block-tree position),
// dense first, each group by size (one shape per thread group); FP32 values, a
// dense leaf's m x n entries row-major, a low-rank leaf's V (k x n) then U (m x k),
// both row-major; per owner its entries (leaf, offset of its local rows in
// row_map), in block-tree order.  Host code only; no kernel lives here.
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
    P.idx = H.P.idx;
    std::vector<size_t> order(L);
    std::iota(order.begin(), order.end(), 0);
    auto shape = [&](size_t l) {
        const HLeaf& lf = H.P.leaves[l];
        return std::make_tuple(H.kind[l], H.P.clusters[lf.row].size, H.P.clusters[lf.col].size);
    };
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return shape(a) < shape(b); });
    std::vector<int> packed_of(L);                   // block-tree leaf -> packed index
    P.leaves.resize(L);
    size_t vals = 0, ts = 0;
    for (size_t q = 0; q < L; ++q) {
        const size_t l = order[q];
        packed_of[l] = (int)q;
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
        e.t_off = ts;
        vals += e.kind ? (size_t)e.rank * (e.m + e.n) : (size_t)e.m * e.n;
        if (e.kind) ts += (size_t)e.rank;
    }
    P.n_t = ts;
    P.values.resize(vals);
    P.values64.resize(vals);
    for (size_t q = 0; q < L; ++q) {
        const size_t l = order[q];
        const HPackedLeaf& e = P.leaves[q];
        const double* src = H.data.data() + H.off[l];
        double* dst = P.values64.data() + e.val;
        if (!e.kind) {
            for (size_t i = 0; i < (size_t)e.m * e.n; ++i) dst[i] = src[i];
        } else {
            const size_t nu = (size_t)e.m * e.rank, nv = (size_t)e.rank * e.n;
            for (size_t i = 0; i < nv; ++i) dst[i] = src[nu + i];        // V first
            for (size_t i = 0; i < nu; ++i) dst[nv + i] = src[i];        // then U
        }
    }
    for (size_t i = 0; i < vals; ++i) P.values[i] = (float)P.values64[i];
    // row owners: the leaves of the cluster tree, in cluster order
    std::vector<int> owner_of_cluster(H.P.clusters.size(), -1);
    for (size_t c = 0; c < H.P.clusters.size(); ++c)
        if (H.P.clusters[c].child[0] < 0) {
            owner_of_cluster[c] = (int)P.owner_begin.size();
            P.owner_begin.push_back(H.P.clusters[c].begin);
            P.owner_size.push_back(H.P.clusters[c].size);
        }
    std::vector<std::vector<HPackedEntry>> per(P.owner_begin.size());
    std::vector<int> stack;
    for (size_t l = 0; l < L; ++l) {                 // block-tree order
        const int tau = H.P.leaves[l].row;
        const HCluster& ct = H.P.clusters[tau];
        const int* tb = H.P.idx.data() + ct.begin;
        stack.assign(1, tau);
        while (!stack.empty()) {                     // the cluster-tree leaves under tau
            const int c = stack.back();
            stack.pop_back();
            const HCluster& cc = H.P.clusters[c];
            if (cc.child[0] >= 0) {
                stack.push_back(cc.child[1]);
                stack.push_back(cc.child[0]);
                continue;
            }
            HPackedEntry en;
            en.leaf = packed_of[l];
            en.rows = P.row_map.size();
            for (int a = 0; a < cc.size; ++a) {      // local row in tau of each owned position
                const int p = H.P.idx[cc.begin + a];
                const int* it = std::lower_bound(tb, tb + ct.size, p);
                if (it == tb + ct.size || *it != p) return "cluster tree is not nested";
                P.row_map.push_back((int)(it - tb));
            }
            per[owner_of_cluster[c]].push_back(en);
        }
    }
    P.owner_ptr.assign(per.size() + 1, 0);
    for (size_t o = 0; o < per.size(); ++o) P.owner_ptr[o + 1] = P.owner_ptr[o] + per[o].size();
    P.entries.reserve(P.owner_ptr.back());
    for (const auto& v : per) P.entries.insert(P.entries.end(), v.begin(), v.end());
    return {};
}

void host_hmatrix_transpose(const HMatrixHost& H, HMatrixHost& T) {
    T = HMatrixHost{};
    T.P = H.P;
    T.kind = H.kind;
    T.rank = H.rank;
    T.fallbacks = H.fallbacks;
    T.off.resize(H.off.size());
    T.data.resize(H.data.size());
    for (size_t l = 0; l < H.P.leaves.size(); ++l) {
        HLeaf& lf = T.P.leaves[l];
        std::swap(lf.row, lf.col);
        const int m = H.P.clusters[H.P.leaves[l].row].size, n = H.P.clusters[H.P.leaves[l].col].size;
        const double* src = H.data.data() + H.off[l];
        double* dst = T.data.data() + H.off[l];
        T.off[l] = H.off[l];
        if (!H.kind[l]) {                               // m x n -> n x m
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < n; ++j) dst[(size_t)j * m + i] = src[(size_t)i * n + j];
        } else {                                        // U (m x k), V (k x n) -> V^T (n x k), U^T (k x m)
            const int k = H.rank[l];
            const double* U = src;
            const double* V = src + (size_t)m * k;
            double* Ut = dst;                           // new U = V^T, n x k
            double* Vt = dst + (size_t)n * k;           // new V = U^T, k x m
            for (int j = 0; j < n; ++j)
                for (int a = 0; a < k; ++a) Ut[(size_t)j * k + a] = V[(size_t)a * n + j];
            for (int a = 0; a < k; ++a)
                for (int i = 0; i < m; ++i) Vt[(size_t)a * m + i] = U[(size_t)i * k + a];
        }
    }
}

}  // namespace lbm
