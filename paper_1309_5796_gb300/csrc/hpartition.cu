// Host set-up of a hierarchical (H-matrix) form of the boundary matrix B:
// support boxes of the surface hat functions, the cluster tree over the boundary
// positions and the leaves of the block tree with their admissibility.
//
// The paper (Sec. 3.1) names hierarchical matrices as the way its comparison
// solver speeds up the boundary element method, without a construction; this is
// the textbook one (geometric bisection, standard admissibility):
//   * a cluster holding more than n_min positions is split in two: its nodes are
//     ordered by their coordinate along the longest side of their bounding box
//     (ties by position) and the first floor(m/2) form the first child;
//   * a block (tau, sigma) is admissible when dist(Q_r(tau), Q_c(sigma)) > 0 and
//     min(diam Q_r(tau), diam Q_c(sigma)) <= eta dist(Q_r(tau), Q_c(sigma)), with
//     Q_r the box of the collocation points and Q_c the box of the supports
//     (surface triangles around each node) of the column hat functions;
//   * from (root, root): admissible -> low-rank leaf; a leaf cluster on either
//     side -> dense leaf; else the four children blocks, (a,a), (a,b), (b,a), (b,b).
// Lengths are sqrt(x*x + y*y + z*z) summed in that order; this file is compiled
// without floating-point contraction so that every decision is the same on any
// host.  Host code only; no kernel lives here.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "lbm_host.h"

namespace lbm {

namespace {

double length3(double x, double y, double z) {
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    return std::sqrt(x2 + y2 + z2);
}

double box_diam(const double* lo, const double* hi) { return length3(hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]); }

double box_dist(const double* lo1, const double* hi1, const double* lo2, const double* hi2) {
    double g[3];
    for (int d = 0; d < 3; ++d) g[d] = std::max(0.0, std::max(lo1[d] - hi2[d], lo2[d] - hi1[d]));
    return length3(g[0], g[1], g[2]);
}

}  // namespace

void host_support_boxes(int N, const double* xyz, int nb, const int* bidx, int F, const int* tris, double* lo,
                        double* hi) {
    std::vector<int> pos((size_t)N, -1);
    for (int j = 0; j < nb; ++j) pos[bidx[j]] = j;
    for (int j = 0; j < nb; ++j)
        for (int d = 0; d < 3; ++d) {
            lo[3 * j + d] = INFINITY;
            hi[3 * j + d] = -INFINITY;
        }
    for (int t = 0; t < F; ++t) {
        const int* v = tris + 3 * t;
        double tlo[3], thi[3];
        for (int d = 0; d < 3; ++d) {
            tlo[d] = std::min(std::min(xyz[3 * v[0] + d], xyz[3 * v[1] + d]), xyz[3 * v[2] + d]);
            thi[d] = std::max(std::max(xyz[3 * v[0] + d], xyz[3 * v[1] + d]), xyz[3 * v[2] + d]);
        }
        for (int k = 0; k < 3; ++k) {
            const int j = pos[v[k]];
            if (j < 0) continue;
            for (int d = 0; d < 3; ++d) {
                lo[3 * j + d] = std::min(lo[3 * j + d], tlo[d]);
                hi[3 * j + d] = std::max(hi[3 * j + d], thi[d]);
            }
        }
    }
}

std::string host_hmatrix_partition(int nb, const double* pts, const double* slo, const double* shi, double eta,
                                   int n_min, HPartition& P) {
    if (nb <= 0) return "no boundary positions";
    if (n_min < 1) return "n_min must be at least 1";
    if (!(eta > 0.0) || !std::isfinite(eta)) return "eta must be positive and finite";
    for (int j = 0; j < nb; ++j)
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(pts[3 * j + d]) || !(slo[3 * j + d] <= pts[3 * j + d]) ||
                !(pts[3 * j + d] <= shi[3 * j + d]))
                return "boundary position " + std::to_string(j) + " lies outside its support box";
    P = HPartition{};
    auto make = [&](std::vector<int> idx) {
        HCluster c;
        c.begin = (int)P.idx.size();
        c.size = (int)idx.size();
        for (int d = 0; d < 3; ++d) {
            c.lo_r[d] = c.lo_c[d] = INFINITY;
            c.hi_r[d] = c.hi_c[d] = -INFINITY;
        }
        for (int j : idx)
            for (int d = 0; d < 3; ++d) {
                c.lo_r[d] = std::min(c.lo_r[d], pts[3 * j + d]);
                c.hi_r[d] = std::max(c.hi_r[d], pts[3 * j + d]);
                c.lo_c[d] = std::min(c.lo_c[d], slo[3 * j + d]);
                c.hi_c[d] = std::max(c.hi_c[d], shi[3 * j + d]);
            }
        P.idx.insert(P.idx.end(), idx.begin(), idx.end());
        P.clusters.push_back(c);
        return (int)P.clusters.size() - 1;
    };
    std::vector<int> all(nb);
    std::iota(all.begin(), all.end(), 0);
    make(all);
    for (size_t c = 0; c < P.clusters.size(); ++c) {      // breadth-first; appends while it walks
        const HCluster cl = P.clusters[c];
        if (cl.size <= n_min) continue;
        int axis = 0;
        for (int d = 1; d < 3; ++d)
            if (cl.hi_r[d] - cl.lo_r[d] > cl.hi_r[axis] - cl.lo_r[axis]) axis = d;
        std::vector<int> order(P.idx.begin() + cl.begin, P.idx.begin() + cl.begin + cl.size);
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            const double xa = pts[3 * a + axis], xb = pts[3 * b + axis];
            return xa < xb || (xa == xb && a < b);
        });
        const int half = cl.size / 2;
        std::vector<int> a(order.begin(), order.begin() + half), b(order.begin() + half, order.end());
        std::sort(a.begin(), a.end());
        std::sort(b.begin(), b.end());
        const int ca = make(std::move(a));
        const int cb = make(std::move(b));
        P.clusters[c].child[0] = ca;
        P.clusters[c].child[1] = cb;
    }
    auto admissible = [&](const HCluster& t, const HCluster& s) {
        const double d = box_dist(t.lo_r, t.hi_r, s.lo_c, s.hi_c);
        return d > 0.0 && std::min(box_diam(t.lo_r, t.hi_r), box_diam(s.lo_c, s.hi_c)) <= eta * d;
    };
    std::vector<std::pair<int, int>> stack{{0, 0}};        // depth-first, children in (a,a) (a,b) (b,a) (b,b) order
    while (!stack.empty()) {
        const auto [t, s] = stack.back();
        stack.pop_back();
        const HCluster &ct = P.clusters[t], &cs = P.clusters[s];
        if (admissible(ct, cs)) {
            P.leaves.push_back({t, s, 1});
        } else if (ct.child[0] < 0 || cs.child[0] < 0) {
            P.leaves.push_back({t, s, 0});
        } else {
            for (int i = 1; i >= 0; --i)
                for (int k = 1; k >= 0; --k) stack.push_back({ct.child[i], cs.child[k]});
        }
    }
    return {};
}

}  // namespace lbm
