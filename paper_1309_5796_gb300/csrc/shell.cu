// Host set-up of the open boundary by space transformation (Sec. 3.1: the
// paper's own steepest-descent solver maps a shell onto the exterior instead of
// using a boundary element method).
//
// Geometry (lattice units h, magnet the cube [0, n]^3, centre c = n/2 (1,1,1),
// rho(x) = max_k |x_k - c_k|): air out to rho = R1 = n/2 + a, shell
// R1 <= rho <= R2 = R1 + s, one Kuhn grid of nt = n + 2(a + s) cells a side
// over all three (node (i,j,k) of the grid at lattice point (i,j,k) - (a+s),
// ids and tetrahedra as for the magnet's own Kuhn cube).  The shell is mapped
// onto rho' >= R1 by x' - c = sig(rho) (x - c), sig = g/rho,
// g = R1 (R2 - R1)/(R2 - rho); in the sector where coordinate k attains the max
// (the first such k), grad rho = sign(x_k - c_k) e_k and
//     J = sig I + sig' (x - c) grad rho^T,    det J = sig^2 g',
//     J^-1 = (I - (sig'/g') (x - c) grad rho^T) / sig   (Sherman-Morrison,
//            using sig + sig' rho = g'),
// and the Laplace form over the exterior becomes the form of the tensor
// M = |det J| J^-1 J^-T over the shell (M = I in the magnet and the air), taken
// at each tetrahedron's centroid.  The stiffness is
//     K_ij = sum_e c_i^T M_e c_j / (6 |det_e|)
// (c the cofactor vectors of the tetrahedron, det = 6 x its signed volume), on
// the CSR pattern of the element adjacency (columns ascending), summed over the
// tetrahedra in their order.  u = 0 on the outer face (rho = R2, the image of
// infinity).  Host code only; no kernel lives here.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "lbm_host.h"

namespace lbm {

namespace {

// M = |det J| J^-1 J^-T at the point d = x - c (lattice units) of the shell.
void shell_tensor_at(const double d[3], double R1, double R2, double M[3][3]) {
    int k = 0;
    for (int q = 1; q < 3; ++q)
        if (std::fabs(d[q]) > std::fabs(d[k])) k = q;
    const double rho = std::fabs(d[k]);
    double gr[3] = {0.0, 0.0, 0.0};
    gr[k] = d[k] > 0.0 ? 1.0 : (d[k] < 0.0 ? -1.0 : 0.0);
    const double g = R1 * (R2 - R1) / (R2 - rho);
    const double dg = R1 * (R2 - R1) / ((R2 - rho) * (R2 - rho));
    const double sig = g / rho;
    const double dsig = (dg * rho - g) / (rho * rho);
    const double detJ = sig * sig * dg;
    double Ji[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ji[i][j] = ((i == j ? 1.0 : 0.0) - (dsig / dg) * d[i] * gr[j]) / sig;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double x = 0.0;
            for (int q = 0; q < 3; ++q) x += Ji[i][q] * Ji[j][q];
            M[i][j] = std::fabs(detJ) * x;
        }
}

}  // namespace

std::string host_shell_setup(int n, int a, int s, double cell, ShellGrid& G) {
    if (n < 1 || a < 1 || s < 1) return "n, a and s must be at least 1";
    if (!(cell > 0.0) || !std::isfinite(cell)) return "cell must be positive";
    const long long nt_ll = (long long)n + 2LL * (a + s);
    if (nt_ll > 400) return "grid too large (n + 2(a + s) > 400)";
    const int nt = (int)nt_ll, n1 = nt + 1, off = a + s;
    const size_t N = (size_t)n1 * n1 * n1;
    G = ShellGrid{};
    G.nt = nt;
    G.R1 = n / 2.0 + a;
    G.R2 = n / 2.0 + a + s;
    const double c = n / 2.0;
    auto id = [&](int i, int j, int k) { return i + n1 * (j + n1 * k); };
    // tetrahedra (cell-major, permutations in lexicographic order, odd ones with
    // their last two vertices swapped so that every volume is positive)
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const size_t T = (size_t)6 * nt * nt * nt;
    std::vector<int> tets(4 * T);
    for (int ck = 0, t = 0; ck < nt; ++ck)
        for (int cj = 0; cj < nt; ++cj)
            for (int ci = 0; ci < nt; ++ci)
                for (int p = 0; p < 6; ++p, ++t) {
                    int v[4][3] = {{ci, cj, ck}};
                    for (int q = 1; q < 4; ++q) {
                        for (int d = 0; d < 3; ++d) v[q][d] = v[q - 1][d];
                        ++v[q][perms[p][q - 1]];
                    }
                    const int* pm = perms[p];
                    const int inv = (pm[0] > pm[1]) + (pm[0] > pm[2]) + (pm[1] > pm[2]);
                    int ids[4] = {id(v[0][0], v[0][1], v[0][2]), id(v[1][0], v[1][1], v[1][2]),
                                  id(v[2][0], v[2][1], v[2][2]), id(v[3][0], v[3][1], v[3][2])};
                    if (inv % 2) std::swap(ids[2], ids[3]);
                    for (int q = 0; q < 4; ++q) tets[4 * (size_t)t + q] = ids[q];
                }
    // CSR pattern of the element adjacency
    std::vector<std::vector<int>> adj(N);
    for (size_t t = 0; t < T; ++t)
        for (int x = 0; x < 4; ++x)
            for (int y = 0; y < 4; ++y) adj[tets[4 * t + x]].push_back(tets[4 * t + y]);
    G.rowptr.assign(N + 1, 0);
    for (size_t i = 0; i < N; ++i) {
        auto& r = adj[i];
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        G.rowptr[i + 1] = G.rowptr[i] + (int)r.size();
    }
    G.col.resize(G.rowptr[N]);
    for (size_t i = 0; i < N; ++i) std::copy(adj[i].begin(), adj[i].end(), G.col.begin() + G.rowptr[i]);
    adj.clear();
    adj.shrink_to_fit();
    G.K.assign(G.col.size(), 0.0);
    G.shell_tets = 0;
    auto lat = [&](int v, int d) {
        const int q = d == 0 ? v % n1 : (d == 1 ? (v / n1) % n1 : v / (n1 * n1));
        return (double)(q - off);
    };
    for (size_t t = 0; t < T; ++t) {
        const int* v = &tets[4 * t];
        double P[4][3], cen[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < 4; ++q)
            for (int d = 0; d < 3; ++d) {
                P[q][d] = lat(v[q], d) * cell;
                cen[d] += lat(v[q], d);
            }
        double dc[3];
        for (int d = 0; d < 3; ++d) dc[d] = cen[d] / 4.0 - c;
        const double rho = std::max(std::fabs(dc[0]), std::max(std::fabs(dc[1]), std::fabs(dc[2])));
        double M[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
        if (rho > G.R1) {
            shell_tensor_at(dc, G.R1, G.R2, M);
            ++G.shell_tets;
        }
        double e[3][3];
        for (int q = 0; q < 3; ++q)
            for (int d = 0; d < 3; ++d) e[q][d] = P[q + 1][d] - P[0][d];
        auto cross = [](const double* x, const double* y, double* z) {
            z[0] = x[1] * y[2] - x[2] * y[1];
            z[1] = x[2] * y[0] - x[0] * y[2];
            z[2] = x[0] * y[1] - x[1] * y[0];
        };
        double cf[4][3];
        cross(e[1], e[2], cf[1]);
        cross(e[2], e[0], cf[2]);
        cross(e[0], e[1], cf[3]);
        for (int d = 0; d < 3; ++d) cf[0][d] = -(cf[1][d] + cf[2][d] + cf[3][d]);
        const double det = e[0][0] * cf[1][0] + e[0][1] * cf[1][1] + e[0][2] * cf[1][2];
        double Mc[4][3];
        for (int q = 0; q < 4; ++q)
            for (int d = 0; d < 3; ++d) Mc[q][d] = M[d][0] * cf[q][0] + M[d][1] * cf[q][1] + M[d][2] * cf[q][2];
        for (int x = 0; x < 4; ++x) {
            const int i = v[x];
            for (int y = 0; y < 4; ++y) {
                const int j = v[y];
                const double val = (cf[x][0] * Mc[y][0] + cf[x][1] * Mc[y][1] + cf[x][2] * Mc[y][2]) /
                                   (6.0 * std::fabs(det));
                const int* b = G.col.data() + G.rowptr[i];
                const int* e2 = G.col.data() + G.rowptr[i + 1];
                G.K[(size_t)(std::lower_bound(b, e2, j) - G.col.data())] += val;
            }
        }
    }
    // Dirichlet rows (the outer face) and the magnet's nodes in the grid
    for (int k = 0; k < n1; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i) {
                const double r = std::max(std::fabs(i - off - c), std::max(std::fabs(j - off - c), std::fabs(k - off - c)));
                if (r == G.R2) G.outer.push_back(id(i, j, k));
            }
    const int m1 = n + 1;
    G.magnet.resize((size_t)m1 * m1 * m1);
    for (int k = 0; k < m1; ++k)
        for (int j = 0; j < m1; ++j)
            for (int i = 0; i < m1; ++i) G.magnet[i + m1 * (j + m1 * (size_t)k)] = id(i + off, j + off, k + off);
    return {};
}

}  // namespace lbm
