// Host construction of the hierarchical (H-matrix) form of the double-layer
// boundary matrix B of the hybrid FEM/BEM open boundary (Sec. 3.1), on the
// partition of csrc/hpartition.cu:
//   * dense leaves hold the exact entries;
//   * admissible leaves are compressed by adaptive cross approximation with
//     partial pivoting (Bebendorf): only the pivot rows and columns are
//     evaluated.  Start from the first row; take the column of the residual
//     row's largest entry as pivot, append u = residual column, v = residual
//     row / pivot, and go on from the unused row where |u| is largest, until
//     |u| |v| <= (eps/2) |S_k|_F (S_k the current approximation, its norm
//     updated exactly from the new terms) or, tested every 8 terms, the
//     residual at 32 sampled entries is that small.  A residual row that
//     vanishes moves on to the next unused row.
//   * partial pivoting can miss a part of a block that none of its pivot rows
//     sees (on a polyhedron the coplanar pairs of a face are exact zeros), so
//     every low-rank leaf is checked at 32 fresh pseudo-random entries (a
//     statistical check, not a bound); when the sampled residual, scaled to
//     the block, exceeds eps |S_k|_F, the
//     approximation resumes from the worst sampled row and is checked again at
//     fresh entries (up to four times); a leaf that still fails is assembled
//     exactly and, if it has at most 65 536 entries, compressed by cross
//     approximation with full pivoting, whose bound |A - U V|_F <= eps |A|_F
//     holds by construction (larger ones stay exact and dense);
//   * the factors of a low-rank leaf are then recompressed to the fewest terms
//     the tolerance needs: U = Qu Ru, V^T = Qv Rv (Gram-Schmidt), the SVD of the
//     k x k core Ru Rv^T by one-sided Jacobi rotations (Hestenes), truncated
//     where the discarded singular values reach eps/2 of the leaf's norm;
//   * a leaf whose factors would not be smaller than the block stays dense.
// Entries: B_ij = (1/4pi) sum_{t contains j} I_t,j(x_i) + (Omega_i/4pi - 1) delta_ij,
// I the closed-form double layer of the linear hat on a flat triangle (the same
// formula as the device assembly in csrc/mesh.cu, written here for the host, with
// the edge integral's logarithm in log1p form:
//   I_k(x) = -phi_k(p) Omega_t + h grad phi_k . sum_e nu_e P_e,
// h the height of x over the plane, p its foot, Omega_t the signed solid angle of
// the triangle (Van Oosterom-Strackee), P_e = int_e dl/|y - x|, nu_e the outward
// in-plane edge normal); the triangles that contain x_i give 0 (excluded by
// index).  Omega_i, the interior solid angle at node i, comes from the incident
// triangles by Girard's theorem (the spherical polygon the cone of the fan cuts
// from the unit sphere: the sum of its dihedral angles minus (m - 2) pi).
// Leaves are independent: they are filled by `threads` host threads, each with
// its own scratch, and concatenated in leaf order, so the result does not depend
// on the thread count.  Host code only; no kernel lives here.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

#include "lbm_host.h"

namespace lbm {

namespace {

constexpr double kPi = 3.14159265358979323846;

void hat_double_layer_host(const double x[3], const double* y0, const double* y1, const double* y2,
                           double I[3]) {
    const double* y[3] = {y0, y1, y2};
    const double e12[3] = {y1[0] - y0[0], y1[1] - y0[1], y1[2] - y0[2]};
    const double e13[3] = {y2[0] - y0[0], y2[1] - y0[1], y2[2] - y0[2]};
    const double cr[3] = {e12[1] * e13[2] - e12[2] * e13[1], e12[2] * e13[0] - e12[0] * e13[2],
                          e12[0] * e13[1] - e12[1] * e13[0]};
    double r[3][3];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) r[k][d] = y[k][d] - x[d];
    const double hnum = r[0][0] * cr[0] + r[0][1] * cr[1] + r[0][2] * cr[2];
    if (hnum == 0.0) {
        I[0] = I[1] = I[2] = 0.0;
        return;
    }
    const double a2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    const double n[3] = {cr[0] / a2, cr[1] / a2, cr[2] / a2};
    const double h = hnum / a2;
    double eta[3];
    for (int k = 0; k < 3; ++k) eta[k] = std::sqrt(r[k][0] * r[k][0] + r[k][1] * r[k][1] + r[k][2] * r[k][2]);
    const double c12[3] = {r[1][1] * r[2][2] - r[1][2] * r[2][1], r[1][2] * r[2][0] - r[1][0] * r[2][2],
                           r[1][0] * r[2][1] - r[1][1] * r[2][0]};
    const double num = r[0][0] * c12[0] + r[0][1] * c12[1] + r[0][2] * c12[2];
    const double d01 = r[0][0] * r[1][0] + r[0][1] * r[1][1] + r[0][2] * r[1][2];
    const double d12 = r[1][0] * r[2][0] + r[1][1] * r[2][1] + r[1][2] * r[2][2];
    const double d20 = r[2][0] * r[0][0] + r[2][1] * r[0][1] + r[2][2] * r[0][2];
    const double den = eta[0] * eta[1] * eta[2] + eta[0] * d12 + eta[1] * d20 + eta[2] * d01;
    const double omega = 2.0 * std::atan2(num, den);
    double es[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3;
        const double e[3] = {y[k1][0] - y[k][0], y[k1][1] - y[k][1], y[k1][2] - y[k][2]};
        const double s = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        const double nu[3] = {(e[1] * n[2] - e[2] * n[1]) / s, (e[2] * n[0] - e[0] * n[2]) / s,
                              (e[0] * n[1] - e[1] * n[0]) / s};
        // ln((a + s)/(a - s)) as log1p(2s/(a - s)): far from the triangle the ratio is
        // 1 + O(s/r), whose logarithm loses a factor r/s of relative accuracy
        const double P = std::log1p(2.0 * s / (eta[k] + eta[k1] - s));
        for (int d = 0; d < 3; ++d) es[d] += nu[d] * P;
    }
    for (int k = 0; k < 3; ++k) {
        const double* a = y[(k + 1) % 3];
        const double* b = y[(k + 2) % 3];
        const double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double ax[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
        const double c[3] = {ab[1] * ax[2] - ab[2] * ax[1], ab[2] * ax[0] - ab[0] * ax[2],
                             ab[0] * ax[1] - ab[1] * ax[0]};
        const double phi = (c[0] * n[0] + c[1] * n[1] + c[2] * n[2]) / a2;
        const double g[3] = {(n[1] * ab[2] - n[2] * ab[1]) / a2, (n[2] * ab[0] - n[0] * ab[2]) / a2,
                             (n[0] * ab[1] - n[1] * ab[0]) / a2};
        I[k] = -phi * omega + h * (g[0] * es[0] + g[1] * es[1] + g[2] * es[2]);
    }
}

uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct Surface {
    const double* xyz;
    int nb;
    const int* bidx;
    const int* tris;
    std::vector<int> pos;                          // node id -> boundary position or -1
    std::vector<int> inc_ptr, inc_tri;             // boundary position -> triangles that contain it
    std::vector<double> omega;                     // interior solid angle per position
    std::vector<int> mark, local, in_cols;         // scratch of the block evaluation
    int stamp = 0, col_stamp = 0;

    // out[a * n + b] = B[rows[a], cols[b]] (boundary positions)
    void eval(const int* rows, int m, const int* cols, int n, double* out) {
        if (m <= 0 || n <= 0) return;
        ++col_stamp;
        for (int b = 0; b < n; ++b) {
            in_cols[cols[b]] = col_stamp;
            local[cols[b]] = b;
        }
        std::fill(out, out + (size_t)m * n, 0.0);
        // the triangles around the columns, in ascending order
        ++stamp;
        std::vector<int> tl;
        for (int b = 0; b < n; ++b)
            for (int q = inc_ptr[cols[b]]; q < inc_ptr[cols[b] + 1]; ++q) {
                const int t = inc_tri[q];
                if (mark[t] != stamp) {
                    mark[t] = stamp;
                    tl.push_back(t);
                }
            }
        std::sort(tl.begin(), tl.end());
        for (int a = 0; a < m; ++a) {
            const int id = bidx[rows[a]];
            const double* x = xyz + 3 * (size_t)id;
            for (int t : tl) {
                const int* v = tris + 3 * (size_t)t;
                if (v[0] == id || v[1] == id || v[2] == id) continue;   // contains x: 0
                double I[3];
                hat_double_layer_host(x, xyz + 3 * (size_t)v[0], xyz + 3 * (size_t)v[1], xyz + 3 * (size_t)v[2], I);
                for (int k = 0; k < 3; ++k) {
                    const int p = pos[v[k]];
                    if (p >= 0 && in_cols[p] == col_stamp) out[(size_t)a * n + local[p]] += I[k];
                }
            }
        }
        const double s = 0.25 / kPi;
        for (size_t e = 0; e < (size_t)m * n; ++e) out[e] *= s;
        for (int a = 0; a < m; ++a)
            if (in_cols[rows[a]] == col_stamp) out[(size_t)a * n + local[rows[a]]] += omega[rows[a]] * s - 1.0;
    }
};

std::string girard(Surface& S, int N, int F) {
    // fan of each boundary node: (a -> b) for every triangle (i, a, b) in its outward order
    std::vector<std::vector<std::pair<int, int>>> fan(S.nb);
    for (int t = 0; t < F; ++t)
        for (int k = 0; k < 3; ++k) {
            const int i = S.tris[3 * t + k];
            if (i < 0 || i >= N || S.pos[i] < 0) return "triangle " + std::to_string(t) + " has a vertex off the surface list";
            fan[S.pos[i]].push_back({S.tris[3 * t + (k + 1) % 3], S.tris[3 * t + (k + 2) % 3]});
        }
    S.omega.assign(S.nb, 0.0);
    for (int q = 0; q < S.nb; ++q) {
        const auto& f = fan[q];
        const int m = (int)f.size();
        if (m < 3) return "surface node " + std::to_string(S.bidx[q]) + " has fewer than 3 triangles";
        const double* x = S.xyz + 3 * (size_t)S.bidx[q];
        double total = 0.0;
        for (const auto& ab : f) {
            int c = -1;
            for (const auto& e : f)
                if (e.first == ab.second) c = e.second;
            if (c < 0) return "open fan at surface node " + std::to_string(S.bidx[q]);
            const double* pa = S.xyz + 3 * (size_t)ab.first;
            const double* pb = S.xyz + 3 * (size_t)ab.second;
            const double* pc = S.xyz + 3 * (size_t)c;
            double u[3] = {pb[0] - x[0], pb[1] - x[1], pb[2] - x[2]};
            const double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            for (double& v : u) v /= un;
            double wa[3] = {pa[0] - x[0], pa[1] - x[1], pa[2] - x[2]};
            double wc[3] = {pc[0] - x[0], pc[1] - x[1], pc[2] - x[2]};
            const double da = wa[0] * u[0] + wa[1] * u[1] + wa[2] * u[2];
            const double dc = wc[0] * u[0] + wc[1] * u[1] + wc[2] * u[2];
            for (int d = 0; d < 3; ++d) {
                wa[d] -= da * u[d];
                wc[d] -= dc * u[d];
            }
            const double cx[3] = {wa[1] * wc[2] - wa[2] * wc[1], wa[2] * wc[0] - wa[0] * wc[2],
                                  wa[0] * wc[1] - wa[1] * wc[0]};
            double th = std::atan2(u[0] * cx[0] + u[1] * cx[1] + u[2] * cx[2],
                                   wa[0] * wc[0] + wa[1] * wc[1] + wa[2] * wc[2]);
            if (th < 0.0) th += 2.0 * kPi;
            total += th;
        }
        S.omega[q] = total - (m - 2) * kPi;
    }
    return {};
}

double dot(const double* a, const double* b, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

// cross approximation with full pivoting of the m x n block A (row-major,
// overwritten); it stops early, one term past the size at which the factors
// stop being smaller than the block.  Returns whether the tolerance was met.
bool full_pivot(double* A, int m, int n, double eps, std::vector<double>& U, std::vector<double>& V, int& k) {
    double norm2 = 0.0;
    for (size_t e = 0; e < (size_t)m * n; ++e) norm2 += A[e] * A[e];
    std::vector<std::vector<double>> us, vs;
    double r2 = norm2;
    const int kcap = std::min(std::min(m, n), (int)(((size_t)m * n - 1) / (size_t)(m + n)) + 1);
    while (r2 > eps * eps * norm2 && (int)us.size() < kcap) {
        size_t best = 0;
        for (size_t e = 1; e < (size_t)m * n; ++e)
            if (std::fabs(A[e]) > std::fabs(A[best])) best = e;
        const int i = (int)(best / n), j = (int)(best % n);
        const double piv = A[best];
        if (piv == 0.0) break;
        std::vector<double> u(m), v(n);
        for (int a = 0; a < m; ++a) u[a] = A[(size_t)a * n + j];
        for (int b = 0; b < n; ++b) v[b] = A[(size_t)i * n + b] / piv;
        r2 = 0.0;
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < n; ++b) {
                double& x = A[(size_t)a * n + b];
                x -= u[a] * v[b];
                r2 += x * x;
            }
        us.push_back(std::move(u));
        vs.push_back(std::move(v));
    }
    k = (int)us.size();
    U.assign((size_t)m * k, 0.0);
    V.assign((size_t)k * n, 0.0);
    for (int l = 0; l < k; ++l) {
        for (int a = 0; a < m; ++a) U[(size_t)a * k + l] = us[l][a];
        for (int b = 0; b < n; ++b) V[(size_t)l * n + b] = vs[l][b];
    }
    return r2 <= eps * eps * norm2;
}

// A = Q R for A (m x k, row-major): Q orthonormal columns (a column that
// vanishes stays zero), R (k x k) upper triangular; classical Gram-Schmidt
// applied twice to every column.
void thin_qr(const std::vector<double>& A, int m, int k, std::vector<double>& Q, std::vector<double>& R) {
    Q = A;
    R.assign((size_t)k * k, 0.0);
    for (int c = 0; c < k; ++c) {
        for (int pass = 0; pass < 2; ++pass)
            for (int p = 0; p < c; ++p) {
                double d = 0.0;
                for (int a = 0; a < m; ++a) d += Q[(size_t)a * k + p] * Q[(size_t)a * k + c];
                R[(size_t)p * k + c] += d;
                for (int a = 0; a < m; ++a) Q[(size_t)a * k + c] -= d * Q[(size_t)a * k + p];
            }
        double nrm = 0.0;
        for (int a = 0; a < m; ++a) nrm += Q[(size_t)a * k + c] * Q[(size_t)a * k + c];
        nrm = std::sqrt(nrm);
        R[(size_t)c * k + c] = nrm;
        for (int a = 0; a < m; ++a) Q[(size_t)a * k + c] = nrm > 0.0 ? Q[(size_t)a * k + c] / nrm : 0.0;
    }
}

// One-sided Jacobi (Hestenes) on C (k x k, row-major): rotations of column
// pairs until all columns are orthogonal, C Z = W with Z orthogonal; the
// singular values are the column norms of W, in any order.
void jacobi_svd(std::vector<double>& W, std::vector<double>& Z, int k) {
    Z.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) Z[(size_t)i * k + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < k; ++i) {
                    const double wp = W[(size_t)i * k + p], wq = W[(size_t)i * k + q];
                    al += wp * wp;
                    be += wq * wq;
                    ga += wp * wq;
                }
                if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
                off = std::max(off, std::fabs(ga) / std::sqrt(al * be));
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < k; ++i) {
                    double& wp = W[(size_t)i * k + p];
                    double& wq = W[(size_t)i * k + q];
                    const double a = wp, b = wq;
                    wp = c * a - s * b;
                    wq = s * a + c * b;
                    double& zp = Z[(size_t)i * k + p];
                    double& zq = Z[(size_t)i * k + q];
                    const double za = zp, zb = zq;
                    zp = c * za - s * zb;
                    zq = s * za + c * zb;
                }
            }
        if (off <= 1e-15) break;
    }
}

// U V (U m x k, V k x n, row-major) recompressed to the fewest singular triplets
// whose discarded tail is at most tol |U V|_F; k updated.
void recompress(std::vector<double>& U, std::vector<double>& V, int m, int n, int& k, double tol) {
    if (k <= 1) return;
    std::vector<double> Vt((size_t)n * k);
    for (int l = 0; l < k; ++l)
        for (int b = 0; b < n; ++b) Vt[(size_t)b * k + l] = V[(size_t)l * n + b];
    std::vector<double> Qu, Ru, Qv, Rv;
    thin_qr(U, m, k, Qu, Ru);
    thin_qr(Vt, n, k, Qv, Rv);
    std::vector<double> C((size_t)k * k, 0.0);         // Ru Rv^T
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double x = 0.0;
            for (int l = 0; l < k; ++l) x += Ru[(size_t)i * k + l] * Rv[(size_t)j * k + l];
            C[(size_t)i * k + j] = x;
        }
    std::vector<double> Z;
    jacobi_svd(C, Z, k);                                  // C now holds W = C_in Z
    std::vector<double> sig(k);
    for (int j = 0; j < k; ++j) {
        double x = 0.0;
        for (int i = 0; i < k; ++i) x += C[(size_t)i * k + j] * C[(size_t)i * k + j];
        sig[j] = std::sqrt(x);
    }
    std::vector<int> ord(k);
    for (int j = 0; j < k; ++j) ord[j] = j;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sig[a] > sig[b]; });
    double total = 0.0;
    for (double v : sig) total += v * v;
    int keep = k;
    double tail = 0.0;
    while (keep > 0 && tail + sig[ord[keep - 1]] * sig[ord[keep - 1]] <= tol * tol * total) {
        tail += sig[ord[keep - 1]] * sig[ord[keep - 1]];
        --keep;
    }
    // U' = Qu W[:, kept] (m x keep), V' = (Qv Z[:, kept])^T (keep x n)
    std::vector<double> U2((size_t)m * keep, 0.0), V2((size_t)keep * n, 0.0);
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < keep; ++c) {
            double x = 0.0;
            for (int l = 0; l < k; ++l) x += Qu[(size_t)a * k + l] * C[(size_t)l * k + ord[c]];
            U2[(size_t)a * keep + c] = x;
        }
    for (int c = 0; c < keep; ++c)
        for (int b = 0; b < n; ++b) {
            double x = 0.0;
            for (int l = 0; l < k; ++l) x += Qv[(size_t)b * k + l] * Z[(size_t)l * k + ord[c]];
            V2[(size_t)c * n + b] = x;
        }
    U.swap(U2);
    V.swap(V2);
    k = keep;
}

struct AcaTerms {
    std::vector<std::vector<double>> us, vs;        // A ~ sum_l us[l] vs[l]^T
    std::vector<char> used;                         // rows that have been pivot (or zero) rows
    double norm2 = 0.0;                             // |sum_l us[l] vs[l]^T|_F^2
};

// Residual of the current terms at 32 pseudo-random entries of the block (seed
// `seed`), scaled to the whole block: an estimate of |A - S_k|_F^2; `worst_row`
// receives the row of the largest sampled residual.
double sampled_residual(Surface& S, const int* R, int m, const int* C, int n, const AcaTerms& T, uint64_t seed,
                        int* worst_row) {
    const int samples = 32, k = (int)T.us.size();
    double res2 = 0.0, worst = -1.0;
    for (int s = 0; s < samples; ++s) {
        const uint64_t hsh = splitmix64(seed + (uint64_t)s);
        const int a = (int)(hsh % (uint64_t)m), b = (int)((hsh >> 32) % (uint64_t)n);
        double exact;
        S.eval(R + a, 1, C + b, 1, &exact);
        double approx = 0.0;
        for (int l = 0; l < k; ++l) approx += T.us[l][a] * T.vs[l][b];
        const double r = exact - approx;
        res2 += r * r;
        if (worst_row && std::fabs(r) > worst) {
            worst = std::fabs(r);
            *worst_row = a;
        }
    }
    return res2 * ((double)m * n / samples);
}

// Partial-pivot cross approximation terms appended to T from row `start` on,
// until |u| |v| <= (eps/2) |S_k|_F or, tested every 8 terms, the residual at 32
// sampled entries (seed `seed`) is within (eps/2) |S_k|_F -- near the tolerance
// the last term overstates the residual by up to sqrt(n) --, or kmax terms, or no
// unused row is left.  Returns true unless it stopped at kmax.
bool aca_extend(Surface& S, const int* R, int m, const int* C, int n, double eps, int kmax, int start,
                uint64_t seed, AcaTerms& T) {
    std::vector<double> row(n), col(m);
    int i = start;
    while ((int)T.us.size() < kmax) {
        T.used[i] = 1;
        S.eval(R + i, 1, C, n, row.data());
        for (size_t l = 0; l < T.us.size(); ++l)
            for (int b = 0; b < n; ++b) row[b] -= T.us[l][i] * T.vs[l][b];
        int j = 0;
        for (int b = 1; b < n; ++b)
            if (std::fabs(row[b]) > std::fabs(row[j])) j = b;
        if (row[j] == 0.0) {
            int nxt = -1;
            for (int a = 0; a < m; ++a)
                if (!T.used[a]) { nxt = a; break; }
            if (nxt < 0) return true;                       // every row is reproduced exactly
            i = nxt;
            continue;
        }
        std::vector<double> v(n), u(m);
        for (int b = 0; b < n; ++b) v[b] = row[b] / row[j];
        S.eval(R, m, C + j, 1, col.data());
        for (int a = 0; a < m; ++a) {
            double x = col[a];
            for (size_t l = 0; l < T.us.size(); ++l) x -= T.vs[l][j] * T.us[l][a];
            u[a] = x;
        }
        const double uu = dot(u.data(), u.data(), m), vv = dot(v.data(), v.data(), n);
        double cross = 0.0;
        for (size_t l = 0; l < T.us.size(); ++l)
            cross += dot(u.data(), T.us[l].data(), m) * dot(T.vs[l].data(), v.data(), n);
        T.norm2 += 2.0 * cross + uu * vv;
        T.us.push_back(std::move(u));
        T.vs.push_back(std::move(v));
        const double goal2 = 0.25 * eps * eps * std::max(T.norm2, 0.0);
        if (uu * vv <= goal2) return true;
        if (T.us.size() % 8 == 0 && sampled_residual(S, R, m, C, n, T, seed, nullptr) <= goal2) return true;
        int nxt = -1;
        double best = -1.0;
        for (int a = 0; a < m; ++a)
            if (!T.used[a] && std::fabs(T.us.back()[a]) > best) { best = std::fabs(T.us.back()[a]); nxt = a; }
        if (nxt < 0) return true;                           // every row has been a pivot row
        i = nxt;
    }
    return false;
}

struct LeafOut {
    int kind = 0, rank = 0, fallback = 0;
    std::vector<double> values;                   // dense m*n, or U (m*k) then V (k*n)
};

// One leaf of the block tree: exact entries (dense), or cross approximation,
// sampled check (resumed from the worst sampled row up to four times), exact
// fallback and recompression (low rank).
void fill_leaf(Surface& S, const HPartition& P, size_t li, double eps, LeafOut& out) {
    const HLeaf& lf = P.leaves[li];
    const HCluster& ct = P.clusters[lf.row];
    const HCluster& cs = P.clusters[lf.col];
    const int m = ct.size, n = cs.size;
    const int* R = P.idx.data() + ct.begin;
    const int* C = P.idx.data() + cs.begin;
    auto store_dense = [&]() {
        out.kind = 0;
        out.rank = 0;
        out.values.resize((size_t)m * n);
        S.eval(R, m, C, n, out.values.data());
    };
    if (!lf.low_rank) {
        store_dense();
        return;
    }
    // adaptive cross approximation with partial pivoting, checked at sampled
    // entries; a failed check resumes it from the worst sampled row
    const int kmax = std::min(std::min(m, n), (int)(((size_t)m * n - 1) / (size_t)(m + n)));
    AcaTerms T;
    T.used.assign(m, 0);
    const uint64_t stop_seed = ((uint64_t)li << 12) | 0xF00u;  // samples of the stopping test
    bool conv = aca_extend(S, R, m, C, n, eps, kmax, 0, stop_seed, T);
    bool ok = false;
    int checks = 0;
    for (int attempt = 0; attempt < 4 && (conv || (int)T.us.size() < kmax); ++attempt) {
        ++checks;
        int worst_row = 0;
        const double est = sampled_residual(S, R, m, C, n, T, ((uint64_t)li << 12) + ((uint64_t)attempt << 6),
                                            &worst_row);
        if (est <= eps * eps * std::max(T.norm2, 0.0) && !(T.us.empty() && est > 0.0)) {
            ok = true;
            break;
        }
        conv = aca_extend(S, R, m, C, n, eps, kmax, worst_row, stop_seed + 0x100u * (uint64_t)(attempt + 1), T);
    }
    std::vector<double> Uf, Vf, exact;
    int k = (int)T.us.size();
    if (!ok) {
        // exact entries; compressed by full pivoting when the block is small enough
        out.fallback = checks > 0;                          // the sampled check failed (else: incompressible)
        exact.resize((size_t)m * n);
        S.eval(R, m, C, n, exact.data());
        std::vector<double> blk(exact);
        if ((size_t)m * n > ((size_t)1 << 16) || !full_pivot(blk.data(), m, n, eps, Uf, Vf, k)) {
            out.kind = 0;
            out.rank = 0;
            out.values.swap(exact);
            return;
        }
    } else {
        Uf.assign((size_t)m * k, 0.0);
        Vf.assign((size_t)k * n, 0.0);
        for (int l = 0; l < k; ++l) {
            for (int a = 0; a < m; ++a) Uf[(size_t)a * k + l] = T.us[l][a];
            for (int b = 0; b < n; ++b) Vf[(size_t)l * n + b] = T.vs[l][b];
        }
    }
    recompress(Uf, Vf, m, n, k, 0.5 * eps);
    if ((size_t)k * (m + n) >= (size_t)m * n) {          // not smaller than the block: dense
        if (exact.empty()) {
            store_dense();
        } else {
            out.kind = 0;
            out.rank = 0;
            out.values.swap(exact);
        }
        return;
    }
    out.kind = 1;
    out.rank = k;
    out.values.reserve(Uf.size() + Vf.size());
    out.values.insert(out.values.end(), Uf.begin(), Uf.end());
    out.values.insert(out.values.end(), Vf.begin(), Vf.end());
}

}  // namespace

std::string host_hmatrix_build(int N, const double* xyz, int nb, const int* bidx, int F, const int* tris, double eta,
                               int n_min, double eps, int threads, HMatrixHost& H) {
    if (!(eps > 0.0) || !(eps < 1.0)) return "eps must lie in (0, 1)";
    if (N <= 0 || nb <= 0 || F <= 0) return "empty surface";
    H = HMatrixHost{};
    Surface S;
    S.xyz = xyz;
    S.nb = nb;
    S.bidx = bidx;
    S.tris = tris;
    S.pos.assign(N, -1);
    for (int q = 0; q < nb; ++q) {
        if (bidx[q] < 0 || bidx[q] >= N) return "surface node id out of range";
        S.pos[bidx[q]] = q;
    }
    if (std::string why = girard(S, N, F); !why.empty()) return why;
    S.inc_ptr.assign(nb + 1, 0);
    for (int t = 0; t < F; ++t)
        for (int k = 0; k < 3; ++k) ++S.inc_ptr[S.pos[tris[3 * t + k]] + 1];
    for (int q = 0; q < nb; ++q) S.inc_ptr[q + 1] += S.inc_ptr[q];
    S.inc_tri.resize(3 * (size_t)F);
    {
        std::vector<int> fill(S.inc_ptr.begin(), S.inc_ptr.end() - 1);
        for (int t = 0; t < F; ++t)
            for (int k = 0; k < 3; ++k) S.inc_tri[fill[S.pos[tris[3 * t + k]]]++] = t;
    }
    S.mark.assign(F, 0);
    S.local.assign(nb, -1);
    S.in_cols.assign(nb, 0);

    std::vector<double> pts(3 * (size_t)nb), lo(3 * (size_t)nb), hi(3 * (size_t)nb);
    host_support_boxes(N, xyz, nb, bidx, F, tris, lo.data(), hi.data());
    for (int q = 0; q < nb; ++q)
        for (int d = 0; d < 3; ++d) pts[3 * q + d] = xyz[3 * (size_t)bidx[q] + d];
    if (std::string why = host_hmatrix_partition(nb, pts.data(), lo.data(), hi.data(), eta, n_min, H.P); !why.empty())
        return why;

    const size_t L = H.P.leaves.size();
    std::vector<LeafOut> outs(L);
    const int nth = std::max(1, std::min(threads, (int)std::min<size_t>(L, 256)));
    std::atomic<size_t> next{0};
    auto work = [&](Surface Sw) {                         // each thread its own scratch
        for (size_t li = next++; li < L; li = next++) fill_leaf(Sw, H.P, li, eps, outs[li]);
    };
    if (nth == 1) {
        work(S);
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < nth; ++t) pool.emplace_back(work, S);
        for (auto& th : pool) th.join();
    }
    H.kind.assign(L, 0);
    H.rank.assign(L, 0);
    H.off.assign(L, 0);
    size_t total = 0;
    for (const LeafOut& o : outs) total += o.values.size();
    H.data.reserve(total);
    for (size_t li = 0; li < L; ++li) {
        H.kind[li] = outs[li].kind;
        H.rank[li] = outs[li].rank;
        H.off[li] = H.data.size();
        H.data.insert(H.data.end(), outs[li].values.begin(), outs[li].values.end());
        H.fallbacks += outs[li].fallback;
    }
    return {};
}

}  // namespace lbm
