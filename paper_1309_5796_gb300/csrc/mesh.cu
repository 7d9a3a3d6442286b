// Mesh set-up on the device: Kuhn-split cube, CSR pattern, integer P1 tables,
// boundary numbering, and the dense double-layer (FEM/BEM) matrix.
//
// Paper: linear tetrahedral finite elements (abstract, Sec. 2.1); the energy
// gradient is a sparse matrix-vector product (Table 2); the stray field comes
// from a scalar potential whose open boundary is a hybrid FEM/BEM (Sec. 3.1).
//
// Exactness: lattice coordinates are integers and every Kuhn tetrahedron has
// det = 1, so the stiffness (h/6 units), divergence coupling (h^2/24) and
// lumped volumes (h^3/24) are small integers assembled without rounding.  Each
// row is assembled by its own thread from the tetrahedra around its node, so
// no atomics are needed and the tables are bit-reproducible.
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <vector>

#include "lbm_internal.cuh"
#include "lbm_host.h"

namespace lbm {

// The 15 lattice offsets of a node's Kuhn neighbourhood, ordered by global id
// delta (lexicographic in dz, dy, dx).
__constant__ int c_stencil[15][3] = {
    {-1, -1, -1}, {0, -1, -1}, {-1, 0, -1}, {0, 0, -1},
    {-1, -1, 0},  {0, -1, 0},  {-1, 0, 0},  {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {1, 1, 0},
    {0, 0, 1},    {1, 0, 1},   {0, 1, 1},   {1, 1, 1}};

__device__ __forceinline__ int stencil_slot(int dx, int dy, int dz) {
    // inverse of c_stencil over the 27 offsets in {-1,0,1}^3
    const int key = (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1));
    switch (key) {
        case 0: return 0;   case 1: return 1;   case 3: return 2;   case 4: return 3;
        case 9: return 4;   case 10: return 5;  case 12: return 6;  case 13: return 7;
        case 14: return 8;  case 16: return 9;  case 17: return 10; case 22: return 11;
        case 23: return 12; case 25: return 13; case 26: return 14;
        default: return -1;
    }
}

// Vertices (lattice coordinates) of Kuhn tetrahedron `perm` of cell (cx,cy,cz):
// {v0, v0+e_a, v0+e_a+e_b, v0+(1,1,1)} for the permutation (a,b,c) in
// lexicographic order, last two swapped for odd permutations (positive volume).
__device__ __forceinline__ void kuhn_tet(int cx, int cy, int cz, int perm, int v[4][3]) {
    const int pa[6] = {0, 0, 1, 1, 2, 2};
    const int pb[6] = {1, 2, 0, 2, 0, 1};
    const bool odd = (perm == 1 || perm == 2 || perm == 5);
    int p0[3] = {cx, cy, cz};
    int p1[3] = {cx, cy, cz};
    p1[pa[perm]] += 1;
    int p2[3] = {p1[0], p1[1], p1[2]};
    p2[pb[perm]] += 1;
    int p3[3] = {cx + 1, cy + 1, cz + 1};
    for (int d = 0; d < 3; ++d) {
        v[0][d] = p0[d];
        v[1][d] = p1[d];
        v[2][d] = odd ? p3[d] : p2[d];
        v[3][d] = odd ? p2[d] : p3[d];
    }
}

__device__ __forceinline__ void cross3i(const int a[3], const int b[3], int c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ bool on_surface(int x, int y, int z, int n) {
    return x == 0 || y == 0 || z == 0 || x == n || y == n || z == n;
}

__global__ void k_row_counts(int n, int* cnt, int* bflag) {
    const int n1 = n + 1, N = n1 * n1 * n1;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int x = id % n1, y = (id / n1) % n1, z = id / (n1 * n1);
        int c = 0;
        for (int s = 0; s < 15; ++s) {
            const int X = x + c_stencil[s][0], Y = y + c_stencil[s][1], Z = z + c_stencil[s][2];
            c += (X >= 0 && X <= n && Y >= 0 && Y <= n && Z >= 0 && Z <= n);
        }
        cnt[id] = c;
        bflag[id] = on_surface(x, y, z, n) ? 1 : 0;
    }
}

// Exclusive prefix sum of in[0..n) into out[0..n], out[n] = total; one block.
__global__ void k_scan_single(const int* in, int* out, int n) {
    __shared__ int s[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int chunk = (n + T - 1) / T;
    const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += in[i];
    s[t] = sum;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {   // inclusive Hillis-Steele scan
        int v = (t >= off) ? s[t - off] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    int run = s[t] - sum;
    for (int i = lo; i < hi; ++i) { out[i] = run; run += in[i]; }
    if (t == T - 1) out[n] = s[t];
}

// One thread per node row: accumulate Kint, Gint, Gint^T and Vint over the
// tetrahedra around the node; write the row in ascending column order.
__global__ void k_assemble(int n, const int* rowptr, const int* bpos, int* col, int* pkA, int* pkB,
                           int* node) {
    const int n1 = n + 1, N = n1 * n1 * n1;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x) {
        const int x = id % n1, y = (id / n1) % n1, z = id / (n1 * n1);
        int K[15], G[15][3], Gt[15][3];
        for (int s = 0; s < 15; ++s) {
            K[s] = 0;
            for (int d = 0; d < 3; ++d) { G[s][d] = 0; Gt[s][d] = 0; }
        }
        int V = 0;
        for (int cz = z - 1; cz <= z; ++cz)
            for (int cy = y - 1; cy <= y; ++cy)
                for (int cx = x - 1; cx <= x; ++cx) {
                    if (cx < 0 || cy < 0 || cz < 0 || cx >= n || cy >= n || cz >= n) continue;
                    for (int p = 0; p < 6; ++p) {
                        int v[4][3];
                        kuhn_tet(cx, cy, cz, p, v);
                        int a = -1;
                        for (int k = 0; k < 4; ++k)
                            if (v[k][0] == x && v[k][1] == y && v[k][2] == z) a = k;
                        if (a < 0) continue;
                        int e1[3], e2[3], e3[3], c[4][3];
                        for (int d = 0; d < 3; ++d) {
                            e1[d] = v[1][d] - v[0][d];
                            e2[d] = v[2][d] - v[0][d];
                            e3[d] = v[3][d] - v[0][d];
                        }
                        cross3i(e2, e3, c[1]);
                        cross3i(e3, e1, c[2]);
                        cross3i(e1, e2, c[3]);
                        for (int d = 0; d < 3; ++d) c[0][d] = -(c[1][d] + c[2][d] + c[3][d]);
                        V += 1;  // det = 1 for every Kuhn tetrahedron
                        for (int b = 0; b < 4; ++b) {
                            const int s = stencil_slot(v[b][0] - x, v[b][1] - y, v[b][2] - z);
                            K[s] += c[a][0] * c[b][0] + c[a][1] * c[b][1] + c[a][2] * c[b][2];
                            for (int d = 0; d < 3; ++d) {
                                G[s][d] += c[a][d];
                                Gt[s][d] += c[b][d];
                            }
                        }
                    }
                }
        int e = rowptr[id];
        for (int s = 0; s < 15; ++s) {
            const int X = x + c_stencil[s][0], Y = y + c_stencil[s][1], Z = z + c_stencil[s][2];
            if (X < 0 || X > n || Y < 0 || Y > n || Z < 0 || Z > n) continue;
            const int j = X + n1 * (Y + n1 * Z);
            const unsigned flag = on_surface(X, Y, Z, n) ? 0x80000000u : 0u;
            col[e] = (int)((unsigned)j | flag);
            pkA[e] = (K[s] & 0xff) | ((G[s][0] & 0xff) << 8) | ((G[s][1] & 0xff) << 16) |
                     ((unsigned)(G[s][2] & 0xff) << 24);
            pkB[e] = (Gt[s][0] & 0xff) | ((Gt[s][1] & 0xff) << 8) | ((Gt[s][2] & 0xff) << 16);
            ++e;
        }
        const int bp = on_surface(x, y, z, n) ? bpos[id] + 1 : 0;
        node[id] = (int)((unsigned)(V & 0xff) | ((unsigned)(K[7] & 0xff) << 8) | ((unsigned)bp << 16));  // slot 7 = diagonal
    }
}

// Stiffness-only CSR for the potential solves: the nonzero Kint entries of each
// row (7 for an interior Kuhn node, whose face- and body-diagonal couplings
// vanish), packed as (column << 8) | (Kint & 0xff).
__global__ void k_kcsr_count(int N, const int* rowptr, const int* pkA, int* cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int c = 0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) c += (pkA[e] & 0xff) != 0;
        cnt[i] = c;
    }
}

__global__ void k_kcsr_fill(int N, const int* rowptr, const int* col, const int* pkA, const int* kptr, int* kent) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int o = kptr[i];
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int k = pkA[e] & 0xff;
            if (k) kent[o++] = (int)(((unsigned)(col[e] & 0x7fffffff) << 8) | (unsigned)k);
        }
    }
}

__global__ void k_boundary_ids(int N, const int* bflag, const int* bpos, int* bidx) {
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < N; id += gridDim.x * blockDim.x)
        if (bflag[id]) bidx[bpos[id]] = id;
}

__global__ void k_tets(int n, int* tets) {
    const int n1 = n + 1, C = n * n * n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 6 * C; t += gridDim.x * blockDim.x) {
        const int cell = t / 6, p = t % 6;
        const int cx = cell % n, cy = (cell / n) % n, cz = cell / (n * n);
        int v[4][3];
        kuhn_tet(cx, cy, cz, p, v);
        for (int k = 0; k < 4; ++k) tets[4 * t + k] = v[k][0] + n1 * (v[k][1] + n1 * v[k][2]);
    }
}

// ---- double-layer potential of hat functions on a flat triangle ------------------
// I_k(x) = int_t phi_k(y) (x-y).n / |x-y|^3 dS_y
//        = -phi_k(p) Omega_t + h grad phi_k . sum_e nu_e P_e
// (h = (y1-x).n, p = foot of x on the plane, Omega_t the signed solid angle by
// Van Oosterom-Strackee, P_e = int_e dl/|y-x|, nu_e the outward edge normal).
// Coplanar points (h = 0) give 0.  Coordinates are lattice units.
__device__ void hat_double_layer(const double x[3], const double y[3][3], double I[3]) {
    double e12[3], e13[3], cr[3];
    for (int d = 0; d < 3; ++d) { e12[d] = y[1][d] - y[0][d]; e13[d] = y[2][d] - y[0][d]; }
    cr[0] = e12[1] * e13[2] - e12[2] * e13[1];
    cr[1] = e12[2] * e13[0] - e12[0] * e13[2];
    cr[2] = e12[0] * e13[1] - e12[1] * e13[0];
    double r[3][3];
    for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) r[k][d] = y[k][d] - x[d];
    const double hnum = r[0][0] * cr[0] + r[0][1] * cr[1] + r[0][2] * cr[2];
    if (hnum == 0.0) { I[0] = I[1] = I[2] = 0.0; return; }
    const double a2 = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    const double nrm[3] = {cr[0] / a2, cr[1] / a2, cr[2] / a2};
    const double h = hnum / a2;
    double eta[3];
    for (int k = 0; k < 3; ++k) eta[k] = sqrt(r[k][0] * r[k][0] + r[k][1] * r[k][1] + r[k][2] * r[k][2]);
    // signed solid angle
    const double c23[3] = {r[1][1] * r[2][2] - r[1][2] * r[2][1], r[1][2] * r[2][0] - r[1][0] * r[2][2],
                           r[1][0] * r[2][1] - r[1][1] * r[2][0]};
    const double num = r[0][0] * c23[0] + r[0][1] * c23[1] + r[0][2] * c23[2];
    const double d12 = r[0][0] * r[1][0] + r[0][1] * r[1][1] + r[0][2] * r[1][2];
    const double d23 = r[1][0] * r[2][0] + r[1][1] * r[2][1] + r[1][2] * r[2][2];
    const double d31 = r[2][0] * r[0][0] + r[2][1] * r[0][1] + r[2][2] * r[0][2];
    const double den = eta[0] * eta[1] * eta[2] + eta[0] * d23 + eta[1] * d31 + eta[2] * d12;
    const double omega = 2.0 * atan2(num, den);
    // sum over edges of nu_e P_e
    double es[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3;
        const double e[3] = {y[k1][0] - y[k][0], y[k1][1] - y[k][1], y[k1][2] - y[k][2]};
        const double s = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        const double nu[3] = {(e[1] * nrm[2] - e[2] * nrm[1]) / s, (e[2] * nrm[0] - e[0] * nrm[2]) / s,
                              (e[0] * nrm[1] - e[1] * nrm[0]) / s};
        const double P = log((eta[k] + eta[k1] + s) / (eta[k] + eta[k1] - s));
        for (int d = 0; d < 3; ++d) es[d] += nu[d] * P;
    }
    for (int k = 0; k < 3; ++k) {
        const int ka = (k + 1) % 3, kb = (k + 2) % 3;   // edge opposite vertex k
        const double ab[3] = {y[kb][0] - y[ka][0], y[kb][1] - y[ka][1], y[kb][2] - y[ka][2]};
        const double ax[3] = {x[0] - y[ka][0], x[1] - y[ka][1], x[2] - y[ka][2]};
        // phi_k(p) = ((b-a) x (p-a)).n / 2A, and (b-a) x (h n) is normal-free
        const double cx[3] = {ab[1] * ax[2] - ab[2] * ax[1], ab[2] * ax[0] - ab[0] * ax[2],
                              ab[0] * ax[1] - ab[1] * ax[0]};
        const double phi_p = (cx[0] * nrm[0] + cx[1] * nrm[1] + cx[2] * nrm[2]) / a2;
        const double g[3] = {(nrm[1] * ab[2] - nrm[2] * ab[1]) / a2, (nrm[2] * ab[0] - nrm[0] * ab[2]) / a2,
                             (nrm[0] * ab[1] - nrm[1] * ab[0]) / a2};
        I[k] = -phi_p * omega + h * (g[0] * es[0] + g[1] * es[1] + g[2] * es[2]);
    }
}

// One block per boundary row i (grid-stride): W[3t+k] = I_k(x_i) for every
// surface triangle t (block scratch), Omega_i = -sum W (Gauss: the closed
// surface seen from a surface point subtends its interior solid angle), then
// B_ij = (1/4pi) sum_{(t,k) at j} W[3t+k] + (Omega_i/4pi - 1) delta_ij in the
// fixed order of the incidence list.
// Coordinates come from the lattice (cube meshes, xyz == nullptr) or from xyz
// (general meshes, units of the mesh's length unit).  A triangle that has the
// collocation node as a vertex contains it and gives 0; with lattice
// coordinates its h is exactly 0, with general ones it is excluded by index.
__global__ void k_bem_assemble(int n, int nb, int F, const int* bidx, const int* tris, const int* inc_ptr,
                               const int* inc_slot, const double* xyz, double* scratch, double* B64, float* B32) {
    __shared__ double s_red[256];
    const int n1 = n + 1;
    double* W = scratch + (size_t)blockIdx.x * 3 * F;
    const double inv4pi = 0.25 / 3.14159265358979323846;
    auto coords = [&](int v, double* c) {
        if (xyz) {
            c[0] = xyz[3 * (size_t)v];
            c[1] = xyz[3 * (size_t)v + 1];
            c[2] = xyz[3 * (size_t)v + 2];
        } else {
            c[0] = (double)(v % n1);
            c[1] = (double)((v / n1) % n1);
            c[2] = (double)(v / (n1 * n1));
        }
    };
    for (int row = blockIdx.x; row < nb; row += gridDim.x) {
        const int id = bidx[row];
        double x[3];
        coords(id, x);
        double om = 0.0;
        for (int t = threadIdx.x; t < F; t += blockDim.x) {
            double y[3][3];
            bool incident = false;
            for (int k = 0; k < 3; ++k) {
                const int v = tris[3 * t + k];
                incident |= (v == id);
                coords(v, y[k]);
            }
            double I[3] = {0.0, 0.0, 0.0};
            if (!incident) hat_double_layer(x, y, I);
            W[3 * t + 0] = I[0];
            W[3 * t + 1] = I[1];
            W[3 * t + 2] = I[2];
            om -= (I[0] + I[1]) + I[2];
        }
        s_red[threadIdx.x] = om;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) s_red[threadIdx.x] += s_red[threadIdx.x + st];
            __syncthreads();
        }
        const double omega = s_red[0];
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            double s = 0.0;
            for (int q = inc_ptr[j]; q < inc_ptr[j + 1]; ++q) s += W[inc_slot[q]];
            double val = s * inv4pi;
            if (j == row) val += omega * inv4pi - 1.0;
            B64[(size_t)row * nb + j] = val;
            if (B32) B32[(size_t)row * nb + j] = (float)val;
        }
        __syncthreads();
    }
}

// ---- general tetrahedral meshes (FP64 assembly) --------------------------------------
// Coordinates in units of the mesh's length unit L.  With the cofactors c_a of
// a tetrahedron and det = e1 . (e2 x e3) (6 x signed volume), the element
// contributions in the units of the integer tables are
//   K (units L/6):    c_a . c_b / |det|
//   G (units L^2/24): sgn(det) c_a          (row a, every column b)
//   G^T:              sgn(det) c_b
//   V (units L^3/24): |det|                 (per incident tetrahedron)
// One thread per row sums the tetrahedra around its node in ascending order.
__global__ void k_assemble_gen(int N, const double* __restrict__ xyz, const int* __restrict__ tets,
                               const int* __restrict__ nt_ptr, const int* __restrict__ nt_idx,
                               const int* __restrict__ rowptr, const int* __restrict__ col, Dbl4* A64,
                               float4* A32, Dbl4* Bt64, float4* Bt32, double* Vn, double* d64, float* d32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int e0 = rowptr[i], e1 = rowptr[i + 1];
        for (int e = e0; e < e1; ++e) {
            A64[e] = Dbl4{0.0, 0.0, 0.0, 0.0};
            Bt64[e] = Dbl4{0.0, 0.0, 0.0, 0.0};
        }
        double V = 0.0;
        for (int q = nt_ptr[i]; q < nt_ptr[i + 1]; ++q) {
            const int t = nt_idx[q];
            int v[4];
            double P[4][3];
            int a = -1;
            for (int k = 0; k < 4; ++k) {
                v[k] = tets[4 * (size_t)t + k];
                if (v[k] == i) a = k;
                for (int d = 0; d < 3; ++d) P[k][d] = xyz[3 * (size_t)v[k] + d];
            }
            double E[3][3], c[4][3];
            for (int k = 0; k < 3; ++k)
                for (int d = 0; d < 3; ++d) E[k][d] = P[k + 1][d] - P[0][d];
            for (int k = 0; k < 3; ++k) {
                const double* u = E[(k + 1) % 3];
                const double* w = E[(k + 2) % 3];
                c[k + 1][0] = u[1] * w[2] - u[2] * w[1];
                c[k + 1][1] = u[2] * w[0] - u[0] * w[2];
                c[k + 1][2] = u[0] * w[1] - u[1] * w[0];
            }
            for (int d = 0; d < 3; ++d) c[0][d] = -(c[1][d] + c[2][d] + c[3][d]);
            const double det = E[0][0] * c[1][0] + E[0][1] * c[1][1] + E[0][2] * c[1][2];
            const double ad = fabs(det), sg = det > 0.0 ? 1.0 : -1.0;
            V += ad;
            for (int b = 0; b < 4; ++b) {
                // slot of column v[b] in row i (columns ascending)
                int lo = e0, hi = e1 - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if ((col[mid] & 0x7fffffff) < v[b]) lo = mid + 1; else hi = mid;
                }
                const double kab = (c[a][0] * c[b][0] + c[a][1] * c[b][1] + c[a][2] * c[b][2]) / ad;
                Dbl4 x = A64[lo];
                x.x += kab;
                x.y += sg * c[a][0];
                x.z += sg * c[a][1];
                x.w += sg * c[a][2];
                A64[lo] = x;
                Dbl4 y = Bt64[lo];
                y.x += sg * c[b][0];
                y.y += sg * c[b][1];
                y.z += sg * c[b][2];
                Bt64[lo] = y;
            }
        }
        Vn[i] = V;
        for (int e = e0; e < e1; ++e) {
            const Dbl4 x = A64[e], y = Bt64[e];
            A32[e] = make_float4((float)x.x, (float)x.y, (float)x.z, (float)x.w);
            Bt32[e] = make_float4((float)y.x, (float)y.y, (float)y.z, 0.f);
            if ((col[e] & 0x7fffffff) == i) {
                d64[i] = x.x;
                d32[i] = (float)x.x;
            }
        }
    }
}

// Stiffness-only CSR of a general mesh: the entries with K != 0, packed as
// (column << 8) | 1 (the low byte only marks a present entry), values apart.
__global__ void k_kcsr_count_gen(int N, const int* rowptr, const Dbl4* A64, int* cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int c = 0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) c += A64[e].x != 0.0;
        cnt[i] = c;
    }
}

__global__ void k_kcsr_fill_gen(int N, const int* rowptr, const int* col, const Dbl4* A64, const int* kptr,
                                int* kent, double* k64, float* k32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        int o = kptr[i];
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const double k = A64[e].x;
            if (k != 0.0) {
                kent[o] = (int)(((unsigned)(col[e] & 0x7fffffff) << 8) | 1u);
                k64[o] = k;
                k32[o] = (float)k;
                ++o;
            }
        }
    }
}

}  // namespace lbm

// ---- host entry points used by the C ABI layer ---------------------------------------
namespace lbm {

static void surface_triangles(int n, std::vector<int>& tris) {
    // Each face square (u,v)-(u+1,v+1) of the six cube faces is split along the
    // same diagonal as the Kuhn cells below it; orientation is made outward.
    const int n1 = n + 1;
    auto id = [n1](int x, int y, int z) { return x + n1 * (y + n1 * z); };
    tris.clear();
    tris.reserve((size_t)36 * n * n);
    for (int d = 0; d < 3; ++d) {
        const int p = (d == 0) ? 1 : 0, q = (d == 2) ? 1 : 2;   // in-plane axes, p < q
        // (e_p x e_q) = +e_d for d = 0, 2 and -e_d for d = 1
        const int sgn = (d == 1) ? -1 : 1;
        for (int side = 0; side < 2; ++side) {
            const int val = side ? n : 0;
            const bool outward_pos = side == 1;
            const bool flip = (sgn > 0) != outward_pos;
            for (int v = 0; v < n; ++v)
                for (int u = 0; u < n; ++u) {
                    int c[4][3];
                    const int uv[4][2] = {{u, v}, {u + 1, v}, {u + 1, v + 1}, {u, v + 1}};
                    for (int k = 0; k < 4; ++k) {
                        c[k][d] = val;
                        c[k][p] = uv[k][0];
                        c[k][q] = uv[k][1];
                    }
                    const int a = id(c[0][0], c[0][1], c[0][2]), b = id(c[1][0], c[1][1], c[1][2]);
                    const int cc = id(c[2][0], c[2][1], c[2][2]), dd = id(c[3][0], c[3][1], c[3][2]);
                    // T1 = (a, b, cc), T2 = (a, cc, dd), both counter-clockwise in (p, q)
                    if (!flip) {
                        tris.insert(tris.end(), {a, b, cc, a, cc, dd});
                    } else {
                        tris.insert(tris.end(), {a, cc, b, a, dd, cc});
                    }
                }
        }
    }
}

void host_boundary_topology(int n, std::vector<int>& tris, const std::vector<int>& bidx,
                            std::vector<int>& inc_ptr, std::vector<int>& inc_slot) {
    surface_triangles(n, tris);
    const int n1 = n + 1;
    host_incidence(n1 * n1 * n1, tris, bidx, inc_ptr, inc_slot);
}

void launch_row_counts(int n, int* cnt, int* bflag, cudaStream_t st) {
    const int N = (n + 1) * (n + 1) * (n + 1);
    k_row_counts<<<(N + 255) / 256, 256, 0, st>>>(n, cnt, bflag);
}
void launch_scan(const int* in, int* out, int count, cudaStream_t st) {
    k_scan_single<<<1, 1024, 0, st>>>(in, out, count);
}
void launch_assemble(int n, const int* rowptr, const int* bpos, int* col, int* pkA, int* pkB, int* node,
                     cudaStream_t st) {
    const int N = (n + 1) * (n + 1) * (n + 1);
    k_assemble<<<(N + 127) / 128, 128, 0, st>>>(n, rowptr, bpos, col, pkA, pkB, node);
}
void launch_kcsr_count(int N, const int* rowptr, const int* pkA, int* cnt, cudaStream_t st) {
    k_kcsr_count<<<(N + 255) / 256, 256, 0, st>>>(N, rowptr, pkA, cnt);
}
void launch_kcsr_fill(int N, const int* rowptr, const int* col, const int* pkA, const int* kptr, int* kent,
                      cudaStream_t st) {
    k_kcsr_fill<<<(N + 255) / 256, 256, 0, st>>>(N, rowptr, col, pkA, kptr, kent);
}
void launch_boundary_ids(int N, const int* bflag, const int* bpos, int* bidx, cudaStream_t st) {
    k_boundary_ids<<<(N + 255) / 256, 256, 0, st>>>(N, bflag, bpos, bidx);
}
void launch_tets(int n, int* tets, cudaStream_t st) {
    const int T = 6 * n * n * n;
    k_tets<<<(T + 255) / 256, 256, 0, st>>>(n, tets);
}
void launch_bem_assemble(int n, int nb, int F, const int* bidx, const int* tris, const int* inc_ptr,
                         const int* inc_slot, const double* xyz, double* scratch, int nblocks, double* B64,
                         float* B32, cudaStream_t st) {
    k_bem_assemble<<<nblocks, 256, 0, st>>>(n, nb, F, bidx, tris, inc_ptr, inc_slot, xyz, scratch, B64, B32);
}
void launch_assemble_gen(int N, const double* xyz, const int* tets, const int* nt_ptr, const int* nt_idx,
                         const int* rowptr, const int* col, Dbl4* A64, float4* A32, Dbl4* Bt64,
                         float4* Bt32, double* Vn, double* d64, float* d32, cudaStream_t st) {
    k_assemble_gen<<<(N + 127) / 128, 128, 0, st>>>(N, xyz, tets, nt_ptr, nt_idx, rowptr, col, A64, A32, Bt64,
                                                   Bt32, Vn, d64, d32);
}
void launch_kcsr_count_gen(int N, const int* rowptr, const Dbl4* A64, int* cnt, cudaStream_t st) {
    k_kcsr_count_gen<<<(N + 255) / 256, 256, 0, st>>>(N, rowptr, A64, cnt);
}
void launch_kcsr_fill_gen(int N, const int* rowptr, const int* col, const Dbl4* A64, const int* kptr, int* kent,
                          double* k64, float* k32, cudaStream_t st) {
    k_kcsr_fill_gen<<<(N + 255) / 256, 256, 0, st>>>(N, rowptr, col, A64, kptr, kent, k64, k32);
}

// ---- general meshes: host topology ---------------------------------------------------
// Validates the tetrahedra, builds the node -> tetrahedron incidence (ascending
// tetrahedron ids), the CSR pattern (per row: the sorted distinct vertices of
// the incident tetrahedra), the surface (faces of exactly one tetrahedron,
// outward: the normal points away from the fourth vertex; smallest id first,
// cyclic order kept, rows sorted), the surface node ids (ascending) and the
// length unit L = (mean |det|)^(1/3).  Returns an empty string or the reason
// the mesh is rejected.
std::string host_general_topology(int N, int T, const int* tets, const double* xyz, GeneralTopology& g) {
    char buf[256];
    for (int t = 0; t < T; ++t) {
        const int* v = tets + 4 * (size_t)t;
        for (int k = 0; k < 4; ++k) {
            if (v[k] < 0 || v[k] >= N) {
                snprintf(buf, sizeof buf, "tetrahedron %d has node id %d outside [0, %d)", t, v[k], N);
                return buf;
            }
            for (int l = 0; l < k; ++l)
                if (v[l] == v[k]) {
                    snprintf(buf, sizeof buf, "tetrahedron %d repeats node %d", t, v[k]);
                    return buf;
                }
        }
    }
    g.nt_ptr.assign(N + 1, 0);
    for (size_t s = 0; s < 4 * (size_t)T; ++s) g.nt_ptr[tets[s] + 1] += 1;
    for (int i = 0; i < N; ++i) {
        if (g.nt_ptr[i + 1] == 0) {
            snprintf(buf, sizeof buf, "node %d belongs to no tetrahedron", i);
            return buf;
        }
        g.nt_ptr[i + 1] += g.nt_ptr[i];
    }
    g.nt_idx.assign(4 * (size_t)T, 0);
    {
        std::vector<int> fill(g.nt_ptr.begin(), g.nt_ptr.end() - 1);
        for (int t = 0; t < T; ++t)
            for (int k = 0; k < 4; ++k) g.nt_idx[fill[tets[4 * (size_t)t + k]]++] = t;
    }
    // determinants and the length unit
    double sum_ad = 0.0;
    g.det.assign(T, 0.0);
    for (int t = 0; t < T; ++t) {
        const int* v = tets + 4 * (size_t)t;
        double e[3][3];
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d) e[k][d] = xyz[3 * (size_t)v[k + 1] + d] - xyz[3 * (size_t)v[0] + d];
        const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) +
                           e[0][1] * (e[1][2] * e[2][0] - e[1][0] * e[2][2]) +
                           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        if (!(det != 0.0) || !std::isfinite(det)) {
            snprintf(buf, sizeof buf, "tetrahedron %d is degenerate (zero or non-finite volume)", t);
            return buf;
        }
        g.det[t] = det;
        sum_ad += fabs(det);
    }
    g.L = cbrt(sum_ad / (double)T);
    // CSR pattern
    g.rowptr.assign(N + 1, 0);
    g.col.clear();
    std::vector<int> nb;
    for (int i = 0; i < N; ++i) {
        nb.clear();
        for (int q = g.nt_ptr[i]; q < g.nt_ptr[i + 1]; ++q)
            for (int k = 0; k < 4; ++k) nb.push_back(tets[4 * (size_t)g.nt_idx[q] + k]);
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        g.col.insert(g.col.end(), nb.begin(), nb.end());
        g.rowptr[i + 1] = (int)g.col.size();
    }
    // surface faces
    struct Face { int k[3]; int t, opp; int v[3]; };
    std::vector<Face> faces(4 * (size_t)T);
    for (int t = 0; t < T; ++t)
        for (int o = 0; o < 4; ++o) {
            Face& f = faces[4 * (size_t)t + o];
            int c = 0;
            for (int k = 0; k < 4; ++k)
                if (k != o) f.v[c++] = tets[4 * (size_t)t + k];
            f.k[0] = f.v[0]; f.k[1] = f.v[1]; f.k[2] = f.v[2];
            std::sort(f.k, f.k + 3);
            f.t = t;
            f.opp = tets[4 * (size_t)t + o];
        }
    std::sort(faces.begin(), faces.end(), [](const Face& a, const Face& b) {
        if (a.k[0] != b.k[0]) return a.k[0] < b.k[0];
        if (a.k[1] != b.k[1]) return a.k[1] < b.k[1];
        if (a.k[2] != b.k[2]) return a.k[2] < b.k[2];
        return a.t < b.t;
    });
    std::vector<std::array<int, 3>> tris;
    for (size_t s = 0; s < faces.size();) {
        size_t e = s + 1;
        while (e < faces.size() && faces[e].k[0] == faces[s].k[0] && faces[e].k[1] == faces[s].k[1] &&
               faces[e].k[2] == faces[s].k[2])
            ++e;
        if (e - s > 2) {
            snprintf(buf, sizeof buf, "face (%d, %d, %d) belongs to %d tetrahedra", faces[s].k[0], faces[s].k[1],
                     faces[s].k[2], (int)(e - s));
            return buf;
        }
        if (e - s == 1) {
            const Face& f = faces[s];
            const double* a = xyz + 3 * (size_t)f.v[0];
            const double* b = xyz + 3 * (size_t)f.v[1];
            const double* c = xyz + 3 * (size_t)f.v[2];
            const double* o = xyz + 3 * (size_t)f.opp;
            const double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            const double ac[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            const double nr[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2],
                                  ab[0] * ac[1] - ab[1] * ac[0]};
            const double side = nr[0] * (o[0] - a[0]) + nr[1] * (o[1] - a[1]) + nr[2] * (o[2] - a[2]);
            std::array<int, 3> tri = {f.v[0], f.v[1], f.v[2]};
            if (side > 0) std::swap(tri[1], tri[2]);
            const int r = (tri[1] < tri[0] && tri[1] < tri[2]) ? 1 : (tri[2] < tri[0] && tri[2] < tri[1]) ? 2 : 0;
            tris.push_back({tri[r], tri[(r + 1) % 3], tri[(r + 2) % 3]});
        }
        s = e;
    }
    if (tris.empty()) return "the mesh has no surface";
    std::sort(tris.begin(), tris.end());
    g.tris.resize(3 * tris.size());
    for (size_t t = 0; t < tris.size(); ++t)
        for (int k = 0; k < 3; ++k) g.tris[3 * t + k] = tris[t][k];
    g.bidx = g.tris;
    std::sort(g.bidx.begin(), g.bidx.end());
    g.bidx.erase(std::unique(g.bidx.begin(), g.bidx.end()), g.bidx.end());
    return std::string();
}

void host_incidence(int N, const std::vector<int>& tris, const std::vector<int>& bidx, std::vector<int>& inc_ptr,
                    std::vector<int>& inc_slot) {
    const int nb = (int)bidx.size(), F = (int)tris.size() / 3;
    std::vector<int> pos(N, -1);
    for (int k = 0; k < nb; ++k) pos[bidx[k]] = k;
    inc_ptr.assign(nb + 1, 0);
    for (int s = 0; s < 3 * F; ++s) inc_ptr[pos[tris[s]] + 1] += 1;
    for (int k = 0; k < nb; ++k) inc_ptr[k + 1] += inc_ptr[k];
    inc_slot.assign(3 * F, 0);
    std::vector<int> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int s = 0; s < 3 * F; ++s) inc_slot[fill[pos[tris[s]]]++] = s;   // ascending slots per node
}

}  // namespace lbm
