// Hot path of one steepest-descent iteration on the device, for a batch of B
// independent instances sharing one mesh (node-major, instance-minor layout:
// value (i, b) at [i*B + b], vector component c at [(i*3 + c)*B + b]).
//
//   trial_update  Eq. (8) curvilinear (Cayley) step from the base point
//   pcg_solve     the scalar-potential solves (Table 2 "solve linear system"):
//                 Jacobi-preconditioned CG, persistent cooperative kernel
//   bem_product   u2|S = B u1|S, the hybrid FEM/BEM open boundary (Sec. 3.1)
//   field_eval    effective field (exchange SpMV + anisotropy + Zeeman + stray
//                 field), H = -m x grad phi (Sec. 2.1), energies, and the
//                 dot products of the BB rule (Sec. 2.3), per-block partials
//   decide        Sec. 2.3 step control: first-step line search, BB1/BB2 with
//                 the adaptive rule, nonmonotone test over the last 20
//                 energies, stop test (Sec. 3.1)
#include <math.h>
#include <stdio.h>

#include "lbm_host.h"

namespace lbm {

constexpr int PCG_THREADS = 512;        // grid-wide (cooperative) variant
constexpr int PCG_SINGLE_THREADS = 1024; // one-CTA variant for small batches
constexpr int FIELD_THREADS = 256;
constexpr int MAXR = 16;                 // row length served by the unrolled gather (Kuhn rows: 15)
constexpr long long SINGLE_CTA_MAX_WORK = 24576;   // N * B up to which one CTA solves

template <typename T, bool CG> __device__ __forceinline__ T ld_vec(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Deterministic per-instance block reduction of NQV values per thread.  Thread
// tid holds row lane rl = tid / B of instance b = tid % B; the totals land in
// out[q*B + b].  Bit q of maxmask selects max instead of sum.
template <int NQV>
__device__ __forceinline__ void block_reduce_inst(double (&v)[NQV], double* scratch, double* out, int B, int RB,
                                                  unsigned maxmask) {
    const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (B <= 32 && (32 % B) == 0) {
        // lanes of one instance differ by multiples of B within the warp
        for (int off = 16; off >= B; off >>= 1)
#pragma unroll
            for (int q = 0; q < NQV; ++q) {
                const double o = __shfl_xor_sync(0xffffffffu, v[q], off);
                v[q] = ((maxmask >> q) & 1u) ? fmax(v[q], o) : v[q] + o;
            }
        if (lane < B)
#pragma unroll
            for (int q = 0; q < NQV; ++q) scratch[q * bd + warp * B + lane] = v[q];
        __syncthreads();
        const int nw = bd >> 5;
        if (tid < B)
#pragma unroll
            for (int q = 0; q < NQV; ++q) {
                double acc = scratch[q * bd + tid];
                for (int w = 1; w < nw; ++w) {
                    const double o = scratch[q * bd + w * B + tid];
                    acc = ((maxmask >> q) & 1u) ? fmax(acc, o) : acc + o;
                }
                out[q * B + tid] = acc;
            }
    } else {
#pragma unroll
        for (int q = 0; q < NQV; ++q) scratch[q * bd + tid] = (tid < RB * B) ? v[q] : 0.0;
        __syncthreads();
        if (tid < B)
#pragma unroll
            for (int q = 0; q < NQV; ++q) {
                double acc = scratch[q * bd + tid];
                for (int r = 1; r < RB; ++r) {
                    const double o = scratch[q * bd + r * B + tid];
                    acc = ((maxmask >> q) & 1u) ? fmax(acc, o) : acc + o;
                }
                out[q * B + tid] = acc;
            }
    }
    __syncthreads();
}

// Totals over blocks of partials part[blk][B][4] (quantities q0..q0+NQV-1), in a
// fixed order, into out[q*B + b].
template <int NQV>
__device__ __forceinline__ void cross_reduce(const double* part, int q0, int nblk, int B, int RB, double* scratch,
                                             double* out) {
    const int tid = threadIdx.x, b = tid % B, rl = tid / B;
    double v[NQV];
#pragma unroll
    for (int q = 0; q < NQV; ++q) v[q] = 0.0;
    if (tid < RB * B) {
#pragma unroll 4
        for (int blk = rl; blk < nblk; blk += RB)
#pragma unroll
            for (int q = 0; q < NQV; ++q) v[q] += __ldcg(&part[((size_t)blk * B + b) * 4 + q0 + q]);
    }
    block_reduce_inst<NQV>(v, scratch, out, B, RB, 0u);
}

// sum_j K_ij (v_j - v_i) (DIFF) or sum_j K_ij v_j over one CSR row; all column
// indices, then all values, are loaded before any arithmetic so the gathers of
// a row are in flight together.
template <typename T, bool CG, bool DIFF>
__device__ __forceinline__ T row_k(const int* __restrict__ col, const int* __restrict__ pkA, int e0, int e1,
                                   const T* v, int B, int b, T vi) {
    int cj[MAXR], kj[MAXR];
#pragma unroll
    for (int t = 0; t < MAXR; ++t) {
        const int e = e0 + t;
        const bool ok = e < e1;
        cj[t] = ok ? (__ldg(&col[e]) & 0x7fffffff) : -1;
        kj[t] = ok ? sbyte(__ldg(&pkA[e]), 0) : 0;
    }
    T vj[MAXR];
#pragma unroll
    for (int t = 0; t < MAXR; ++t) vj[t] = cj[t] >= 0 ? ld_vec<T, CG>(&v[(size_t)cj[t] * B + b]) : vi;
    T acc = T(0);
#pragma unroll
    for (int t = 0; t < MAXR; ++t) acc += T(kj[t]) * (DIFF ? (vj[t] - vi) : vj[t]);
    for (int e = e0 + MAXR; e < e1; ++e) {
        const T x = ld_vec<T, CG>(&v[(size_t)(col[e] & 0x7fffffff) * B + b]);
        acc += T(sbyte(pkA[e], 0)) * (DIFF ? (x - vi) : x);
    }
    return acc;
}

template <typename T>
struct PcgArgs {
    MeshView M;
    BatchView<T> V;
    int mode;          // 0: Neumann (u1), 1: Dirichlet (u2)
    double tol2;       // squared relative residual
    int max_iter;
    unsigned* bar;
    int* err;
    unsigned long long* sweeps;
};

template <bool SINGLE>
__device__ __forceinline__ bool pcg_sync(unsigned* bar, unsigned& epoch, int* err) {
    if constexpr (SINGLE) {
        __syncthreads();
        return true;
    } else {
        return grid_sync(bar, gridDim.x, epoch, err);
    }
}

// Jacobi-PCG on Kint for B instances at once, fused so that every iteration
// needs two synchronisations (grid barriers, or __syncthreads in the one-CTA
// variant):
//   A: w = K z, p = z + beta p, q = w + beta q (= K p), partial p.q
//   B: alpha = rho/p.q, x += alpha p, r -= alpha q, z = r / K_ii, partials r.z, r.r
// Neumann: rhs = (1/4) Gint m at the trial point, made consistent (mean
// removed); the residual is tested without its mean; the solution is gauged to
// zero V-weighted mean and its surface values are gathered for the BEM.
// Dirichlet: the surface values come from the BEM product; surface rows are
// frozen (r = z = p = q = 0).
template <typename T, bool SINGLE>
__global__ void __launch_bounds__(SINGLE ? PCG_SINGLE_THREADS : PCG_THREADS, 1) k_pcg(PcgArgs<T> A) {
    extern __shared__ double sm[];
    constexpr bool CG = !SINGLE;
    const int bd = blockDim.x, tid = threadIdx.x;
    const int B = A.V.B, RB = bd / B;
    const bool lane = tid < RB * B;
    const int b = tid % B, rl = tid / B;
    double* scratch = sm;                // [4][bd]
    double* out = scratch + 4 * bd;      // [4][B]
    double* s_rho = out + 4 * B;         // [B]
    double* s_rhop = s_rho + B;
    double* s_ab = s_rhop + B;
    double* s_tol = s_ab + B;
    int* s_flag = (int*)(s_tol + B);
    int* s_act = s_flag + B;
    int* s_cur = s_act + B;
    int* s_it = s_cur + B;
    __shared__ int s_all;

    for (int i = tid; i < B; i += bd) {
        s_act[i] = A.V.st[i].phase != PH_DONE;
        s_cur[i] = A.V.st[i].cur;
        s_it[i] = 0;
        s_rhop[i] = 1.0;
    }
    __syncthreads();
    const int N = A.M.N;
    const bool dir = A.mode == 1;
    const bool act = lane && s_act[b];
    const int row0 = blockIdx.x * RB + rl, rstride = gridDim.x * RB;
    const int* __restrict__ rowptr = A.M.rowptr;
    const int* __restrict__ col = A.M.col;
    const int* __restrict__ pkA = A.M.pkA;
    const int* __restrict__ node = A.M.node;
    T* __restrict__ x = dir ? A.V.u2 : A.V.u1;
    T* __restrict__ r = A.V.r;
    T* __restrict__ z = A.V.z;
    T* __restrict__ p = A.V.p;
    T* __restrict__ q = A.V.q;
    double* part_rz = A.V.part;
    double* part_pq = A.V.part + (size_t)gridDim.x * B * 4;
    unsigned epoch = 0;
    const double* meval = A.V.m + (size_t)(1 - s_cur[b]) * N * 3 * B;

    if (dir) {
        if (act)
            for (int row = row0; row < N; row += rstride) {
                const int bp = (int)((unsigned)node[row] >> 16);
                if (bp) x[(size_t)row * B + b] = A.V.ub2[(size_t)(bp - 1) * B + b];
            }
        if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;
    }
    {   // residual of the warm start
        // Neumann: the system is singular with null space span{1}; the right-hand
        // side is made consistent (sum zero) by removing its mean before use.
        double psum[1] = {0.0};
        if (act)
            for (int row = row0; row < N; row += rstride) {
                const int nd = node[row];
                const size_t ib = (size_t)row * B + b;
                if (dir && ((unsigned)nd >> 16)) { r[ib] = T(0); z[ib] = T(0); p[ib] = T(0); q[ib] = T(0); continue; }
                const int e0 = rowptr[row], e1 = rowptr[row + 1];
                const T xi = x[ib];
                const T kx = row_k<T, CG, true>(col, pkA, e0, e1, x, B, b, xi);
                T rhs = T(0);
                if (!dir) {
                    double acc = 0.0;
                    for (int e = e0; e < e1; ++e) {
                        const int w = pkA[e];
                        const size_t mj = (size_t)(col[e] & 0x7fffffff) * 3 * B + b;
                        acc += sbyte(w, 1) * meval[mj] + sbyte(w, 2) * meval[mj + B] + sbyte(w, 3) * meval[mj + 2 * B];
                    }
                    rhs = T(0.25 * acc);
                } else {
                    for (int e = e0; e < e1; ++e) {
                        const int c = col[e];
                        if (c < 0) rhs -= T(sbyte(pkA[e], 0)) * ld_vec<T, CG>(&x[(size_t)(c & 0x7fffffff) * B + b]);
                    }
                }
                r[ib] = dir ? -kx : rhs - kx;
                z[ib] = rhs;                          // kept for the second pass
                p[ib] = T(0);
                q[ib] = T(0);
                psum[0] += (double)rhs;
            }
        double mean = 0.0;
        if (!dir) {
            block_reduce_inst<1>(psum, scratch, out, B, RB, 0u);
            if (SINGLE) {
                if (tid < B) s_ab[tid] = out[tid] / (double)N;
            } else {
                if (tid < B) part_pq[((size_t)blockIdx.x * B + tid) * 4 + 2] = out[tid];
                if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;
                cross_reduce<1>(part_pq, 2, gridDim.x, B, RB, scratch, out);
                if (tid < B) s_ab[tid] = out[tid] / (double)N;
            }
            __syncthreads();
            mean = s_ab[b];
        }
        double v4[4] = {0.0, 0.0, 0.0, 0.0};   // r.z, r.r, rhs.rhs, sum r
        if (act)
            for (int row = row0; row < N; row += rstride) {
                const int nd = node[row];
                if (dir && ((unsigned)nd >> 16)) continue;
                const size_t ib = (size_t)row * B + b;
                const T rhs = z[ib] - T(mean);
                const T ri = r[ib] - T(mean);
                const T zi = ri / T((nd >> 8) & 0xff);
                r[ib] = ri;
                z[ib] = zi;
                v4[0] += (double)ri * (double)zi;
                v4[1] += (double)ri * (double)ri;
                v4[2] += (double)rhs * (double)rhs;
                v4[3] += (double)ri;
            }
        block_reduce_inst<4>(v4, scratch, out, B, RB, 0u);
        if (!SINGLE) {
            if (tid < B)
                for (int k = 0; k < 4; ++k) part_rz[((size_t)blockIdx.x * B + tid) * 4 + k] = out[k * B + tid];
            if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;
        }
    }
    for (int k = 0;; ++k) {
        if (!SINGLE) cross_reduce<4>(part_rz, 0, gridDim.x, B, RB, scratch, out);
        if (tid < B) {
            const double rho = out[tid];
            // Neumann: test the residual without its null-space (mean) component,
            // which rounding feeds and CG cannot remove
            const double sr = out[3 * B + tid];
            const double rr = dir ? out[B + tid] : fmax(out[B + tid] - sr * sr / (double)N, 0.0);
            if (k == 0) s_tol[tid] = A.tol2 * out[2 * B + tid];
            const int conv = !s_act[tid] || rr <= s_tol[tid] || k >= A.max_iter;
            s_ab[tid] = (k == 0 || conv) ? 0.0 : rho / s_rhop[tid];
            s_rho[tid] = rho;
            s_flag[tid] = conv;
        }
        __syncthreads();
        if (tid == 0) {
            int all = 1;
            for (int i = 0; i < B; ++i) all &= s_flag[i];
            s_all = all;
        }
        __syncthreads();
        if (s_all) break;
        const bool run = act && !s_flag[b];
        double ppq[1] = {0.0};
        if (run) {
            const T beta = T(s_ab[b]);
            for (int row = row0; row < N; row += rstride) {
                const int nd = node[row];
                if (dir && ((unsigned)nd >> 16)) continue;
                const size_t ib = (size_t)row * B + b;
                const T w = row_k<T, CG, false>(col, pkA, rowptr[row], rowptr[row + 1], z, B, b, T(0));
                const T pi = z[ib] + beta * p[ib];
                const T qi = w + beta * q[ib];
                p[ib] = pi;
                q[ib] = qi;
                ppq[0] += (double)pi * (double)qi;
            }
        }
        block_reduce_inst<1>(ppq, scratch, out, B, RB, 0u);
        if (!SINGLE) {
            if (tid < B) part_pq[((size_t)blockIdx.x * B + tid) * 4] = out[tid];
            if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;
            cross_reduce<1>(part_pq, 0, gridDim.x, B, RB, scratch, out);
        }
        if (tid < B) s_ab[tid] = s_flag[tid] ? 0.0 : s_rho[tid] / out[tid];
        __syncthreads();
        double v4[4] = {0.0, 0.0, 0.0, 0.0};
        if (run) {
            const T alpha = T(s_ab[b]);
            for (int row = row0; row < N; row += rstride) {
                const int nd = node[row];
                if (dir && ((unsigned)nd >> 16)) continue;
                const size_t ib = (size_t)row * B + b;
                const T xi = x[ib] + alpha * p[ib];
                const T ri = r[ib] - alpha * q[ib];
                const T zi = ri / T((nd >> 8) & 0xff);
                x[ib] = xi;
                r[ib] = ri;
                z[ib] = zi;
                v4[0] += (double)ri * (double)zi;
                v4[1] += (double)ri * (double)ri;
                v4[3] += (double)ri;
            }
        }
        block_reduce_inst<4>(v4, scratch, out, B, RB, 0u);
        if (!SINGLE) {
            if (tid < B)
                for (int kk = 0; kk < 4; ++kk)
                    if (kk != 2) part_rz[((size_t)blockIdx.x * B + tid) * 4 + kk] = out[kk * B + tid];
            if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;
        } else {
            __syncthreads();
        }
        if (tid < B) {
            s_rhop[tid] = s_rho[tid];
            if (!s_flag[tid]) s_it[tid] += 1;
        }
    }
    if (blockIdx.x == 0) {
        for (int i = tid; i < B; i += bd) {
            if (dir) A.V.st[i].cg2 += s_it[i];
            else A.V.st[i].cg1 += s_it[i];
        }
        if (tid == 0 && A.sweeps) {
            int kmax = 0;
            for (int i = 0; i < B; ++i) kmax = max(kmax, s_it[i]);
            A.sweeps[dir ? 1 : 0] += (unsigned long long)kmax;
        }
    }
    if (dir) return;
    // gauge: remove the V-weighted mean; gather the surface values
    {
        double pv[1] = {0.0};
        if (act)
            for (int row = row0; row < N; row += rstride)
                pv[0] += (double)(node[row] & 0xff) * (double)x[(size_t)row * B + b];
        block_reduce_inst<1>(pv, scratch, out, B, RB, 0u);
        if (!SINGLE) {
            if (tid < B) part_pq[((size_t)blockIdx.x * B + tid) * 4 + 1] = out[tid];
            if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;
            cross_reduce<1>(part_pq, 1, gridDim.x, B, RB, scratch, out);
        }
        if (tid < B) s_ab[tid] = out[tid] / A.M.vsum;
        __syncthreads();
        if (act) {
            const T mean = T(s_ab[b]);
            for (int row = row0; row < N; row += rstride) {
                const size_t ib = (size_t)row * B + b;
                const T xi = x[ib] - mean;
                x[ib] = xi;
                const int bp = (int)((unsigned)node[row] >> 16);
                if (bp) A.V.ub1[(size_t)(bp - 1) * B + b] = xi;
            }
        }
    }
}

size_t pcg_part_elems(int num_sms, int B) { return (size_t)2 * num_sms * B * 4; }

template <typename T>
int pcg_solve(const Launch& L, const MeshView& M, const BatchView<T>& V, int mode, double tol, int max_iter,
              int* iters_dev) {
    (void)iters_dev;
    const int B = V.B;
    PcgArgs<T> a{M, V, mode, tol * tol, max_iter, L.bar, L.err, L.sweeps};
    void* args[] = {&a};
    cudaError_t e;
    if ((long long)M.N * B <= SINGLE_CTA_MAX_WORK) {
        const size_t smem = sizeof(double) * (4 * PCG_SINGLE_THREADS + 8 * B) + sizeof(int) * 4 * B;
        static bool attr_set[2] = {false, false};
        if (!attr_set[sizeof(T) == 8]) {
            cudaFuncSetAttribute(k_pcg<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            attr_set[sizeof(T) == 8] = true;
        }
        e = cudaLaunchKernel((void*)k_pcg<T, true>, dim3(1), dim3(PCG_SINGLE_THREADS), args, smem, L.stream);
    } else {
        const int RB = PCG_THREADS / B;
        const size_t smem = sizeof(double) * (4 * PCG_THREADS + 8 * B) + sizeof(int) * 4 * B;
        static int occ_cache[2] = {0, 0};
        int& occ = occ_cache[sizeof(T) == 8];
        if (!occ) {
            cudaFuncSetAttribute(k_pcg<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg<T, false>, PCG_THREADS, 64 * 1024);
            if (occ < 1) occ = 1;
            if (occ > 1) occ = 1;
        }
        int nblk = (M.N + RB - 1) / RB;
        const int maxblk = occ * L.num_sms;
        if (nblk > maxblk) nblk = maxblk;
        cudaMemsetAsync(L.bar, 0, sizeof(unsigned), L.stream);
        e = cudaLaunchCooperativeKernel((void*)k_pcg<T, false>, dim3(nblk), dim3(PCG_THREADS), args, smem, L.stream);
    }
    *L.launches += 1;
    return e == cudaSuccess ? 0 : (int)e;
}

// ---- BEM product -------------------------------------------------------------------
template <typename T>
__global__ void k_gemv(const T* __restrict__ A, const T* __restrict__ x, T* __restrict__ y, int nb) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int row = warp; row < nb; row += nw) {
        const T* a = A + (size_t)row * nb;
        double acc = 0.0;
        for (int j = lane; j < nb; j += 32) acc += (double)(a[j] * x[j]);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[row] = T(acc);
    }
}

// Y[nb][B] = A[nb][nb] X[nb][B]; 64x64 tiles, 256 threads, 4x4 outputs each.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const T* __restrict__ A, const T* __restrict__ X, T* __restrict__ Y,
                                              int nb, int B) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 4];
    __shared__ T Xs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    T acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < nb; k0 += BK) {
        for (int l = tid; l < BM * BK; l += 256) {
            const int mm = l / BK, kk = l % BK;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < nb && gk < nb) ? A[(size_t)gm * nb + gk] : T(0);
        }
        for (int l = tid; l < BK * BN; l += 256) {
            const int kk = l / BN, nn = l % BN;
            const int gk = k0 + kk, gn = n0 + nn;
            Xs[kk][nn] = (gk < nb && gn < B) ? X[(size_t)gk * B + gn] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], xv[4];
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
            for (int j = 0; j < 4; ++j) xv[j] = Xs[kk][tx * 4 + j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * xv[j];
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < nb && gn < B) Y[(size_t)gm * B + gn] = acc[i][j];
        }
}

template <typename T> __host__ __device__ inline const T* bem_ptr(const MeshView& M);
template <> __host__ __device__ inline const double* bem_ptr<double>(const MeshView& M) { return M.B64; }
template <> __host__ __device__ inline const float* bem_ptr<float>(const MeshView& M) { return M.B32; }

template <typename T>
void bem_product(const Launch& L, const MeshView& M, const BatchView<T>& V) {
    const T* Bm = bem_ptr<T>(M);
    if (V.B == 1) {
        const int warps = M.nb;
        int blocks = (warps * 32 + 255) / 256;
        if (blocks > 8 * L.num_sms) blocks = 8 * L.num_sms;
        k_gemv<T><<<blocks, 256, 0, L.stream>>>(Bm, V.ub1, V.ub2, M.nb);
    } else {
        dim3 grid((M.nb + 63) / 64, (V.B + 63) / 64);
        k_gemm<T><<<grid, 256, 0, L.stream>>>(Bm, V.ub1, V.ub2, M.nb, V.B);
    }
    *L.launches += 1;
}

// ---- effective field, gradient, energies and step dot products -----------------------
int field_blocks(const Launch& L, const MeshView& M, int B) {
    const int RB = FIELD_THREADS / B;
    int nblk = (M.N + RB - 1) / RB;
    const int maxblk = 4 * L.num_sms;
    return nblk < maxblk ? nblk : maxblk;
}

template <typename T>
__global__ void __launch_bounds__(FIELD_THREADS) k_field(MeshView M, BatchView<T> V, int demag) {
    extern __shared__ double fsm[];
    double* scratch = fsm;                        // [Q_COUNT][bd]
    double* out = fsm + Q_COUNT * FIELD_THREADS;  // [Q_COUNT][B]
    const int tid = threadIdx.x;
    const int B = V.B, RB = FIELD_THREADS / B;
    const bool lane = tid < RB * B;
    const int b = tid % B, rl = tid / B;
    const int N = M.N;
    double acc[Q_COUNT];
#pragma unroll
    for (int k = 0; k < Q_COUNT; ++k) acc[k] = 0.0;
    const int phase = lane ? V.st[b].phase : PH_DONE;
    if (lane && phase != PH_DONE) {
        const int cur = V.st[b].cur;
        const InstConst ic = V.ic[b];
        const double* mt = V.m + (size_t)(1 - cur) * N * 3 * B;
        const double* mb = V.m + (size_t)cur * N * 3 * B;
        double* Ht = V.H + (size_t)(1 - cur) * N * 3 * B;
        const double* Hb = V.H + (size_t)cur * N * 3 * B;
        for (int row = blockIdx.x * RB + rl; row < N; row += gridDim.x * RB) {
            const int nd = M.node[row];
            const double vi = (double)(nd & 0xff);
            const size_t i3 = (size_t)row * 3 * B + b;
            const double mx = mt[i3], my = mt[i3 + B], mz = mt[i3 + 2 * B];
            T ex0 = T(0), ex1 = T(0), ex2 = T(0), hd0 = T(0), hd1 = T(0), hd2 = T(0);
            const int e0 = M.rowptr[row], e1 = M.rowptr[row + 1];
            for (int e = e0; e < e1; ++e) {
                const int j = __ldg(&M.col[e]) & 0x7fffffff;
                const T k = T(sbyte(__ldg(&M.pkA[e]), 0));
                const size_t j3 = (size_t)j * 3 * B + b;
                // difference form: exact zero for a uniform state, no cancellation
                ex0 += k * T(mt[j3] - mx);
                ex1 += k * T(mt[j3 + B] - my);
                ex2 += k * T(mt[j3 + 2 * B] - mz);
                if (demag) {
                    const int wb = __ldg(&M.pkB[e]);
                    const T u = V.u1[(size_t)j * B + b] + V.u2[(size_t)j * B + b];
                    hd0 += T(sbyte(wb, 0)) * u;
                    hd1 += T(sbyte(wb, 1)) * u;
                    hd2 += T(sbyte(wb, 2)) * u;
                }
            }
            const double m[3] = {mx, my, mz};
            const double kx[3] = {(double)ex0, (double)ex1, (double)ex2};
            const double ma = m[0] * ic.a[0] + m[1] * ic.a[1] + m[2] * ic.a[2];
            const double hd[3] = {-(double)hd0 / vi, -(double)hd1 / vi, -(double)hd2 / vi};
            double h[3];
            for (int c = 0; c < 3; ++c) h[c] = -4.0 * ic.lam * kx[c] / vi + ic.Q * ma * ic.a[c] + ic.hz[c] + hd[c];
            // H = -m x grad phi = (V/12) m x h ;  g = m x H
            const double mh[3] = {m[1] * h[2] - m[2] * h[1], m[2] * h[0] - m[0] * h[2], m[0] * h[1] - m[1] * h[0]};
            const double Hv[3] = {vi / 12.0 * mh[0], vi / 12.0 * mh[1], vi / 12.0 * mh[2]};
            Ht[i3] = Hv[0];
            Ht[i3 + B] = Hv[1];
            Ht[i3 + 2 * B] = Hv[2];
            if (V.hout) {
                V.hout[i3] = h[0];
                V.hout[i3 + B] = h[1];
                V.hout[i3 + 2 * B] = h[2];
            }
            const double g[3] = {m[1] * Hv[2] - m[2] * Hv[1], m[2] * Hv[0] - m[0] * Hv[2],
                                 m[0] * Hv[1] - m[1] * Hv[0]};
            const double bm[3] = {mb[i3], mb[i3 + B], mb[i3 + 2 * B]};
            const double bH[3] = {Hb[i3], Hb[i3 + B], Hb[i3 + 2 * B]};
            const double gb[3] = {bm[1] * bH[2] - bm[2] * bH[1], bm[2] * bH[0] - bm[0] * bH[2],
                                  bm[0] * bH[1] - bm[1] * bH[0]};
            const double mxa[3] = {m[1] * ic.a[2] - m[2] * ic.a[1], m[2] * ic.a[0] - m[0] * ic.a[2],
                                   m[0] * ic.a[1] - m[1] * ic.a[0]};
            acc[Q_EEX] += ic.lam / 6.0 * (m[0] * kx[0] + m[1] * kx[1] + m[2] * kx[2]);
            acc[Q_EAN] += ic.Q / 24.0 * vi * (mxa[0] * mxa[0] + mxa[1] * mxa[1] + mxa[2] * mxa[2]);
            acc[Q_EZ] -= vi / 12.0 * (m[0] * ic.hz[0] + m[1] * ic.hz[1] + m[2] * ic.hz[2]);
            acc[Q_ED] -= vi / 24.0 * (m[0] * hd[0] + m[1] * hd[1] + m[2] * hd[2]);
            acc[Q_TORQUE] = fmax(acc[Q_TORQUE], sqrt(mh[0] * mh[0] + mh[1] * mh[1] + mh[2] * mh[2]));
            acc[Q_HMAX] = fmax(acc[Q_HMAX], sqrt(Hv[0] * Hv[0] + Hv[1] * Hv[1] + Hv[2] * Hv[2]));
            double ss = 0.0, sy = 0.0, yy = 0.0, gg = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double sc = m[c] - bm[c], yc = g[c] - gb[c];
                ss += sc * sc;
                sy += sc * yc;
                yy += yc * yc;
                gg += g[c] * g[c];
            }
            acc[Q_GG] += gg;
            acc[Q_SS] += ss;
            acc[Q_SY] += sy;
            acc[Q_YY] += yy;
            acc[Q_MX] += vi * m[0];
            acc[Q_MY] += vi * m[1];
            acc[Q_MZ] += vi * m[2];
            if (!(isfinite(h[0]) && isfinite(h[1]) && isfinite(h[2]))) acc[Q_BAD] = 1.0;
        }
    }
    const unsigned maxmask = (1u << Q_TORQUE) | (1u << Q_HMAX) | (1u << Q_BAD);
    block_reduce_inst<Q_COUNT>(acc, scratch, out, B, RB, maxmask);
    if (tid < B)
        for (int k = 0; k < Q_COUNT; ++k) V.part[((size_t)blockIdx.x * B + tid) * NQ + k] = out[k * B + tid];
}

template <typename T>
void field_eval(const Launch& L, const MeshView& M, const BatchView<T>& V, int demag) {
    const int nblk = field_blocks(L, M, V.B);
    const size_t smem = sizeof(double) * Q_COUNT * (FIELD_THREADS + V.B);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_field<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr_set = true;
    }
    k_field<T><<<nblk, FIELD_THREADS, smem, L.stream>>>(M, V, demag);
    *L.launches += 1;
}

// ---- Sec. 2.3 step control, one warp per instance ---------------------------------------
__device__ double hist_max(const InstState& s) {
    double e = s.hist[0];
    for (int k = 1; k < s.nhist; ++k) e = fmax(e, s.hist[k]);
    return e;
}

__global__ void k_decide(const double* __restrict__ part, int nblk, InstState* st, const InstConst* ic, StepOpts so,
                         double vsum, int B) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    const int b = warp;
    double v[Q_COUNT];
    for (int k = 0; k < Q_COUNT; ++k) {
        const bool mx = (k == Q_TORQUE || k == Q_HMAX || k == Q_BAD);
        double acc = 0.0;
        for (int blk = lane; blk < nblk; blk += 32) {
            const double x = part[((size_t)blk * B + b) * NQ + k];
            acc = mx ? fmax(acc, x) : acc + x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, acc, o);
            acc = mx ? fmax(acc, y) : acc + y;
        }
        v[k] = acc;
    }
    if (lane != 0) return;
    InstState& s = st[b];
    if (s.phase == PH_DONE) return;
    const double E = ((v[Q_EEX] + v[Q_EAN]) + v[Q_EZ]) + v[Q_ED];
    s.evals += 1;
    if (v[Q_BAD] > 0.0 || !isfinite(E)) {
        s.status = 4;   // LBM_E_NAN
        s.phase = PH_DONE;
        return;
    }
    const double gg = v[Q_GG], torque = v[Q_TORQUE];
    const bool conv = so.grad_tol > 0.0 ? (gg < so.grad_tol) : (torque < so.tol);
    bool accept;
    if (s.phase == PH_INIT) {
        accept = true;
    } else if (s.phase == PH_SEARCH) {
        accept = E <= s.E_ref - so.c1 * s.tau * s.gg_base;
    } else {
        const double emax = hist_max(s);
        accept = !(E > emax);
        if (!accept) {
            s.phase = PH_SEARCH;
            s.E_ref = emax;
            s.line_searches += 1;
            s.backtracks = 0;
        }
    }
    if (!accept) {
        s.backtracks += 1;
        if (s.backtracks > so.max_backtracks) {
            s.status = 6;   // LBM_E_LINESEARCH
            s.phase = PH_DONE;
        } else {
            s.tau *= 0.5;
        }
        return;
    }
    // accepted: the trial becomes the base point
    const bool init = s.phase == PH_INIT;
    s.cur ^= 1;
    s.E = E;
    s.terms[0] = v[Q_EEX];
    s.terms[1] = v[Q_EAN];
    s.terms[2] = v[Q_EZ];
    s.terms[3] = v[Q_ED];
    s.torque = torque;
    s.gg = gg;
    s.gg_base = gg;
    s.mean_m[0] = v[Q_MX] / vsum;
    s.mean_m[1] = v[Q_MY] / vsum;
    s.mean_m[2] = v[Q_MZ] / vsum;
    const int mem = so.memory < HIST_MAX ? so.memory : HIST_MAX;
    if (init) {
        s.hist[0] = E;
        s.nhist = 1;
        s.hpos = 1 % mem;
        s.iters = 0;
        s.line_searches = 0;
        s.backtracks = 0;
        s.ntau2 = 0;
        s.kappa = so.kappa0;
        if (conv) { s.status = 0; s.phase = PH_DONE; return; }
        if (so.max_iter <= 0) { s.status = 3; s.phase = PH_DONE; return; }
        s.tau = 1.0 / v[Q_HMAX];
        s.phase = PH_SEARCH;
        s.E_ref = E;
        s.line_searches = 1;
        return;
    }
    s.hist[s.hpos] = E;
    s.hpos = (s.hpos + 1) % mem;
    if (s.nhist < mem) s.nhist += 1;
    s.iters += 1;
    if (conv) { s.status = 0; s.phase = PH_DONE; return; }
    if (s.iters >= so.max_iter) { s.status = 3; s.phase = PH_DONE; return; }
    const double ss = v[Q_SS], sy = v[Q_SY], yy = v[Q_YY];
    double tau = s.tau;
    if (sy > 0.0) {
        const double t1 = ss / sy, t2 = sy / yy;
        const int ma = so.m_alpha < MALPHA_MAX ? so.m_alpha : MALPHA_MAX;
        if (s.ntau2 < ma) {
            s.tau2[s.ntau2++] = t2;
        } else {
            for (int k = 1; k < ma; ++k) s.tau2[k - 1] = s.tau2[k];
            s.tau2[ma - 1] = t2;
        }
        if (t2 / t1 <= s.kappa) {
            double mn = s.tau2[0];
            for (int k = 1; k < s.ntau2; ++k) mn = fmin(mn, s.tau2[k]);
            tau = mn;
            s.kappa *= 0.9;
        } else {
            tau = t1;
            s.kappa *= 1.1;
        }
    }
    s.tau = fmin(fmax(tau, so.tau_min), so.tau_max);
    s.phase = PH_BB;
    s.backtracks = 0;
}

template <typename T>
void decide(const Launch& L, const MeshView& M, const BatchView<T>& V, const StepOpts& so, int nblk_field) {
    const int threads = 128;
    const int blocks = (V.B * 32 + threads - 1) / threads;
    k_decide<<<blocks, threads, 0, L.stream>>>(V.part, nblk_field, V.st, V.ic, so, M.vsum, V.B);
    *L.launches += 1;
}

// ---- Eq. (8): the curvilinear step ------------------------------------------------------
template <typename T>
__global__ void k_trial(int N, BatchView<T> V) {
    const int B = V.B;
    const size_t total = (size_t)N * B;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        const size_t row = t / B;
        const int phase = V.st[b].phase;
        if (phase == PH_DONE) continue;
        const int cur = V.st[b].cur;
        const size_t i3 = row * 3 * B + b;
        const double* mb = V.m + (size_t)cur * N * 3 * B;
        double* mt = V.m + (size_t)(1 - cur) * N * 3 * B;
        if (phase == PH_INIT) {
            mt[i3] = mb[i3];
            mt[i3 + B] = mb[i3 + B];
            mt[i3 + 2 * B] = mb[i3 + 2 * B];
            continue;
        }
        // x = [(1 - |w|^2) m - 2 m x w + 2 (m.w) w] / (1 + |w|^2),  w = tau H / 2
        const double* Hb = V.H + (size_t)cur * N * 3 * B;
        const double ht = 0.5 * V.st[b].tau;
        const double m0 = mb[i3], m1 = mb[i3 + B], m2 = mb[i3 + 2 * B];
        const double w0 = ht * Hb[i3], w1 = ht * Hb[i3 + B], w2 = ht * Hb[i3 + 2 * B];
        const double ww = w0 * w0 + w1 * w1 + w2 * w2;
        const double mw = m0 * w0 + m1 * w1 + m2 * w2;
        const double c0 = m1 * w2 - m2 * w1, c1 = m2 * w0 - m0 * w2, c2 = m0 * w1 - m1 * w0;
        const double den = 1.0 + ww;
        mt[i3] = ((1.0 - ww) * m0 - 2.0 * c0 + 2.0 * mw * w0) / den;
        mt[i3 + B] = ((1.0 - ww) * m1 - 2.0 * c1 + 2.0 * mw * w1) / den;
        mt[i3 + 2 * B] = ((1.0 - ww) * m2 - 2.0 * c2 + 2.0 * mw * w2) / den;
    }
}

template <typename T>
void trial_update(const Launch& L, const MeshView& M, const BatchView<T>& V) {
    const size_t total = (size_t)M.N * V.B;
    size_t blocks = (total + 255) / 256;
    if (blocks > (size_t)8 * L.num_sms) blocks = (size_t)8 * L.num_sms;
    k_trial<T><<<(unsigned)blocks, 256, 0, L.stream>>>(M.N, V);
    *L.launches += 1;
}

// ---- state reset and layout conversion -------------------------------------------------
__global__ void k_reset(InstState* st, int B, int set_cur0) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    InstState& s = st[b];
    s.phase = PH_INIT;
    s.status = 3;
    if (set_cur0) s.cur = 0;
    s.iters = s.evals = s.line_searches = s.backtracks = 0;
    s.nhist = s.hpos = s.ntau2 = 0;
    s.cg1 = s.cg2 = 0;
}

void reset_states(const Launch& L, InstState* st, int B, const StepOpts& so, int set_cur0) {
    (void)so;
    k_reset<<<(B + 127) / 128, 128, 0, L.stream>>>(st, B, set_cur0);
    *L.launches += 1;
}

template <typename T>
__global__ void k_pack_m(int N, BatchView<T> V, const double* __restrict__ in) {
    const int B = V.B;
    const size_t total = (size_t)B * N * 3;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        const size_t ic = t / B;   // i*3 + c
        const size_t i = ic / 3, c = ic % 3;
        const int cur = V.st[b].cur;
        V.m[(size_t)cur * N * 3 * B + t] = in[((size_t)b * N + i) * 3 + c];
    }
}

template <typename T>
__global__ void k_unpack_m(int N, BatchView<T> V, double* __restrict__ out) {
    const int B = V.B;
    const size_t total = (size_t)B * N * 3;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        const size_t ic = t / B;
        const size_t i = ic / 3, c = ic % 3;
        const int cur = V.st[b].cur;
        out[((size_t)b * N + i) * 3 + c] = V.m[(size_t)cur * N * 3 * B + t];
    }
}

template <typename T>
__global__ void k_unpack_field(int N, BatchView<T> V, double* __restrict__ h, double* __restrict__ u, double cell) {
    const int B = V.B;
    const size_t total = (size_t)B * N;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        const size_t i = t / B;
        const double Js = V.ic[b].Js;
        if (h)
            for (int c = 0; c < 3; ++c) h[((size_t)b * N + i) * 3 + c] = Js * V.hout[(i * 3 + c) * B + b];
        if (u) {
            u[((size_t)b * 2 + 0) * N + i] = cell * (double)V.u1[t];
            u[((size_t)b * 2 + 1) * N + i] = cell * (double)V.u2[t];
        }
    }
}

template <typename T>
void pack_m(const Launch& L, const MeshView& M, const BatchView<T>& V, const double* staged) {
    k_pack_m<T><<<4 * L.num_sms, 256, 0, L.stream>>>(M.N, V, staged);
    *L.launches += 1;
}
template <typename T>
void unpack_m(const Launch& L, const MeshView& M, const BatchView<T>& V, double* staged) {
    k_unpack_m<T><<<4 * L.num_sms, 256, 0, L.stream>>>(M.N, V, staged);
    *L.launches += 1;
}
template <typename T>
void unpack_field(const Launch& L, const MeshView& M, const BatchView<T>& V, double* h, double* u) {
    k_unpack_field<T><<<4 * L.num_sms, 256, 0, L.stream>>>(M.N, V, h, u, M.cell);
    *L.launches += 1;
}

#define LBM_INSTANTIATE(T)                                                                               \
    template int pcg_solve<T>(const Launch&, const MeshView&, const BatchView<T>&, int, double, int, int*); \
    template void bem_product<T>(const Launch&, const MeshView&, const BatchView<T>&);                     \
    template void field_eval<T>(const Launch&, const MeshView&, const BatchView<T>&, int);                 \
    template void trial_update<T>(const Launch&, const MeshView&, const BatchView<T>&);                    \
    template void decide<T>(const Launch&, const MeshView&, const BatchView<T>&, const StepOpts&, int);    \
    template void pack_m<T>(const Launch&, const MeshView&, const BatchView<T>&, const double*);           \
    template void unpack_m<T>(const Launch&, const MeshView&, const BatchView<T>&, double*);               \
    template void unpack_field<T>(const Launch&, const MeshView&, const BatchView<T>&, double*, double*);

LBM_INSTANTIATE(float)
LBM_INSTANTIATE(double)

}  // namespace lbm
