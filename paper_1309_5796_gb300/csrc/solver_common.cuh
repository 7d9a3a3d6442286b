// Device helpers shared by the potential-solve kernels (solver.cu: one-CTA and
// cooperative-grid variants; pcg_cluster.cu: thread-block-cluster variant):
// vector loads and stores, deterministic block reductions, the stiffness row
// products, the divergence right-hand side and the kernel arguments.
#pragma once

#include <type_traits>

#include "lbm_host.h"

namespace lbm {

constexpr int MAXR = 16;                 // row length served by the unrolled gather (Kuhn rows: 15)

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

// Column sums for threads that each hold VEC consecutive columns: thread tid is
// row lane rl = tid / G of column group g = tid % G (columns g*VEC .. +VEC-1,
// C = G*VEC).  Fixed summation order; totals in out[q*C + c] (FP64).  The sums
// inside the block are taken in R (FP32 for the per-iteration dot products of
// the FP32 solves, whose per-thread partials are FP32 already: GB300 issues
// FP64 at a small fraction of the FP32 rate).  `scratch` holds at least
// NQV * max(bd/32, RB) * C values of R.
template <int NQV, int VEC, typename R = double>
__device__ __forceinline__ void block_reduce_cols(R (&v)[NQV][VEC], R* scratch, double* out, int C, int G,
                                                  int RB) {
    const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, g = tid % G;
    int nrow;
    if (G <= 32 && (32 % G) == 0) {
        // lanes of one column group differ by multiples of G within the warp
        for (int off = 16; off >= G; off >>= 1)
#pragma unroll
            for (int q = 0; q < NQV; ++q)
#pragma unroll
                for (int k = 0; k < VEC; ++k) v[q][k] += __shfl_xor_sync(0xffffffffu, v[q][k], off);
        nrow = bd >> 5;
        if (lane < G)
#pragma unroll
            for (int q = 0; q < NQV; ++q)
#pragma unroll
                for (int k = 0; k < VEC; ++k) scratch[(q * nrow + warp) * C + g * VEC + k] = v[q][k];
    } else {
        nrow = RB;
        const int rl = tid / G;
        if (tid < RB * G)
#pragma unroll
            for (int q = 0; q < NQV; ++q)
#pragma unroll
                for (int k = 0; k < VEC; ++k) scratch[(q * nrow + rl) * C + g * VEC + k] = v[q][k];
    }
    __syncthreads();
    for (int t = tid; t < NQV * C; t += bd) {
        const int q = t / C, c = t % C;
        R acc = R(0);
        for (int r = 0; r < nrow; ++r) acc += scratch[(q * nrow + r) * C + c];
        out[q * C + c] = (double)acc;
    }
    __syncthreads();
}

// Totals over blocks of partials part[blk][C][4] (quantities q0..q0+NQV-1), in a
// fixed order, into out[q*C + c] (threads hold VEC columns each, as above).
template <int NQV, int VEC>
__device__ __forceinline__ void cross_reduce_cols(const double* part, int q0, int nblk, int C, int G, int RB,
                                                  double* scratch, double* out) {
    const int tid = threadIdx.x, g = tid % G, rl = tid / G;
    double v[NQV][VEC];
#pragma unroll
    for (int q = 0; q < NQV; ++q)
#pragma unroll
        for (int k = 0; k < VEC; ++k) v[q][k] = 0.0;
    if (tid < RB * G) {
#pragma unroll 2
        for (int blk = rl; blk < nblk; blk += RB)
#pragma unroll
            for (int k = 0; k < VEC; ++k)
#pragma unroll
                for (int q = 0; q < NQV; ++q) v[q][k] += __ldcg(&part[((size_t)blk * C + g * VEC + k) * 4 + q0 + q]);
    }
    block_reduce_cols<NQV, VEC>(v, scratch, out, C, G, RB);
}

template <typename T, int VEC> struct VecOf;
template <> struct VecOf<float, 4> { using type = float4; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<double, 2> { using type = double2; };

template <typename T, int VEC, bool CG>
__device__ __forceinline__ void vload(T (&d)[VEC], const T* p) {
    if constexpr (std::is_same<T, double>::value && VEC == 4) {   // four doubles: two 16-byte loads
        double2 a, b;
        if constexpr (CG) { a = __ldcg(reinterpret_cast<const double2*>(p)); b = __ldcg(reinterpret_cast<const double2*>(p + 2)); }
        else { a = *reinterpret_cast<const double2*>(p); b = *reinterpret_cast<const double2*>(p + 2); }
        d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
    } else {
        using V = typename VecOf<T, VEC>::type;
        V x;
        if constexpr (CG) x = __ldcg(reinterpret_cast<const V*>(p));
        else x = *reinterpret_cast<const V*>(p);
        if constexpr (VEC == 4) { d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w; }
        else { d[0] = x.x; d[1] = x.y; }
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void vstore(T* p, const T (&d)[VEC]) {
    if constexpr (std::is_same<T, double>::value && VEC == 4) {
        *reinterpret_cast<double2*>(p) = make_double2(d[0], d[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(d[2], d[3]);
    } else {
        using V = typename VecOf<T, VEC>::type;
        V x;
        if constexpr (VEC == 4) { x.x = d[0]; x.y = d[1]; x.z = d[2]; x.w = d[3]; }
        else { x.x = d[0]; x.y = d[1]; }
        *reinterpret_cast<V*>(p) = x;
    }
}

constexpr double MP_INNER = 1e-4;   // residual reduction of one FP32 cycle of a mixed-iteration solve
constexpr int MP_MAX_CYCLES = 16;
constexpr int MAXK = 8;   // stiffness entries served by the unrolled gather (interior Kuhn rows: 7)

// Value tables of a general mesh in the precision of the kernel.
template <typename T> struct GenTab;
template <> struct GenTab<float> {
    using V4 = float4;
    static __device__ __forceinline__ const float4* A(const MeshView& M) { return M.gA32; }
    static __device__ __forceinline__ const float4* Bt(const MeshView& M) { return M.gB32; }
    static __device__ __forceinline__ const float* k(const MeshView& M) { return M.gk32; }
    static __device__ __forceinline__ const float* d(const MeshView& M) { return M.gd32; }
};
template <> struct GenTab<double> {
    using V4 = Dbl4;
    static __device__ __forceinline__ const Dbl4* A(const MeshView& M) { return M.gA64; }
    static __device__ __forceinline__ const Dbl4* Bt(const MeshView& M) { return M.gB64; }
    static __device__ __forceinline__ const double* k(const MeshView& M) { return M.gk64; }
    static __device__ __forceinline__ const double* d(const MeshView& M) { return M.gd64; }
};

// acc[k] = sum_j K_ij (v_j - v_i) (DIFF) or sum_j K_ij v_j for VEC consecutive
// columns of one row of the stiffness-only CSR.  The packed entries are read
// first -- one load per lane and a warp broadcast when the whole warp works on
// this row (warp_row) -- then every vector gather of the row is issued before
// any arithmetic.  warp_row requires the full warp to take part.
// General meshes (GEN): the values come from kval, and rows of any length are
// served MAXK entries at a time.
template <typename T, int VEC, bool CG, bool DIFF, bool GEN>
__device__ __forceinline__ void row_kv(const int* __restrict__ kent, const T* __restrict__ kval, int e0, int e1,
                                       const T* v, int C, int c0, const T (&vi)[VEC], T (&acc)[VEC],
                                       bool warp_row) {
    if constexpr (GEN) {
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] = T(0);
        for (int base = e0; base < e1; base += MAXK) {
            int w[MAXK];
            T kv[MAXK];
            if (warp_row) {
                const int lane = threadIdx.x & 31;
                const bool has = lane < MAXK && base + lane < e1;
                const int mine = has ? __ldg(&kent[base + lane]) : 0;
                const T mk = has ? __ldg(&kval[base + lane]) : T(0);
#pragma unroll
                for (int t = 0; t < MAXK; ++t) {
                    w[t] = __shfl_sync(0xffffffffu, mine, t);
                    kv[t] = __shfl_sync(0xffffffffu, mk, t);
                }
            } else {
#pragma unroll
                for (int t = 0; t < MAXK; ++t) {
                    const bool has = base + t < e1;
                    w[t] = has ? __ldg(&kent[base + t]) : 0;
                    kv[t] = has ? __ldg(&kval[base + t]) : T(0);
                }
            }
            T vj[MAXK][VEC];
#pragma unroll
            for (int t = 0; t < MAXK; ++t) {
                if (w[t] != 0) vload<T, VEC, CG>(vj[t], &v[(size_t)((unsigned)w[t] >> 8) * C + c0]);
                else
#pragma unroll
                    for (int k = 0; k < VEC; ++k) vj[t][k] = vi[k];
            }
#pragma unroll
            for (int t = 0; t < MAXK; ++t)
#pragma unroll
                for (int k = 0; k < VEC; ++k) acc[k] += kv[t] * (DIFF ? (vj[t][k] - vi[k]) : vj[t][k]);
        }
        return;
    }
    int w[MAXK];
    if (warp_row) {
        const int lane = threadIdx.x & 31;
        const int mine = (lane < MAXK && e0 + lane < e1) ? __ldg(&kent[e0 + lane]) : 0;
#pragma unroll
        for (int t = 0; t < MAXK; ++t) w[t] = __shfl_sync(0xffffffffu, mine, t);
    } else {
#pragma unroll
        for (int t = 0; t < MAXK; ++t) w[t] = (e0 + t < e1) ? __ldg(&kent[e0 + t]) : 0;
    }
    T vj[MAXK][VEC];
#pragma unroll
    for (int t = 0; t < MAXK; ++t) {
        if (w[t] != 0) vload<T, VEC, CG>(vj[t], &v[(size_t)((unsigned)w[t] >> 8) * C + c0]);
        else
#pragma unroll
            for (int k = 0; k < VEC; ++k) vj[t][k] = vi[k];
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) acc[k] = T(0);
#pragma unroll
    for (int t = 0; t < MAXK; ++t) {
        const T kk = T(sbyte(w[t], 0));
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] += kk * (DIFF ? (vj[t][k] - vi[k]) : vj[t][k]);
    }
    for (int e = e0 + MAXK; e < e1; ++e) {
        const int ww = __ldg(&kent[e]);
        T x[VEC];
        vload<T, VEC, CG>(x, &v[(size_t)((unsigned)ww >> 8) * C + c0]);
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] += T(sbyte(ww, 0)) * (DIFF ? (x[k] - vi[k]) : x[k]);
    }
}

// As row_kv for a warp that owns the row, with the row's packed entries
// already in registers (lane l holds entry e0 + l, l < 32: `mine`, and its
// value `mk` for general meshes), so that no index load sits on the row's
// critical path; entries beyond the 32nd are loaded here.
template <typename T, int VEC, bool CG, bool DIFF, bool GEN>
__device__ __forceinline__ void row_kv_warp(int mine, T mk, int e0, int e1, const int* __restrict__ kent,
                                            const T* __restrict__ kval, const T* v, int C, int c0,
                                            const T (&vi)[VEC], T (&acc)[VEC]) {
#pragma unroll
    for (int k = 0; k < VEC; ++k) acc[k] = T(0);
    const int cnt = e1 - e0;
    for (int base = 0; base < cnt; base += MAXK) {
        int w[MAXK];
        T kv[MAXK];
#pragma unroll
        for (int t = 0; t < MAXK; ++t) {
            const int idx = base + t;   // warp-uniform
            if (idx < 32) {
                w[t] = __shfl_sync(0xffffffffu, mine, idx);
                kv[t] = GEN ? __shfl_sync(0xffffffffu, mk, idx) : T(0);
            } else {
                const bool has = idx < cnt;
                w[t] = has ? __ldg(&kent[e0 + idx]) : 0;
                kv[t] = (GEN && has) ? __ldg(&kval[e0 + idx]) : T(0);
            }
            if (!GEN) kv[t] = T(sbyte(w[t], 0));
        }
        T vj[MAXK][VEC];
#pragma unroll
        for (int t = 0; t < MAXK; ++t) {
            if (w[t] != 0) vload<T, VEC, CG>(vj[t], &v[(size_t)((unsigned)w[t] >> 8) * C + c0]);
            else
#pragma unroll
                for (int k = 0; k < VEC; ++k) vj[t][k] = vi[k];
        }
#pragma unroll
        for (int t = 0; t < MAXK; ++t)
#pragma unroll
            for (int k = 0; k < VEC; ++k) acc[k] += kv[t] * (DIFF ? (vj[t][k] - vi[k]) : vj[t][k]);
    }
}

// The trial point of an instance whose base point is `cur`, in T.
template <typename T>
__device__ __forceinline__ const T* trial_m(const BatchView<T>& V, int cur, int N) {
    if constexpr (sizeof(T) == 4) {
        (void)cur;
        (void)N;
        return V.m32;
    } else {
        return V.m + (size_t)(1 - cur) * N * 3 * V.B;
    }
}

template <typename T>
struct PcgArgs {
    MeshView M;
    BatchView<T> V;
    int mode;          // 0: stage 1 (u1 | w), 1: stage 2 (u2 | uT)
    double tol2;       // squared relative residual
    int max_iter;
    unsigned* bar;
    int* err;
    unsigned long long* sweeps;
    double* fin;
};

// b_i = (1/4) sum_j Gint_ij . m_j (the divergence right-hand side) at the trial point
// meval: the trial point in T (FP32 kernels: its FP32 copy)
template <typename T, bool GEN>
__device__ __forceinline__ double rhs_b(const int* __restrict__ col, const int* __restrict__ pkA,
                                        const typename GenTab<T>::V4* __restrict__ gA, int e0, int e1,
                                        const T* meval, int B, int b) {
    T acc = T(0);
    for (int e = e0; e < e1; ++e) {
        const size_t mj = (size_t)(__ldg(&col[e]) & 0x7fffffff) * 3 * B + b;
        if constexpr (GEN) {
            const typename GenTab<T>::V4 a = gA[e];
            acc += a.y * meval[mj] + a.z * meval[mj + B] + a.w * meval[mj + 2 * B];
        } else {
            const int w = __ldg(&pkA[e]);
            acc += T(sbyte(w, 1)) * meval[mj] + T(sbyte(w, 2)) * meval[mj + B] + T(sbyte(w, 3)) * meval[mj + 2 * B];
        }
    }
    return 0.25 * (double)acc;
}

// Grid-wide totals of per-block partials part[blk][C][4] (quantities
// q0..q0+NQV-1) into out[q*C + c] of every block: after a barrier one warp of
// the grid sums each (column, quantity) over the blocks (lanes stride the
// blocks, then a fixed xor tree) into fin; after a second barrier every block
// copies fin.  Fixed order, so all blocks and all runs get the same bits.
template <int NQV>
__device__ __forceinline__ bool grid_reduce(const double* part, int q0, int C, double* fin, double* out,
                                            unsigned* bar, unsigned& epoch, int* err) {
    if (!grid_sync(bar, gridDim.x, epoch, err)) return false;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int gw = blockIdx.x * nw + (threadIdx.x >> 5), tw = gridDim.x * nw;
    const int P = C * NQV;
    for (int pidx = gw; pidx < P; pidx += tw) {
        const int c = pidx / NQV, q = pidx % NQV;
        double acc = 0.0;
        for (int blk = lane; blk < (int)gridDim.x; blk += 32) acc += __ldcg(&part[((size_t)blk * C + c) * 4 + q0 + q]);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) fin[pidx] = acc;
    }
    if (!grid_sync(bar, gridDim.x, epoch, err)) return false;
    for (int t = threadIdx.x; t < P; t += blockDim.x) out[(t % NQV) * C + t / NQV] = __ldcg(&fin[t]);
    __syncthreads();
    return true;
}

// rhs_b for the four consecutive instances b0..b0+3 (b0 a multiple of 4, B too):
// the row's column and coupling entries are read once, the trial point as
// 16-byte vectors of four instances; per instance the sum of rhs_b.
template <typename T, bool GEN>
__device__ __forceinline__ void rhs_b4(const int* __restrict__ col, const int* __restrict__ pkA,
                                       const typename GenTab<T>::V4* __restrict__ gA, int e0, int e1,
                                       const T* meval, int B, int b0, double (&f)[4]) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int e = e0; e < e1; ++e) {
        const size_t mj = (size_t)(__ldg(&col[e]) & 0x7fffffff) * 3 * B + b0;
        T gx, gy, gz;
        if constexpr (GEN) {
            const typename GenTab<T>::V4 a = gA[e];
            gx = a.y; gy = a.z; gz = a.w;
        } else {
            const int w = __ldg(&pkA[e]);
            gx = T(sbyte(w, 1)); gy = T(sbyte(w, 2)); gz = T(sbyte(w, 3));
        }
        const T g3[3] = {gx, gy, gz};
#pragma unroll
        for (int c = 0; c < 3; ++c) {   // one component at a time (few live registers)
            T mc[4];
            vload<T, 4, false>(mc, meval + mj + (size_t)c * B);
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += g3[c] * mc[k];
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) f[k] = 0.25 * (double)acc[k];
}

}  // namespace lbm
