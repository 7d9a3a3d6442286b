// Potential solves (Table 2 "solve linear system"; Sec. 3.1 "magnetic scalar
// potential") by Jacobi-preconditioned CG with one thread-block cluster per
// group of CPC systems, for batches with many systems.
//
// The systems of a batch are independent, so nothing needs to be shared across
// the whole grid: cluster k (CL = 4, 8 or 16 CTAs) solves the k-th group of CPC
// columns [g*CPC, (g+1)*CPC) of the [N][2B] system layout that still has an
// active instance, over all N rows, CTA r of the cluster owning the contiguous
// rows [r*rpc, (r+1)*rpc); when few groups remain active (the end of a batch)
// the host picks a shape with more CTAs per cluster.  Every reduction of the
// iteration (p.q; r.z, r.r, sum r; the Neumann mean and the gauge) is a block
// sum in a fixed order, then a fixed-order sum over the cluster's CTAs read
// through distributed shared memory after one hardware cluster barrier: every
// CTA gets the same bits, so every CTA takes the same decisions, and no CTA
// ever waits on a memory flag (no software grid barrier, no time limit needed).
//
// The preconditioned residual z of the cluster's systems lives in the CTAs'
// shared memory (rows of a CTA in its own, neighbours in other CTAs of the
// cluster read by ld.shared::cluster), so the stiffness product's gathers never
// touch L2; p, q, r and x stay in global memory in the batch layout.
//
// Iteration and numerics are those of the grid-wide kernel k_pcg (solver.cu):
//   A: w = K z, p = z + beta p, q = w + beta q (= K p), partial p.q
//   B: alpha = rho/p.q, x += alpha p, r -= alpha q, z = r / K_ii, partials r.z, r.r, sum r
// with the Neumann mean removal, the null-space-free residual test, the
// V-weighted gauge, Dirichlet surface rows frozen, and (MP) FP64 potentials
// iterated in FP32 with the FP64 residual recomputed at every restart.
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "solver_common.cuh"

namespace lbm {
namespace {

// threads per CTA (8 systems per cluster: 768 threads, 80 registers; 4
// systems: 1024, 64 registers) and rows per thread and pass of the iteration
// loops (all loads of a pass are issued before its arithmetic).  Measured on
// the 30^3-cell cube with 64 instances: 1024 threads and one row (29 us per
// iteration) beat 512 threads and two rows (36 us): more warps hide the
// shared-memory and barrier latency better than more rows per warp
template <int CPC> constexpr int cl_threads() { return CPC == 8 ? 768 : 1024; }
template <int CPC> constexpr int cl_rows() { return 1; }
constexpr int CL_NW = 32;           // warps of the largest CTA (reduction scratch)
constexpr size_t CL_SMEM_MAX = 227 * 1024;
constexpr int CHK = 4;             // stiffness entries gathered per step of the row product

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_index() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// All threads of all CTAs of the cluster; release/acquire at cluster scope, so
// shared (local and distributed) and global writes before it are visible to
// the cluster's threads after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t peer_u32(uint32_t a, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float4 ld_peer4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}
__device__ __forceinline__ double ld_peer_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}

// Shared-memory layout of one CTA (offsets in bytes).
struct ClSmem {
    size_t z, dtab, scratch, out, slots, cold, coldf, coli, total;
};
__host__ __device__ inline ClSmem cl_smem(int rpc, int cpc) {
    ClSmem s;
    size_t o = 0;
    auto take = [&o](size_t b) { const size_t at = o; o = (o + b + 15) & ~(size_t)15; return at; };
    s.z = take(sizeof(float) * (size_t)rpc * cpc);
    s.dtab = take(sizeof(float) * (size_t)rpc);
    s.scratch = take(sizeof(double) * 4 * CL_NW * cpc);
    s.out = take(sizeof(double) * 4 * cpc);
    s.slots = take(sizeof(double) * 2 * 4 * cpc);
    s.cold = take(sizeof(double) * 5 * cpc);
    s.coldf = take(sizeof(float) * cpc);
    s.coli = take(sizeof(int) * 5 * cpc);
    s.total = o;
    return s;
}

template <typename T, bool MP, bool GEN, int CPC, int CL>
__global__ void __launch_bounds__(cl_threads<CPC>(), 1) k_pcg_cluster(PcgArgs<T> A, int rpc) {
    static_assert(sizeof(T) == 4 || MP, "FP32 work vectors: FP32 solves, or FP64 solves iterated in FP32");
    using W = float;
    constexpr int CL_THREADS = cl_threads<CPC>();
    constexpr int VEC = 4, G = CPC / VEC, RB = CL_THREADS / G, U = cl_rows<CPC>();
    extern __shared__ __align__(16) unsigned char smraw[];
    const ClSmem lay = cl_smem(rpc, CPC);
    float* zs = reinterpret_cast<float*>(smraw + lay.z);           // [rpc][CPC]
    // per own row: 1/K_ii (the Jacobi preconditioner), negative on surface rows
    float* dtab = reinterpret_cast<float*>(smraw + lay.dtab);       // [rpc]
    double* scratch = reinterpret_cast<double*>(smraw + lay.scratch);
    double* out = reinterpret_cast<double*>(smraw + lay.out);       // [4][CPC]
    double* slots = reinterpret_cast<double*>(smraw + lay.slots);   // [2][4][CPC]
    double* s_rho = reinterpret_cast<double*>(smraw + lay.cold);
    double* s_rhop = s_rho + CPC;
    double* s_ab = s_rhop + CPC;
    double* s_tol = s_ab + CPC;
    double* s_tin = s_tol + CPC;
    // alpha or beta of the current step as FP32 for the row loops (a conversion
    // from FP64 per thread would issue at GB300's FP64 rate)
    float* s_abf = reinterpret_cast<float*>(smraw + lay.coldf);
    int* s_flag = reinterpret_cast<int*>(smraw + lay.coli);
    int* s_act = s_flag + CPC;
    int* s_cur = s_act + CPC;
    int* s_it = s_cur + CPC;
    int* s_done = s_it + CPC;

    const int tid = threadIdx.x;
    const int g = tid % G, rl = tid / G;
    const unsigned rank = cluster_rank();
    const int B = A.V.B, C = 2 * B, N = A.M.N;
    // The cluster's group of CPC systems: the k-th group with an active
    // instance (k = the cluster's index), so that a launch with fewer, larger
    // clusters serves the groups still iterating; clusters beyond the active
    // groups have nothing to do.  Every CTA reads the same phases (no kernel of
    // this launch changes them), so all agree.
    __shared__ unsigned s_bal[8];
    __shared__ int s_grp;
    int grp;
    {
        const int ng = 2 * B / CPC;   // <= 256: B <= 512
        bool a = false;
        if (tid < ng)
            for (int i = 0; i < CPC; ++i) a |= A.V.st[(tid * CPC + i) % B].phase != PH_DONE;
        const unsigned bal = __ballot_sync(0xffffffffu, a);
        if ((tid & 31) == 0 && tid < 256) s_bal[tid >> 5] = bal;
        if (tid == 0) s_grp = -1;
        __syncthreads();
        if (a) {
            int k = __popc(bal & ((1u << (tid & 31)) - 1u));
            for (int w = 0; w < (tid >> 5); ++w) k += __popc(s_bal[w]);
            if (k == (int)cluster_index()) s_grp = tid;
        }
        if (tid == 0 && rank == 0 && cluster_index() == 0) {
            int nact = 0;
            for (int w = 0; w < (ng + 31) / 32; ++w) nact += __popc(s_bal[w]);
            if (nact > (int)(gridDim.x / CL)) atomicOr(A.err, DEV_ERR_SHAPE);   // groups left unsolved
        }
        __syncthreads();
        grp = s_grp;
    }
    const int col0 = (grp < 0 ? 0 : grp) * CPC;
    const int c0 = col0 + g * VEC;                 // first column of this thread
    const int cl0 = g * VEC;                       // the same within the cluster's columns
    const int mode = A.mode;
    const bool neu = (mode == col0 / B);           // B % CPC == 0: one kind of system per cluster
    const int lo = (int)rank * rpc, hi = min(N, lo + rpc);
    const uint32_t zbase = smem_u32(zs);

    for (int i = tid; i < CPC; i += CL_THREADS) {
        const int b = (col0 + i) % B;
        s_act[i] = grp >= 0 && A.V.st[b].phase != PH_DONE;
        s_cur[i] = A.V.st[b].cur;
        s_it[i] = 0;
        s_done[i] = 0;
        s_tin[i] = 0.0;
        s_rhop[i] = 1.0;
    }
    {
        const int lo0 = (int)cluster_rank() * rpc, hi0 = min(A.M.N, lo0 + rpc);
        for (int row = lo0 + (int)threadIdx.x; row < hi0; row += CL_THREADS) {
            const int nd = A.M.node[row];
            const float dinv = 1.f / (GEN ? GenTab<float>::d(A.M)[row] : float((nd >> 8) & 0xff));
            dtab[row - lo0] = ((unsigned)nd >> 16) ? -dinv : dinv;
        }
    }
    __syncthreads();
    bool actk[VEC], any_act = false;
    int bk[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        actk[k] = s_act[cl0 + k] != 0;
        any_act |= actk[k];
        bk[k] = (c0 + k) % B;
    }
    int cluster_act = 0;
    for (int i = 0; i < CPC; ++i) cluster_act |= s_act[i];

    const int* __restrict__ rowptr = A.M.rowptr;
    const int* __restrict__ col = A.M.col;
    const int* __restrict__ pkA = A.M.pkA;
    const int* __restrict__ node = A.M.node;
    const int* __restrict__ kptr = A.M.kptr;
    const int* __restrict__ kent = A.M.kent;
    const T* __restrict__ kvalT = GEN ? GenTab<T>::k(A.M) : nullptr;
    const W* __restrict__ kvalW = GEN ? GenTab<W>::k(A.M) : nullptr;
    const W* __restrict__ kdiagW = GEN ? GenTab<W>::d(A.M) : nullptr;
    const typename GenTab<T>::V4* __restrict__ gA = GEN ? GenTab<T>::A(A.M) : nullptr;
    T* __restrict__ x = mode ? A.V.U2 : A.V.U1;
    // The work vectors r, p, q and d of this cluster's systems use a grouped
    // layout: the cluster's slice [N][CPC] is contiguous, so the rows a warp
    // touches are one contiguous run (the [N][2B] layout would give every row
    // its own cache line).  d, the FP32 correction that alpha p accumulates into
    // (folded into x at the end of every cycle), lives in the upper half of r's
    // FP64 storage (MP) or in the global z array (z itself is in shared memory).
    const size_t gbase = (size_t)(grp < 0 ? 0 : grp) * N * CPC;
    W* __restrict__ r = reinterpret_cast<W*>(A.V.r) + gbase;
    W* __restrict__ xacc = (MP ? reinterpret_cast<W*>(A.V.r) + (size_t)N * C : reinterpret_cast<W*>(A.V.z)) + gbase;
    W* __restrict__ p = reinterpret_cast<W*>(A.V.p) + gbase;
    W* __restrict__ q = reinterpret_cast<W*>(A.V.q) + gbase;
    int par = 0;
    const double* last = nullptr;   // slot of the latest r.z, r.r, ref.ref, sum r partials

    // Cluster reductions of NQV quantities (per-thread values of VEC columns):
    // partial() sums the CTA's values (warp shuffles, then the warps in order)
    // into this CTA's slot slots[par] and passes the cluster barrier; totals()
    // then adds the CL slots of the cluster (the same bits in every CTA);
    // reduce() does both and leaves every total in out[q*CPC + c] for all threads.
    // The slots alternate, so a slot is rewritten only after two more cluster
    // barriers, when every CTA has read it.
    auto partial = [&](auto& vals) -> double* {
        constexpr int NQV = sizeof(vals) / sizeof(vals[0]);
        using R = typename std::remove_reference<decltype(vals[0][0])>::type;
        R* scr = reinterpret_cast<R*>(scratch);
        const int lane = tid & 31, warp = tid >> 5;
        constexpr int NWC = CL_THREADS / 32;
        for (int off = 16; off >= G; off >>= 1)
#pragma unroll
            for (int qq = 0; qq < NQV; ++qq)
#pragma unroll
                for (int k = 0; k < VEC; ++k) vals[qq][k] += __shfl_xor_sync(0xffffffffu, vals[qq][k], off);
        if (lane < G)
#pragma unroll
            for (int qq = 0; qq < NQV; ++qq)
#pragma unroll
                for (int k = 0; k < VEC; ++k) scr[(qq * NWC + warp) * CPC + cl0 + k] = vals[qq][k];
        __syncthreads();
        double* mine = slots + par * 4 * CPC;
        if (tid < NQV * CPC) {
            const int qq = tid / CPC, c = tid % CPC;
            R acc = R(0);
            for (int w = 0; w < NWC; ++w) acc += scr[(qq * NWC + w) * CPC + c];
            mine[tid] = (double)acc;
        }
        par ^= 1;
        cluster_sync();
        return mine;
    };
    // totals(slot, nq): every total of the first nq quantities into out[q*CPC + c],
    // all at once: thread t loads rank t % CL's partial of value t / CL, and the
    // CL consecutive lanes of a value add theirs in a fixed butterfly (the same
    // bits in every lane and every CTA of the cluster)
    auto totals = [&](const double* slot, int nq) {
        const int nv = nq * CPC;
        if ((tid >> 5) <= ((nv * CL - 1) >> 5)) {   // only the warps holding values (FP64 issues slowly)
            double v = 0.0;
            if (tid < nv * CL) v = ld_peer_f64(peer_u32(smem_u32(slot + tid / CL), (unsigned)(tid % CL)));
#pragma unroll
            for (int off = CL / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (tid < nv * CL && tid % CL == 0) out[tid / CL] = v;
        }
        __syncthreads();
    };
    auto reduce = [&](auto& vals) {
        constexpr int NQV = sizeof(vals) / sizeof(vals[0]);
        totals(partial(vals), NQV);
    };
    // z of row j (this thread's VEC columns): own rows from this CTA's shared
    // memory, others from the owning CTA's through the cluster window
    // On the Kuhn cube a row's couplings reach at most 1 + (n+1) + (n+1)^2 rows
    // away; when a CTA's slab is at least that long, a row outside this CTA's
    // slab lies in a neighbouring CTA's (no division for the owner).
    const int s2k = A.M.n + 1, halo = 1 + s2k + s2k * s2k;
    const bool adj_only = !GEN && rpc >= halo;
    auto zrow = [&](int j) -> float4 {
        if (j >= lo && j < lo + rpc) return *reinterpret_cast<const float4*>(zs + (j - lo) * CPC + cl0);
        const unsigned o = adj_only ? (j < lo ? rank - 1u : rank + 1u) : (unsigned)(j / rpc);
        return ld_peer4(peer_u32(zbase + (uint32_t)(((j - (int)o * rpc) * CPC + cl0) * 4), o));
    };

    if (cluster_act) {
        // Dirichlet systems: surface values (stage 1 adjoint: zero; stage 2 forward: B u1_S)
        if (!neu && any_act)
            for (int row = lo + rl; row < hi; row += RB) {
                const int bp = (int)((unsigned)node[row] >> 16);
                if (!bp) continue;
#pragma unroll
                for (int k = 0; k < VEC; ++k)
                    if (actk[k]) x[(size_t)row * C + c0 + k] = mode ? A.V.ub_out[(size_t)(bp - 1) * C + bk[k]] : T(0);
            }
        {
            const W zero[VEC] = {};
            for (int row = lo + rl; row < hi; row += RB) vstore<W, VEC>(&xacc[row * CPC + cl0], zero);
        }
        cluster_sync();
        for (int cycle = 0;; ++cycle) {
            {   // residual of the current x (gathers of other CTAs' rows bypass L1)
                double psum[1][VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) psum[0][k] = 0.0;
                for (int row = lo + rl; row < hi; row += RB) {
                    const int bp = (int)((unsigned)node[row] >> 16);
                    const unsigned ib = (unsigned)row * (unsigned)C + (unsigned)c0;   // < 2^31: checked at launch
                    const unsigned go = (unsigned)(row * CPC + cl0);               // grouped work vectors
                    T xi[VEC], kx[VEC];
                    W rv[VEC];
                    float zr[VEC];
                    vload<T, VEC, false>(xi, &x[ib]);
                    row_kv<T, VEC, true, true, GEN>(kent, kvalT, kptr[row], kptr[row + 1], x, C, c0, xi, kx, false);
                    // right-hand side: b (computed once per evaluation, four consecutive
                    // instances), none for the stage-2 forward system; plus the BEM term
                    // c on the surface rows of the stage-2 adjoint (Neumann) system
                    double fb[VEC] = {0.0, 0.0, 0.0, 0.0};
                    if (!(mode == 1 && !neu) && !(!neu && bp) && any_act)
                        vload<double, VEC, false>(fb, &A.V.bvec[(size_t)row * B + bk[0]]);
                    // norm reference of Dirichlet systems: f - K_IS x_S
                    double kxs[VEC] = {0.0, 0.0, 0.0, 0.0};
                    if (!neu && !bp)
                        for (int e = kptr[row]; e < kptr[row + 1]; ++e) {
                            const int ww = kent[e];
                            const int j = (int)((unsigned)ww >> 8);
                            if ((unsigned)node[j] >> 16) {
                                T xs[VEC];
                                vload<T, VEC, true>(xs, &x[(size_t)j * C + c0]);
                                const double kk = GEN ? (double)kvalT[e] : (double)sbyte(ww, 0);
#pragma unroll
                                for (int k = 0; k < VEC; ++k) kxs[k] += kk * (double)xs[k];
                            }
                        }
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        if (!neu && bp) { rv[k] = W(0); zr[k] = 0.f; continue; }
                        double f = actk[k] ? fb[k] : 0.0;
                        if (mode == 1 && neu && bp) f += (double)A.V.ub_out[(size_t)(bp - 1) * C + c0 + k];
                        const double ref = neu ? f : f - kxs[k];   // norm reference
                        rv[k] = W(T(f) - kx[k]);
                        zr[k] = (float)ref;   // kept for the second pass
                        if (actk[k]) psum[0][k] += f;
                    }
                    vstore<W, VEC>(&r[go], rv);
                    *reinterpret_cast<float4*>(zs + (row - lo) * CPC + cl0) = make_float4(zr[0], zr[1], zr[2], zr[3]);
                }
                reduce(psum);   // Neumann: consistent right-hand side (sum zero)
                W mean[VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) mean[k] = neu ? W(out[cl0 + k] / (double)N) : W(0);
                double v4[4][VEC];   // r.z, r.r, ref.ref, sum r
#pragma unroll
                for (int k = 0; k < VEC; ++k) v4[0][k] = v4[1][k] = v4[2][k] = v4[3][k] = 0.0;
                for (int row = lo + rl; row < hi; row += RB) {
                    const float dt = dtab[row - lo];
                    const bool surf = dt < 0.f;
                    const unsigned go = (unsigned)(row * CPC + cl0);               // grouped work vectors
                    float* zp = zs + (row - lo) * CPC + cl0;
                    const W dinv = fabsf(dt);
                    W rv[VEC], zv[VEC];
                    vload<W, VEC, false>(rv, &r[go]);
                    const float4 zr = *reinterpret_cast<const float4*>(zp);
                    zv[0] = zr.x; zv[1] = zr.y; zv[2] = zr.z; zv[3] = zr.w;
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        if (!neu && surf) continue;
                        const W refk = zv[k] - mean[k];
                        rv[k] -= mean[k];
                        zv[k] = rv[k] * dinv;
                        if (actk[k]) {
                            v4[0][k] += (double)rv[k] * (double)zv[k];
                            v4[1][k] += (double)rv[k] * (double)rv[k];
                            v4[2][k] += (double)refk * (double)refk;
                            v4[3][k] += (double)rv[k];
                        }
                    }
                    const W zero[VEC] = {};
                    vstore<W, VEC>(&r[go], rv);
                    *reinterpret_cast<float4*>(zp) = make_float4(zv[0], zv[1], zv[2], zv[3]);
                    vstore<W, VEC>(&p[go], zero);
                    vstore<W, VEC>(&q[go], zero);
                }
                last = partial(v4);
            }
            for (int it = 0;; ++it) {
                // the slot `last` holds the CTAs' r.z, r.r, (ref.ref: first pass
                // only), sum r
                totals(last, 4);
                if (tid < CPC) {
                    if (it > 0) {   // bookkeeping of the iteration just finished
                        s_rhop[tid] = s_rho[tid];
                        if (!s_flag[tid]) s_it[tid] += 1;
                    }
                    const double rho = out[tid];
                    // Neumann: the residual without its null-space (mean) component
                    const double sr = out[3 * CPC + tid];
                    const double rr0 = out[CPC + tid];
                    const double rr = neu ? fmax(rr0 - sr * sr / (double)N, 0.0) : rr0;
                    int conv;
                    if constexpr (MP) {
                        if (it == 0) {   // rr is the true (FP64) residual of this cycle
                            s_tol[tid] = A.tol2 * out[2 * CPC + tid];
                            s_done[tid] = !s_act[tid] || rr <= s_tol[tid] || s_it[tid] >= A.max_iter;
                            s_tin[tid] = fmax(s_tol[tid], MP_INNER * MP_INNER * rr);
                        }
                        conv = s_done[tid] || rr <= s_tin[tid] || s_it[tid] >= A.max_iter;
                    } else {
                        if (it == 0) s_tol[tid] = A.tol2 * out[2 * CPC + tid];
                        conv = !s_act[tid] || rr <= s_tol[tid] || it >= A.max_iter;
                    }
                    s_ab[tid] = (it == 0 || conv) ? 0.0 : rho / s_rhop[tid];
                    s_abf[tid] = (float)s_ab[tid];
                    s_rho[tid] = rho;
                    s_flag[tid] = conv;
                }
                // the same totals in every CTA of the cluster: every CTA leaves together
                if (__syncthreads_and(tid < CPC ? s_flag[tid] : 1)) break;
                bool run = false;
                W beta[VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    run |= actk[k] && !s_flag[cl0 + k];
                    beta[k] = s_abf[cl0 + k];
                }
                W tpq[1][VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) tpq[0][k] = W(0);
                if (run)
                    for (int rb = lo + rl; rb < hi; rb += U * RB) {
                        // U rows per pass: every row's loads are issued before any arithmetic
                        W pvu[U][VEC], qvu[U][VEC];
                        bool surfu[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int row = rb + u * RB;
                            if (row < hi) {
                                const unsigned go = (unsigned)(row * CPC + cl0);   // grouped work vectors
                                vload<W, VEC, false>(pvu[u], &p[go]);
                                vload<W, VEC, false>(qvu[u], &q[go]);
                                surfu[u] = dtab[row - lo] < 0.f;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int row = rb + u * RB;
                            if (row >= hi) break;
                            const unsigned go = (unsigned)(row * CPC + cl0);
                            W (&pv)[VEC] = pvu[u];
                            W (&qv)[VEC] = qvu[u];
                            const bool surf = surfu[u];
                            const float* zp = zs + (row - lo) * CPC + cl0;
                            const float4 zi = *reinterpret_cast<const float4*>(zp);
                            float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
                            auto add = [&w4](float kk, const float4& zj) {
                                w4.x += kk * zj.x;
                                w4.y += kk * zj.y;
                                w4.z += kk * zj.z;
                                w4.w += kk * zj.w;
                            };
                            if (!GEN && !surf) {
                                // interior node of the Kuhn cube: the 7-point stencil of P1 on
                                // this triangulation (36 on the diagonal, -6 for the six axis
                                // neighbours), in the CSR's ascending column order
                                const int s2 = A.M.n + 1, s3 = s2 * s2;
                                float4 z0, z1, z2, z4, z5, z6;
                                if (row - s3 >= lo && row + s3 < hi) {   // all in this CTA's slab
                                    z0 = *reinterpret_cast<const float4*>(zp - s3 * CPC);
                                    z1 = *reinterpret_cast<const float4*>(zp - s2 * CPC);
                                    z2 = *reinterpret_cast<const float4*>(zp - CPC);
                                    z4 = *reinterpret_cast<const float4*>(zp + CPC);
                                    z5 = *reinterpret_cast<const float4*>(zp + s2 * CPC);
                                    z6 = *reinterpret_cast<const float4*>(zp + s3 * CPC);
                                } else {
                                    z0 = zrow(row - s3);
                                    z1 = zrow(row - s2);
                                    z2 = zrow(row - 1);
                                    z4 = zrow(row + 1);
                                    z5 = zrow(row + s2);
                                    z6 = zrow(row + s3);
                                }
                                add(-6.f, z0);
                                add(-6.f, z1);
                                add(-6.f, z2);
                                add(36.f, zi);
                                add(-6.f, z4);
                                add(-6.f, z5);
                                add(-6.f, z6);
                            } else {
                                const int e0 = kptr[row], e1 = kptr[row + 1];
                                for (int base = e0; base < e1; base += CHK) {
                                    int wj[CHK];
                                    W kv[CHK];
#pragma unroll
                                    for (int t = 0; t < CHK; ++t) {
                                        const bool has = base + t < e1;
                                        wj[t] = has ? __ldg(&kent[base + t]) : 0;
                                        if constexpr (GEN) kv[t] = has ? __ldg(&kvalW[base + t]) : W(0);
                                        else kv[t] = W(sbyte(wj[t], 0));
                                    }
                                    float4 zj[CHK];
#pragma unroll
                                    for (int t = 0; t < CHK; ++t)
                                        zj[t] = wj[t] != 0 ? zrow((int)((unsigned)wj[t] >> 8)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                                    for (int t = 0; t < CHK; ++t) add(kv[t], zj[t]);
                                }
                            }
                            const float zv[VEC] = {zi.x, zi.y, zi.z, zi.w}, wv[VEC] = {w4.x, w4.y, w4.z, w4.w};
                            const bool frozen = !neu && surf;
#pragma unroll
                            for (int k = 0; k < VEC; ++k) {
                                pv[k] = zv[k] + beta[k] * pv[k];
                                qv[k] = frozen ? W(0) : wv[k] + beta[k] * qv[k];
                                tpq[0][k] += pv[k] * qv[k];
                            }
                            vstore<W, VEC>(&p[go], pv);
                            vstore<W, VEC>(&q[go], qv);
                        }
                    }
                {
                    totals(partial(tpq), 1);
                    if (tid < CPC) {
                        s_ab[tid] = s_flag[tid] ? 0.0 : s_rho[tid] / out[tid];
                        s_abf[tid] = (float)s_ab[tid];
                    }
                    __syncthreads();
                }
                W alpha[VEC];
#pragma unroll
                for (int k = 0; k < VEC; ++k) alpha[k] = s_abf[cl0 + k];
                W v4[4][VEC];   // r.z, r.r, (unused), sum r: thread and block sums in W, cluster sums in FP64
#pragma unroll
                for (int k = 0; k < VEC; ++k) v4[0][k] = v4[1][k] = v4[2][k] = v4[3][k] = W(0);
                if (run)
                    for (int rb = lo + rl; rb < hi; rb += U * RB) {
                        W xau[U][VEC], rau[U][VEC], pau[U][VEC], qau[U][VEC];
                        W dinvu[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int row = rb + u * RB;
                            if (row < hi) {
                                const unsigned go = (unsigned)(row * CPC + cl0);   // grouped work vectors
                                vload<W, VEC, false>(xau[u], &xacc[go]);
                                vload<W, VEC, false>(rau[u], &r[go]);
                                vload<W, VEC, false>(pau[u], &p[go]);
                                vload<W, VEC, false>(qau[u], &q[go]);
                                dinvu[u] = fabsf(dtab[row - lo]);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int row = rb + u * RB;
                            if (row >= hi) break;
                            const unsigned go = (unsigned)(row * CPC + cl0);
                            W (&xa)[VEC] = xau[u];
                            W (&ra)[VEC] = rau[u];
                            W za[VEC];
                            const W dinv = dinvu[u];
#pragma unroll
                            for (int k = 0; k < VEC; ++k) {
                                xa[k] += alpha[k] * pau[u][k];
                                ra[k] -= alpha[k] * qau[u][k];
                                za[k] = ra[k] * dinv;
                                v4[0][k] += ra[k] * za[k];
                                v4[1][k] += ra[k] * ra[k];
                                v4[3][k] += ra[k];
                            }
                            vstore<W, VEC>(&xacc[go], xa);
                            vstore<W, VEC>(&r[go], ra);
                            *reinterpret_cast<float4*>(zs + (row - lo) * CPC + cl0) = make_float4(za[0], za[1], za[2], za[3]);
                        }
                    }
                last = partial(v4);
            }
            // fold the cycle's FP32 correction into x before anything reads x
            for (int row = lo + rl; row < hi; row += RB) {
                const unsigned ib = (unsigned)row * (unsigned)C + (unsigned)c0;
                const unsigned go = (unsigned)(row * CPC + cl0);
                T xv[VEC];
                W dv[VEC];
                const W zero[VEC] = {};
                vload<T, VEC, false>(xv, &x[ib]);
                vload<W, VEC, false>(dv, &xacc[go]);
#pragma unroll
                for (int k = 0; k < VEC; ++k) xv[k] += T(dv[k]);
                vstore<T, VEC>(&x[ib], xv);
                vstore<W, VEC>(&xacc[go], zero);
            }
            cluster_sync();
            if constexpr (!MP) {
                break;
            } else {
                // done when every column met the tolerance on its true residual at
                // the start of this cycle (or ran out of iterations or cycles)
                if (__syncthreads_and(tid < CPC ? s_done[tid] : 1) || cycle + 1 >= MP_MAX_CYCLES) break;
            }
        }
        // epilogue: Neumann systems are gauged to zero V-weighted mean and (stage 1)
        // hand u1_S to the BEM product; stage-1 Dirichlet (adjoint) systems hand
        // t = b_S - K_SI w (w vanishes on the surface, so K_SI w = (K w)_S)
        if (neu) {
            double pv[1][VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) pv[0][k] = 0.0;
            for (int row = lo + rl; row < hi; row += RB) {
                const double vi = GEN ? A.M.gV[row] : (double)(node[row] & 0xff);
                T xv[VEC];
                vload<T, VEC, false>(xv, &x[(size_t)row * C + c0]);
#pragma unroll
                for (int k = 0; k < VEC; ++k) pv[0][k] += vi * (double)xv[k];
            }
            reduce(pv);
            T mean[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) mean[k] = T(out[cl0 + k] / A.M.vsum);
            if (any_act)
                for (int row = lo + rl; row < hi; row += RB) {
                    const unsigned ib = (unsigned)row * (unsigned)C + (unsigned)c0;   // < 2^31: checked at launch
                    const int bp = (int)((unsigned)node[row] >> 16);
                    T xv[VEC];
                    vload<T, VEC, false>(xv, &x[ib]);
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        if (!actk[k]) continue;
                        xv[k] -= mean[k];
                        if (mode == 0 && bp) A.V.ub_in[(size_t)(bp - 1) * C + c0 + k] = xv[k];
                    }
                    vstore<T, VEC>(&x[ib], xv);
                }
        } else if (mode == 0 && any_act) {
            for (int row = lo + rl; row < hi; row += RB) {
                const int bp = (int)((unsigned)node[row] >> 16);
                if (!bp) continue;
                const unsigned ib = (unsigned)row * (unsigned)C + (unsigned)c0;   // < 2^31: checked at launch
                T xv[VEC], kw[VEC];
                vload<T, VEC, false>(xv, &x[ib]);
                row_kv<T, VEC, true, false, GEN>(kent, kvalT, kptr[row], kptr[row + 1], x, C, c0, xv, kw, false);
                double fb[VEC];
                vload<double, VEC, false>(fb, &A.V.bvec[(size_t)row * B + bk[0]]);
#pragma unroll
                for (int k = 0; k < VEC; ++k)
                    if (actk[k]) A.V.ub_in[(size_t)(bp - 1) * C + c0 + k] = T(fb[k]) - kw[k];
            }
        }
        if (rank == 0 && tid < CPC) {
            const int c = col0 + tid;
            if (neu) atomicAdd((unsigned long long*)&A.V.st[c % B].cg1, (unsigned long long)s_it[tid]);
            else atomicAdd((unsigned long long*)&A.V.st[c % B].cg2, (unsigned long long)s_it[tid]);
        }
    }
    // sweep counter: the largest iteration count of the launch (the last
    // cluster to finish adds it and clears the two counter words)
    if (rank == 0 && tid == 0) {
        unsigned kmax = 0;
        if (cluster_act)
            for (int i = 0; i < CPC; ++i) kmax = max(kmax, (unsigned)s_it[i]);
        atomicMax(&A.bar[2], kmax);
        __threadfence();
        const unsigned ncl = gridDim.x / CL;
        if (atomicAdd(&A.bar[3], 1u) == ncl - 1) {
            __threadfence();
            const unsigned km = atomicExch(&A.bar[2], 0u);
            atomicExch(&A.bar[3], 0u);
            if (A.sweeps) A.sweeps[mode + (sizeof(T) == 8 ? 2 : 0)] += (unsigned long long)km;
        }
    }
    cluster_sync();   // no CTA leaves while another may still read its shared memory
}

// Clusters of one shape (CL CTAs, CPC systems) that can be resident at once,
// queried once per (kernel, device, shared memory) and cached, so that no query
// runs while a chunk of iterations is being captured.
template <typename T, bool MP, bool GEN, int CPC, int CL>
int resident_clusters(int N, size_t* smem_out) {
    const int rpc = (N + CL - 1) / CL;
    const size_t smem = cl_smem(rpc, CPC).total;
    *smem_out = smem;
    if (smem > CL_SMEM_MAX) return 0;
    auto fn = k_pcg_cluster<T, MP, GEN, CPC, CL>;
    static std::mutex mu;
    static std::map<std::tuple<int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int ncl = 0;
    if (kernel_smem_attr((const void*)fn, (int)smem) == cudaSuccess &&
        (CL <= 8 || cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                        cudaSuccess)) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)CL);
        cfg.blockDim = dim3(cl_threads<CPC>());
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&ncl, (const void*)fn, &cfg) != cudaSuccess) ncl = 0;
    }
    cudaGetLastError();
    cache.emplace(key, ncl);
    return ncl;
}

// Launch nclusters clusters of one shape (the caller has checked that they can
// all be resident at once: otherwise they would run in waves).
template <typename T, bool MP, bool GEN, int CPC, int CL>
cudaError_t launch_cluster(const Launch& L, PcgArgs<T>& a, int nclusters) {
    const int N = a.M.N;
    const int rpc = (N + CL - 1) / CL;
    size_t smem = 0;
    resident_clusters<T, MP, GEN, CPC, CL>(N, &smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * CL));
    cfg.blockDim = dim3(cl_threads<CPC>());
    cfg.dynamicSmemBytes = smem;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg_cluster<T, MP, GEN, CPC, CL>, a, rpc);
}

// The shape for a batch of B instances of which active[b] (host flags at the
// start of the chunk; null: all) are iterating: the groups of CPC systems with
// an active instance must all fit in the resident clusters.  Preference: 4
// systems on 16 CTAs, on 8 CTAs (fewer rows per CTA: shorter iterations for the
// few instances still running at the end of a batch), 8 systems on 8 CTAs,
// 4 systems on 4 CTAs.  Returns the shape's code (CPC * 100 + CL; 0: none) and
// its cluster count (the groups a full batch has, or all resident clusters of
// the shape, whichever is fewer).
template <typename T, bool MP, bool GEN>
int choose_shape(const Launch& L, int N, int B, int* nclusters) {
    auto groups = [&](int cpc) {
        int n = 0;
        for (int gidx = 0; gidx < 2 * B / cpc; ++gidx) {
            bool a = L.active == nullptr;
            for (int i = 0; i < cpc && !a; ++i) a = L.active[(gidx * cpc + i) % B] != 0;
            n += a;
        }
        return n;
    };
    size_t smem = 0;
    // a shape serves n active groups if its resident clusters (and the caller's
    // cap on CTAs, L.max_blocks) hold them all
    auto fits = [&](int cpc, int cl, int r, int n) {
        int cap = r;
        if (L.max_blocks > 0) cap = std::min(cap, L.max_blocks / cl);
        if (n > cap) return false;
        *nclusters = std::min(cap, 2 * B / cpc);
        return true;
    };
    const int n4 = groups(4);
    if (fits(4, 16, resident_clusters<T, MP, GEN, 4, 16>(N, &smem), n4)) return 416;
    if (fits(4, 8, resident_clusters<T, MP, GEN, 4, 8>(N, &smem), n4)) return 408;
    if (B >= 32 && B % 8 == 0 && fits(8, 8, resident_clusters<T, MP, GEN, 8, 8>(N, &smem), groups(8))) return 808;
    if (fits(4, 4, resident_clusters<T, MP, GEN, 4, 4>(N, &smem), n4)) return 404;
    return 0;
}

template <typename T, bool MP, bool GEN>
cudaError_t launch_any(const Launch& L, PcgArgs<T>& a, bool* ok) {
    int ncl = 0;
    const int shape = choose_shape<T, MP, GEN>(L, a.M.N, a.V.B, &ncl);
    *ok = shape != 0;
    switch (shape) {
        case 416: return launch_cluster<T, MP, GEN, 4, 16>(L, a, ncl);
        case 408: return launch_cluster<T, MP, GEN, 4, 8>(L, a, ncl);
        case 808: return launch_cluster<T, MP, GEN, 8, 8>(L, a, ncl);
        case 404: return launch_cluster<T, MP, GEN, 4, 4>(L, a, ncl);
        default: return cudaSuccess;
    }
}

bool cluster_qualifies(const MeshView& M, int B, bool fp64, bool mixed_iter) {
    if (fp64 && !mixed_iter) return false;
    if (B % 4 != 0 || B < 16 || B > 512) return false;
    return (size_t)M.N * 2 * B < ((size_t)1 << 31);   // 32-bit element offsets in the kernel
}

}  // namespace

int pcg_cluster_shape(const Launch& L, const MeshView& M, int B, bool fp64, bool mixed_iter) {
    if (L.pcg_kernel == 1 || !cluster_qualifies(M, B, fp64, mixed_iter)) return 0;
    int ncl = 0;
    if (fp64) return M.gen ? choose_shape<double, true, true>(L, M.N, B, &ncl)
                           : choose_shape<double, true, false>(L, M.N, B, &ncl);
    return M.gen ? choose_shape<float, false, true>(L, M.N, B, &ncl) : choose_shape<float, false, false>(L, M.N, B, &ncl);
}

// The cluster variant when the batch has enough systems (B a multiple of 4,
// 16 <= B <= 512), its work vectors are FP32 (FP32 solves, or FP64 solves
// iterated in FP32), z of a cluster's systems fits its CTAs' shared memory and
// the clusters serving the active groups can be resident together.  Returns 1
// when launched (*err: the launch's status), 0 when no shape qualifies.
template <typename T>
int pcg_solve_cluster(const Launch& L, const MeshView& M, const BatchView<T>& V, int mode, double tol, int max_iter,
                      bool mixed_iter, cudaError_t* err) {
    *err = cudaSuccess;
    const bool mp = sizeof(T) == 8;
    if (!cluster_qualifies(M, V.B, mp, mixed_iter)) return 0;
    PcgArgs<T> a{M, V, mode, tol * tol, max_iter, L.bar, L.err, L.sweeps, L.fin};
    bool ok = false;
    cudaError_t e;
    if constexpr (sizeof(T) == 8) e = M.gen ? launch_any<T, true, true>(L, a, &ok) : launch_any<T, true, false>(L, a, &ok);
    else e = M.gen ? launch_any<T, false, true>(L, a, &ok) : launch_any<T, false, false>(L, a, &ok);
    *err = e;
    if (!ok && e == cudaSuccess) return 0;
    *L.launches += 1;
    return 1;
}

template int pcg_solve_cluster<float>(const Launch&, const MeshView&, const BatchView<float>&, int, double, int, bool,
                                      cudaError_t*);
template int pcg_solve_cluster<double>(const Launch&, const MeshView&, const BatchView<double>&, int, double, int,
                                       bool, cudaError_t*);

}  // namespace lbm
