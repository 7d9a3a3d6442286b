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

#include <algorithm>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <type_traits>

#include "solver_common.cuh"

namespace lbm {

constexpr int PCG_THREADS = 512;        // grid-wide (cooperative) variant
constexpr int PCG_SINGLE_THREADS = 512;  // one-CTA variant for small batches
constexpr int FIELD_THREADS = 256;
constexpr long long SINGLE_CTA_MAX_WORK = 24576;   // N * B up to which one CTA solves

cudaError_t kernel_smem_attr(const void* fn, int smem_limit, int threads, size_t smem, int* blocks_per_sm) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, size_t>, int> occ_cache;
    static std::map<std::pair<const void*, int>, int> limit_set;   // largest limit set so far
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto it = limit_set.find({fn, dev});
    if (it == limit_set.end() || it->second < smem_limit) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
        if (e != cudaSuccess) return e;
        limit_set[{fn, dev}] = smem_limit;
    }
    if (blocks_per_sm) {
        const auto key = std::make_tuple(fn, dev, threads, smem);
        auto oc = occ_cache.find(key);
        if (oc == occ_cache.end()) {
            int occ = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
            if (e != cudaSuccess) return e;
            oc = occ_cache.emplace(key, occ).first;
        }
        *blocks_per_sm = oc->second;
    }
    return cudaSuccess;
}

template <bool SINGLE>
__device__ __forceinline__ bool pcg_sync(unsigned* bar, unsigned& epoch, int* err) {
    if constexpr (SINGLE) {
        __syncthreads();
        return true;
    } else {
        return grid_sync(bar, gridDim.x, epoch, err);
    }
}


// Jacobi-PCG on Kint for the 2B systems of one stage of the forward and adjoint
// FEM/BEM chains (column c: instance c % B, adjoint if c >= B):
//   stage 1: forward  K u1 = b               (Neumann)
//            adjoint  K_II w_I = b_I, w_S = 0 (Dirichlet)
//   stage 2: forward  K_II u2_I = -K_IS u2_S, u2_S = B u1_S   (Dirichlet)
//            adjoint  K uT = b + S^T B^T t,  t = b_S - K_SI w  (Neumann)
// Each thread owns VEC consecutive columns of a row (one 8- or 16-byte vector),
// so every neighbour gather of the SpMV moves VEC values per lane.  Fused so
// that every iteration needs two synchronisations (grid barriers, or
// __syncthreads in the one-CTA variant):
//   A: w = K z, p = z + beta p, q = w + beta q (= K p), partial p.q
//   B: alpha = rho/p.q, x += alpha p, r -= alpha q, z = r / K_ii, partials r.z, r.r
// Neumann systems: the right-hand side is made consistent (mean removed), the
// residual is tested without its mean, and the solution is gauged to zero
// V-weighted mean.  Dirichlet systems freeze the surface rows (p = q = r = z = 0).
template <typename T, bool SINGLE, int VEC, bool GEN, bool MP>
__global__ void __launch_bounds__(SINGLE ? PCG_SINGLE_THREADS : PCG_THREADS, 1) k_pcg(PcgArgs<T> A) {
    extern __shared__ double sm[];
    constexpr bool CG = !SINGLE;
    using W = typename std::conditional<MP, float, T>::type;   // precision of the iteration
    const int bd = blockDim.x, tid = threadIdx.x;
    const int B = A.V.B, C = 2 * B, G = C / VEC, RB = bd / G;
    const bool lane = tid < RB * G;
    const int g = tid % G, rl = tid / G, c0 = g * VEC;
    const int mode = A.mode;
    // a warp works on one row when the column groups of a row fill whole warps
    const bool warp_row = (G % 32) == 0;
    const int nrow_red = (G <= 32 && (32 % G) == 0) ? (bd >> 5) : RB;
    double* scratch = sm;                               // [4][nrow_red][C]
    double* out = scratch + 4 * nrow_red * C;           // [4][C]
    double* s_rho = out + 4 * C;                        // [C]
    double* s_rhop = s_rho + C;
    double* s_ab = s_rhop + C;
    double* s_tol = s_ab + C;
    double* s_tin = s_tol + C;                          // MP: tolerance of the current cycle
    int* s_flag = (int*)(s_tin + C);
    int* s_act = s_flag + C;
    int* s_cur = s_act + C;
    int* s_it = s_cur + C;
    int* s_done = s_it + C;                             // MP: true residual met the tolerance

    for (int i = tid; i < C; i += bd) {
        s_act[i] = A.V.st[i % B].phase != PH_DONE;
        s_cur[i] = A.V.st[i % B].cur;
        s_it[i] = 0;
        s_done[i] = 0;
        s_tin[i] = 0.0;
        s_rhop[i] = 1.0;
    }
    __syncthreads();
    const int N = A.M.N;
    int bk[VEC];
    bool neu[VEC], actk[VEC];
    bool any_act = false;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const int c = c0 + k;
        bk[k] = c % B;
        neu[k] = (mode == c / B);
        actk[k] = lane && s_act[c];
        any_act |= actk[k];
    }
    // row loops are entered by whole warps when warp_row (the gather broadcasts)
    const bool do_rows = warp_row ? (__any_sync(0xffffffffu, any_act) != 0) : any_act;
    const int row0 = blockIdx.x * RB + rl, rstride = gridDim.x * RB;
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
    // work vectors in W (MP: FP32 values in the FP64 arrays' storage)
    W* __restrict__ r = reinterpret_cast<W*>(A.V.r);
    // where the update phase accumulates alpha p: x itself, or (MP) an FP32
    // correction d in the unused upper half of r's FP64 storage, folded into the
    // FP64 x once per cycle (no FP64 arithmetic in the iterations)
    using XA = typename std::conditional<MP, W, T>::type;
    XA* __restrict__ xacc = MP ? reinterpret_cast<XA*>(reinterpret_cast<W*>(A.V.r) + (size_t)A.M.N * C)
                               : reinterpret_cast<XA*>(mode ? A.V.U2 : A.V.U1);
    W* __restrict__ z = reinterpret_cast<W*>(A.V.z);
    W* __restrict__ p = reinterpret_cast<W*>(A.V.p);
    W* __restrict__ q = reinterpret_cast<W*>(A.V.q);
    double* part = A.V.part;
    unsigned epoch = 0;

    // partials of this block -> totals in `out` (a grid reduction unless SINGLE).
    // Few partials (small batches): one barrier, then every block sums all of
    // them; the two halves of `part` alternate so that a block writing the next
    // partials never overwrites ones another block is still reading.  Many
    // partials: the two-level reduction (one warp per total, two barriers).
    const bool few = (size_t)gridDim.x * C * 4 <= (size_t)8 * bd;
    unsigned red_idx = 0;
    auto reduce = [&](auto& vals, int q0) -> bool {
        constexpr int NQV = sizeof(vals) / sizeof(vals[0]);
        using R = typename std::remove_reference<decltype(vals[0][0])>::type;
        block_reduce_cols<NQV, VEC, R>(vals, reinterpret_cast<R*>(scratch), out, C, G, RB);
        if constexpr (SINGLE) {
            return true;
        } else {
            double* pr = part + (size_t)(red_idx & 1u) * gridDim.x * C * 4;
            red_idx += 1;
            if (tid < C)
                for (int k = 0; k < NQV; ++k) pr[((size_t)blockIdx.x * C + tid) * 4 + q0 + k] = out[k * C + tid];
            if (few) {
                if (!grid_sync(A.bar, gridDim.x, epoch, A.err)) return false;
                cross_reduce_cols<NQV, VEC>(pr, q0, gridDim.x, C, G, RB, scratch, out);
                return true;
            }
            return grid_reduce<NQV>(pr, q0, C, A.fin, out, A.bar, epoch, A.err);
        }
    };

    // Dirichlet systems: surface values (stage 1 adjoint: zero; stage 2 forward: B u1_S)
    if (any_act)
        for (int row = row0; row < N; row += rstride) {
            const int bp = (int)((unsigned)node[row] >> 16);
            if (!bp) continue;
#pragma unroll
            for (int k = 0; k < VEC; ++k)
                if (actk[k] && !neu[k])
                    x[(size_t)row * C + c0 + k] = mode ? A.V.ub_out[(size_t)(bp - 1) * C + bk[k]] : T(0);
        }
    if constexpr (MP) {
        const W zero[VEC] = {};
        if (lane)
            for (int row = row0; row < N; row += rstride) vstore<W, VEC>(&xacc[(size_t)row * C + c0], zero);
    }
    if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;
    // One cycle: the residual of the current x in the precision of x (T), then
    // preconditioned CG iterations in the work precision W.  MP (FP64 x, FP32
    // work vectors): a cycle ends when the FP32 recurrence has reduced the
    // residual by MP_INNER (or reached the tolerance); the next cycle replaces it
    // by the true FP64 residual and restarts CG from there, so the test that
    // ends the solve is always taken on the FP64 residual.
    for (int cycle = 0;; ++cycle) {
    {   // residual of the current x
        double psum[1][VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) psum[0][k] = 0.0;
        if (do_rows)
            for (int row = row0; row < N; row += rstride) {
                const int nd = node[row];
                const int bp = (int)((unsigned)nd >> 16);
                const size_t ib = (size_t)row * C + c0;
                T xi[VEC], kx[VEC];
                W rv[VEC], zv[VEC];
                vload<T, VEC, false>(xi, &x[ib]);
                row_kv<T, VEC, CG, true, GEN>(kent, kvalT, kptr[row], kptr[row + 1], x, C, c0, xi, kx, warp_row);
                const int e0 = rowptr[row], e1 = rowptr[row + 1];
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    if (!neu[k] && bp) { rv[k] = W(0); zv[k] = W(0); continue; }
                    // f: the right-hand side (b in every system but the stage-2 forward one)
                    double f = 0.0;
                    if (!(mode == 1 && !neu[k]) && actk[k])
                        f = A.V.bvec[(size_t)row * B + bk[k]];
                    if (mode == 1 && neu[k] && bp) f += (double)A.V.ub_out[(size_t)(bp - 1) * C + c0 + k];
                    double ref = f;   // norm reference: f (Neumann), f - K_IS x_S (Dirichlet)
                    if (!neu[k])
                        for (int e = kptr[row]; e < kptr[row + 1]; ++e) {
                            const int ww = kent[e];
                            const int j = (int)((unsigned)ww >> 8);
                            if ((unsigned)node[j] >> 16)
                                ref -= (GEN ? (double)kvalT[e] : (double)sbyte(ww, 0)) *
                                       (double)ld_vec<T, CG>(&x[(size_t)j * C + c0 + k]);
                        }
                    rv[k] = W(T(f) - kx[k]);
                    zv[k] = W(ref);                       // kept for the second pass
                    if (actk[k]) psum[0][k] += f;
                }
                const W zero[VEC] = {};
                vstore<W, VEC>(&r[ib], rv);
                vstore<W, VEC>(&z[ib], zv);
                vstore<W, VEC>(&p[ib], zero);
                vstore<W, VEC>(&q[ib], zero);
            }
        // Neumann: consistent right-hand side (sum zero)
        if (!reduce(psum, 2)) return;
        if (tid < C) s_ab[tid] = out[tid] / (double)N;
        __syncthreads();
        W mean[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) mean[k] = neu[k] ? W(s_ab[c0 + k]) : W(0);
        double v4[4][VEC];   // r.z, r.r, ref.ref, sum r
#pragma unroll
        for (int k = 0; k < VEC; ++k) v4[0][k] = v4[1][k] = v4[2][k] = v4[3][k] = 0.0;
        if (any_act)
            for (int row = row0; row < N; row += rstride) {
                const int nd = node[row];
                const bool surf = ((unsigned)nd >> 16) != 0;
                const size_t ib = (size_t)row * C + c0;
                const W dinv = W(1) / (GEN ? kdiagW[row] : W((nd >> 8) & 0xff));
                W rv[VEC], zv[VEC];
                vload<W, VEC, false>(rv, &r[ib]);
                vload<W, VEC, false>(zv, &z[ib]);
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    if (!neu[k] && surf) continue;
                    const W ref = zv[k] - mean[k];
                    rv[k] -= mean[k];
                    zv[k] = rv[k] * dinv;
                    if (actk[k]) {
                        v4[0][k] += (double)rv[k] * (double)zv[k];
                        v4[1][k] += (double)rv[k] * (double)rv[k];
                        v4[2][k] += (double)ref * (double)ref;
                        v4[3][k] += (double)rv[k];
                    }
                }
                vstore<W, VEC>(&r[ib], rv);
                vstore<W, VEC>(&z[ib], zv);
            }
        if (!reduce(v4, 0)) return;
    }
    for (int it = 0;; ++it) {
        // `out` holds the totals of r.z, r.r, (ref.ref), sum r of the last pass
        if (tid < C) {
            const bool nn = (mode == tid / B);
            const double rho = out[tid];
            // Neumann: test the residual without its null-space (mean) component,
            // which rounding feeds and CG cannot remove
            const double sr = out[3 * C + tid];
            const double rr = nn ? fmax(out[C + tid] - sr * sr / (double)N, 0.0) : out[C + tid];
            int conv;
            if constexpr (MP) {
                if (it == 0) {   // rr is the true (FP64) residual of this cycle
                    s_tol[tid] = A.tol2 * out[2 * C + tid];
                    s_done[tid] = !s_act[tid] || rr <= s_tol[tid] || s_it[tid] >= A.max_iter;
                    s_tin[tid] = fmax(s_tol[tid], MP_INNER * MP_INNER * rr);
                }
                conv = s_done[tid] || rr <= s_tin[tid] || s_it[tid] >= A.max_iter;
            } else {
                if (it == 0) s_tol[tid] = A.tol2 * out[2 * C + tid];
                conv = !s_act[tid] || rr <= s_tol[tid] || it >= A.max_iter;
            }
            s_ab[tid] = (it == 0 || conv) ? 0.0 : rho / s_rhop[tid];
            s_rho[tid] = rho;
            s_flag[tid] = conv;
        }
        // C <= blockDim.x: one flag per thread, combined by the barrier itself
        if (__syncthreads_and(tid < C ? s_flag[tid] : 1)) break;
        bool run = false;
        W beta[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            run |= actk[k] && !s_flag[c0 + k];
            beta[k] = W(s_ab[c0 + k]);
        }
        const bool run_rows = warp_row ? (__any_sync(0xffffffffu, run) != 0) : run;
        W tpq[1][VEC];   // per-thread and block partial sums in W; grid sums in FP64
#pragma unroll
        for (int k = 0; k < VEC; ++k) tpq[0][k] = W(0);
        if (run_rows && warp_row) {
            // software-pipelined rows: the row pointers two rows ahead and the
            // packed entries and node word one row ahead are in flight while
            // the current row gathers, so each row waits on its gathers only
            const int lane = threadIdx.x & 31;
            int row = row0, rown = row0 + rstride;
            int kp0 = 0, kp1 = 0, kn0 = 0, kn1 = 0;
            if (row < N) { kp0 = kptr[row]; kp1 = kptr[row + 1]; }
            if (rown < N) { kn0 = kptr[rown]; kn1 = kptr[rown + 1]; }
            int mine = (row < N && kp0 + lane < kp1) ? __ldg(&kent[kp0 + lane]) : 0;
            W mk = (GEN && row < N && kp0 + lane < kp1) ? __ldg(&kvalW[kp0 + lane]) : W(0);
            int nd = row < N ? node[row] : 0;
            for (; row < N; row = rown, rown += rstride) {
                const int rown2 = rown + rstride;
                int kf0 = 0, kf1 = 0;
                if (rown2 < N) { kf0 = kptr[rown2]; kf1 = kptr[rown2 + 1]; }
                const int minen = (rown < N && kn0 + lane < kn1) ? __ldg(&kent[kn0 + lane]) : 0;
                const W mkn = (GEN && rown < N && kn0 + lane < kn1) ? __ldg(&kvalW[kn0 + lane]) : W(0);
                const int ndn = rown < N ? node[rown] : 0;
                const bool surf = ((unsigned)nd >> 16) != 0;
                const size_t ib = (size_t)row * C + c0;
                W zi[VEC], w[VEC], pv[VEC], qv[VEC];
                vload<W, VEC, false>(zi, &z[ib]);
                vload<W, VEC, false>(pv, &p[ib]);
                vload<W, VEC, false>(qv, &q[ib]);
                row_kv_warp<W, VEC, CG, false, GEN>(mine, mk, kp0, kp1, kent, kvalW, z, C, c0, zi, w);
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    pv[k] = zi[k] + beta[k] * pv[k];
                    qv[k] = (!neu[k] && surf) ? W(0) : w[k] + beta[k] * qv[k];
                    tpq[0][k] += pv[k] * qv[k];
                }
                vstore<W, VEC>(&p[ib], pv);
                vstore<W, VEC>(&q[ib], qv);
                kp0 = kn0; kp1 = kn1; kn0 = kf0; kn1 = kf1;
                mine = minen; mk = mkn; nd = ndn;
            }
        } else if (run_rows) {
            for (int row = row0; row < N; row += rstride) {
                const int nd = node[row];
                const bool surf = ((unsigned)nd >> 16) != 0;
                const size_t ib = (size_t)row * C + c0;
                W zi[VEC], w[VEC], pv[VEC], qv[VEC];
                vload<W, VEC, false>(zi, &z[ib]);
                row_kv<W, VEC, CG, false, GEN>(kent, kvalW, kptr[row], kptr[row + 1], z, C, c0, zi, w, warp_row);
                vload<W, VEC, false>(pv, &p[ib]);
                vload<W, VEC, false>(qv, &q[ib]);
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    pv[k] = zi[k] + beta[k] * pv[k];
                    qv[k] = (!neu[k] && surf) ? W(0) : w[k] + beta[k] * qv[k];
                    tpq[0][k] += pv[k] * qv[k];
                }
                vstore<W, VEC>(&p[ib], pv);
                vstore<W, VEC>(&q[ib], qv);
            }
        }
        if (!reduce(tpq, 0)) return;
        if (tid < C) s_ab[tid] = s_flag[tid] ? 0.0 : s_rho[tid] / out[tid];
        __syncthreads();
        XA alpha[VEC];
        W alphaw[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            alpha[k] = XA(s_ab[c0 + k]);
            alphaw[k] = W(s_ab[c0 + k]);
        }
        W v4[4][VEC];   // r.z, r.r, (unused), sum r: per-thread and block sums in W, grid sums in FP64
#pragma unroll
        for (int k = 0; k < VEC; ++k) v4[0][k] = v4[1][k] = v4[2][k] = v4[3][k] = W(0);
        // two rows per pass: both rows' loads are in flight together
        if (run)
            for (int row = row0; row < N; row += 2 * rstride) {
                const int rowb = row + rstride;
                const bool two = rowb < N;
                const size_t ia = (size_t)row * C + c0, ibb = (size_t)(two ? rowb : row) * C + c0;
                const int nda = node[row], ndb = node[two ? rowb : row];
                XA xa[VEC], xb[VEC];
                W ra[VEC], pa[VEC], qa[VEC], rb[VEC], pb[VEC], qb[VEC], za[VEC], zb[VEC];
                vload<XA, VEC, false>(xa, &xacc[ia]);
                vload<W, VEC, false>(ra, &r[ia]);
                vload<W, VEC, false>(pa, &p[ia]);
                vload<W, VEC, false>(qa, &q[ia]);
                vload<XA, VEC, false>(xb, &xacc[ibb]);
                vload<W, VEC, false>(rb, &r[ibb]);
                vload<W, VEC, false>(pb, &p[ibb]);
                vload<W, VEC, false>(qb, &q[ibb]);
                const W dinva = W(1) / (GEN ? kdiagW[row] : W((nda >> 8) & 0xff));
                const W dinvb = W(1) / (GEN ? kdiagW[two ? rowb : row] : W((ndb >> 8) & 0xff));
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    xa[k] += alpha[k] * XA(pa[k]);
                    ra[k] -= alphaw[k] * qa[k];
                    za[k] = ra[k] * dinva;
                    v4[0][k] += ra[k] * za[k];
                    v4[1][k] += ra[k] * ra[k];
                    v4[3][k] += ra[k];
                }
                vstore<XA, VEC>(&xacc[ia], xa);
                vstore<W, VEC>(&r[ia], ra);
                vstore<W, VEC>(&z[ia], za);
                if (two) {
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        xb[k] += alpha[k] * XA(pb[k]);
                        rb[k] -= alphaw[k] * qb[k];
                        zb[k] = rb[k] * dinvb;
                        v4[0][k] += rb[k] * zb[k];
                        v4[1][k] += rb[k] * rb[k];
                        v4[3][k] += rb[k];
                    }
                    vstore<XA, VEC>(&xacc[ibb], xb);
                    vstore<W, VEC>(&r[ibb], rb);
                    vstore<W, VEC>(&z[ibb], zb);
                }
            }
        // quantity 2 (ref.ref) is carried over from the prologue in `out`
        double keep2[1];
        if (tid < C) keep2[0] = out[2 * C + tid];
        if (!reduce(v4, 0)) return;
        if (tid < C) {
            s_rhop[tid] = s_rho[tid];
            if (!s_flag[tid]) s_it[tid] += 1;
            out[2 * C + tid] = keep2[0];
        }
        __syncthreads();
    }
    if constexpr (!MP) {
        break;
    } else {
        // fold the cycle's FP32 correction into the FP64 x before anything reads x
        if (lane)
            for (int row = row0; row < N; row += rstride) {
                const size_t ib = (size_t)row * C + c0;
                T xv[VEC];
                W dv[VEC];
                const W zero[VEC] = {};
                vload<T, VEC, false>(xv, &x[ib]);
                vload<W, VEC, false>(dv, &xacc[ib]);
#pragma unroll
                for (int k = 0; k < VEC; ++k) xv[k] += T(dv[k]);
                vstore<T, VEC>(&x[ib], xv);
                vstore<W, VEC>(&xacc[ib], zero);
            }
        if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;
        // done when every column met the tolerance on its true residual at the
        // start of this cycle (or ran out of iterations or cycles)
        if (__syncthreads_and(tid < C ? s_done[tid] : 1) || cycle + 1 >= MP_MAX_CYCLES) break;
    }
    }
    if (blockIdx.x == 0) {
        for (int i = tid; i < C; i += bd) {
            const bool nn = (mode == i / B);
            if (nn) atomicAdd((unsigned long long*)&A.V.st[i % B].cg1, (unsigned long long)s_it[i]);
            else atomicAdd((unsigned long long*)&A.V.st[i % B].cg2, (unsigned long long)s_it[i]);
        }
        if (tid == 0 && A.sweeps) {
            int kmax = 0;
            for (int i = 0; i < C; ++i) kmax = max(kmax, s_it[i]);
            A.sweeps[mode + (sizeof(T) == 8 ? 2 : 0)] += (unsigned long long)kmax;
        }
    }
    // epilogue: Neumann systems are gauged to zero V-weighted mean; stage 1 then
    // hands the surface values to the BEM products: u1_S (forward) and
    // t = b_S - K_SI w (adjoint; w vanishes on the surface, so K_SI w = (K w)_S).
    double pv[1][VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) pv[0][k] = 0.0;
    if (any_act)
        for (int row = row0; row < N; row += rstride) {
            const double vi = GEN ? A.M.gV[row] : (double)(node[row] & 0xff);
            T xv[VEC];
            vload<T, VEC, false>(xv, &x[(size_t)row * C + c0]);
#pragma unroll
            for (int k = 0; k < VEC; ++k)
                if (neu[k]) pv[0][k] += vi * (double)xv[k];
        }
    if (!reduce(pv, 1)) return;
    if (tid < C) s_ab[tid] = out[tid] / A.M.vsum;
    __syncthreads();
    if (!pcg_sync<SINGLE>(A.bar, epoch, A.err)) return;   // every block has read `out` of x
    bool need_kw = false;
#pragma unroll
    for (int k = 0; k < VEC; ++k) need_kw |= (mode == 0 && !neu[k] && actk[k]);
    const bool kw_rows = warp_row ? (__any_sync(0xffffffffu, need_kw) != 0) : need_kw;
    if (do_rows)
        for (int row = row0; row < N; row += rstride) {
            const size_t ib = (size_t)row * C + c0;
            const int bp = (int)((unsigned)node[row] >> 16);
            T xv[VEC];
            vload<T, VEC, false>(xv, &x[ib]);
            T kw[VEC];
            if (kw_rows && bp)
                row_kv<T, VEC, CG, false, GEN>(kent, kvalT, kptr[row], kptr[row + 1], x, C, c0, xv, kw, warp_row);
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                if (!actk[k]) continue;
                if (neu[k]) {
                    xv[k] -= T(s_ab[c0 + k]);
                    if (mode == 0 && bp) A.V.ub_in[(size_t)(bp - 1) * C + c0 + k] = xv[k];
                } else if (mode == 0 && bp) {
                    A.V.ub_in[(size_t)(bp - 1) * C + c0 + k] =
                        T(A.V.bvec[(size_t)row * B + bk[k]]) - kw[k];
                }
            }
            vstore<T, VEC>(&x[ib], xv);
        }
}

// b_i = (1/4) sum_j Gint_ij . m_j at the trial point of every active instance
// (one thread per row and instance, instances fastest): computed once per
// evaluation and read by both potential-solve stages (forward and adjoint
// right-hand sides, the adjoint's surface hand-off), by the same arithmetic
// (rhs_b) the solves used inline before.
template <typename T, bool GEN>
__global__ void k_rhs(MeshView M, BatchView<T> V) {
    const int B = V.B;
    const size_t total = (size_t)M.N * B;
    const typename GenTab<T>::V4* __restrict__ gA = GEN ? GenTab<T>::A(M) : nullptr;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        const int row = (int)(t / B);
        const InstState& s = V.st[b];
        if (s.phase == PH_DONE) continue;
        V.bvec[t] = rhs_b<T, GEN>(M.col, M.pkA, gA, M.rowptr[row], M.rowptr[row + 1], trial_m(V, s.cur, M.N), B, b);
    }
}

template <typename T>
void rhs_eval(const Launch& L, const MeshView& M, const BatchView<T>& V) {
    const size_t total = (size_t)M.N * V.B;
    size_t blocks = (total + 255) / 256;
    if (blocks > (size_t)8 * L.num_sms) blocks = (size_t)8 * L.num_sms;
    if (M.gen) k_rhs<T, true><<<(unsigned)blocks, 256, 0, L.stream>>>(M, V);
    else k_rhs<T, false><<<(unsigned)blocks, 256, 0, L.stream>>>(M, V);
    *L.launches += 1;
}

size_t pcg_part_elems(int num_sms, int B) { return (size_t)2 * num_sms * (2 * B) * 4; }

template <typename T, bool SINGLE, int VEC, bool GEN, bool MP>
static cudaError_t launch_pcg(const Launch& L, const MeshView& M, PcgArgs<T>& a, int C) {
    const int bd = SINGLE ? PCG_SINGLE_THREADS : PCG_THREADS;
    const int G = C / VEC, RB = bd / G;
    const int nrow_red = (G <= 32 && (32 % G) == 0) ? (bd >> 5) : RB;
    const size_t smem = sizeof(double) * (4 * (size_t)nrow_red * C + 9 * (size_t)C) + sizeof(int) * 5 * C;
    const void* fn = (const void*)k_pcg<T, SINGLE, VEC, GEN, MP>;
    int occ = 1;
    cudaError_t ea = kernel_smem_attr(fn, 200 * 1024, bd, 200 * 1024, SINGLE ? nullptr : &occ);
    if (ea != cudaSuccess) return ea;
    occ = 1;   // the partials buffer holds one block per SM
    void* args[] = {&a};
    if (SINGLE) return cudaLaunchKernel((void*)k_pcg<T, SINGLE, VEC, GEN, MP>, dim3(1), dim3(bd), args, smem, L.stream);
    int nblk = (M.N + RB - 1) / RB;
    int maxblk = occ * L.num_sms;
    if (L.max_blocks > 0 && L.max_blocks < maxblk) maxblk = L.max_blocks;
    if (nblk > maxblk) nblk = maxblk;
    cudaMemsetAsync(L.bar, 0, sizeof(unsigned), L.stream);
    return cudaLaunchCooperativeKernel((void*)k_pcg<T, SINGLE, VEC, GEN, MP>, dim3(nblk), dim3(bd), args, smem, L.stream);
}

template <typename T, bool GEN, bool MP>
static cudaError_t dispatch_pcg(const Launch& L, const MeshView& M, PcgArgs<T>& a, int C, bool single) {
    constexpr int V4 = sizeof(T) == 4 ? 4 : 2;
    const bool vec4 = (sizeof(T) == 4) && (C % 4 == 0);
    if (single) return vec4 ? launch_pcg<T, true, V4, GEN, MP>(L, M, a, C) : launch_pcg<T, true, 2, GEN, MP>(L, M, a, C);
    return vec4 ? launch_pcg<T, false, V4, GEN, MP>(L, M, a, C) : launch_pcg<T, false, 2, GEN, MP>(L, M, a, C);
}

// mixed_iter (FP64 only): iterate in FP32 with FP64 residual replacement.
template <typename T>
int pcg_solve(const Launch& L, const MeshView& M, const BatchView<T>& V, int mode, double tol, int max_iter,
              bool mixed_iter) {
    if (L.pcg_kernel != 1) {
        cudaError_t ce;
        if (pcg_solve_cluster<T>(L, M, V, mode, tol, max_iter, mixed_iter, &ce)) return ce == cudaSuccess ? 0 : (int)ce;
    }
    const int C = 2 * V.B;
    PcgArgs<T> a{M, V, mode, tol * tol, max_iter, L.bar, L.err, L.sweeps, L.fin};
    // one CTA is fastest for small FP32 work (no grid barriers); FP64 arithmetic
    // issues at a small fraction of the FP32 rate, so plain FP64 solves spread
    // over the grid from a much smaller size on
    const long long work = (long long)M.N * C * ((sizeof(T) == 8 && !mixed_iter) ? 16 : 1);
    const bool single = work <= SINGLE_CTA_MAX_WORK;
    cudaError_t e;
    if constexpr (sizeof(T) == 8) {
        if (mixed_iter) {
            e = M.gen ? dispatch_pcg<T, true, true>(L, M, a, C, single)
                      : dispatch_pcg<T, false, true>(L, M, a, C, single);
            *L.launches += 1;
            return e == cudaSuccess ? 0 : (int)e;
        }
    }
    e = M.gen ? dispatch_pcg<T, true, false>(L, M, a, C, single) : dispatch_pcg<T, false, false>(L, M, a, C, single);
    *L.launches += 1;
    return e == cudaSuccess ? 0 : (int)e;
}

// ---- BEM products: forward u2_S = B u1_S, adjoint c_S = B^T t_S ------------------------
// Columns 0..B-1 of the [nb][2B] surface arrays belong to the forward chain,
// columns B..2B-1 to the adjoint chain.

// Per-lane accumulator of a matrix-vector product, chosen by the VECTOR type:
// FP32 vectors (the FP32 phase) use a compensated (Kahan) FP32 sum, so that the
// product stays bound by memory bandwidth rather than by GB300's FP64 units;
// FP64 vectors (FP64 runs and the FP64 phase of mixed runs, whose matrix may be
// the FP32 copy) keep every vector value in FP64 and sum in FP64.
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double x) { s = fma(a, x, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float x) {
        const float y = __fmaf_rn(a, x, -c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// y[row*inc] = sum_j A[row][j] x[j*inc]; one warp per row
template <typename TA, typename T>
__global__ void k_gemv(const TA* __restrict__ A, const T* __restrict__ x, T* __restrict__ y, int nb, int inc) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int row = warp; row < nb; row += nw) {
        const TA* a = A + (size_t)row * nb;
        DotAcc<T> acc;
        for (int j = lane; j < nb; j += 32) acc.add(T(a[j]), x[(size_t)j * inc]);
        double v = acc.value();
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) y[(size_t)row * inc] = T(v);
    }
}

// part[s][j] = sum_{i in chunk s} A[i][j] x[i*inc]: column-parallel, coalesced rows
template <typename TA, typename T>
__global__ void k_gemv_t_part(const TA* __restrict__ A, const T* __restrict__ x, double* __restrict__ part, int nb,
                              int inc, int rows_per_chunk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i0 = blockIdx.y * rows_per_chunk, i1 = min(nb, i0 + rows_per_chunk);
    if (j >= nb) return;
    DotAcc<T> acc;
#pragma unroll 4
    for (int i = i0; i < i1; ++i) acc.add(T(A[(size_t)i * nb + j]), x[(size_t)i * inc]);
    part[(size_t)blockIdx.y * nb + j] = acc.value();
}

template <typename T>
__global__ void k_sum_parts(const double* __restrict__ part, int S, int nb, T* __restrict__ y, int inc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb) return;
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += part[(size_t)s * nb + j];
    y[(size_t)j * inc] = T(acc);
}

// Y[:, 0:ncols] = op(A) X[:, 0:ncols] with row strides ldx, ldy; 64x64 tiles,
// 256 threads, 4x4 outputs each.  TRANS: op(A) = A^T.  Arithmetic in the
// matrix type TA (vectors of type T are converted on load and store).
template <typename TA, typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_gemm(const TA* __restrict__ A, const T* __restrict__ X, int ldx,
                                              T* __restrict__ Y, int ldy, int nb, int ncols) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ TA As[BK][BM + 4];
    __shared__ TA Xs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    TA acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = TA(0);
    for (int k0 = 0; k0 < nb; k0 += BK) {
        for (int l = tid; l < BM * BK; l += 256) {
            int mm, kk;
            if (TRANS) { kk = l / BM; mm = l % BM; } else { mm = l / BK; kk = l % BK; }
            const int gm = m0 + mm, gk = k0 + kk;
            TA v = TA(0);
            if (gm < nb && gk < nb) v = TRANS ? A[(size_t)gk * nb + gm] : A[(size_t)gm * nb + gk];
            As[kk][mm] = v;
        }
        for (int l = tid; l < BK * BN; l += 256) {
            const int kk = l / BN, nn = l % BN;
            const int gk = k0 + kk, gn = n0 + nn;
            Xs[kk][nn] = (gk < nb && gn < ncols) ? TA(X[(size_t)gk * ldx + gn]) : TA(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            TA a[4], xv[4];
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
            if (gm < nb && gn < ncols) Y[(size_t)gm * ldy + gn] = T(acc[i][j]);
        }
}

// ---- FP64-accurate batched BEM products on the FP32 units ------------------------------
// Y = op(B) X for the FP64 vectors of FP64 batches (the FP64 phase of mixed
// runs included), with B = B_hi + B_lo (B_hi the FP32 copy of B, B_lo the FP32
// rounding of B - B_hi: together B to about 2^-48 relative) and x = x_hi + x_lo
// the same way.  Per term a_hi x_hi is exact as p + e (e = fma(a_hi, x_hi, -p));
// p is added to the high word of a double-FP32 accumulator with Knuth's TwoSum,
// whose rounding error is exact; that error, e and the cross terms a_hi x_lo +
// a_lo x_hi go into the low word (the a_lo x_lo term is 2^-48 of the term); the
// two words are combined in FP64.  (Kahan compensation in FP32 is not enough:
// it keeps each term to about FP32 precision.)  GB300 issues FP32 arithmetic
// at many times its FP64 rate, so twelve FP32 instructions per term beat one
// FP64 fused multiply-add.  The sum over K is split across blocks (blockIdx.z); the
// partials part[z][row][c] (FP64) are added in a fixed order by k_sum_splits.
__global__ void k_bem_lo(const double* __restrict__ B64, const float* __restrict__ B32, float* __restrict__ lo,
                         size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        lo[i] = (float)(B64[i] - (double)B32[i]);
}

void launch_bem_lo(const double* B64, const float* B32, float* B32lo, size_t n, cudaStream_t st) {
    k_bem_lo<<<1024, 256, 0, st>>>(B64, B32, B32lo, n);
}

template <bool TRANS>
__global__ void __launch_bounds__(256) k_gemm_df(const float* __restrict__ Ahi, const float* __restrict__ Alo,
                                                 const double* __restrict__ X, int ldx, double* __restrict__ part,
                                                 int ldp, int nb, int ncols, int kchunk) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float Ah[BK][BM + 4], Al[BK][BM + 4], Xh[BK][BN + 4], Xl[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk, kend = min(nb, kbeg + kchunk);
    float sh[4][4], sl[4][4];   // high and low words of the accumulators
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int l = tid; l < BM * BK; l += 256) {
            int mm, kk;
            if (TRANS) { kk = l / BM; mm = l % BM; } else { mm = l / BK; kk = l % BK; }
            const int gm = m0 + mm, gk = k0 + kk;
            float h = 0.f, w = 0.f;
            if (gm < nb && gk < kend) {
                const size_t idx = TRANS ? (size_t)gk * nb + gm : (size_t)gm * nb + gk;
                h = Ahi[idx];
                w = Alo[idx];
            }
            Ah[kk][mm] = h;
            Al[kk][mm] = w;
        }
        for (int l = tid; l < BK * BN; l += 256) {
            const int kk = l / BN, nn = l % BN;
            const int gk = k0 + kk, gn = n0 + nn;
            const double v = (gk < kend && gn < ncols) ? X[(size_t)gk * ldx + gn] : 0.0;
            const float h = (float)v;
            Xh[kk][nn] = h;
            Xl[kk][nn] = (float)(v - (double)h);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float ah[4], al[4], xh[4], xl[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ah[i] = Ah[kk][ty * 4 + i];
                al[i] = Al[kk][ty * 4 + i];
                xh[i] = Xh[kk][tx * 4 + i];
                xl[i] = Xl[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = __fmul_rn(ah[i], xh[j]);
                    float e = __fmaf_rn(ah[i], xh[j], -p);   // exact: a_hi x_hi = p + e
                    e = __fmaf_rn(ah[i], xl[j], e);
                    e = __fmaf_rn(al[i], xh[j], e);
                    // TwoSum: t + err = sh + p exactly
                    const float t = __fadd_rn(sh[i][j], p);
                    const float bp = __fsub_rn(t, sh[i][j]);
                    const float ap = __fsub_rn(t, bp);
                    const float err = __fadd_rn(__fsub_rn(sh[i][j], ap), __fsub_rn(p, bp));
                    sh[i][j] = t;
                    sl[i][j] = __fadd_rn(sl[i][j], __fadd_rn(err, e));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < nb && gn < ncols)
                part[((size_t)blockIdx.z * nb + gm) * ldp + gn] = (double)sh[i][j] + (double)sl[i][j];
        }
}

// y[row][c] = sum over the S splits of part[s][row][c], in split order (C = 2B columns)
__global__ void k_sum_splits(const double* __restrict__ part, int S, int nb, int C, double* __restrict__ y) {
    const size_t total = (size_t)nb * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int z = 0; z < S; ++z) acc += part[(size_t)z * total + i];
        y[i] = acc;
    }
}

// K splits so that the two products fill about four waves of two blocks per SM
int bem_df_splits(int nb, int B, int num_sms) {
    const int tiles = ((nb + 63) / 64) * ((B + 63) / 64) * 2;
    int S = (8 * num_sms + tiles - 1) / tiles;
    if (S > 16) S = 16;
    if (S < 1) S = 1;
    return S;
}

template <typename T> __host__ __device__ inline const T* bem_ptr(const MeshView& M);
template <> __host__ __device__ inline const double* bem_ptr<double>(const MeshView& M) { return M.B64; }
template <> __host__ __device__ inline const float* bem_ptr<float>(const MeshView& M) { return M.B32; }

// Row chunks of the column-parallel transposed product: enough blocks for about
// eight per SM, so that the column loads of many warps are in flight (at most
// 32 chunks: the partial sums are 32 x nb).
int bem_chunks(int nb, int num_sms) {
    const int colblocks = (nb + 255) / 256;
    int S = (8 * num_sms + colblocks - 1) / colblocks;
    if (S > 32) S = 32;
    if (S < 1) S = 1;
    return S;
}

// ---- autotuner: row chunks of the transposed single-instance product ------------------
// At the first product of a (nb, matrix type, vector type, SM count) the
// column-parallel kernel is timed with 4, 8, 16 and 32 row chunks (CUDA events
// on the launching stream; it reads the live input and writes only the
// partial-sum scratch); the fastest is kept for the process.
static std::mutex g_chunks_mu;
static std::map<std::tuple<int, int, int, int>, int> g_chunks;

template <typename F>
static int tuned_chunks(const Launch& L, int nb, int key_a, int key_b, F&& launch_with) {
    const auto key = std::make_tuple(nb, key_a, key_b, L.num_sms);
    // without tuning (a call that must not wait) the default shape, whatever an
    // earlier call tuned: its summation order then does not depend on history
    if (!L.tune) return bem_chunks(nb, L.num_sms);
    {
        std::lock_guard<std::mutex> lk(g_chunks_mu);
        auto it = g_chunks.find(key);
        if (it != g_chunks.end()) return it->second;
    }
    int best = bem_chunks(nb, L.num_sms);
    float best_ms = -1.f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int S : {4, 8, 16, 32}) {
        float t[3];
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, L.stream);
            launch_with(S);
            cudaEventRecord(e1, L.stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&t[rep], e0, e1);
            *L.launches += 1;
        }
        const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
        if (best_ms < 0.f || med < best_ms) {
            best = S;
            best_ms = med;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_chunks_mu);
    g_chunks[key] = best;
    return best;
}

int gemv_chunks_chosen(int nb, int key_a, int key_b, int num_sms) {
    std::lock_guard<std::mutex> lk(g_chunks_mu);
    auto it = g_chunks.find(std::make_tuple(nb, key_a, key_b, num_sms));
    return it == g_chunks.end() ? 0 : it->second;
}

template <typename TA, typename T>
static void bem_launch(const Launch& L, const TA* Bm, const MeshView& M, const BatchView<T>& V) {
    const int B = V.B, C = 2 * B, nb = M.nb;
    if (B == 1) {
        int blocks = (nb * 32 + 255) / 256;
        if (blocks > 8 * L.num_sms) blocks = 8 * L.num_sms;
        k_gemv<TA, T><<<blocks, 256, 0, L.stream>>>(Bm, V.ub_in, V.ub_out, nb, C);
        const int S = tuned_chunks(L, nb, (int)sizeof(TA), (int)sizeof(T), [&](int s) {
            k_gemv_t_part<TA, T><<<dim3((nb + 255) / 256, s), 256, 0, L.stream>>>(Bm, V.ub_in + 1,
                                                                                 (double*)V.bem_part, nb, C,
                                                                                 (nb + s - 1) / s);
        });
        const int rpc = (nb + S - 1) / S;
        k_gemv_t_part<TA, T><<<dim3((nb + 255) / 256, S), 256, 0, L.stream>>>(Bm, V.ub_in + 1, (double*)V.bem_part,
                                                                             nb, C, rpc);
        k_sum_parts<T><<<(nb + 255) / 256, 256, 0, L.stream>>>((const double*)V.bem_part, S, nb, V.ub_out + 1, C);
        *L.launches += 3;
    } else if constexpr (std::is_same<TA, double>::value && std::is_same<T, double>::value) {
        if (M.B32lo) {
            // FP64 batches: the FP64-accurate product on the FP32 units
            const int S = bem_df_splits(nb, B, L.num_sms);
            const int kchunk = (((nb + S - 1) / S) + 15) / 16 * 16;
            dim3 grid((nb + 63) / 64, (B + 63) / 64, S);
            double* part = reinterpret_cast<double*>(V.bem_part);
            k_gemm_df<false><<<grid, 256, 0, L.stream>>>(M.B32, M.B32lo, V.ub_in, C, part, C, nb, B, kchunk);
            k_gemm_df<true><<<grid, 256, 0, L.stream>>>(M.B32, M.B32lo, V.ub_in + B, C, part + B, C, nb, B, kchunk);
            size_t blocks = ((size_t)nb * C + 255) / 256;
            if (blocks > (size_t)8 * L.num_sms) blocks = (size_t)8 * L.num_sms;
            k_sum_splits<<<(unsigned)blocks, 256, 0, L.stream>>>(part, S, nb, C, V.ub_out);
            *L.launches += 3;
        } else {
            dim3 grid((nb + 63) / 64, (B + 63) / 64);
            k_gemm<TA, T, false><<<grid, 256, 0, L.stream>>>(Bm, V.ub_in, C, V.ub_out, C, nb, B);
            k_gemm<TA, T, true><<<grid, 256, 0, L.stream>>>(Bm, V.ub_in + B, C, V.ub_out + B, C, nb, B);
            *L.launches += 2;
        }
    } else {
        dim3 grid((nb + 63) / 64, (B + 63) / 64);
        k_gemm<TA, T, false><<<grid, 256, 0, L.stream>>>(Bm, V.ub_in, C, V.ub_out, C, nb, B);
        k_gemm<TA, T, true><<<grid, 256, 0, L.stream>>>(Bm, V.ub_in + B, C, V.ub_out + B, C, nb, B);
        *L.launches += 2;
    }
}

// ---- BEM products with the hierarchical (H-matrix) form of B -------------------------
// y = B_H x on columns [coff, coff + B) of the [nb][2B] surface arrays, in the
// two passes the packed layout is made for: (1) t = V x_sigma for every row of
// every low-rank leaf; (2) every position's row of y is the sum, over the
// entries of its row owner in block-tree order, of a dense leaf's row times
// x_sigma or a U row times t, written once (no atomics, a fixed order).  Values
// in the vector precision (FP32 or FP64), sums in DotAcc (compensated in FP32).
template <typename T, typename VT, bool WARP>
__global__ void k_hm_v(HMView H, const VT* __restrict__ vals, const T* __restrict__ x, int ldx, int coff, int B,
                       T* __restrict__ t) {
    if constexpr (WARP) {   // one instance: a warp per row of t, lanes over the columns of V
        const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
        if (g >= H.n_t) return;
        const HLeafDev lf = H.leaves[H.trow_leaf[g]];
        const int l = H.trow_l[g];
        const VT* Vr = vals + lf.val + (long long)l * lf.n;
        const int* cols = H.idx + lf.col_begin;
        DotAcc<T> acc;
        for (int b = lane; b < lf.n; b += 32) acc.add(T(Vr[b]), x[(size_t)cols[b] * ldx + coff]);
        double v = acc.value();
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) t[g] = T(v);
    } else {                // a thread per (row of t, instance): the row of V is broadcast
        const long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        if (tt >= (long long)H.n_t * B) return;
        const int g = (int)(tt / B), c = (int)(tt % B);
        const HLeafDev lf = H.leaves[H.trow_leaf[g]];
        const VT* Vr = vals + lf.val + (long long)H.trow_l[g] * lf.n;
        const int* cols = H.idx + lf.col_begin;
        DotAcc<T> acc;
        for (int b = 0; b < lf.n; ++b) acc.add(T(Vr[b]), x[(size_t)cols[b] * ldx + coff + c]);
        t[(size_t)g * B + c] = T(acc.value());
    }
}

template <typename T, typename VT>
__global__ void k_hm_own(HMView H, const VT* __restrict__ vals, const T* __restrict__ x, int ldx, int coff, int B,
                         const T* __restrict__ t, T* __restrict__ y) {
    const long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tt >= (long long)H.nb * B) return;
    const int sl = (int)(tt / B), c = (int)(tt % B);   // output row (owners in order) and instance
    const int o = H.slot_owner[sl];
    const int a = H.slot_a[sl];                        // local row within the owner
    DotAcc<T> acc;
    for (long long e = H.owner_ptr[o]; e < H.owner_ptr[o + 1]; ++e) {
        const HLeafDev lf = H.leaves[H.ent_leaf[e]];
        const int r = H.row_map[H.ent_rows[e] + a];    // row within the leaf's row cluster
        if (lf.kind == 0) {
            const VT* D = vals + lf.val + (long long)r * lf.n;
            const int* cols = H.idx + lf.col_begin;
            for (int b = 0; b < lf.n; ++b) acc.add(T(D[b]), x[(size_t)cols[b] * ldx + coff + c]);
        } else {
            const VT* U = vals + lf.val + (long long)lf.rank * lf.n + (long long)r * lf.rank;
            const T* tl = t + (size_t)lf.t_off * B + c;
            for (int l = 0; l < lf.rank; ++l) acc.add(T(U[l]), tl[(size_t)l * B]);
        }
    }
    y[(size_t)H.idx[H.owner_begin[o] + a] * ldx + coff + c] = T(acc.value());
}

template <typename T>
static void hm_apply(const Launch& L, const HMView& H, const T* x, T* y, int ldx, int coff, int B, T* t) {
    using VT = T;
    const VT* vals;
    if constexpr (sizeof(T) == 4) vals = reinterpret_cast<const VT*>(H.v32);
    else vals = reinterpret_cast<const VT*>(H.v64);
    if (H.n_t > 0) {
        if (B == 1) {
            const long long threads = (long long)H.n_t * 32;
            k_hm_v<T, VT, true><<<(unsigned)((threads + 255) / 256), 256, 0, L.stream>>>(H, vals, x, ldx, coff, B, t);
        } else {
            const long long threads = (long long)H.n_t * B;
            k_hm_v<T, VT, false><<<(unsigned)((threads + 255) / 256), 256, 0, L.stream>>>(H, vals, x, ldx, coff, B, t);
        }
        *L.launches += 1;
    }
    const long long threads = (long long)H.nb * B;
    k_hm_own<T, VT><<<(unsigned)((threads + 255) / 256), 256, 0, L.stream>>>(H, vals, x, ldx, coff, B, t, y);
    *L.launches += 1;
}

template <typename T>
void hm_product(const Launch& L, const HMDevice& H, const T* x, T* y, int B) {
    T* t0 = reinterpret_cast<T*>(H.t);
    T* t1 = t0 + (size_t)H.fwd.n_t * B;
    hm_apply<T>(L, H.fwd, x, y, 2 * B, 0, B, t0);   // u2_S = B u1_S
    hm_apply<T>(L, H.adj, x, y, 2 * B, B, B, t1);   // c_S = B^T t_S
}

// FP32 vectors use the FP32 copy of B, FP64 vectors the FP64 matrix (the FP64
// phase of a mixed run included: FP32 arithmetic in its products perturbed the
// stray field enough to keep the true torque of the final state near 4e-5).
// With a hierarchical form of B on the mesh, both products use it.
template <typename T>
void bem_product(const Launch& L, const MeshView& M, const BatchView<T>& V) {
    if (M.hm) {
        hm_product<T>(L, *M.hm, V.ub_in, V.ub_out, V.B);
        return;
    }
    if constexpr (sizeof(T) == 4) bem_launch<float, T>(L, M.B32, M, V);
    else bem_launch<double, T>(L, M.B64, M, V);
}

// ---- effective field, gradient, energies and step dot products -----------------------
int field_blocks(const Launch& L, const MeshView& M, int B) {
    const int RB = FIELD_THREADS / B;
    int nblk = (M.N + RB - 1) / RB;
    const int maxblk = 4 * L.num_sms;
    return nblk < maxblk ? nblk : maxblk;
}

template <typename T, bool GEN>
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
        const double lam6 = ic.lam / 6.0, q24 = ic.Q / 24.0;
        const double* mt = V.m + (size_t)(1 - cur) * N * 3 * B;
        const double* mb = V.m + (size_t)cur * N * 3 * B;
        double* Gt = V.H + (size_t)(1 - cur) * N * 3 * B;        // grad phi at the trial point
        const double* Gb = V.H + (size_t)cur * N * 3 * B;   // grad phi at the base point
        for (int row = blockIdx.x * RB + rl; row < N; row += gridDim.x * RB) {
            const double vi = GEN ? M.gV[row] : (double)(M.node[row] & 0xff);
            const size_t i3 = (size_t)row * 3 * B + b;
            const double mx = mt[i3], my = mt[i3 + B], mz = mt[i3 + 2 * B];
            T ex0 = T(0), ex1 = T(0), ex2 = T(0), hd0 = T(0), hd1 = T(0), hd2 = T(0);
            // neighbour values in T: the FP32 kernel reads the FP32 copy of the trial
            // point (exact zero differences for equal values are kept)
            const T* mn = (sizeof(T) == 4) ? reinterpret_cast<const T*>(V.m32) : reinterpret_cast<const T*>(mt);
            const T tx = mn[i3], ty = mn[i3 + B], tz = mn[i3 + 2 * B];
            const int e0 = M.rowptr[row], e1 = M.rowptr[row + 1];
            for (int e = e0; e < e1; ++e) {
                const int j = __ldg(&M.col[e]) & 0x7fffffff;
                const T k = GEN ? T(GenTab<T>::A(M)[e].x) : T(sbyte(__ldg(&M.pkA[e]), 0));
                const size_t j3 = (size_t)j * 3 * B + b;
                // difference form: exact zero for a uniform state, no cancellation
                ex0 += k * (mn[j3] - tx);
                ex1 += k * (mn[j3 + B] - ty);
                ex2 += k * (mn[j3 + 2 * B] - tz);
                if (demag) {
                    // (forward + adjoint)/2: the potential whose lumped gradient is the
                    // exact gradient of the stray-field energy
                    const size_t jc = (size_t)j * 2 * B + b;
                    const T u = T(0.5) * (V.U1[jc] + V.U2[jc] + V.U2[jc + B]);
                    if constexpr (GEN) {
                        const typename GenTab<T>::V4 gb = GenTab<T>::Bt(M)[e];
                        hd0 += gb.x * u;
                        hd1 += gb.y * u;
                        hd2 += gb.z * u;
                    } else {
                        const int wb = __ldg(&M.pkB[e]);
                        hd0 += T(sbyte(wb, 0)) * u;
                        hd1 += T(sbyte(wb, 1)) * u;
                        hd2 += T(sbyte(wb, 2)) * u;
                    }
                }
            }
            const double m[3] = {mx, my, mz};
            const double kx[3] = {(double)ex0, (double)ex1, (double)ex2};
            const double ma = m[0] * ic.a[0] + m[1] * ic.a[1] + m[2] * ic.a[2];
            // GB300 issues FP64 at a small fraction of its FP32 rate: one division
            // per node (1/V_i), constant factors as products, squared maxima
            // (the square roots are taken once, on the totals, by k_decide)
            const double ivi = 1.0 / vi;
            const double cex = -4.0 * ic.lam * ivi;
            const double hd[3] = {-(double)hd0 * ivi, -(double)hd1 * ivi, -(double)hd2 * ivi};
            double h[3];
            for (int c = 0; c < 3; ++c) h[c] = cex * kx[c] + ic.Q * ma * ic.a[c] + ic.hz[c] + hd[c];
            // grad phi = -(V/12) h ;  H = -m x grad phi = (V/12) m x h ;  g = m x H
            const double v12 = vi * (1.0 / 12.0), v24 = vi * (1.0 / 24.0);
            const double gr[3] = {-v12 * h[0], -v12 * h[1], -v12 * h[2]};
            const double mh[3] = {m[1] * h[2] - m[2] * h[1], m[2] * h[0] - m[0] * h[2], m[0] * h[1] - m[1] * h[0]};
            const double Hv[3] = {v12 * mh[0], v12 * mh[1], v12 * mh[2]};
            Gt[i3] = gr[0];
            Gt[i3 + B] = gr[1];
            Gt[i3 + 2 * B] = gr[2];
            if (V.hout) {
                V.hout[i3] = h[0];
                V.hout[i3 + B] = h[1];
                V.hout[i3 + 2 * B] = h[2];
            }
            const double g[3] = {m[1] * Hv[2] - m[2] * Hv[1], m[2] * Hv[0] - m[0] * Hv[2],
                                 m[0] * Hv[1] - m[1] * Hv[0]};
            const double bm[3] = {mb[i3], mb[i3 + B], mb[i3 + 2 * B]};
            const double bg[3] = {Gb[i3], Gb[i3 + B], Gb[i3 + 2 * B]};
            // g_b = m_b x (-m_b x grad_b) = grad_b - (m_b . grad_b) m_b  (|m_b| = 1)
            const double bmg = bm[0] * bg[0] + bm[1] * bg[1] + bm[2] * bg[2];
            const double gb[3] = {bg[0] - bmg * bm[0], bg[1] - bmg * bm[1], bg[2] - bmg * bm[2]};
            // E is quadratic in m, so E_t - E_b = (grad_t + grad_b) . (m_t - m_b) / 2 exactly
            acc[Q_DE] += 0.5 * ((gr[0] + bg[0]) * (m[0] - bm[0]) + (gr[1] + bg[1]) * (m[1] - bm[1]) +
                                (gr[2] + bg[2]) * (m[2] - bm[2]));
            const double mxa[3] = {m[1] * ic.a[2] - m[2] * ic.a[1], m[2] * ic.a[0] - m[0] * ic.a[2],
                                   m[0] * ic.a[1] - m[1] * ic.a[0]};
            acc[Q_EEX] += lam6 * (m[0] * kx[0] + m[1] * kx[1] + m[2] * kx[2]);
            acc[Q_EAN] += q24 * vi * (mxa[0] * mxa[0] + mxa[1] * mxa[1] + mxa[2] * mxa[2]);
            acc[Q_EZ] -= v12 * (m[0] * ic.hz[0] + m[1] * ic.hz[1] + m[2] * ic.hz[2]);
            acc[Q_ED] -= v24 * (m[0] * hd[0] + m[1] * hd[1] + m[2] * hd[2]);
            acc[Q_TORQUE] = fmax(acc[Q_TORQUE], mh[0] * mh[0] + mh[1] * mh[1] + mh[2] * mh[2]);
            acc[Q_HMAX] = fmax(acc[Q_HMAX], Hv[0] * Hv[0] + Hv[1] * Hv[1] + Hv[2] * Hv[2]);
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
    kernel_smem_attr((const void*)k_field<T, false>, 96 * 1024);
    kernel_smem_attr((const void*)k_field<T, true>, 96 * 1024);
    if (M.gen) k_field<T, true><<<nblk, FIELD_THREADS, smem, L.stream>>>(M, V, demag);
    else k_field<T, false><<<nblk, FIELD_THREADS, smem, L.stream>>>(M, V, demag);
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
    const double Edirect = ((v[Q_EEX] + v[Q_EAN]) + v[Q_EZ]) + v[Q_ED];
    // Decisions use E(base) + (E(trial) - E(base)) with the difference from the
    // gradients (exact for the quadratic energy): its rounding scales with the
    // step, not with |E|, so tiny decreases near the minimum stay resolvable.
    const double E = s.phase == PH_INIT ? Edirect : s.Eacc + v[Q_DE];
    s.evals += 1;
    if (v[Q_BAD] > 0.0 || !isfinite(E) || !isfinite(Edirect)) {
        s.status = 4;   // LBM_E_NAN
        s.phase = PH_DONE;
        return;
    }
    v[Q_TORQUE] = sqrt(v[Q_TORQUE]);   // the field kernel keeps squared maxima
    v[Q_HMAX] = sqrt(v[Q_HMAX]);
    const double gg = v[Q_GG], torque = v[Q_TORQUE];
    const bool conv = so.grad_tol > 0.0 ? (gg < so.grad_tol) : (torque < so.tol);
    bool accept;
    if (s.phase == PH_INIT || s.phase == PH_LB) {
        accept = true;   // LaBonte's iteration takes every step
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
    s.E = Edirect;
    s.Eacc = E;
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
        const bool warm = s.warm != 0 && so.method == 0;
        s.warm = 0;
        s.hist[0] = E;
        s.nhist = 1;
        s.hpos = 1 % mem;
        s.iters = 0;
        s.line_searches = 0;
        s.backtracks = 0;
        if (!warm) {
            s.ntau2 = 0;
            s.kappa = so.kappa0;
        }
        s.best_torque = torque;
        s.best_iter = 0;
        if (conv) { s.status = 0; s.phase = PH_DONE; return; }
        if (warm) {
            // a new precision phase at the point where the previous one stopped:
            // its next BB step (and kappa, tau^2 memory) continues the iteration;
            // the nonmonotone test against this evaluation's energy guards it
            s.tau = fmin(fmax(s.tau, so.tau_min), so.tau_max);
            s.phase = PH_BB;
        } else if (so.method == 1) {
            s.tau = so.omega;
            s.phase = PH_LB;
            s.line_searches = 0;
        } else {
            s.tau = 1.0 / v[Q_HMAX];
            s.phase = PH_SEARCH;
            s.E_ref = E;
            s.line_searches = 1;
        }
        // the iteration limit stops after the next step is prepared: a resumed
        // run continues from next_phase exactly where this one would have gone on
        if (so.max_iter <= 0) { s.next_phase = s.phase; s.status = 3; s.phase = PH_DONE; }
        return;
    }
    s.hist[s.hpos] = E;
    s.hpos = (s.hpos + 1) % mem;
    if (s.nhist < mem) s.nhist += 1;
    s.iters += 1;
    if (conv) { s.status = 0; s.phase = PH_DONE; return; }
    // the iteration limit and a stall stop after the next step is prepared (tau,
    // kappa, tau^2 memory), so that a resumed run continues from next_phase
    // exactly as this one would have gone on
    bool stop = s.iters >= so.max_iter;
    // progress = the smallest torque so far halved; a phase that creeps (new
    // minima, but no halving within stall_iters steps) has stalled
    if (torque < 0.5 * s.best_torque) {
        s.best_torque = torque;
        s.best_iter = s.iters;
    } else if (so.stall_iters > 0 && s.iters - s.best_iter >= so.stall_iters) {
        stop = true;
    }
    if (s.phase == PH_LB) {   // LaBonte: the next step uses the same relaxation
        if (stop) { s.next_phase = PH_LB; s.status = 3; s.phase = PH_DONE; }
        return;
    }
    const double ss = v[Q_SS], sy = v[Q_SY], yy = v[Q_YY];
    double tau = 1.0 / v[Q_HMAX];   // s.y <= 0: restart with the first-step trial
    if (sy > 0.0 && so.bb_rule != 0) {
        // plain rules: BB1, BB2, or BB1 and BB2 on alternate steps
        const double t1 = ss / sy, t2 = sy / yy;
        const bool first = so.bb_rule == 1 || (so.bb_rule == 3 && ((s.iters - 1) & 1) == 0);
        tau = first ? t1 : t2;
    } else if (sy > 0.0) {
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
    if (stop) { s.next_phase = PH_BB; s.status = 3; s.phase = PH_DONE; }
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
        // the trial point, and its FP32 copy for the FP32 kernels (one conversion
        // per node instead of one per neighbour entry)
        auto put = [&](double x0, double x1, double x2) {
            mt[i3] = x0;
            mt[i3 + B] = x1;
            mt[i3 + 2 * B] = x2;
            if (V.m32) {
                V.m32[i3] = (float)x0;
                V.m32[i3 + B] = (float)x1;
                V.m32[i3 + 2 * B] = (float)x2;
            }
        };
        if (phase == PH_INIT) {
            put(mb[i3], mb[i3 + B], mb[i3 + 2 * B]);
            continue;
        }
        if (phase == PH_LB) {
            // LaBonte, all nodes at once: m <- normalize((1 - omega) m + omega h/|h|);
            // h is parallel to -grad phi (positive nodal volumes)
            const double* Gb = V.H + (size_t)cur * N * 3 * B;
            const double om = V.st[b].tau;
            const double m0 = mb[i3], m1 = mb[i3 + B], m2 = mb[i3 + 2 * B];
            const double g0 = Gb[i3], g1 = Gb[i3 + B], g2 = Gb[i3 + 2 * B];
            const double gn = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
            double x0 = m0, x1 = m1, x2 = m2;
            if (gn > 0.0) {
                x0 = (1.0 - om) * m0 - om * g0 / gn;
                x1 = (1.0 - om) * m1 - om * g1 / gn;
                x2 = (1.0 - om) * m2 - om * g2 / gn;
            }
            const double xn = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
            put(x0 / xn, x1 / xn, x2 / xn);
            continue;
        }
        // x = [(1 - |w|^2) m - 2 m x w + 2 (m.w) w] / (1 + |w|^2),  w = tau H / 2
        const double* Gb = V.H + (size_t)cur * N * 3 * B;   // grad phi at the base point
        const double ht = 0.5 * V.st[b].tau;
        const double m0 = mb[i3], m1 = mb[i3 + B], m2 = mb[i3 + 2 * B];
        const double g0 = Gb[i3], g1 = Gb[i3 + B], g2 = Gb[i3 + 2 * B];
        // w = (tau/2) H with H = -m x grad phi
        const double w0 = -ht * (m1 * g2 - m2 * g1), w1 = -ht * (m2 * g0 - m0 * g2), w2 = -ht * (m0 * g1 - m1 * g0);
        const double ww = w0 * w0 + w1 * w1 + w2 * w2;
        const double mw = m0 * w0 + m1 * w1 + m2 * w2;
        const double c0 = m1 * w2 - m2 * w1, c1 = m2 * w0 - m0 * w2, c2 = m0 * w1 - m1 * w0;
        const double iden = 1.0 / (1.0 + ww);   // one FP64 division per node
        put(((1.0 - ww) * m0 - 2.0 * c0 + 2.0 * mw * w0) * iden, ((1.0 - ww) * m1 - 2.0 * c1 + 2.0 * mw * w1) * iden,
            ((1.0 - ww) * m2 - 2.0 * c2 + 2.0 * mw * w2) * iden);
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
__global__ void k_reset(InstState* st, int B, int set_cur0, int warm) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    InstState& s = st[b];
    s.phase = PH_INIT;
    s.status = 3;
    if (set_cur0) s.cur = 0;
    s.iters = s.evals = s.line_searches = s.backtracks = 0;
    s.nhist = s.hpos = 0;
    if (!warm) s.ntau2 = 0;   // warm: tau, kappa and the tau^2 memory are kept
    s.warm = warm;
    s.next_phase = PH_DONE;
    s.cg1 = s.cg2 = 0;
}

void reset_states(const Launch& L, InstState* st, int B, const StepOpts& so, int set_cur0, int warm) {
    (void)so;
    k_reset<<<(B + 127) / 128, 128, 0, L.stream>>>(st, B, set_cur0, warm);
    *L.launches += 1;
}

// Continue instances that the iteration limit (or a stall) stopped, from the
// step they had prepared; converged and failed instances stay done.
__global__ void k_resume(InstState* st, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    InstState& s = st[b];
    if (s.phase == PH_DONE && s.status == 3 && s.next_phase != PH_DONE) s.phase = s.next_phase;
}

void resume_states(const Launch& L, InstState* st, int B) {
    k_resume<<<(B + 127) / 128, 128, 0, L.stream>>>(st, B);
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
            u[((size_t)b * 2 + 0) * N + i] = cell * (double)V.U1[i * 2 * B + b];
            u[((size_t)b * 2 + 1) * N + i] = cell * (double)V.U2[i * 2 * B + b];
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
    template int pcg_solve<T>(const Launch&, const MeshView&, const BatchView<T>&, int, double, int, bool); \
    template void bem_product<T>(const Launch&, const MeshView&, const BatchView<T>&);                     \
    template void rhs_eval<T>(const Launch&, const MeshView&, const BatchView<T>&);                        \
    template void hm_product<T>(const Launch&, const HMDevice&, const T*, T*, int);                         \
    template void field_eval<T>(const Launch&, const MeshView&, const BatchView<T>&, int);                 \
    template void trial_update<T>(const Launch&, const MeshView&, const BatchView<T>&);                    \
    template void decide<T>(const Launch&, const MeshView&, const BatchView<T>&, const StepOpts&, int);    \
    template void pack_m<T>(const Launch&, const MeshView&, const BatchView<T>&, const double*);           \
    template void unpack_m<T>(const Launch&, const MeshView&, const BatchView<T>&, double*);               \
    template void unpack_field<T>(const Launch&, const MeshView&, const BatchView<T>&, double*, double*);

LBM_INSTANTIATE(float)
LBM_INSTANTIATE(double)

}  // namespace lbm
