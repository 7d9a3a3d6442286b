// Scalar potential with the open boundary by space transformation (Sec. 3.1:
// the scheme of the paper's own steepest-descent solver): the magnet, an air
// box and a shell mapped onto the rest of space share one Kuhn grid; the
// shell's tetrahedra carry the tensor M = |det J| J^-1 J^-T of the map, the
// outer face (the image of infinity) has u = 0, and one symmetric solve
//     K_grid u = b      (b = (1/4) Gint m at the magnet's nodes, 0 elsewhere)
// gives the total potential, whose lumped gradient at the magnet's nodes is
// exactly the gradient field of the stray-field energy (no boundary matrix, no
// adjoint chain).  The host set-up (csrc/shell.cu) builds the grid and its
// stiffness; here the solve runs on the device for all instances of a batch
// at once: Jacobi-preconditioned CG, one persistent cooperative kernel per
// solve (grid barriers with the context's time limit), the grid potential
// warm-started from the instance's previous solve.
//
// Every row that is not on the outer face is an interior node of the grid, and
// the Kuhn split couples a node only to the 14 neighbours along +-x, +-y, +-z,
// +-(x+y), +-(x+z), +-(y+z), +-(x+y+z).  The operator is therefore applied as a
// stencil with per-row coefficients (no column indices): a 16-value record per
// row (diagonal, the 14 couplings in that order, 1/K_ii).  Where M = I (the
// magnet and the air) the diagonal couplings vanish and the row takes the
// 7-point form.
#include <type_traits>

#include "solver_common.cuh"

namespace lbm {
namespace {

template <typename W>
struct ShellArgs {
    ShellDev S;
    int B;
    const InstState* st;
    const double* bvec;           // [N][B] divergence right-hand side of the magnet
    double* x;                    // [Ng][B] FP64 grid potential
    W *r, *z, *p, *q, *d;         // [Ng][B] work vectors (d: this solve's correction of x)
    double tol2;
    int max_iter;
    unsigned* bar;
    int* err;
    double* part;
    double* fin;
    unsigned long long* sweeps;
};

template <typename C> struct CoefLoad;
template <> struct CoefLoad<float> {
    __device__ static void row(const float* p, float (&c)[16]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p) + k);
            c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
        }
    }
};
template <> struct CoefLoad<double> {
    __device__ static void row(const double* p, double (&c)[16]) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const double2 v = __ldg(reinterpret_cast<const double2*>(p) + k);
            c[2 * k] = v.x; c[2 * k + 1] = v.y;
        }
    }
};

// VEC consecutive values (instances c0 .. c0+VEC-1 of one row), L2-only loads
// (CG) for values other blocks write during the kernel.
template <int VEC, bool CG, typename W>
__device__ __forceinline__ void ldv(W (&d)[VEC], const W* p) {
    if constexpr (VEC == 1) {
        d[0] = CG ? __ldcg(p) : *p;
    } else if constexpr (std::is_same<W, float>::value && VEC == 4) {
        const float4 v = CG ? __ldcg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    } else if constexpr (std::is_same<W, float>::value && VEC == 2) {
        const float2 v = CG ? __ldcg(reinterpret_cast<const float2*>(p)) : *reinterpret_cast<const float2*>(p);
        d[0] = v.x; d[1] = v.y;
    } else {   // doubles, VEC = 2 or 4: 16-byte loads
#pragma unroll
        for (int k = 0; k < VEC; k += 2) {
            const double2 v = CG ? __ldcg(reinterpret_cast<const double2*>(p + k)) : *reinterpret_cast<const double2*>(p + k);
            d[k] = v.x; d[k + 1] = v.y;
        }
    }
}
template <int VEC, typename W>
__device__ __forceinline__ void stv(W* p, const W (&d)[VEC]) {
    if constexpr (VEC == 1) {
        *p = d[0];
    } else if constexpr (std::is_same<W, float>::value && VEC == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(d[0], d[1], d[2], d[3]);
    } else if constexpr (std::is_same<W, float>::value && VEC == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(d[0], d[1]);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; k += 2) *reinterpret_cast<double2*>(p + k) = make_double2(d[k], d[k + 1]);
    }
}

// (K v)_row for VEC instances: v points at the row's first value; sx, sy, sz
// are the strides of one grid step along x, y, z in v.
template <int VEC, typename R, typename C, typename V>
__device__ __forceinline__ void kuhn_apply(const C (&c)[16], const V* v, ptrdiff_t sx, ptrdiff_t sy, ptrdiff_t sz,
                                           bool full, R (&w)[VEC]) {
    const ptrdiff_t off[15] = {0, sx, -sx, sy, -sy, sz, -sz, sx + sy, -sx - sy, sx + sz, -sx - sz, sy + sz, -sy - sz,
                               sx + sy + sz, -sx - sy - sz};
#pragma unroll
    for (int k = 0; k < VEC; ++k) w[k] = R(0);
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        V t[VEC];
        ldv<VEC, true>(t, v + off[j]);
#pragma unroll
        for (int k = 0; k < VEC; ++k) w[k] += R(c[j]) * R(t[k]);
    }
    if (full) {
#pragma unroll
        for (int j = 7; j < 15; ++j) {
            V t[VEC];
            ldv<VEC, true>(t, v + off[j]);
#pragma unroll
            for (int k = 0; k < VEC; ++k) w[k] += R(c[j]) * R(t[k]);
        }
    }
}

// Threads hold VEC consecutive instances of one row: thread tid works on
// instances c0 = (tid % G) VEC .. c0 + VEC - 1 (G = B / VEC) of row lane tid / G.
// W is the type of the CG work vectors and of the per-thread and per-block
// dot-product sums (grid totals in FP64):
//   W = double: plain FP64 CG on K d = f - K x, then x += d;
//   W = float, RES64 = false (the FP32 phase of a mixed run): the residual of
//     the warm start in FP32 arithmetic, FP32 CG to the tolerance, x += d;
//   W = float, RES64 = true (FP64 solves with mixed iterations): cycles of the
//     FP64 residual f - K x, FP32 CG until it has reduced that residual by
//     MP_INNER (or met the tolerance), x += d; the solve ends on the FP64
//     residual test (restarted CG, as the magnet's mixed-iteration solves).
// Per CG iteration (the same fused form as the magnet's solves):
//   A: w = K z, p = z + beta p, q = w + beta q (= K p), partial p.q
//   B: alpha = rho / p.q, d += alpha p, r -= alpha q, z = r / K_ii, partials r.z, r.r
// Outer-face rows keep zero in every vector (and 1/K_ii = 0 there), so they
// drop out of every product.
template <typename W, bool RES64, int THREADS, int VEC>
__global__ void __launch_bounds__(THREADS, 1) k_shell_pcg(ShellArgs<W> A) {
    using R0 = typename std::conditional<RES64 || std::is_same<W, double>::value, double, float>::type;
    extern __shared__ double sm[];
    const int B = A.B, tid = threadIdx.x, bd = blockDim.x;
    const int G = B / VEC, RB = bd / G;
    const bool lane = tid < RB * G;
    const int g = tid % G, c0 = g * VEC, rl = tid / G;
    const int nrow = (G <= 32 && (32 % G) == 0) ? (bd >> 5) : RB;
    double* scratch = sm;                          // [4][nrow][B] doubles (or floats in the same room)
    double* out = scratch + 4 * (size_t)nrow * B;  // [4][B]
    double* s_rho = out + 4 * B;
    double* s_rhop = s_rho + B;
    double* s_ab = s_rhop + B;
    double* s_tol = s_ab + B;
    double* s_tin = s_tol + B;
    int* s_flag = (int*)(s_tin + B);
    int* s_act = s_flag + B;
    int* s_it = s_act + B;
    int* s_done = s_it + B;
    // alpha or beta of the current step in W for the row loops (a conversion from
    // FP64 per thread would issue at GB300's FP64 rate)
    W* s_abw = reinterpret_cast<W*>(s_done + B);   // 8-byte aligned: four int arrays of B
    for (int i = tid; i < B; i += bd) {
        s_act[i] = A.st[i].phase != PH_DONE;
        s_it[i] = 0;
        s_done[i] = 0;
    }
    __syncthreads();
    bool act[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) act[k] = lane && s_act[c0 + k];
    const int Ng = A.S.Ng, n1 = A.S.n1;
    const ptrdiff_t sx = B, sy = (ptrdiff_t)n1 * B, sz = (ptrdiff_t)n1 * n1 * B;
    const W* coefW;
    if constexpr (std::is_same<W, double>::value) coefW = A.S.coef64;
    else coefW = A.S.coef32;
    const int row0 = blockIdx.x * RB + rl, rstride = gridDim.x * RB;
    unsigned epoch = 0;
    auto publish = [&]() -> bool {
        if (tid < B)
            for (int k = 0; k < 4; ++k) A.part[((size_t)blockIdx.x * B + tid) * 4 + k] = out[k * B + tid];
        return grid_reduce<4>(A.part, 0, B, A.fin, out, A.bar, epoch, A.err);
    };
    const W zero[VEC] = {};
    for (int cycle = 0;; ++cycle) {
        // residual of the current x: r = f - K x, z = r / K_ii, d = p = q = 0
        {
            R0 v[4][VEC];   // r.z, r.r, f.f
#pragma unroll
            for (int k = 0; k < VEC; ++k) v[0][k] = v[1][k] = v[2][k] = v[3][k] = R0(0);
            if (lane)
                for (int row = row0; row < Ng; row += rstride) {
                    const size_t i = (size_t)row * B + c0;
                    const int kind = __ldg(&A.S.kind[row]);
                    stv<VEC>(A.p + i, zero);
                    stv<VEC>(A.q + i, zero);
                    stv<VEC>(A.d + i, zero);
                    if (kind == 0) {   // outer face: u = 0
                        stv<VEC>(A.r + i, zero);
                        stv<VEC>(A.z + i, zero);
                        continue;
                    }
                    const int gn = __ldg(&A.S.gnode[row]);
                    double f[VEC];
#pragma unroll
                    for (int k = 0; k < VEC; ++k) f[k] = 0.0;
                    if (gn >= 0) ldv<VEC, false>(f, A.bvec + (size_t)gn * B + c0);
                    R0 kx[VEC];
                    W dinv;
                    if constexpr (std::is_same<R0, double>::value) {
                        double c[16];
                        CoefLoad<double>::row(A.S.coef64 + (size_t)row * 16, c);
                        kuhn_apply<VEC>(c, A.x + i, sx, sy, sz, kind == 2, kx);
                        dinv = W(c[15]);
                    } else {
                        float c[16];
                        CoefLoad<float>::row(A.S.coef32 + (size_t)row * 16, c);
                        kuhn_apply<VEC>(c, A.x + i, sx, sy, sz, kind == 2, kx);
                        dinv = c[15];
                    }
                    W rw[VEC], zw[VEC];
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        if (!act[k]) f[k] = 0.0;
                        const R0 rv = R0(f[k]) - kx[k];
                        rw[k] = W(rv);
                        zw[k] = rw[k] * dinv;
                        if (act[k]) {
                            v[0][k] += R0(rw[k]) * R0(zw[k]);
                            v[1][k] += rv * rv;
                            v[2][k] += R0(f[k]) * R0(f[k]);
                        }
                    }
                    stv<VEC>(A.r + i, rw);
                    stv<VEC>(A.z + i, zw);
                }
            block_reduce_cols<4, VEC, R0>(v, reinterpret_cast<R0*>(scratch), out, B, G, RB);
            if (!publish()) return;
        }
        if (tid < B) {
            const double rr = out[B + tid];
            if (cycle == 0) s_tol[tid] = A.tol2 * out[2 * B + tid];
            s_done[tid] = !s_act[tid] || rr <= s_tol[tid] || s_it[tid] >= A.max_iter;
            s_tin[tid] = RES64 ? fmax(s_tol[tid], MP_INNER * MP_INNER * rr) : s_tol[tid];
            s_rhop[tid] = 1.0;
        }
        if (__syncthreads_and(tid < B ? s_done[tid] : 1)) break;
        for (int it = 0;; ++it) {
            if (tid < B) {
                const double rho = out[tid], rr = out[B + tid];
                const int conv = s_done[tid] || rr <= s_tin[tid] || s_it[tid] >= A.max_iter;
                s_ab[tid] = (it == 0 || conv) ? 0.0 : rho / s_rhop[tid];
                s_abw[tid] = W(s_ab[tid]);
                s_rho[tid] = rho;
                s_flag[tid] = conv;
            }
            if (__syncthreads_and(tid < B ? s_flag[tid] : 1)) break;
            bool run[VEC];
            W beta[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                run[k] = act[k] && !s_flag[c0 + k];
                beta[k] = s_abw[c0 + k];
            }
            W v[4][VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) v[0][k] = v[1][k] = v[2][k] = v[3][k] = W(0);
            // outer-face rows (kind 0) skip the stencil and keep zero
            if (lane)
                for (int row = row0; row < Ng; row += rstride) {
                    const int kind = __ldg(&A.S.kind[row]);
                    if (kind == 0) continue;
                    const size_t i = (size_t)row * B + c0;
                    W c[16];
                    CoefLoad<W>::row(coefW + (size_t)row * 16, c);
                    W w[VEC], zi[VEC], pv[VEC], qv[VEC];
                    ldv<VEC, false>(zi, A.z + i);
                    ldv<VEC, false>(pv, A.p + i);
                    ldv<VEC, false>(qv, A.q + i);
                    kuhn_apply<VEC>(c, A.z + i, sx, sy, sz, kind == 2, w);
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        pv[k] = zi[k] + beta[k] * pv[k];
                        qv[k] = w[k] + beta[k] * qv[k];
                        if (run[k]) v[0][k] += pv[k] * qv[k];
                    }
                    stv<VEC>(A.p + i, pv);
                    stv<VEC>(A.q + i, qv);
                }
            block_reduce_cols<4, VEC, W>(v, reinterpret_cast<W*>(scratch), out, B, G, RB);
            if (!publish()) return;
            if (tid < B) {
                s_ab[tid] = s_flag[tid] ? 0.0 : s_rho[tid] / out[tid];
                s_abw[tid] = W(s_ab[tid]);
            }
            __syncthreads();
            W alpha[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                alpha[k] = s_abw[c0 + k];
                v[0][k] = v[1][k] = v[2][k] = v[3][k] = W(0);
            }
            // two rows per pass (a stream: every load first); outer-face rows
            // need no test: their vectors and 1/K_ii are zero, and stay so
            if (lane)
                for (int row = row0; row < Ng; row += 2 * rstride) {
                    const int rowb = row + rstride;
                    const bool two = rowb < Ng;
                    const size_t ia = (size_t)row * B + c0, ib = (size_t)(two ? rowb : row) * B + c0;
                    const W da = __ldg(coefW + (size_t)row * 16 + 15);
                    const W db = __ldg(coefW + (size_t)(two ? rowb : row) * 16 + 15);
                    W xa[VEC], pa[VEC], ra[VEC], qa[VEC], xb[VEC], pb[VEC], rb[VEC], qb[VEC];
                    ldv<VEC, false>(xa, A.d + ia);
                    ldv<VEC, false>(pa, A.p + ia);
                    ldv<VEC, false>(ra, A.r + ia);
                    ldv<VEC, false>(qa, A.q + ia);
                    ldv<VEC, false>(xb, A.d + ib);
                    ldv<VEC, false>(pb, A.p + ib);
                    ldv<VEC, false>(rb, A.r + ib);
                    ldv<VEC, false>(qb, A.q + ib);
#pragma unroll
                    for (int k = 0; k < VEC; ++k) {
                        xa[k] += alpha[k] * pa[k];
                        ra[k] -= alpha[k] * qa[k];
                        pa[k] = ra[k] * da;   // z
                        if (run[k]) {
                            v[0][k] += ra[k] * pa[k];
                            v[1][k] += ra[k] * ra[k];
                        }
                    }
                    stv<VEC>(A.d + ia, xa);
                    stv<VEC>(A.r + ia, ra);
                    stv<VEC>(A.z + ia, pa);
                    if (two) {
#pragma unroll
                        for (int k = 0; k < VEC; ++k) {
                            xb[k] += alpha[k] * pb[k];
                            rb[k] -= alpha[k] * qb[k];
                            pb[k] = rb[k] * db;
                            if (run[k]) {
                                v[0][k] += rb[k] * pb[k];
                                v[1][k] += rb[k] * rb[k];
                            }
                        }
                        stv<VEC>(A.d + ib, xb);
                        stv<VEC>(A.r + ib, rb);
                        stv<VEC>(A.z + ib, pb);
                    }
                }
            block_reduce_cols<4, VEC, W>(v, reinterpret_cast<W*>(scratch), out, B, G, RB);
            if (!publish()) return;
            if (tid < B) {
                s_rhop[tid] = s_rho[tid];
                if (!s_flag[tid]) s_it[tid] += 1;
            }
            __syncthreads();
        }
        // fold the cycle's correction into x before anything reads x
        if (lane)
            for (int row = row0; row < Ng; row += rstride) {
                const size_t i = (size_t)row * B + c0;
                double xv[VEC];
                W dv[VEC];
                ldv<VEC, false>(xv, A.x + i);
                ldv<VEC, false>(dv, A.d + i);
#pragma unroll
                for (int k = 0; k < VEC; ++k) xv[k] += (double)dv[k];
                stv<VEC>(A.x + i, xv);
            }
        if (!RES64 || cycle + 1 >= MP_MAX_CYCLES) break;
        if (!grid_sync(A.bar, gridDim.x, epoch, A.err)) return;
    }
    if (blockIdx.x == 0) {
        for (int i = tid; i < B; i += bd)
            atomicAdd((unsigned long long*)&((InstState*)A.st)[i].cg1, (unsigned long long)s_it[i]);
        if (tid == 0 && A.sweeps) {
            int kmax = 0;
            for (int i = 0; i < B; ++i) kmax = max(kmax, s_it[i]);
            A.sweeps[std::is_same<W, float>::value && !RES64 ? 0 : 2] += (unsigned long long)kmax;
        }
    }
}

// The magnet's potential for the field kernel, which reads (U1 + U2 + U2adj)/2:
// U1 = u, U2 = 0 (forward columns), U2adj = u (the operator is symmetric).
template <typename T>
__global__ void k_shell_scatter(ShellDev S, int N, int B, const double* __restrict__ x, T* U1, T* U2) {
    const size_t total = (size_t)N * B;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        const size_t i = t / B;
        const T u = T(x[(size_t)S.magnet[i] * B + b]);
        U1[i * 2 * B + b] = u;
        U2[i * 2 * B + b] = T(0);
        U2[i * 2 * B + B + b] = u;
    }
}

template <typename W, bool RES64, int THREADS, int VEC>
int launch_shell(const Launch& L, const ShellDev& S, const double* bvec, double* shx, double* part, int B,
                 const InstState* st, double tol, int max_iter) {
    const int G = B / VEC, RB = THREADS / G;
    const int nrow = (G <= 32 && (32 % G) == 0) ? (THREADS >> 5) : RB;
    const size_t smem = sizeof(double) * (4 * (size_t)nrow * B + 9 * (size_t)B) + sizeof(int) * 4 * B + sizeof(W) * B;
    const void* fn = (const void*)k_shell_pcg<W, RES64, THREADS, VEC>;
    int occ = 1;
    cudaError_t e = kernel_smem_attr(fn, 160 * 1024, THREADS, smem, &occ);
    if (e != cudaSuccess) return (int)e;
    if (occ < 1) return (int)cudaErrorInvalidConfiguration;
    int nblk = (S.Ng + RB - 1) / RB;
    if (nblk > L.num_sms) nblk = L.num_sms;   // one block per SM (the partials hold one block per SM)
    const size_t Gv = (size_t)S.Ng * B;
    ShellArgs<W> a;
    a.S = S;
    a.B = B;
    a.st = st;
    a.bvec = bvec;
    a.x = shx;
    W* w = reinterpret_cast<W*>(shx + Gv);   // five work vectors after x
    a.r = w;
    a.z = w + Gv;
    a.p = w + 2 * Gv;
    a.q = w + 3 * Gv;
    a.d = w + 4 * Gv;
    a.tol2 = tol * tol;
    a.max_iter = max_iter;
    a.bar = L.bar;
    a.err = L.err;
    a.part = part;
    a.fin = L.fin;
    a.sweeps = L.sweeps;
    void* args[] = {&a};
    e = cudaMemsetAsync(L.bar, 0, sizeof(unsigned), L.stream);
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(fn, dim3(nblk), dim3(THREADS), args, smem, L.stream);
    return (int)e;
}

template <typename W, bool RES64, int THREADS>
int launch_shell_vec(const Launch& L, const ShellDev& S, const double* bvec, double* shx, double* part, int B,
                     const InstState* st, double tol, int max_iter) {
    // the widest vectors the batch allows (FP64 work vectors at most two wide)
    if constexpr (sizeof(W) == 4)
        if (B % 4 == 0) return launch_shell<W, RES64, THREADS, 4>(L, S, bvec, shx, part, B, st, tol, max_iter);
    if (B % 2 == 0) return launch_shell<W, RES64, THREADS, 2>(L, S, bvec, shx, part, B, st, tol, max_iter);
    return launch_shell<W, RES64, THREADS, 1>(L, S, bvec, shx, part, B, st, tol, max_iter);
}

}  // namespace

template <typename T>
int shell_solve(const Launch& L, const MeshView& M, const BatchView<T>& V, double tol, int max_iter, bool mixed_iter) {
    const ShellDev& S = *M.shell;
    const int B = V.B;
    if (B < 1 || B > 512) return (int)cudaErrorInvalidValue;
    int e;
    // FP32 iterations for FP32 batches and for FP64 solves with mixed iterations
    if (sizeof(T) == 4) e = launch_shell_vec<float, false, 512>(L, S, V.bvec, V.shx, V.part, B, V.st, tol, max_iter);
    else if (mixed_iter) e = launch_shell_vec<float, true, 512>(L, S, V.bvec, V.shx, V.part, B, V.st, tol, max_iter);
    else e = launch_shell_vec<double, false, 512>(L, S, V.bvec, V.shx, V.part, B, V.st, tol, max_iter);
    if (e) return e;
    size_t blocks = ((size_t)M.N * B + 255) / 256;
    if (blocks > (size_t)8 * L.num_sms) blocks = (size_t)8 * L.num_sms;
    k_shell_scatter<T><<<(unsigned)blocks, 256, 0, L.stream>>>(S, M.N, B, V.shx, V.U1, V.U2);
    *L.launches += 2;
    return 0;
}

template int shell_solve<float>(const Launch&, const MeshView&, const BatchView<float>&, double, int, bool);
template int shell_solve<double>(const Launch&, const MeshView&, const BatchView<double>&, double, int, bool);

}  // namespace lbm
