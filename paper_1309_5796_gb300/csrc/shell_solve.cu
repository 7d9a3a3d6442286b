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
// at once: Jacobi-preconditioned CG in FP64, one persistent cooperative
// kernel per solve (grid barriers with the context's time limit), the grid
// potential warm-started from the instance's previous solve.
#include "solver_common.cuh"

namespace lbm {
namespace {

constexpr int SH_THREADS = 512;

struct ShellArgs {
    ShellDev S;
    int B;
    const InstState* st;
    const double* bvec;                       // [N][B] divergence right-hand side of the magnet
    double *x, *r, *z, *p, *q;                // [Ng][B]
    double tol2;
    int max_iter;
    unsigned* bar;
    int* err;
    double* part;
    double* fin;
    unsigned long long* sweeps;
};

// One instance per column: thread tid works on instance b = tid % B of row
// lane tid / B.  Per iteration (the same fused form as the magnet's solves):
//   A: w = K z, p = z + beta p, q = w + beta q (= K p), partial p.q
//   B: alpha = rho / p.q, x += alpha p, r -= alpha q, z = r / K_ii, partials r.z, r.r
// Outer-face rows are frozen at zero (x, r, z, p, q), so they drop out of
// every product.
__global__ void __launch_bounds__(SH_THREADS, 1) k_shell_pcg(ShellArgs A) {
    extern __shared__ double sm[];
    const int B = A.B, tid = threadIdx.x, bd = blockDim.x;
    const int RB = bd / B;
    const bool lane = tid < RB * B;
    const int b = tid % B, rl = tid / B;
    const int nrow = (B <= 32 && (32 % B) == 0) ? (bd >> 5) : RB;
    double* scratch = sm;                          // [4][nrow][B]
    double* out = scratch + 4 * (size_t)nrow * B;  // [4][B]
    double* s_rho = out + 4 * B;
    double* s_rhop = s_rho + B;
    double* s_ab = s_rhop + B;
    double* s_tol = s_ab + B;
    int* s_flag = (int*)(s_tol + B);
    int* s_act = s_flag + B;
    int* s_it = s_act + B;
    for (int i = tid; i < B; i += bd) {
        s_act[i] = A.st[i].phase != PH_DONE;
        s_it[i] = 0;
        s_rhop[i] = 1.0;
    }
    __syncthreads();
    const bool act = lane && s_act[b];
    const int Ng = A.S.Ng;
    const int row0 = blockIdx.x * RB + rl, rstride = gridDim.x * RB;
    unsigned epoch = 0;
    unsigned red = 0;
    auto reduce = [&](double (&v)[4][1], int nq) -> bool {
        (void)nq;
        block_reduce_cols<4, 1, double>(v, scratch, out, B, B, RB);
        double* pr = A.part + (size_t)(red & 1u) * gridDim.x * B * 4;
        red += 1;
        if (tid < B)
            for (int k = 0; k < 4; ++k) pr[((size_t)blockIdx.x * B + tid) * 4 + k] = out[k * B + tid];
        return grid_reduce<4>(pr, 0, B, A.fin, out, A.bar, epoch, A.err);
    };
    // residual of the warm start, r = f - K x
    {
        double v[4][1] = {{0.0}, {0.0}, {0.0}, {0.0}};   // r.z, r.r, f.f, -
        if (lane)
            for (int row = row0; row < Ng; row += rstride) {
                const size_t i = (size_t)row * B + b;
                const int gn = A.S.gnode[row];
                if (gn == -2) {   // outer face: u = 0
                    A.r[i] = A.z[i] = A.p[i] = A.q[i] = 0.0;
                    continue;
                }
                const double f = (gn >= 0 && act) ? A.bvec[(size_t)gn * B + b] : 0.0;
                double kx = 0.0;
                for (int e = A.S.rowptr[row]; e < A.S.rowptr[row + 1]; ++e)
                    kx += A.S.val[e] * __ldcg(&A.x[(size_t)A.S.col[e] * B + b]);
                const double rv = f - kx, zv = rv * A.S.dinv[row];
                A.r[i] = rv;
                A.z[i] = zv;
                A.p[i] = 0.0;
                A.q[i] = 0.0;
                if (act) {
                    v[0][0] += rv * zv;
                    v[1][0] += rv * rv;
                    v[2][0] += f * f;
                }
            }
        if (!reduce(v, 3)) return;
    }
    if (tid < B) s_tol[tid] = A.tol2 * out[2 * B + tid];
    __syncthreads();
    for (int it = 0;; ++it) {
        if (tid < B) {
            const double rho = out[tid], rr = out[B + tid];
            const int conv = !s_act[tid] || rr <= s_tol[tid] || it >= A.max_iter;
            s_ab[tid] = (it == 0 || conv) ? 0.0 : rho / s_rhop[tid];
            s_rho[tid] = rho;
            s_flag[tid] = conv;
        }
        if (__syncthreads_and(tid < B ? s_flag[tid] : 1)) break;
        const bool run = act && !s_flag[b];
        const double beta = s_ab[b];
        double v[4][1] = {{0.0}, {0.0}, {0.0}, {0.0}};
        if (lane)
            for (int row = row0; row < Ng; row += rstride) {
                if (A.S.gnode[row] == -2) continue;
                const size_t i = (size_t)row * B + b;
                double w = 0.0;
                for (int e = A.S.rowptr[row]; e < A.S.rowptr[row + 1]; ++e)
                    w += A.S.val[e] * __ldcg(&A.z[(size_t)A.S.col[e] * B + b]);
                const double pv = A.z[i] + beta * A.p[i];
                const double qv = w + beta * A.q[i];
                A.p[i] = pv;
                A.q[i] = qv;
                if (run) v[0][0] += pv * qv;
            }
        if (!reduce(v, 1)) return;
        if (tid < B) s_ab[tid] = s_flag[tid] ? 0.0 : s_rho[tid] / out[tid];
        __syncthreads();
        const double alpha = s_ab[b];
        double u[4][1] = {{0.0}, {0.0}, {0.0}, {0.0}};
        if (lane)
            for (int row = row0; row < Ng; row += rstride) {
                if (A.S.gnode[row] == -2) continue;
                const size_t i = (size_t)row * B + b;
                A.x[i] += alpha * A.p[i];
                const double rv = A.r[i] - alpha * A.q[i];
                const double zv = rv * A.S.dinv[row];
                A.r[i] = rv;
                A.z[i] = zv;
                if (run) {
                    u[0][0] += rv * zv;
                    u[1][0] += rv * rv;
                }
            }
        if (!reduce(u, 2)) return;
        if (tid < B) {
            s_rhop[tid] = s_rho[tid];
            if (!s_flag[tid]) s_it[tid] += 1;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int i = tid; i < B; i += bd)
            atomicAdd((unsigned long long*)&((InstState*)A.st)[i].cg1, (unsigned long long)s_it[i]);
        if (tid == 0 && A.sweeps) {
            int kmax = 0;
            for (int i = 0; i < B; ++i) kmax = max(kmax, s_it[i]);
            A.sweeps[2] += (unsigned long long)kmax;
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

}  // namespace

template <typename T>
int shell_solve(const Launch& L, const MeshView& M, const BatchView<T>& V, double tol, int max_iter) {
    const ShellDev& S = *M.shell;
    const int B = V.B;
    if (B > SH_THREADS) return (int)cudaErrorInvalidValue;
    const int RB = SH_THREADS / B;
    const int nrow = (B <= 32 && (32 % B) == 0) ? (SH_THREADS >> 5) : RB;
    const size_t smem = sizeof(double) * (4 * (size_t)nrow * B + 8 * (size_t)B) + sizeof(int) * 3 * B;
    int occ = 1;
    cudaError_t e = kernel_smem_attr((const void*)k_shell_pcg, 64 * 1024, SH_THREADS, smem, &occ);
    if (e != cudaSuccess) return (int)e;
    int nblk = (S.Ng + RB - 1) / RB;
    if (nblk > L.num_sms) nblk = L.num_sms;   // one block per SM (the partials hold one block per SM)
    ShellArgs a;
    a.S = S;
    a.B = B;
    a.st = V.st;
    a.bvec = V.bvec;
    a.x = V.shx;
    a.r = V.shx + (size_t)S.Ng * B;
    a.z = V.shx + 2 * (size_t)S.Ng * B;
    a.p = V.shx + 3 * (size_t)S.Ng * B;
    a.q = V.shx + 4 * (size_t)S.Ng * B;
    a.tol2 = tol * tol;
    a.max_iter = max_iter;
    a.bar = L.bar;
    a.err = L.err;
    a.part = V.part;
    a.fin = L.fin;
    a.sweeps = L.sweeps;
    void* args[] = {&a};
    e = cudaMemsetAsync(L.bar, 0, sizeof(unsigned), L.stream);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((void*)k_shell_pcg, dim3(nblk), dim3(SH_THREADS), args, smem, L.stream);
    if (e != cudaSuccess) return (int)e;
    size_t blocks = ((size_t)M.N * B + 255) / 256;
    if (blocks > (size_t)8 * L.num_sms) blocks = (size_t)8 * L.num_sms;
    k_shell_scatter<T><<<(unsigned)blocks, 256, 0, L.stream>>>(S, M.N, B, V.shx, V.U1, V.U2);
    *L.launches += 2;
    return 0;
}

template int shell_solve<float>(const Launch&, const MeshView&, const BatchView<float>&, double, int);
template int shell_solve<double>(const Launch&, const MeshView&, const BatchView<double>&, double, int);

}  // namespace lbm
