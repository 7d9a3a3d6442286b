// Internal declarations shared by the CUDA translation units of liblbm.
//
// Reduced units used on the device (cell edge h, Kd = Js^2/(2 mu0)):
//   lattice coordinates (unit h); integer FEM tables Kint, Gint, Vint with
//   K = (h/6) Kint, G = (h^2/24) Gint, V = (h^3/24) Vint;
//   fields h~ = mu0 H / Js; potential u~ = u / h with Kint u1~ = (1/4) Gint m;
//   energies in Kd h^3; gradient grad_i phi = -(Vint_i/12) h~_i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---- per-block partial quantities of the field kernel (one set per instance) ----
enum {
    Q_EEX = 0, Q_EAN, Q_EZ, Q_ED,      // energy terms (sum)
    Q_TORQUE, Q_HMAX,                  // max |m x h~|, max |H| (max)
    Q_GG, Q_SS, Q_SY, Q_YY,            // sum |g|^2, s.s, s.y, y.y (sum)
    Q_MX, Q_MY, Q_MZ,                  // sum Vint m (sum)
    Q_BAD,                             // non-finite flag (max)
    Q_DE,                              // E(trial) - E(base) by the trapezoid rule (sum)
    Q_COUNT
};
constexpr int NQ = 16;                 // stride of the partials array

enum { PH_INIT = 0, PH_SEARCH = 1, PH_BB = 2, PH_DONE = 3, PH_LB = 4 };   // PH_LB: LaBonte iteration
constexpr int HIST_MAX = 64;
constexpr int MALPHA_MAX = 8;

// Device status bits (context-wide error word).
constexpr int DEV_ERR_TIMEOUT = 1;
constexpr int DEV_ERR_SHAPE = 2;     // a cluster solve launched fewer clusters than active groups

// Four doubles on a 32-byte boundary (general-mesh value tables).
struct __align__(32) Dbl4 {
    double x, y, z, w;
};

struct InstConst {
    double lam;        // A / (Kd h^2): h_ex~ = -4 lam (Kint m)_i / Vint_i
    double Q;          // K1 / Kd:      h_an~ = Q (m.a) a
    double a[3];       // easy axis
    double hz[3];      // mu0 H_ext / Js
    double Eunit;      // Kd h^3 (J)
    double Js;
};

struct StepOpts {
    double tol, grad_tol, c1, kappa0, tau_min, tau_max;
    int max_iter, max_backtracks, memory, m_alpha;
    int bb_rule;     // 0 adaptive, 1 BB1, 2 BB2, 3 BB1/BB2 alternation
    int stall_iters; // give up after this many accepted steps without a new smallest torque (0: never)
    int method;      // 0 curvilinear steepest descent (Sec. 2), 1 LaBonte rotate-to-field
    double omega;    // LaBonte relaxation factor
};

struct InstState {
    int phase, status, cur, iters, evals, line_searches, backtracks, nhist, hpos, ntau2;
    long long cg1, cg2;
    double tau, E_ref, gg_base, E, kappa, torque, gg;
    double Eacc;                   // base energy carried by exact differences (decisions)
    double best_torque;            // smallest torque of the accepted points so far
    int best_iter;                 // the iteration where it was reached
    int warm;                      // 1: the first evaluation resumes the step state (tau, kappa,
                                   // tau^2 memory) of a previous phase instead of a line search
    int next_phase;                // after a stop by the iteration limit or a stall: the phase the
                                   // iteration would have continued in (lbm_solve_opts.resume)
    double terms[4];
    double mean_m[3];
    double hist[HIST_MAX];
    double tau2[MALPHA_MAX];
};

// ---- small device helpers ---------------------------------------------------
__device__ __forceinline__ int sbyte(int w, int k) { return (int)(signed char)((w >> (8 * k)) & 0xff); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Software grid barrier for cooperative launches.  `count` must be zero at
// launch; each block's thread 0 keeps its own epoch.  The wait gives up after
// err[1] milliseconds (2 s when err[1] is 0), or when another block has flagged
// an error, sets DEV_ERR_TIMEOUT and returns false; callers then leave the
// kernel.  err[2] is a test hook: when nonzero every barrier waits for one
// arrival more than the grid makes, so the wait runs out by design (the error
// path is then exercised without any fault).  err points at >= 4 ints.
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned nblocks, unsigned& epoch, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        epoch += 1u;
        const int lim_ms = *(volatile int*)(err + 1);
        const unsigned extra = *(volatile int*)(err + 2) ? 1u : 0u;
        const uint64_t limit = lim_ms > 0 ? (uint64_t)lim_ms * 1000000ull : 2000000000ull;
        const unsigned target = epoch * nblocks + extra;
        // release: the block's writes (ordered before this by the barrier above)
        // become visible to every block whose acquire load sees the increment
        red_release_add(count, 1u);
        int ok = 1;
        const uint64_t t0 = globaltimer_ns();
        unsigned spins = 0;
        while (ld_acquire_u32(count) < target) {
            if ((++spins & 31u) == 0u) {
                if (*(volatile int*)err) { ok = 0; break; }
                if (globaltimer_ns() - t0 > limit) { atomicOr(err, DEV_ERR_TIMEOUT); ok = 0; break; }
            }
        }
        s_ok = ok;   // the acquire loads above order the other blocks' writes before the barrier below
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace lbm
