// Batched BEM products on the 5th-generation tensor cores (tcgen05, kind::tf32,
// "3xTF32": A_hi X_hi + A_hi X_lo + A_lo X_hi with FP32 accumulation in TMEM).
//
// The same-mesh batch turns u2_S = B u1_S (forward chain) and c_S = B^T t_S
// (adjoint chain) of the hybrid FEM/BEM open boundary (Sec. 3.1) into two dense
// GEMMs with the batch as the N dimension.  Both are computed as
//     Y[m][n] = sum_k A[m][k] X[n][k]        (A = B or B^T, both K-major)
// from padded FP32 copies of B and B^T and a transposed, hi/lo-split copy of the
// surface vectors.  One CTA computes a 128 x 64 tile over a K range (split-K,
// partials summed in a fixed order by a second kernel).
//
// Warp roles (192 threads): warp 0 issues TMA loads (one elected lane), warp 1
// owns the TMEM accumulator and issues the MMAs (one elected lane), warps 2-5
// split each A tile into its TF32 head (bits kept in place) and tail (A - head)
// in shared memory, and finally read the accumulator back (each warp its lane
// quadrant).  Every wait on an mbarrier gives up after one second, sets the
// context's error word and leaves the CTA through the common exit that frees
// the TMEM columns.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cuda.h>
#include <stdint.h>

#include "lbm_host.h"

namespace lbm {

namespace tc {

constexpr int BM = 128, BN = 64, BK = 32, STAGES = 4, THREADS = 192;
constexpr int A_BYTES = BM * BK * 4;   // 16 KB
constexpr int X_BYTES = BN * BK * 4;   // 8 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * X_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 64;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Wait for the phase with the given parity; false after 1 s (error word set).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t spin = 0;; ++spin) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((spin & 63u) == 63u) {
            if (*(volatile int*)err) return false;
            if (globaltimer_ns() - t0 > 1000000000ull) {
                atomicOr(err, DEV_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile written by TMA with 128-byte
// swizzling (rows of 128 B, 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t sw128_desc(const void* tile) {
    const uint32_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);    // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Ypart[split][m][n] = sum_{k in split} A[m][k] X[xrow0 + n][k],  m < nb, n < ncols
__global__ void __launch_bounds__(THREADS, 1)
    k_bem_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapXhi,
             const __grid_constant__ CUtensorMap mapXlo, int xrow0, int nb, int ncols, int kblocks_per_split,
             float* __restrict__ Ypart, int* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* full = bars;                 // [STAGES] TMA landed
    uint64_t* conv = bars + STAGES;        // [STAGES] tail split written
    uint64_t* empty = bars + 2 * STAGES;   // [STAGES] MMAs of the stage done
    uint64_t* done = bars + 3 * STAGES;    // accumulator complete
    uint32_t* s_taddr = (uint32_t*)(bars + 3 * STAGES + 1);
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM;
    const int kb0 = blockIdx.y * kblocks_per_split;
    const int nkb_total = (nb + BK - 1) / BK;
    const int nkb = max(0, min(kblocks_per_split, nkb_total - kb0));

    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 128);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_taddr)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_taddr;

    if (nkb > 0) {
        if (warp == 0 && lane == 0) {
            // ---- producer: TMA loads of A, X_hi, X_lo per stage -----------------
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES;
                if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1, err)) { s_fail = 1; break; }
                uint8_t* st = smem + s * STAGE_BYTES;
                mbar_expect_tx(&full[s], A_BYTES + 2 * X_BYTES);
                const int k = (kb0 + kb) * BK;
                tma_load_2d(st, &mapA, &full[s], k, m0);
                tma_load_2d(st + 2 * A_BYTES, &mapXhi, &full[s], k, xrow0);
                tma_load_2d(st + 2 * A_BYTES + X_BYTES, &mapXlo, &full[s], k, xrow0);
            }
        } else if (warp == 1 && lane == 0) {
            // ---- MMA issuer ----------------------------------------------------------
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES;
                if (!mbar_wait(&conv[s], (kb / STAGES) & 1, err)) { s_fail = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint8_t* st = smem + s * STAGE_BYTES;
                const uint64_t dAh = sw128_desc(st), dAl = sw128_desc(st + A_BYTES);
                const uint64_t dXh = sw128_desc(st + 2 * A_BYTES), dXl = sw128_desc(st + 2 * A_BYTES + X_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    const uint64_t o = (uint64_t)(kk * 32) >> 4;   // 8 TF32 = 32 B along K
                    mma_tf32(tmem, dAh + o, dXh + o, (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_tf32(tmem, dAh + o, dXl + o, 1u);
                    mma_tf32(tmem, dAl + o, dXh + o, 1u);
                }
                mma_commit(&empty[s]);
            }
            mma_commit(done);
        } else if (warp >= 2) {
            // ---- converters: A -> TF32 head (in place) + tail (A - head) --------------
            const int ct = tid - 64;   // 0..127
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES;
                if (!mbar_wait(&full[s], (kb / STAGES) & 1, err)) { s_fail = 1; break; }
                float4* a = (float4*)(smem + s * STAGE_BYTES);
                float4* t = (float4*)(smem + s * STAGE_BYTES + A_BYTES);
#pragma unroll
                for (int i = 0; i < A_BYTES / 16 / 128; ++i) {
                    float4 v = a[ct + 128 * i];
                    float4 h, l;
                    h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
                    h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
                    h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
                    h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
                    l.x = v.x - h.x;
                    l.y = v.y - h.y;
                    l.z = v.z - h.z;
                    l.w = v.w - h.w;
                    a[ct + 128 * i] = h;
                    t[ct + 128 * i] = l;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&conv[s]);
            }
            // ---- epilogue: accumulator rows of this warp's lane quadrant -----------------
            if (!s_fail && mbar_wait(done, 0, err)) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int quad = warp & 3;
                const int m = m0 + quad * 32 + lane;
                float* yrow = Ypart + ((size_t)blockIdx.y * nb + (m < nb ? m : 0)) * BN;
#pragma unroll
                for (int half = 0; half < BN / 32; ++half) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 32), v);
                    if (m < nb)
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (half * 32 + j < ncols) yrow[half * 32 + j] = v[j];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Y[m * ldy + n] = sum_s Ypart[s][m][n] (fixed order)
template <typename T>
__global__ void k_tc_sum(const float* __restrict__ Ypart, int splits, int nb, int ncols, T* __restrict__ Y, int ldy) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * ncols) return;
    const int m = t / ncols, n = t % ncols;
    float acc = 0.f;
    for (int s = 0; s < splits; ++s) acc += Ypart[((size_t)s * nb + m) * BN + n];
    Y[(size_t)m * ldy + n] = T(acc);
}

// XT_hi / XT_lo [2B][ldp]: the surface vectors, transposed (column c of the
// [nb][2B] array becomes row c) and split into TF32 head and tail.
template <typename T>
__global__ void k_tc_split(const T* __restrict__ X, int nb, int C, int ldp, float* __restrict__ hi,
                           float* __restrict__ lo) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * C) return;
    const int k = t / C, c = t % C;
    const float v = (float)X[t];
    const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    hi[(size_t)c * ldp + k] = h;
    lo[(size_t)c * ldp + k] = v - h;
}

}  // namespace tc

// ---- host side --------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The tensor-map encoder is a driver-API function; it is looked up through the
// runtime so that the library itself does not link against libcuda.
static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

static int make_map(CUtensorMap* map, const float* base, int inner, int outer, int ld, int box_inner, int box_outer) {
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    const cuuint32_t estr[2] = {1, 1};
    EncodeTiledFn enc = encode_fn();
    if (!enc) return -3;
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}

int tc_ld(int nb) { return (nb + 31) & ~31; }

constexpr int TC_MAX_SPLITS = 8;   // largest split-K count the autotuner tries

size_t tc_scratch_floats(int nb, int B, int num_sms) {
    (void)num_sms;
    const int ldp = tc_ld(nb);
    return (size_t)2 * (2 * B) * ldp + (size_t)TC_MAX_SPLITS * nb * tc::BN + 64;
}

// ---- autotuner: split-K count of the tensor-core product ----------------------------
// At the first product of a (nb, B, SM count) the kernel is timed with every
// candidate split count (K blocks per split rounded so that every split has
// work) on the operands in scratch, with CUDA events on the launching stream;
// the fastest is kept for the process.  Only scratch is written while tuning.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tc_splits;

int splits_for(int nkb, int want, int* kps_out) {
    int splits = want < 1 ? 1 : (want > nkb ? nkb : want);
    const int kps = (nkb + splits - 1) / splits;
    *kps_out = kps;
    return (nkb + kps - 1) / kps;   // every split has at least one K block
}
}  // namespace

static int tc_tuned_splits(const Launch& L, const CUtensorMap& mA, const CUtensorMap& mXh, const CUtensorMap& mXl,
                           int nb, int B, float* ypart) {
    const auto key = std::make_tuple(nb, B, L.num_sms);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tc_splits.find(key);
        if (it != g_tc_splits.end()) return it->second;
    }
    const int mt = (nb + tc::BM - 1) / tc::BM, nkb = (nb + tc::BK - 1) / tc::BK;
    if (!L.tune) return (L.num_sms + mt - 1) / mt;
    int best = 0;
    float best_ms = 0.f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int want = 1; want <= TC_MAX_SPLITS; ++want) {
        int kps;
        const int splits = splits_for(nkb, want, &kps);
        if (splits != want) continue;
        float t[3];
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, L.stream);
            tc::k_bem_tc<<<dim3(mt, splits), tc::THREADS, tc::SMEM_BYTES, L.stream>>>(mA, mXh, mXl, 0, nb, B, kps,
                                                                                      ypart, L.err);
            cudaEventRecord(e1, L.stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&t[rep], e0, e1);
            *L.launches += 1;
        }
        const float med = std::max(std::min(t[0], t[1]), std::min(std::max(t[0], t[1]), t[2]));
        if (best == 0 || med < best_ms) {
            best = splits;
            best_ms = med;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best == 0) best = 1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tc_splits[key] = best;
    return best;
}

int tc_splits_chosen(int nb, int B, int num_sms) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tc_splits.find(std::make_tuple(nb, B, num_sms));
    return it == g_tc_splits.end() ? 0 : it->second;
}

// Both BEM products of the batch on the tensor cores.  A32 / A32T: padded FP32
// copies of B and B^T (ld = tc_ld(nb)); scratch: tc_scratch_floats(...) floats.
template <typename T>
int bem_product_tc(const Launch& L, int nb, const float* A32, const float* A32T, const T* ub_in, T* ub_out, int B,
                   float* scratch) {
    if (B > tc::BN) return -1;
    const int C = 2 * B, ldp = tc_ld(nb);
    float* xhi = scratch;
    float* xlo = scratch + (size_t)C * ldp;
    float* ypart = scratch + (size_t)2 * C * ldp;
    if (kernel_smem_attr((const void*)tc::k_bem_tc, tc::SMEM_BYTES) != cudaSuccess) return -3;
    const int total = nb * C;
    tc::k_tc_split<T><<<(total + 255) / 256, 256, 0, L.stream>>>(ub_in, nb, C, ldp, xhi, xlo);
    const int mt = (nb + tc::BM - 1) / tc::BM, nkb = (nb + tc::BK - 1) / tc::BK;
    CUtensorMap mA, mAT, mXh, mXl;
    int e = make_map(&mA, A32, nb, nb, ldp, tc::BK, tc::BM);
    if (!e) e = make_map(&mAT, A32T, nb, nb, ldp, tc::BK, tc::BM);
    if (!e) e = make_map(&mXh, xhi, nb, C, ldp, tc::BK, tc::BN);
    if (!e) e = make_map(&mXl, xlo, nb, C, ldp, tc::BK, tc::BN);
    if (e) return e;
    int kps;
    const int splits = splits_for(nkb, tc_tuned_splits(L, mA, mXh, mXl, nb, B, ypart), &kps);
    const dim3 grid(mt, splits);
    // forward: rows 0..B-1 of X; adjoint: rows B..2B-1 with B^T
    tc::k_bem_tc<<<grid, tc::THREADS, tc::SMEM_BYTES, L.stream>>>(mA, mXh, mXl, 0, nb, B, kps, ypart, L.err);
    tc::k_tc_sum<T><<<(nb * B + 255) / 256, 256, 0, L.stream>>>(ypart, splits, nb, B, ub_out, C);
    tc::k_bem_tc<<<grid, tc::THREADS, tc::SMEM_BYTES, L.stream>>>(mAT, mXh, mXl, B, nb, B, kps, ypart, L.err);
    tc::k_tc_sum<T><<<(nb * B + 255) / 256, 256, 0, L.stream>>>(ypart, splits, nb, B, ub_out + B, C);
    *L.launches += 5;
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// padded FP32 copies of B and B^T for the tensor-core path
__global__ void k_tc_pad(const float* __restrict__ B32, int nb, int ldp, float* __restrict__ A, float* __restrict__ AT) {
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)nb * nb) return;
    const int i = (int)(t / nb), j = (int)(t % nb);
    const float v = B32[t];
    A[(size_t)i * ldp + j] = v;
    AT[(size_t)j * ldp + i] = v;
}

void tc_prepare(const Launch& L, const float* B32, int nb, float* A, float* AT) {
    const int ldp = tc_ld(nb);
    cudaMemsetAsync(A, 0, sizeof(float) * (size_t)nb * ldp, L.stream);
    cudaMemsetAsync(AT, 0, sizeof(float) * (size_t)nb * ldp, L.stream);
    const size_t total = (size_t)nb * nb;
    k_tc_pad<<<(unsigned)((total + 255) / 256), 256, 0, L.stream>>>(B32, nb, ldp, A, AT);
    *L.launches += 1;
}

template int bem_product_tc<float>(const Launch&, int, const float*, const float*, const float*, float*, int, float*);
template int bem_product_tc<double>(const Launch&, int, const float*, const float*, const double*, double*, int,
                                    float*);

}  // namespace lbm
