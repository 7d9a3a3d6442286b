// C ABI of liblbm: contexts, meshes, instance batches, and the host loop that
// drives the device-resident minimiser (Sec. 2.2-2.3) and the hysteresis
// continuation (Sec. 1.1, 3.1).  Every decision of the iteration (step length,
// acceptance, line search, stop test) is taken on the device; the host only
// enqueues kernels and polls the instance phases every `check_every` steps.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <array>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_host.h"

using namespace lbm;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_E_OOM : LBM_E_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

constexpr double MU0 = 4e-7 * 3.14159265358979323846;
// The FP64 phase of a mixed run stops at this fraction of the requested torque
constexpr double POLISH_MARGIN = 0.9;

// No C++ exception crosses the C interface: every entry point runs inside
// LBM_TRY / LBM_CATCH, which turn host allocation failures into LBM_E_OOM and
// anything else (e.g. a thread that cannot be started) into LBM_E_INVALID.
#define LBM_TRY try {
#define LBM_CATCH                                                                    \
    }                                                                                \
    catch (const std::bad_alloc&) {                                                  \
        return fail(LBM_E_OOM, "host memory allocation failed");                     \
    }                                                                                \
    catch (const std::exception& ex_) {                                              \
        return fail(LBM_E_INVALID, "%s", ex_.what());                                \
    }                                                                                \
    catch (...) {                                                                    \
        return fail(LBM_E_INVALID, "unexpected error");                              \
    }

struct Mesh {
    int n = 0, N = 0, nb = 0, nnz = 0, F = 0, T = 0;
    int num_sms = 0;                         // of the context's device (sizes split-K scratch)
    double cell = 0;
    int *rowptr = nullptr, *col = nullptr, *pkA = nullptr, *pkB = nullptr, *node = nullptr, *bidx = nullptr;
    int *tris = nullptr, *inc_ptr = nullptr, *inc_slot = nullptr;
    int *kptr = nullptr, *kent = nullptr;
    int nnzK = 0;
    double* B64 = nullptr;
    float* B32 = nullptr;
    float* B32lo = nullptr;                   // fp32(B64 - B32) for FP64 batches of >1 instance (lazy)
    HMDevice* hm = nullptr;                   // hierarchical form of B (lbm_mesh_hmatrix), or null
    std::vector<void*> hm_mem;                // its device allocations
    ShellDev* shell = nullptr;                // space-transformation boundary (lbm_mesh_shell), or null
    std::vector<void*> shell_mem;             // its device allocations
    float *tcA = nullptr, *tcAT = nullptr;   // padded FP32 B and B^T for the tensor-core path (lazy)
    // general meshes (lbm_mesh_upload; n == 0)
    bool gen = false;
    double vsum = 0.0;
    int* tets = nullptr;                     // T*4 as uploaded (orientation kept)
    double* xyz = nullptr;                   // N*3 in units of L
    Dbl4 *gA64 = nullptr, *gB64 = nullptr;
    float4 *gA32 = nullptr, *gB32 = nullptr;
    double *gk64 = nullptr, *gV = nullptr, *gd64 = nullptr;
    float *gk32 = nullptr, *gd32 = nullptr;
    size_t bytes = 0;
    MeshView view() const {
        MeshView v;
        v.n = n; v.N = N; v.nb = nb; v.nnz = nnz; v.F = F;
        v.rowptr = rowptr; v.col = col; v.pkA = pkA; v.pkB = pkB; v.node = node; v.bidx = bidx;
        v.kptr = kptr; v.kent = kent;
        v.B64 = B64; v.B32 = B32; v.B32lo = B32lo;
        v.hm = hm;
        v.shell = shell;
        v.vsum = gen ? vsum : 24.0 * (double)n * n * n;
        v.cell = cell;
        v.gen = gen ? 1 : 0;
        v.gA64 = gA64; v.gA32 = gA32; v.gB64 = gB64; v.gB32 = gB32;
        v.gk64 = gk64; v.gk32 = gk32; v.gV = gV; v.gd64 = gd64; v.gd32 = gd32;
        return v;
    }
};

// One captured chunk of iterations of a batch (check_every calls of the trial
// update, field evaluation and step decision), replayed as a CUDA graph.  Valid
// for the batch, options and mesh operators it was captured with (`key`).
struct ChunkGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<char> key;
    int64_t launches = 0;                                  // kernel launches per replay
    bool failed = false;                                   // capture not possible for `key`
    std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> prof;   // profiling event nodes
    void clear() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        for (auto& e : prof) {
            cudaEventDestroy(std::get<1>(e));
            cudaEventDestroy(std::get<2>(e));
        }
        prof.clear();
        key.clear();
        launches = 0;
        failed = false;
    }
};

struct Inst {
    int64_t mesh = 0;
    int B = 0, precision = 0, tsize = 8;
    void* vec = nullptr;           // all T-typed vectors in one allocation
    double* part = nullptr;
    InstState* st = nullptr;
    InstConst* ic = nullptr;
    double* staged = nullptr;      // B*N*3 doubles (host <-> device layout conversion)
    double* staged_u = nullptr;    // B*2*N doubles
    Inst* polish = nullptr;        // FP64 shadow batch finishing mixed-precision runs
    bool use_tc = false;           // BEM products on the tensor cores (LBM_MIXED_TC, 2 <= batch <= 64)
    float* tc_scratch = nullptr;
    bool owns_tc_scratch = true;
    std::vector<lbm_material> mats;
    std::vector<double> h;         // B*3 tesla
    size_t bytes = 0;
    ChunkGraph graph;              // the batch's captured chunk of iterations
};

}  // namespace

struct ProfEvent {
    int kind;
    cudaEvent_t a, b;
};

namespace { struct Server; }

struct lbm_ctx {
    Server* server = nullptr;
    int device = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<ProfEvent> ev_live;
    int64_t prof_launches[LBM_PROF_KINDS] = {0};
    double prof_ms[LBM_PROF_KINDS] = {0};
    int64_t prof_cg[2] = {0, 0};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    unsigned* bar = nullptr;
    int* err = nullptr;
    int64_t launches = 0;
    int64_t next_id = 1;
    std::map<int64_t, Mesh*> meshes;
    std::map<int64_t, Inst*> insts;
    unsigned long long* sweeps = nullptr;   // device [4]
    double* fin = nullptr;                  // device [4096] grid-reduction results
    cudaStream_t cap_stream = nullptr;      // where chunks are captured (lazy)
    ChunkGraph* capturing = nullptr;        // the chunk being captured (profiling events become nodes)
    int64_t graph_stats[3] = {0, 0, 0};     // replays, captures, captures refused
    Launch launch() { return Launch{stream, num_sms, bar, err, &launches, sweeps, fin, 0}; }
};

namespace {

cudaEvent_t pool_get(lbm_ctx* ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Brackets one launch of `kind` with events on the launching stream (the
// context's stream; launches on other streams are not profiled).
struct ProfScope {
    lbm_ctx* ctx;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(lbm_ctx* c, int k, cudaStream_t s) : ctx(c), kind(k), st(s) {
        if (ctx->prof && ctx->capturing && st == ctx->cap_stream) {
            // captured: an event-record node of the graph, timed after each replay
            cudaEventCreate(&a);
            cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
        } else if (ctx->prof && st == ctx->stream) {
            a = pool_get(ctx);
            cudaEventRecord(a, st);
        }
    }
    ~ProfScope() {
        if (!a) return;
        if (ctx->prof && ctx->capturing && st == ctx->cap_stream) {
            cudaEvent_t b;
            cudaEventCreate(&b);
            cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
            ctx->capturing->prof.emplace_back(kind, a, b);
        } else {
            cudaEvent_t b = pool_get(ctx);
            cudaEventRecord(b, st);
            ctx->ev_live.push_back(ProfEvent{kind, a, b});
        }
    }
};

// After a replay of a captured chunk and a synchronisation: its event nodes' times.
void prof_harvest_graph(lbm_ctx* ctx, const ChunkGraph& g) {
    for (const auto& e : g.prof) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, std::get<1>(e), std::get<2>(e)) == cudaSuccess) {
            ctx->prof_ms[std::get<0>(e)] += ms;
            ctx->prof_launches[std::get<0>(e)] += 1;
        }
    }
}

// After a stream synchronisation: fold the recorded event pairs into the totals.
void prof_harvest(lbm_ctx* ctx) {
    for (const ProfEvent& e : ctx->ev_live) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
            ctx->prof_ms[e.kind] += ms;
            ctx->prof_launches[e.kind] += 1;
        }
        ctx->ev_pool.push_back(e.a);
        ctx->ev_pool.push_back(e.b);
    }
    ctx->ev_live.clear();
}

// Byte offsets of the per-instance arrays inside one allocation; every array
// starts on a 256-byte boundary (the PCG reads 8- and 16-byte vectors).
struct VecLayout {
    size_t m, g, hout, U1, U2, r, z, p, q, ub_in, ub_out, bem_part, m32, bvec, shx, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

VecLayout vec_layout(const Mesh& M, int B, int tsize) {
    const size_t N = M.N, nb = M.nb, C = 2 * (size_t)B;
    VecLayout L;
    size_t o = 0;
    auto take = [&o](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
    L.m = take(8 * 2 * N * 3 * B);
    L.g = take(8 * 2 * N * 3 * B);
    L.hout = take(8 * N * 3 * B);
    L.U1 = take(tsize * N * C);
    L.U2 = take(tsize * N * C);
    L.r = take(tsize * N * C);
    L.z = take(tsize * N * C);
    L.p = take(tsize * N * C);
    L.q = take(tsize * N * C);
    L.ub_in = take(tsize * nb * C);
    L.ub_out = take(tsize * nb * C);
    // 32 x nb partial sums of the transposed single-instance product; FP64
    // batches also the K-split partials of the batched product (S x nb x 2B)
    const size_t df = (tsize == 8 && B > 1) ? (size_t)bem_df_splits((int)nb, B, M.num_sms) * nb * C : 0;
    L.bem_part = take(8 * (32 * nb > df ? 32 * nb : df));
    L.m32 = tsize == 4 ? take(4 * N * 3 * B) : 0;
    L.bvec = take(8 * N * B);
    // space-transformation boundary: grid potential and CG vectors, FP64 in every mode
    L.shx = M.shell ? take(8 * 6 * (size_t)M.shell->Ng * B) : 0;
    L.total = o;
    return L;
}

template <typename T>
BatchView<T> batch_view(const lbm_ctx* ctx, const Mesh& M, const Inst& I, bool with_hout) {
    (void)ctx;
    const VecLayout L = vec_layout(M, I.B, sizeof(T));
    char* base = (char*)I.vec;
    BatchView<T> v;
    v.B = I.B;
    v.m = (double*)(base + L.m);
    v.H = (double*)(base + L.g);
    v.hout = with_hout ? (double*)(base + L.hout) : nullptr;
    v.U1 = (T*)(base + L.U1);
    v.U2 = (T*)(base + L.U2);
    v.r = (T*)(base + L.r);
    v.z = (T*)(base + L.z);
    v.p = (T*)(base + L.p);
    v.q = (T*)(base + L.q);
    v.ub_in = (T*)(base + L.ub_in);
    v.ub_out = (T*)(base + L.ub_out);
    v.bem_part = (T*)(base + L.bem_part);
    v.m32 = sizeof(T) == 4 ? (float*)(base + L.m32) : nullptr;
    v.bvec = (double*)(base + L.bvec);
    v.shx = M.shell ? (double*)(base + L.shx) : nullptr;
    v.part = I.part;
    v.st = I.st;
    v.ic = I.ic;
    return v;
}

size_t vec_bytes(const Mesh& M, int B, int tsize) { return vec_layout(M, B, tsize).total; }

// A new magnetisation starts its potential solves from zero (not from the
// previous solve's potentials), so that a solve depends only on its inputs.
int zero_potentials(lbm_ctx* ctx, const Mesh& M, const Inst& I) {
    const VecLayout L = vec_layout(M, I.B, I.tsize);
    const size_t bytes = (size_t)I.tsize * M.N * 2 * I.B;
    CK(cudaMemsetAsync((char*)I.vec + L.U1, 0, bytes, ctx->stream));
    CK(cudaMemsetAsync((char*)I.vec + L.U2, 0, bytes, ctx->stream));
    if (M.shell) CK(cudaMemsetAsync((char*)I.vec + L.shx, 0, sizeof(double) * M.shell->Ng * I.B, ctx->stream));
    return LBM_OK;
}

size_t part_elems(const lbm_ctx* ctx, int B) {
    const size_t a = (size_t)4 * ctx->num_sms * B * NQ;   // field kernel partials
    const size_t b = pcg_part_elems(ctx->num_sms, B);          // PCG (two regions, 2B systems)
    return a > b ? a : b;
}

Mesh* get_mesh(lbm_ctx* ctx, lbm_mesh h) {
    auto it = ctx->meshes.find(h);
    return it == ctx->meshes.end() ? nullptr : it->second;
}
Inst* get_inst(lbm_ctx* ctx, lbm_inst h) {
    auto it = ctx->insts.find(h);
    return it == ctx->insts.end() ? nullptr : it->second;
}

void free_hm(Mesh* m) {
    for (void* p : m->hm_mem) cudaFree(p);
    m->hm_mem.clear();
    if (m->hm && m->hm->t) cudaFree(m->hm->t);
    delete m->hm;
    m->hm = nullptr;
}

// The first-pass scratch of the hierarchical products for batches of B instances.
int hm_reserve(lbm_ctx* ctx, Mesh* M, int B) {
    if (!M->hm) return LBM_OK;
    const size_t need = sizeof(double) * 2 * (size_t)(M->hm->fwd.n_t > 0 ? M->hm->fwd.n_t : 1) * B;
    if (M->hm->t_bytes >= need) return LBM_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    if (M->hm->t) cudaFree(M->hm->t);
    M->hm->t = nullptr;
    M->hm->t_bytes = 0;
    CK(cudaMalloc(&M->hm->t, need));
    M->hm->t_bytes = need;
    return LBM_OK;
}

void free_shell(Mesh* m) {
    for (void* p : m->shell_mem) cudaFree(p);
    m->shell_mem.clear();
    delete m->shell;
    m->shell = nullptr;
}

void free_mesh(Mesh* m) {
    free_hm(m);
    free_shell(m);
    void* ptrs[] = {m->rowptr, m->col, m->pkA, m->pkB, m->node, m->bidx, m->tris, m->inc_ptr, m->inc_slot,
                    m->kptr, m->kent, m->B64, m->B32, m->B32lo, m->tcA, m->tcAT, m->tets, m->xyz, m->gA64, m->gB64,
                    m->gA32, m->gB32, m->gk64, m->gV, m->gd64, m->gk32, m->gd32};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

void free_inst(Inst* I) {
    I->graph.clear();
    if (I->polish) free_inst(I->polish);
    if (I->tc_scratch && I->owns_tc_scratch) cudaFree(I->tc_scratch);
    void* ptrs[] = {I->vec, I->part, I->st, I->ic, I->staged, I->staged_u};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete I;
}

int upload_consts(lbm_ctx* ctx, Inst* I, const Mesh& M) {
    std::vector<InstConst> ic(I->B);
    const double h = M.cell;
    for (int b = 0; b < I->B; ++b) {
        const lbm_material& mt = I->mats[b];
        const double Kd = mt.Js * mt.Js / (2.0 * MU0);
        double an = sqrt(mt.axis[0] * mt.axis[0] + mt.axis[1] * mt.axis[1] + mt.axis[2] * mt.axis[2]);
        if (!(an > 0)) an = 1.0;
        InstConst& c = ic[b];
        c.lam = mt.A / (Kd * h * h);
        c.Q = mt.K1 / Kd;
        for (int d = 0; d < 3; ++d) {
            c.a[d] = mt.axis[d] / an;
            c.hz[d] = I->h[3 * b + d] / mt.Js;
        }
        c.Eunit = Kd * h * h * h;
        c.Js = mt.Js;
    }
    CK(cudaMemcpyAsync(I->ic, ic.data(), sizeof(InstConst) * I->B, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

StepOpts step_opts(const lbm_solve_opts& o) {
    StepOpts s;
    s.tol = o.tol;
    s.grad_tol = o.grad_tol;
    s.c1 = o.c1;
    s.kappa0 = o.kappa0;
    s.tau_min = o.tau_min;
    s.tau_max = o.tau_max;
    s.max_iter = o.max_iter;
    s.max_backtracks = o.max_backtracks;
    s.memory = o.memory;
    s.m_alpha = o.m_alpha;
    s.bb_rule = o.bb_rule;
    s.method = o.method;
    s.omega = o.omega;
    s.stall_iters = o.stall_iters;
    return s;
}

int check_opts(const lbm_solve_opts& o) {
    if (!(o.tol >= 0) || o.max_iter < 0 || o.memory < 1 || o.memory > HIST_MAX || o.m_alpha < 1 ||
        o.m_alpha > MALPHA_MAX || o.max_backtracks < 0 || o.cg_max_iter < 1 || !(o.cg_tol > 0) ||
        o.check_every < 1 || !(o.tau_min > 0) || !(o.tau_max >= o.tau_min) || !(o.switch_tol >= 0) ||
        !(o.cg_tol_polish > 0) || o.bb_rule < 0 || o.bb_rule > 3 || o.method < 0 || o.method > 1 ||
        (o.method == 1 && !(o.omega > 0.0 && o.omega <= 2.0)) || o.stall_iters < 0 || o.pcg_kernel < 0 ||
        o.pcg_kernel > 2 || o.use_graphs < 0 || o.use_graphs > 1 || !(o.cg_tol_fp32 >= 0) || o.resume < 0 ||
        o.resume > 1)
        return fail(LBM_E_INVALID, "invalid solve options");
    return LBM_OK;
}

// One field evaluation of every active instance at its trial point.
template <typename T>
int eval_trial(lbm_ctx* ctx, const Launch& L, const Mesh& M, const Inst& I, const BatchView<T>& V,
               const lbm_solve_opts& o) {
    MeshView mv = M.view();
    if (o.demag && M.shell) {
        // open boundary by space transformation: one symmetric solve on the grid
        ProfScope ps(ctx, 1 + (sizeof(T) == 8 ? 5 : 0), L.stream);
        rhs_eval<T>(L, mv, V);
        const int e = shell_solve<T>(L, mv, V, o.cg_tol, o.cg_max_iter, o.cg_mixed_iter != 0);
        if (e) return fail(LBM_E_CUDA, "cooperative launch failed: %s", cudaGetErrorString((cudaError_t)e));
    } else if (o.demag) {
        int e;
        const int k64 = sizeof(T) == 8 ? 5 : 0;
        {
            ProfScope ps(ctx, 1 + k64, L.stream);
            rhs_eval<T>(L, mv, V);
            e = pcg_solve<T>(L, mv, V, 0, o.cg_tol, o.cg_max_iter, o.cg_mixed_iter != 0);
        }
        if (e) return fail(LBM_E_CUDA, "cooperative launch failed: %s", cudaGetErrorString((cudaError_t)e));
        {
            ProfScope ps(ctx, 2, L.stream);
            if (I.use_tc && M.tcA && I.tc_scratch && !M.hm) {
                e = bem_product_tc<T>(L, M.nb, M.tcA, M.tcAT, V.ub_in, V.ub_out, V.B, I.tc_scratch);
                if (e) return fail(LBM_E_CUDA, "tensor-core BEM product failed (%d)", e);
            } else {
                bem_product<T>(L, mv, V);
            }
        }
        {
            ProfScope ps(ctx, 3 + (k64 ? 4 : 0), L.stream);
            e = pcg_solve<T>(L, mv, V, 1, o.cg_tol, o.cg_max_iter, o.cg_mixed_iter != 0);
        }
        if (e) return fail(LBM_E_CUDA, "cooperative launch failed: %s", cudaGetErrorString((cudaError_t)e));
    }
    {
        ProfScope ps(ctx, 4, L.stream);
        field_eval<T>(L, mv, V, o.demag);
    }
    return LBM_OK;
}

// One iteration of every active instance: trial point (Eq. 8), field
// evaluation at it, step decision (Sec. 2.3).
template <typename T>
int iterate_once(lbm_ctx* ctx, const Launch& L, const Mesh& M, const Inst& I, const BatchView<T>& V,
                 const lbm_solve_opts& o, const StepOpts& so, int nblk_field) {
    const MeshView mv = M.view();
    {
        ProfScope ps(ctx, 0, L.stream);
        trial_update<T>(L, mv, V);
    }
    int e = eval_trial<T>(ctx, L, M, I, V, o);
    if (e) return e;
    ProfScope ps(ctx, 5, L.stream);
    decide<T>(L, mv, V, so, nblk_field);
    return LBM_OK;
}

// `chunk` iterations of a batch: captured once as a CUDA graph (on the
// context's capture stream, or on `cap` when given) and replayed, or launched
// one by one (use_graphs == 0, the first chunk of a run -- it performs any
// one-time set-up: kernel attributes, occupancy queries, autotuning -- or a
// capture that the driver refused).  The graph is valid for the batch, options
// and the mesh's operators it was captured with; *replayed tells the caller
// to read the graph's profiling nodes after its synchronisation.
template <typename T>
int run_chunk(lbm_ctx* ctx, const Launch& L, const Mesh& M, Inst* I, const BatchView<T>& V, const lbm_solve_opts& o,
              const StepOpts& so, int nblk_field, int chunk, bool first, cudaStream_t cap, bool* replayed) {
    *replayed = false;
    ChunkGraph& g = I->graph;
    std::vector<char> key(sizeof(lbm_solve_opts) + 10 * sizeof(int64_t));
    {
        // the launch shape of the cluster potential solves (it follows the active
        // instances; querying it here also caches its occupancy before a capture)
        const int64_t shape = pcg_cluster_shape(L, M.view(), I->B, sizeof(T) == 8, o.cg_mixed_iter != 0);
        const int64_t k[10] = {chunk, (int64_t)sizeof(T), I->B, (int64_t)(intptr_t)M.hm, (int64_t)(intptr_t)M.B32lo,
                               (int64_t)(intptr_t)M.tcA, ctx->prof ? 1 : 0, (int64_t)(intptr_t)V.m,
                               (int64_t)(intptr_t)M.shell, shape};
        memcpy(key.data(), &o, sizeof(lbm_solve_opts));
        memcpy(key.data() + sizeof(lbm_solve_opts), k, sizeof k);
    }
    const bool use = o.use_graphs != 0 && !first && chunk > 1 && !(g.failed && g.key == key);
    if (use && !(g.exec && g.key == key)) {
        g.clear();
        if (!cap) {
            if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            cap = ctx->cap_stream;
        }
        Launch Lc = L;
        Lc.stream = cap;
        const int64_t l0 = ctx->launches;
        ctx->capturing = &g;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int rc = LBM_OK;
        if (e == cudaSuccess)
            for (int k = 0; k < chunk && rc == LBM_OK; ++k) rc = iterate_once<T>(ctx, Lc, M, *I, V, o, so, nblk_field);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cap, &graph) : e;
        ctx->capturing = nullptr;
        const int64_t per = ctx->launches - l0;
        ctx->launches = l0;
        if (e2 == cudaSuccess && rc == LBM_OK && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
        else e = e2 != cudaSuccess ? e2 : cudaErrorStreamCaptureInvalidated;
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();   // a refused capture leaves its error here
        g.key = key;
        ctx->graph_stats[1] += 1;
        if (e != cudaSuccess || !g.exec) {
            ctx->graph_stats[2] += 1;
            for (auto& pe : g.prof) {
                cudaEventDestroy(std::get<1>(pe));
                cudaEventDestroy(std::get<2>(pe));
            }
            g.prof.clear();
            g.exec = nullptr;
            g.failed = true;   // plain launches for these settings from now on
        } else {
            g.launches = per;
        }
    }
    if (use && g.exec && g.key == key) {
        CK(cudaGraphLaunch(g.exec, L.stream));
        ctx->launches += g.launches;
        ctx->graph_stats[0] += 1;
        *replayed = true;
        return LBM_OK;
    }
    for (int k = 0; k < chunk; ++k) {
        const int e = iterate_once<T>(ctx, L, M, *I, V, o, so, nblk_field);
        if (e) return e;
    }
    return LBM_OK;
}

void fill_result(const InstState& s, const InstConst& c, lbm_result& r, double wall_ms) {
    r.status = s.status;
    r.iterations = s.iters;
    r.evaluations = s.evals;
    r.line_searches = s.line_searches;
    r.cg_iters1 = s.cg1;
    r.cg_iters2 = s.cg2;
    for (int k = 0; k < 4; ++k) r.energy[k] = s.terms[k] * c.Eunit;
    r.energy[4] = s.E * c.Eunit;
    r.torque = s.torque;
    r.gg = s.gg;
    for (int k = 0; k < 3; ++k) r.mean_m[k] = s.mean_m[k];
    r.wall_ms = wall_ms;
}

template <typename T>
int run_minimise(lbm_ctx* ctx, Inst* I, const lbm_solve_opts& o, lbm_result* res, bool evaluate_only,
                 double* hout, double* uout, std::vector<InstState>* states_out = nullptr, bool warm = false) {
    Mesh& M = *ctx->meshes[I->mesh];
    const auto t0 = std::chrono::steady_clock::now();
    BatchView<T> V = batch_view<T>(ctx, M, *I, evaluate_only && hout);
    Launch L = ctx->launch();
    L.pcg_kernel = o.pcg_kernel;
    MeshView mv = M.view();
    lbm_solve_opts oo = o;
    if (evaluate_only) oo.max_iter = 0;
    const StepOpts so = step_opts(oo);
    if (oo.resume && !evaluate_only) resume_states(L, I->st, I->B);
    else reset_states(L, I->st, I->B, so, 0, warm ? 1 : 0);
    const int nblk_field = field_blocks(L, mv, I->B);
    std::vector<InstState> hs(I->B);
    // instances iterating at the start of each chunk (all after the reset); the
    // cluster potential solves launch only for the groups among them
    std::vector<unsigned char> active(I->B, 1);
    L.active = active.data();
    const int64_t max_loops = (int64_t)(oo.max_iter + 1) * (oo.max_backtracks + 2) + 2;
    int64_t loops = 0;
    int rc = LBM_OK;
    bool first = true;
    while (true) {
        const int chunk = evaluate_only ? 1 : oo.check_every;
        bool replayed = false;
        int e = run_chunk<T>(ctx, L, M, I, V, oo, so, nblk_field, chunk, first, nullptr, &replayed);
        if (e) return e;
        first = false;
        loops += chunk;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hs.data(), I->st, sizeof(InstState) * I->B, cudaMemcpyDeviceToHost, ctx->stream));
        int errw = 0;
        CK(cudaMemcpyAsync(&errw, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        prof_harvest(ctx);
        if (replayed && ctx->prof) prof_harvest_graph(ctx, I->graph);
        if (errw) {
            cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream);
            if (errw & DEV_ERR_SHAPE)
                return fail(LBM_E_CUDA, "a potential solve launched fewer clusters than active systems");
            return fail(LBM_E_TIMEOUT, "a device-side wait ran out of time (error word %d)", errw);
        }
        bool all = true;
        for (int b = 0; b < I->B; ++b) {
            all &= hs[b].phase == PH_DONE;
            active[b] = hs[b].phase != PH_DONE;
        }
        if (all) break;
        if (loops > max_loops) { rc = LBM_E_NOT_CONVERGED; break; }
    }
    if (evaluate_only && (hout || uout)) {
        // the evaluated trial is now the base point; h was written at that point
        unpack_field<T>(L, mv, V, hout ? I->staged : nullptr, uout ? I->staged_u : nullptr);
        if (hout) CK(cudaMemcpyAsync(hout, I->staged, sizeof(double) * I->B * M.N * 3, cudaMemcpyDeviceToHost,
                                     ctx->stream));
        if (uout) CK(cudaMemcpyAsync(uout, I->staged_u, sizeof(double) * I->B * M.N * 2,
                                     cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (res) {
        std::vector<InstConst> hc(I->B);
        CK(cudaMemcpy(hc.data(), I->ic, sizeof(InstConst) * I->B, cudaMemcpyDeviceToHost));
        for (int b = 0; b < I->B; ++b) {
            fill_result(hs[b], hc[b], res[b], ms);
            if (evaluate_only && hs[b].status == 3) res[b].status = LBM_OK;
        }
    }
    if (ctx->prof)
        for (int b = 0; b < I->B; ++b) ctx->prof_cg[sizeof(T) == 8 ? 1 : 0] += hs[b].cg1 + hs[b].cg2;
    if (states_out) *states_out = hs;
    (void)rc;
    return LBM_OK;
}

__global__ void k_widen(const float* __restrict__ src, double* __restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

// Mixed precision: an FP32 phase (FP32 potentials, BEM product and SpMV; FP64
// state, reductions and step decisions) to switch_tol, then an FP64 phase on a
// shadow batch warm-started from the FP32 state and potentials, to tol.
int minimise_mixed(lbm_ctx* ctx, Inst* I, const lbm_solve_opts& o, lbm_result* res) {
    Mesh& M = *ctx->meshes[I->mesh];
    const auto t0 = std::chrono::steady_clock::now();
    lbm_solve_opts o1 = o;
    if (o.cg_tol_fp32 > 0) o1.cg_tol = o.cg_tol_fp32;
    o1.tol = o.tol > o.switch_tol ? o.tol : o.switch_tol;   // FP32 phase; it hands a stalled
                                                            // instance to the FP64 phase
    std::vector<InstState> s1, s2;
    int rc = run_minimise<float>(ctx, I, o1, nullptr, false, nullptr, nullptr, &s1);
    if (rc) return rc;
    bool need = false;
    for (int b = 0; b < I->B; ++b)
        need |= s1[b].status != 4 && !(s1[b].status == 0 && s1[b].torque < o.tol);
    const size_t N = M.N, B = I->B;
    if (need) {
        if (!I->polish) {
            Inst* P = new Inst();
            P->mesh = I->mesh;
            P->B = I->B;
            P->precision = LBM_FP64;
            P->tsize = 8;
            // The FP64 phase fixes the final accuracy: its BEM products stay on the
            // SIMT path (FP32 matrix).  The tensor cores' FP32 accumulation is not
            // round-to-nearest, and over the long reductions of the product
            // (K = nb) it biases the stray-field energy by ~1e-6 relative.
            P->use_tc = false;
            P->tc_scratch = nullptr;
            P->owns_tc_scratch = false;
            const size_t vb = vec_bytes(M, I->B, 8), pe = part_elems(ctx, I->B);
            if (cudaMalloc(&P->vec, vb) != cudaSuccess || cudaMalloc(&P->part, pe * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&P->st, sizeof(InstState) * B) != cudaSuccess ||
                cudaMalloc(&P->ic, sizeof(InstConst) * B) != cudaSuccess ||
                cudaMalloc(&P->staged, sizeof(double) * B * N * 3) != cudaSuccess ||
                cudaMalloc(&P->staged_u, sizeof(double) * B * N * 2) != cudaSuccess) {
                free_inst(P);
                return fail(LBM_E_OOM, "allocation of the FP64 phase of a mixed run failed");
            }
            CK(cudaMemsetAsync(P->vec, 0, vb, ctx->stream));
            I->polish = P;
        }
        Inst* P = I->polish;
        P->mats = I->mats;
        P->h = I->h;
        // state (m at base and trial, cur) and constants; potentials widened to FP64
        CK(cudaMemcpyAsync(P->vec, I->vec, sizeof(double) * 2 * N * 3 * B, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(P->st, I->st, sizeof(InstState) * B, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(P->ic, I->ic, sizeof(InstConst) * B, cudaMemcpyDeviceToDevice, ctx->stream));
        const VecLayout L32 = vec_layout(M, I->B, 4), L64 = vec_layout(M, I->B, 8);
        const size_t npot = N * 2 * B;
        k_widen<<<4 * ctx->num_sms, 256, 0, ctx->stream>>>((const float*)((const char*)I->vec + L32.U1),
                                                           (double*)((char*)P->vec + L64.U1), npot);
        k_widen<<<4 * ctx->num_sms, 256, 0, ctx->stream>>>((const float*)((const char*)I->vec + L32.U2),
                                                           (double*)((char*)P->vec + L64.U2), npot);
        ctx->launches += 2;
        if (M.shell)   // the grid potential (FP64 in both phases) warm-starts the FP64 phase's solves
            CK(cudaMemcpyAsync((char*)P->vec + L64.shx, (const char*)I->vec + L32.shx,
                               sizeof(double) * M.shell->Ng * B, cudaMemcpyDeviceToDevice, ctx->stream));
        lbm_solve_opts o2 = o;
        o2.cg_tol = o.cg_tol_polish;
        o2.stall_iters = 0;   // the FP64 phase runs to tol or max_iter
        // a 10 % margin below tol: the phase's torque comes from solves to
        // cg_tol_polish, the exact problem's may differ by that much
        o2.tol = POLISH_MARGIN * o.tol;
        // the FP64 phase continues the FP32 phase's step state (BB step, kappa,
        // tau^2 memory) after one FP64 evaluation of the point, instead of
        // starting over with a line search
        rc = run_minimise<double>(ctx, P, o2, nullptr, false, nullptr, nullptr, &s2, true);
        if (rc) return rc;
        CK(cudaMemcpyAsync(I->vec, P->vec, sizeof(double) * 2 * N * 3 * B, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(I->st, P->st, sizeof(InstState) * B, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (res) {
        std::vector<InstConst> hc(I->B);
        CK(cudaMemcpy(hc.data(), I->ic, sizeof(InstConst) * I->B, cudaMemcpyDeviceToHost));
        for (int b = 0; b < I->B; ++b) {
            const bool two = need && s1[b].status != 4;
            fill_result(two ? s2[b] : s1[b], hc[b], res[b], ms);
            if (two) {
                res[b].iterations += s1[b].iters;
                res[b].evaluations += s1[b].evals;
                res[b].line_searches += s1[b].line_searches;
                res[b].cg_iters1 += s1[b].cg1;
                res[b].cg_iters2 += s1[b].cg2;
            }
        }
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_opts(lbm_solve_opts* o, int32_t precision) {
    memset(o, 0, sizeof *o);
    o->tol = 1e-6;
    o->grad_tol = 0.0;
    o->max_iter = 100000;
    o->cg_tol = precision == LBM_FP64 ? 1e-13 : 1e-7;
    o->cg_max_iter = 5000;
    o->c1 = 1e-4;
    o->max_backtracks = 30;
    o->memory = 20;
    o->kappa0 = 0.5;
    o->m_alpha = 3;
    o->tau_min = 1e-10;
    o->tau_max = 1e10;
    o->demag = 1;
    o->check_every = 16;
    o->switch_tol = 1e-4;
    o->cg_tol_polish = 1e-10;
    o->cg_mixed_iter = precision == LBM_FP64 ? 0 : 1;
    o->bb_rule = 0;
    o->method = 0;
    o->omega = 1.0;
    o->stall_iters = precision == LBM_FP64 ? 0 : 200;
    o->pcg_kernel = 0;
    o->use_graphs = 1;
    o->cg_tol_fp32 = precision == LBM_FP64 ? 0.0 : 3e-5;
    o->resume = 0;
    if (precision != LBM_FP64) o->cg_tol = 1e-6;
}

const char* lbm_last_error(void) { return g_err.c_str(); }

int lbm_create(lbm_ctx** out, int32_t device, void* stream) {
    LBM_TRY
    if (!out) return fail(LBM_E_INVALID, "null output pointer");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(LBM_E_INVALID, "device %d not present (%d devices)", device, ndev);
    CK(cudaSetDevice(device));
    lbm_ctx* c = new lbm_ctx();
    c->device = device;
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, device);
    c->num_sms = prop.multiProcessorCount;
    if (!prop.cooperativeLaunch) {
        delete c;
        return fail(LBM_E_CUDA, "device does not support cooperative launches");
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return fail(LBM_E_CUDA, "stream: %s", cudaGetErrorString(e)); }
        c->own_stream = true;
    }
    if (cudaMalloc(&c->bar, 64) != cudaSuccess || cudaMalloc(&c->err, 64) != cudaSuccess) {
        delete c;
        return fail(LBM_E_OOM, "context allocation failed");
    }
    cudaMemset(c->bar, 0, 64);
    cudaMemset(c->err, 0, 64);
    if (cudaMalloc(&c->sweeps, 64) != cudaSuccess || cudaMalloc(&c->fin, sizeof(double) * 4096) != cudaSuccess) {
        delete c;
        return fail(LBM_E_OOM, "context allocation failed");
    }
    cudaMemset(c->sweeps, 0, 64);
    *out = c;
    return LBM_OK;
    LBM_CATCH
}

int lbm_destroy(lbm_ctx* ctx) {
    LBM_TRY
    if (!ctx) return LBM_OK;
    if (ctx->server) lbm_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->insts) free_inst(kv.second);
    for (auto& kv : ctx->meshes) free_mesh(kv.second);
    prof_harvest(ctx);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    cudaFree(ctx->bar);
    cudaFree(ctx->err);
    cudaFree(ctx->sweeps);
    cudaFree(ctx->fin);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return LBM_OK;
    LBM_CATCH
}

int lbm_launch_count(lbm_ctx* ctx, int64_t* count) {
    LBM_TRY
    if (!ctx || !count) return fail(LBM_E_INVALID, "null argument");
    *count = ctx->launches;
    return LBM_OK;
    LBM_CATCH
}

int lbm_graph_stats(lbm_ctx* ctx, int64_t out[3]) {
    LBM_TRY
    if (!ctx || !out) return fail(LBM_E_INVALID, "null argument");
    for (int k = 0; k < 3; ++k) out[k] = ctx->graph_stats[k];
    return LBM_OK;
    LBM_CATCH
}

int lbm_mesh_cube(lbm_ctx* ctx, double cell_m, int32_t n, lbm_mesh* out) {
    LBM_TRY
    if (!ctx || !out || n < 1 || n > 96 || !(cell_m > 0)) return fail(LBM_E_INVALID, "lbm_mesh_cube: bad argument");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    Mesh* M = new Mesh();
    M->num_sms = ctx->num_sms;
    M->n = n;
    M->cell = cell_m;
    const int n1 = n + 1, N = n1 * n1 * n1;
    M->N = N;
    M->T = 6 * n * n * n;
    int *cnt = nullptr, *bflag = nullptr, *bpos = nullptr;
    auto cleanup = [&]() {
        if (cnt) cudaFree(cnt);
        if (bflag) cudaFree(bflag);
        if (bpos) cudaFree(bpos);
    };
#define CKM(call)                   \
    do {                            \
        cudaError_t e_ = (call);    \
        if (e_ != cudaSuccess) {    \
            cleanup();              \
            free_mesh(M);           \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_E_OOM : LBM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
        }                           \
    } while (0)
    CKM(cudaMalloc(&cnt, sizeof(int) * N));
    CKM(cudaMalloc(&bflag, sizeof(int) * N));
    CKM(cudaMalloc(&bpos, sizeof(int) * (N + 1)));
    CKM(cudaMalloc(&M->rowptr, sizeof(int) * (N + 1)));
    launch_row_counts(n, cnt, bflag, st);
    launch_scan(cnt, M->rowptr, N, st);
    launch_scan(bflag, bpos, N, st);
    ctx->launches += 3;
    int tot[2];
    CKM(cudaMemcpyAsync(&tot[0], M->rowptr + N, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKM(cudaMemcpyAsync(&tot[1], bpos + N, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKM(cudaStreamSynchronize(st));
    M->nnz = tot[0];
    M->nb = tot[1];
    CKM(cudaMalloc(&M->col, sizeof(int) * M->nnz));
    CKM(cudaMalloc(&M->pkA, sizeof(int) * M->nnz));
    CKM(cudaMalloc(&M->pkB, sizeof(int) * M->nnz));
    CKM(cudaMalloc(&M->node, sizeof(int) * N));
    CKM(cudaMalloc(&M->bidx, sizeof(int) * M->nb));
    launch_assemble(n, M->rowptr, bpos, M->col, M->pkA, M->pkB, M->node, st);
    launch_boundary_ids(N, bflag, bpos, M->bidx, st);
    CKM(cudaMalloc(&M->kptr, sizeof(int) * (N + 1)));
    launch_kcsr_count(N, M->rowptr, M->pkA, cnt, st);
    launch_scan(cnt, M->kptr, N, st);
    CKM(cudaMemcpyAsync(&tot[0], M->kptr + N, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKM(cudaStreamSynchronize(st));
    M->nnzK = tot[0];
    CKM(cudaMalloc(&M->kent, sizeof(int) * M->nnzK));
    launch_kcsr_fill(N, M->rowptr, M->col, M->pkA, M->kptr, M->kent, st);
    ctx->launches += 5;
    std::vector<int> hb(M->nb), tris, incp, incs;
    CKM(cudaMemcpyAsync(hb.data(), M->bidx, sizeof(int) * M->nb, cudaMemcpyDeviceToHost, st));
    CKM(cudaStreamSynchronize(st));
    host_boundary_topology(n, tris, hb, incp, incs);
    M->F = (int)tris.size() / 3;
    CKM(cudaMalloc(&M->tris, sizeof(int) * tris.size()));
    CKM(cudaMalloc(&M->inc_ptr, sizeof(int) * incp.size()));
    CKM(cudaMalloc(&M->inc_slot, sizeof(int) * incs.size()));
    CKM(cudaMemcpyAsync(M->tris, tris.data(), sizeof(int) * tris.size(), cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->inc_ptr, incp.data(), sizeof(int) * incp.size(), cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->inc_slot, incs.data(), sizeof(int) * incs.size(), cudaMemcpyHostToDevice, st));
    const size_t nb2 = (size_t)M->nb * M->nb;
    CKM(cudaMalloc(&M->B64, sizeof(double) * nb2));
    CKM(cudaMalloc(&M->B32, sizeof(float) * nb2));
    int nblocks = 2 * ctx->num_sms;
    if (nblocks > M->nb) nblocks = M->nb;
    double* scratch = nullptr;
    CKM(cudaMalloc(&scratch, sizeof(double) * 3 * (size_t)M->F * nblocks));
    launch_bem_assemble(n, M->nb, M->F, M->bidx, M->tris, M->inc_ptr, M->inc_slot, nullptr, scratch, nblocks,
                        M->B64, M->B32, st);
    ctx->launches += 1;
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(scratch);
    CKM(e);
    CKM(cudaGetLastError());
    cleanup();
    cnt = bflag = bpos = nullptr;
#undef CKM
    M->bytes = sizeof(int) * ((size_t)3 * N + 2 + 3 * (size_t)M->nnz + M->nnzK + M->nb + tris.size() +
                              incp.size() + incs.size()) + 12 * nb2;
    const int64_t id = ctx->next_id++;
    ctx->meshes[id] = M;
    *out = id;
    return LBM_OK;
    LBM_CATCH
}

int lbm_mesh_upload(lbm_ctx* ctx, const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                    lbm_mesh* out) {
    LBM_TRY
    if (!ctx || !out || !xyz || !tets) return fail(LBM_E_INVALID, "lbm_mesh_upload: null argument");
    if (n_nodes < 4 || n_nodes > LBM_UPLOAD_MAX_NODES || n_tets < 1 || n_tets > LBM_UPLOAD_MAX_TETS)
        return fail(LBM_E_INVALID, "lbm_mesh_upload: need 4 <= n_nodes <= %d and 1 <= n_tets <= %d",
                    LBM_UPLOAD_MAX_NODES, LBM_UPLOAD_MAX_TETS);
    for (int64_t k = 0; k < 3 * n_nodes; ++k)
        if (!std::isfinite(xyz[k])) return fail(LBM_E_INVALID, "lbm_mesh_upload: non-finite coordinate");
    const int N = (int)n_nodes, T = (int)n_tets;
    GeneralTopology g;
    const std::string why = host_general_topology(N, T, tets, xyz, g);
    if (!why.empty()) return fail(LBM_E_INVALID, "lbm_mesh_upload: %s", why.c_str());
    const int nb = (int)g.bidx.size();
    if (nb > 65534) return fail(LBM_E_INVALID, "lbm_mesh_upload: %d surface nodes (at most 65534)", nb);
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    Mesh* M = new Mesh();
    M->num_sms = ctx->num_sms;
    M->gen = true;
    M->n = 0;
    M->N = N;
    M->T = T;
    M->nb = nb;
    M->nnz = (int)g.col.size();
    M->F = (int)g.tris.size() / 3;
    M->cell = g.L;
    // coordinates in units of L, surface flags on the columns, node words
    std::vector<double> xl(3 * (size_t)N);
    for (size_t k = 0; k < xl.size(); ++k) xl[k] = xyz[k] / g.L;
    std::vector<int> bpos(N, 0), colf(g.col.size()), nodew(N);
    for (int k = 0; k < nb; ++k) bpos[g.bidx[k]] = k + 1;
    for (size_t e = 0; e < g.col.size(); ++e) colf[e] = (int)((unsigned)g.col[e] | (bpos[g.col[e]] ? 0x80000000u : 0u));
    for (int i = 0; i < N; ++i) nodew[i] = (int)((unsigned)bpos[i] << 16);
    double vsum = 0.0;
    for (int t = 0; t < T; ++t) vsum += 4.0 * fabs(g.det[t]) / (g.L * g.L * g.L);
    M->vsum = vsum;
    std::vector<int> incp, incs;
    host_incidence(N, g.tris, g.bidx, incp, incs);
    int *nt_ptr = nullptr, *nt_idx = nullptr, *cnt = nullptr;
    double* scratch = nullptr;
    auto cleanup = [&]() {
        if (nt_ptr) cudaFree(nt_ptr);
        if (nt_idx) cudaFree(nt_idx);
        if (cnt) cudaFree(cnt);
        if (scratch) cudaFree(scratch);
    };
#define CKM(call)                   \
    do {                            \
        cudaError_t e_ = (call);    \
        if (e_ != cudaSuccess) {    \
            cudaStreamSynchronize(st); \
            cleanup();              \
            free_mesh(M);           \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_E_OOM : LBM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
        }                           \
    } while (0)
    const size_t nnz = M->nnz;
    CKM(cudaMalloc(&M->rowptr, sizeof(int) * (N + 1)));
    CKM(cudaMalloc(&M->col, sizeof(int) * nnz));
    CKM(cudaMalloc(&M->node, sizeof(int) * N));
    CKM(cudaMalloc(&M->bidx, sizeof(int) * nb));
    CKM(cudaMalloc(&M->tets, sizeof(int) * 4 * (size_t)T));
    CKM(cudaMalloc(&M->xyz, sizeof(double) * 3 * (size_t)N));
    CKM(cudaMalloc(&M->tris, sizeof(int) * g.tris.size()));
    CKM(cudaMalloc(&M->inc_ptr, sizeof(int) * incp.size()));
    CKM(cudaMalloc(&M->inc_slot, sizeof(int) * incs.size()));
    CKM(cudaMalloc(&nt_ptr, sizeof(int) * (N + 1)));
    CKM(cudaMalloc(&nt_idx, sizeof(int) * g.nt_idx.size()));
    CKM(cudaMalloc(&cnt, sizeof(int) * N));
    CKM(cudaMalloc(&M->gA64, sizeof(Dbl4) * nnz));
    CKM(cudaMalloc(&M->gB64, sizeof(Dbl4) * nnz));
    CKM(cudaMalloc(&M->gA32, sizeof(float4) * nnz));
    CKM(cudaMalloc(&M->gB32, sizeof(float4) * nnz));
    CKM(cudaMalloc(&M->gV, sizeof(double) * N));
    CKM(cudaMalloc(&M->gd64, sizeof(double) * N));
    CKM(cudaMalloc(&M->gd32, sizeof(float) * N));
    CKM(cudaMalloc(&M->kptr, sizeof(int) * (N + 1)));
    CKM(cudaMemcpyAsync(M->rowptr, g.rowptr.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->col, colf.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->node, nodew.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->bidx, g.bidx.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->tets, tets, sizeof(int) * 4 * (size_t)T, cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->xyz, xl.data(), sizeof(double) * xl.size(), cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->tris, g.tris.data(), sizeof(int) * g.tris.size(), cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->inc_ptr, incp.data(), sizeof(int) * incp.size(), cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(M->inc_slot, incs.data(), sizeof(int) * incs.size(), cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(nt_ptr, g.nt_ptr.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st));
    CKM(cudaMemcpyAsync(nt_idx, g.nt_idx.data(), sizeof(int) * g.nt_idx.size(), cudaMemcpyHostToDevice, st));
    launch_assemble_gen(N, M->xyz, M->tets, nt_ptr, nt_idx, M->rowptr, M->col, M->gA64, M->gA32, M->gB64, M->gB32,
                        M->gV, M->gd64, M->gd32, st);
    launch_kcsr_count_gen(N, M->rowptr, M->gA64, cnt, st);
    launch_scan(cnt, M->kptr, N, st);
    ctx->launches += 3;
    int tot = 0;
    CKM(cudaMemcpyAsync(&tot, M->kptr + N, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKM(cudaStreamSynchronize(st));
    M->nnzK = tot;
    CKM(cudaMalloc(&M->kent, sizeof(int) * (size_t)M->nnzK));
    CKM(cudaMalloc(&M->gk64, sizeof(double) * (size_t)M->nnzK));
    CKM(cudaMalloc(&M->gk32, sizeof(float) * (size_t)M->nnzK));
    launch_kcsr_fill_gen(N, M->rowptr, M->col, M->gA64, M->kptr, M->kent, M->gk64, M->gk32, st);
    ctx->launches += 1;
    const size_t nb2 = (size_t)nb * nb;
    CKM(cudaMalloc(&M->B64, sizeof(double) * nb2));
    CKM(cudaMalloc(&M->B32, sizeof(float) * nb2));
    int nblocks = 2 * ctx->num_sms;
    if (nblocks > nb) nblocks = nb;
    CKM(cudaMalloc(&scratch, sizeof(double) * 3 * (size_t)M->F * nblocks));
    launch_bem_assemble(0, nb, M->F, M->bidx, M->tris, M->inc_ptr, M->inc_slot, M->xyz, scratch, nblocks, M->B64,
                        M->B32, st);
    ctx->launches += 1;
    CKM(cudaStreamSynchronize(st));
    CKM(cudaGetLastError());
    cleanup();
#undef CKM
    M->bytes = sizeof(int) * ((size_t)3 * N + 2 + nnz + M->nnzK + nb + g.tris.size() + incp.size() + incs.size() +
                              4 * (size_t)T) +
               sizeof(double) * (3 * (size_t)N + 3 * (size_t)N + M->nnzK) + (32 + 32 + 16 + 16) * nnz +
               4 * ((size_t)N + M->nnzK) + 12 * nb2;
    const int64_t id = ctx->next_id++;
    ctx->meshes[id] = M;
    *out = id;
    return LBM_OK;
    LBM_CATCH
}

int lbm_mesh_values(lbm_ctx* ctx, lbm_mesh mesh, double* K, double* G, double* Gt, double* V, double* unit_m) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M) return fail(LBM_E_INVALID, "unknown mesh");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const double L = M->cell;
    const double sK = L / 6.0, sG = L * L / 24.0, sV = L * L * L / 24.0;
    if (unit_m) *unit_m = L;
    if (M->gen) {
        std::vector<Dbl4> a(M->nnz), b(M->nnz);
        std::vector<double> v(M->N);
        CK(cudaMemcpyAsync(a.data(), M->gA64, sizeof(Dbl4) * M->nnz, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(b.data(), M->gB64, sizeof(Dbl4) * M->nnz, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(v.data(), M->gV, sizeof(double) * M->N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int e = 0; e < M->nnz; ++e) {
            if (K) K[e] = sK * a[e].x;
            if (G) { G[3 * e] = sG * a[e].y; G[3 * e + 1] = sG * a[e].z; G[3 * e + 2] = sG * a[e].w; }
            if (Gt) { Gt[3 * e] = sG * b[e].x; Gt[3 * e + 1] = sG * b[e].y; Gt[3 * e + 2] = sG * b[e].z; }
        }
        if (V)
            for (int i = 0; i < M->N; ++i) V[i] = sV * v[i];
        return LBM_OK;
    }
    std::vector<int> a(M->nnz), b(M->nnz), nd(M->N);
    CK(cudaMemcpyAsync(a.data(), M->pkA, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(b.data(), M->pkB, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(nd.data(), M->node, sizeof(int) * M->N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    auto sb = [](int w, int k) { return (double)(signed char)((w >> (8 * k)) & 0xff); };
    for (int e = 0; e < M->nnz; ++e) {
        if (K) K[e] = sK * sb(a[e], 0);
        for (int d = 0; d < 3; ++d) {
            if (G) G[3 * e + d] = sG * sb(a[e], 1 + d);
            if (Gt) Gt[3 * e + d] = sG * sb(b[e], d);
        }
    }
    if (V)
        for (int i = 0; i < M->N; ++i) V[i] = sV * (double)(nd[i] & 0xff);
    return LBM_OK;
    LBM_CATCH
}

int lbm_mesh_destroy(lbm_ctx* ctx, lbm_mesh mesh) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M) return fail(LBM_E_INVALID, "unknown mesh");
    for (auto& kv : ctx->insts)
        if (kv.second->mesh == mesh) return fail(LBM_E_INVALID, "mesh still has instances");
    cudaStreamSynchronize(ctx->stream);
    free_mesh(M);
    ctx->meshes.erase(mesh);
    return LBM_OK;
    LBM_CATCH
}

int lbm_mesh_info(lbm_ctx* ctx, lbm_mesh mesh, int64_t info[8]) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M || !info) return fail(LBM_E_INVALID, "unknown mesh");
    info[0] = M->N;
    info[1] = M->nb;
    info[2] = M->nnz;
    info[3] = M->T;
    info[4] = M->F;
    info[5] = (int64_t)M->bytes;
    info[6] = M->n;
    info[7] = 0;
    return LBM_OK;
    LBM_CATCH
}

int lbm_mesh_export(lbm_ctx* ctx, lbm_mesh mesh, int32_t* tets, int32_t* rowptr, int32_t* col, int32_t* kval,
                    int32_t* gval, int32_t* gtval, int32_t* vol, int32_t* bnd, int32_t* tris) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M) return fail(LBM_E_INVALID, "unknown mesh");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    if (M->gen && (kval || gval || gtval || vol))
        return fail(LBM_E_INVALID, "lbm_mesh_export: integer tables exist for cube meshes only (use lbm_mesh_values)");
    if (tets && M->gen) {
        CK(cudaMemcpyAsync(tets, M->tets, sizeof(int) * 4 * (size_t)M->T, cudaMemcpyDeviceToHost, st));
    } else if (tets) {
        int* d = nullptr;
        CK(cudaMalloc(&d, sizeof(int) * 4 * (size_t)M->T));
        launch_tets(M->n, d, st);
        ctx->launches += 1;
        cudaError_t e = cudaMemcpyAsync(tets, d, sizeof(int) * 4 * (size_t)M->T, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(d);
        CK(e);
    }
    if (rowptr) CK(cudaMemcpyAsync(rowptr, M->rowptr, sizeof(int) * (M->N + 1), cudaMemcpyDeviceToHost, st));
    if (bnd) CK(cudaMemcpyAsync(bnd, M->bidx, sizeof(int) * M->nb, cudaMemcpyDeviceToHost, st));
    if (tris) CK(cudaMemcpyAsync(tris, M->tris, sizeof(int) * 3 * M->F, cudaMemcpyDeviceToHost, st));
    std::vector<int> c(M->nnz), a(M->nnz), b(M->nnz), nd(M->N);
    CK(cudaMemcpyAsync(c.data(), M->col, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost, st));
    if (!M->gen) {
        CK(cudaMemcpyAsync(a.data(), M->pkA, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(b.data(), M->pkB, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaMemcpyAsync(nd.data(), M->node, sizeof(int) * M->N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    auto sb = [](int w, int k) { return (int)(signed char)((w >> (8 * k)) & 0xff); };
    for (int e = 0; e < M->nnz; ++e) {
        if (col) col[e] = c[e] & 0x7fffffff;
        if (kval) kval[e] = sb(a[e], 0);
        for (int d = 0; d < 3; ++d) {
            if (gval) gval[3 * e + d] = sb(a[e], 1 + d);
            if (gtval) gtval[3 * e + d] = sb(b[e], d);
        }
    }
    if (vol)
        for (int i = 0; i < M->N; ++i) vol[i] = nd[i] & 0xff;
    return LBM_OK;
    LBM_CATCH
}

int lbm_bem_rows(lbm_ctx* ctx, lbm_mesh mesh, int64_t row0, int64_t nrows, double* out) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M || !out || row0 < 0 || nrows < 0 || row0 + nrows > M->nb) return fail(LBM_E_INVALID, "bad rows");
    CK(cudaMemcpyAsync(out, M->B64 + (size_t)row0 * M->nb, sizeof(double) * nrows * M->nb,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
    LBM_CATCH
}

int lbm_hmatrix_plan(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets, double eps, double eta,
                     int32_t n_min, int32_t threads, int64_t out[4]) {
    LBM_TRY
    if (!xyz || !tets || !out) return fail(LBM_E_INVALID, "lbm_hmatrix_plan: null argument");
    if (n_nodes < 4 || n_nodes > LBM_UPLOAD_MAX_NODES || n_tets < 1 || n_tets > LBM_UPLOAD_MAX_TETS)
        return fail(LBM_E_INVALID, "lbm_hmatrix_plan: mesh size out of range");
    for (int64_t k = 0; k < 3 * n_nodes; ++k)
        if (!std::isfinite(xyz[k])) return fail(LBM_E_INVALID, "lbm_hmatrix_plan: non-finite coordinate");
    if (!(eps > 0.0 && eps < 1.0) || !(eta > 0.0) || !std::isfinite(eta) || n_min < 1 || threads < 1)
        return fail(LBM_E_INVALID,
                    "lbm_hmatrix_plan: eps must lie in (0, 1), eta be positive, n_min and threads at least 1");
    GeneralTopology g;
    const std::string why = host_general_topology((int)n_nodes, (int)n_tets, tets, xyz, g);
    if (!why.empty()) return fail(LBM_E_INVALID, "lbm_hmatrix_plan: %s", why.c_str());
    std::vector<double> xl(3 * (size_t)n_nodes);                 // in units of the length unit, as uploads
    for (size_t k = 0; k < xl.size(); ++k) xl[k] = xyz[k] / g.L;
    HMatrixHost H;
    const int nb = (int)g.bidx.size(), F = (int)(g.tris.size() / 3);
    const std::string w2 = host_hmatrix_build((int)n_nodes, xl.data(), nb, g.bidx.data(), F, g.tris.data(), eta,
                                              n_min, eps, threads, H);
    if (!w2.empty()) return fail(LBM_E_INVALID, "lbm_hmatrix_plan: %s", w2.c_str());
    int64_t low = 0;
    for (int k : H.kind) low += k;
    out[0] = (int64_t)H.data.size();
    out[1] = (int64_t)nb * nb;
    out[2] = (int64_t)H.kind.size();
    out[3] = low;
    return LBM_OK;
    LBM_CATCH
}

// Upload one packed operator: leaf table, positions, values (FP32 and FP64),
// the first pass's row table, the owners' slots and entries.
static int hm_upload(lbm_ctx* ctx, Mesh* M, const HPacked& P, HMView& v) {
    auto up = [&](const void* src, size_t bytes) -> void* {
        void* d = nullptr;
        if (bytes == 0) bytes = 16;
        if (cudaMalloc(&d, bytes) != cudaSuccess) return nullptr;
        M->hm_mem.push_back(d);
        if (src && cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) return nullptr;
        return d;
    };
    std::vector<HLeafDev> lv(P.leaves.size());
    std::vector<int> trow_leaf, trow_l;
    for (size_t q = 0; q < P.leaves.size(); ++q) {
        const HPackedLeaf& e = P.leaves[q];
        lv[q] = HLeafDev{e.row_begin, e.m, e.col_begin, e.n, e.kind, e.rank, (long long)e.val, (long long)e.t_off};
        if (e.kind)
            for (int l = 0; l < e.rank; ++l) {
                trow_leaf.push_back((int)q);
                trow_l.push_back(l);
            }
    }
    // output rows: every owner's positions, owners in order; they must cover
    // every surface position exactly once
    std::vector<int> slot_owner, slot_a, seen(P.nb, 0);
    for (size_t o = 0; o < P.owner_begin.size(); ++o)
        for (int a = 0; a < P.owner_size[o]; ++a) {
            const size_t at = (size_t)P.owner_begin[o] + a;
            const int pos = at < P.idx.size() ? P.idx[at] : -1;
            if (pos < 0 || pos >= P.nb || seen[pos]++)
                return fail(LBM_E_INVALID, "lbm_mesh_hmatrix: row owners do not partition the surface");
            slot_owner.push_back((int)o);
            slot_a.push_back(a);
        }
    if ((int)slot_owner.size() != P.nb) return fail(LBM_E_INVALID, "lbm_mesh_hmatrix: row owners do not cover the surface");
    std::vector<long long> optr(P.owner_ptr.begin(), P.owner_ptr.end()), erows(P.entries.size());
    std::vector<int> eleaf(P.entries.size());
    for (size_t e = 0; e < P.entries.size(); ++e) {
        eleaf[e] = P.entries[e].leaf;
        erows[e] = (long long)P.entries[e].rows;
    }
    v.nb = P.nb;
    v.nleaf = (int)lv.size();
    v.n_t = (int)P.n_t;
    v.leaves = (const HLeafDev*)up(lv.data(), sizeof(HLeafDev) * lv.size());
    v.idx = (const int*)up(P.idx.data(), sizeof(int) * P.idx.size());
    v.v32 = (const float*)up(P.values.data(), sizeof(float) * P.values.size());
    v.v64 = (const double*)up(P.values64.data(), sizeof(double) * P.values64.size());
    v.trow_leaf = (const int*)up(trow_leaf.data(), sizeof(int) * trow_leaf.size());
    v.trow_l = (const int*)up(trow_l.data(), sizeof(int) * trow_l.size());
    v.slot_owner = (const int*)up(slot_owner.data(), sizeof(int) * slot_owner.size());
    v.slot_a = (const int*)up(slot_a.data(), sizeof(int) * slot_a.size());
    v.owner_begin = (const int*)up(P.owner_begin.data(), sizeof(int) * P.owner_begin.size());
    v.owner_ptr = (const long long*)up(optr.data(), sizeof(long long) * optr.size());
    v.ent_leaf = (const int*)up(eleaf.data(), sizeof(int) * eleaf.size());
    v.ent_rows = (const long long*)up(erows.data(), sizeof(long long) * erows.size());
    v.row_map = (const int*)up(P.row_map.data(), sizeof(int) * P.row_map.size());
    if (!v.leaves || !v.idx || !v.v32 || !v.v64 || !v.trow_leaf || !v.trow_l || !v.slot_owner || !v.slot_a || !v.owner_begin ||
        !v.owner_ptr || !v.ent_leaf || !v.ent_rows || !v.row_map)
        return fail(LBM_E_OOM, "lbm_mesh_hmatrix: device allocation failed");
    CK(cudaStreamSynchronize(ctx->stream));   // the host vectors go out of scope
    return LBM_OK;
}

int lbm_mesh_hmatrix(lbm_ctx* ctx, lbm_mesh mesh, double eps, double eta, int32_t n_min, int32_t threads,
                     int64_t info[4]) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M) return fail(LBM_E_INVALID, "lbm_mesh_hmatrix: unknown mesh");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    free_hm(M);
    if (eps <= 0.0) {   // back to the dense matrix
        if (info) info[0] = info[1] = info[2] = info[3] = 0;
        return LBM_OK;
    }
    if (!(eps < 1.0) || !(eta > 0.0) || !std::isfinite(eta) || n_min < 1 || threads < 1)
        return fail(LBM_E_INVALID, "lbm_mesh_hmatrix: eps must lie in (0, 1), eta be positive, n_min and threads at "
                    "least 1");
    // the surface as the mesh holds it: node coordinates (lattice units for a
    // Kuhn cube, the length unit for an upload), surface ids, triangles
    const int N = M->N, nb = M->nb, F = M->F;
    std::vector<double> xyz(3 * (size_t)N);
    if (M->gen) {
        CK(cudaMemcpy(xyz.data(), M->xyz, sizeof(double) * xyz.size(), cudaMemcpyDeviceToHost));
    } else {
        const int s = M->n + 1;
        for (int id = 0; id < N; ++id) {
            xyz[3 * (size_t)id] = id % s;
            xyz[3 * (size_t)id + 1] = (id / s) % s;
            xyz[3 * (size_t)id + 2] = id / (s * s);
        }
    }
    std::vector<int> bidx(nb), tris(3 * (size_t)F);
    CK(cudaMemcpy(bidx.data(), M->bidx, sizeof(int) * nb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(tris.data(), M->tris, sizeof(int) * tris.size(), cudaMemcpyDeviceToHost));
    HMatrixHost H, Ht;
    std::string why = host_hmatrix_build(N, xyz.data(), nb, bidx.data(), F, tris.data(), eta, n_min, eps, threads, H);
    if (!why.empty()) return fail(LBM_E_INVALID, "lbm_mesh_hmatrix: %s", why.c_str());
    host_hmatrix_transpose(H, Ht);
    HPacked Pf, Pa;
    why = host_hmatrix_pack(H, nb, Pf);
    if (why.empty()) why = host_hmatrix_pack(Ht, nb, Pa);
    if (!why.empty()) return fail(LBM_E_INVALID, "lbm_mesh_hmatrix: %s", why.c_str());
    M->hm = new HMDevice();
    int rc = hm_upload(ctx, M, Pf, M->hm->fwd);
    if (!rc) rc = hm_upload(ctx, M, Pa, M->hm->adj);
    int bmax = 1;
    for (auto& kv : ctx->insts)
        if (kv.second->mesh == mesh) bmax = std::max(bmax, kv.second->B);
    if (!rc) rc = hm_reserve(ctx, M, bmax);
    if (rc) {
        free_hm(M);
        return rc;
    }
    if (info) {
        int64_t low = 0;
        for (int k : H.kind) low += k;
        info[0] = (int64_t)H.data.size();
        info[1] = (int64_t)nb * nb;
        info[2] = (int64_t)H.kind.size();
        info[3] = low;
    }
    return LBM_OK;
    LBM_CATCH
}

int lbm_mesh_shell(lbm_ctx* ctx, lbm_mesh mesh, int32_t a, int32_t s, int64_t info[3]) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M) return fail(LBM_E_INVALID, "lbm_mesh_shell: unknown mesh");
    if (M->gen) return fail(LBM_E_INVALID, "lbm_mesh_shell: only Kuhn-cube meshes (lbm_mesh_create)");
    for (auto& kv : ctx->insts)
        if (kv.second->mesh == mesh)
            return fail(LBM_E_INVALID, "lbm_mesh_shell: the mesh has instances (attach or detach before creating them)");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    if (a == 0 && s == 0) {   // back to the FEM/BEM coupling
        free_shell(M);
        if (info) info[0] = info[1] = info[2] = 0;
        return LBM_OK;
    }
    if (a < 1 || s < 1) return fail(LBM_E_INVALID, "lbm_mesh_shell: a and s must be at least 1 (or both 0)");
    if ((int64_t)M->n + 2 * ((int64_t)a + s) > 200)
        return fail(LBM_E_INVALID, "lbm_mesh_shell: grid too large (n + 2(a + s) > 200)");
    ShellGrid G;
    const std::string why = host_shell_setup(M->n, a, s, 1.0, G);   // K in units of h
    if (!why.empty()) return fail(LBM_E_INVALID, "lbm_mesh_shell: %s", why.c_str());
    const int Ng = (int)(G.rowptr.size() - 1), nnz = (int)G.col.size(), n1 = G.nt + 1;
    // the per-row stencil records: every coupling of a row off the outer face
    // lies along one of the 14 Kuhn directions
    const int dir[15][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
                            {1, 1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1}, {1, 1, 1},
                            {-1, -1, -1}};
    std::vector<double> c64((size_t)Ng * 16, 0.0);
    std::vector<float> c32((size_t)Ng * 16, 0.0f);
    std::vector<unsigned char> kind(Ng, 1);
    std::vector<int> gnode(Ng, -1);
    for (int v : G.outer) kind[v] = 0;
    for (size_t i = 0; i < G.magnet.size(); ++i) gnode[G.magnet[i]] = (int)i;
    for (int r = 0; r < Ng; ++r) {
        if (kind[r] == 0) continue;
        double* c = c64.data() + (size_t)r * 16;
        const int ri = r % n1, rj = (r / n1) % n1, rk = r / (n1 * n1);
        for (int e = G.rowptr[r]; e < G.rowptr[r + 1]; ++e) {
            const int cidx = G.col[e];
            const int di = cidx % n1 - ri, dj = (cidx / n1) % n1 - rj, dk = cidx / (n1 * n1) - rk;
            int k = 0;
            while (k < 15 && !(dir[k][0] == di && dir[k][1] == dj && dir[k][2] == dk)) ++k;
            if (k == 15 || ri == 0 || rj == 0 || rk == 0 || ri == n1 - 1 || rj == n1 - 1 || rk == n1 - 1)
                return fail(LBM_E_INVALID, "lbm_mesh_shell: grid stiffness outside the Kuhn stencil");
            c[k] = 6.0 * G.K[e];
        }
        if (!(c[0] > 0.0)) return fail(LBM_E_INVALID, "lbm_mesh_shell: stiffness without a positive diagonal");
        c[15] = 1.0 / c[0];
        for (int k = 7; k < 15; ++k)
            if (c[k] != 0.0) kind[r] = 2;
    }
    for (size_t k = 0; k < c64.size(); ++k) c32[k] = (float)c64[k];
    free_shell(M);
    ShellDev* S = new ShellDev();
    M->shell = S;
    auto up = [&](const void* src, size_t bytes) -> void* {
        void* d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) return nullptr;
        M->shell_mem.push_back(d);
        if (cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) return nullptr;
        return d;
    };
    S->Ng = Ng;
    S->n1 = n1;
    S->coef64 = (const double*)up(c64.data(), sizeof(double) * c64.size());
    S->coef32 = (const float*)up(c32.data(), sizeof(float) * c32.size());
    S->kind = (const unsigned char*)up(kind.data(), kind.size());
    S->gnode = (const int*)up(gnode.data(), sizeof(int) * gnode.size());
    S->magnet = (const int*)up(G.magnet.data(), sizeof(int) * G.magnet.size());
    if (!S->coef64 || !S->coef32 || !S->kind || !S->gnode || !S->magnet) {
        free_shell(M);
        return fail(LBM_E_OOM, "lbm_mesh_shell: device allocation failed");
    }
    CK(cudaStreamSynchronize(ctx->stream));   // the host vectors go out of scope
    if (info) {
        info[0] = Ng;
        info[1] = nnz;
        info[2] = (int64_t)G.shell_tets;
    }
    return LBM_OK;
    LBM_CATCH
}

int lbm_bem_apply(lbm_ctx* ctx, lbm_mesh mesh, int32_t precision, int32_t batch, const double* x, double* y,
                  double* yt) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M || !x || batch < 1 || batch > 256 || (precision != LBM_FP64 && precision != LBM_MIXED))
        return fail(LBM_E_INVALID, "lbm_bem_apply: bad argument");
    CK(cudaSetDevice(ctx->device));
    if (int rc = hm_reserve(ctx, M, batch)) return rc;
    const int nb = M->nb, B = batch, C = 2 * B;
    const size_t tsize = precision == LBM_FP64 ? 8 : 4;
    const size_t S = (size_t)bem_df_splits(nb, B, ctx->num_sms);
    const size_t part = std::max((size_t)32 * nb, S * nb * C);
    std::vector<double> xin((size_t)nb * C);
    for (int q = 0; q < nb; ++q)
        for (int c = 0; c < B; ++c) xin[(size_t)q * C + c] = xin[(size_t)q * C + B + c] = x[(size_t)q * B + c];
    void *din = nullptr, *dout = nullptr, *dpart = nullptr;
    auto cleanup = [&]() {
        if (din) cudaFree(din);
        if (dout) cudaFree(dout);
        if (dpart) cudaFree(dpart);
    };
    if (cudaMalloc(&din, tsize * nb * C) != cudaSuccess || cudaMalloc(&dout, tsize * nb * C) != cudaSuccess ||
        cudaMalloc(&dpart, sizeof(double) * part) != cudaSuccess) {
        cleanup();
        return fail(LBM_E_OOM, "lbm_bem_apply: device allocation failed");
    }
    std::vector<float> xin32;
    if (tsize == 4) xin32.assign(xin.begin(), xin.end());
    const void* src = tsize == 8 ? (const void*)xin.data() : (const void*)xin32.data();
    cudaError_t e = cudaMemcpyAsync(din, src, tsize * nb * C, cudaMemcpyHostToDevice, ctx->stream);
    Launch L = ctx->launch();
    const MeshView mv = M->view();
    if (tsize == 8) {
        BatchView<double> V{};
        V.B = B;
        V.ub_in = (double*)din;
        V.ub_out = (double*)dout;
        V.bem_part = (double*)dpart;
        bem_product<double>(L, mv, V);
    } else {
        BatchView<float> V{};
        V.B = B;
        V.ub_in = (float*)din;
        V.ub_out = (float*)dout;
        V.bem_part = (float*)dpart;
        bem_product<float>(L, mv, V);
    }
    std::vector<double> out((size_t)nb * C);
    std::vector<float> out32(tsize == 4 ? (size_t)nb * C : 0);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tsize == 8 ? (void*)out.data() : (void*)out32.data(), dout, tsize * nb * C,
                            cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cleanup();
    if (e != cudaSuccess) return fail(LBM_E_CUDA, "lbm_bem_apply: %s", cudaGetErrorString(e));
    if (tsize == 4) out.assign(out32.begin(), out32.end());
    for (int q = 0; q < nb; ++q)
        for (int c = 0; c < B; ++c) {
            if (y) y[(size_t)q * B + c] = out[(size_t)q * C + c];
            if (yt) yt[(size_t)q * B + c] = out[(size_t)q * C + B + c];
        }
    return LBM_OK;
    LBM_CATCH
}

int lbm_instance_create(lbm_ctx* ctx, lbm_mesh mesh, int32_t batch, int32_t precision, lbm_inst* out) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M || !out) return fail(LBM_E_INVALID, "unknown mesh");
    if (batch < 1 || batch > 256) return fail(LBM_E_INVALID, "batch must be in [1, 256]");
    if (precision < LBM_FP64 || precision > LBM_MIXED_TC) return fail(LBM_E_INVALID, "unknown precision");
    CK(cudaSetDevice(ctx->device));
    Inst* I = new Inst();
    I->mesh = mesh;
    I->B = batch;
    I->precision = precision;
    I->tsize = precision == LBM_FP64 ? 8 : 4;
    const size_t vb = vec_bytes(*M, batch, precision == LBM_FP64 ? 8 : 4), pe = part_elems(ctx, batch);
    const size_t N = M->N;
#define CKI(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            free_inst(I);                                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_E_OOM : LBM_E_CUDA, "%s: %s", #call,   \
                        cudaGetErrorString(e_));                                                    \
        }                                                                                           \
    } while (0)
    CKI(cudaMalloc(&I->vec, vb));
    CKI(cudaMalloc(&I->part, pe * sizeof(double)));
    CKI(cudaMalloc(&I->st, sizeof(InstState) * batch));
    CKI(cudaMalloc(&I->ic, sizeof(InstConst) * batch));
    CKI(cudaMalloc(&I->staged, sizeof(double) * batch * N * 3));
    CKI(cudaMalloc(&I->staged_u, sizeof(double) * batch * N * 2));
    CKI(cudaMemsetAsync(I->vec, 0, vb, ctx->stream));
    CKI(cudaMemsetAsync(I->st, 0, sizeof(InstState) * batch, ctx->stream));
#undef CKI
    I->bytes = vb + pe * 8 + (sizeof(InstState) + sizeof(InstConst)) * batch + 40 * batch * N;
    if (precision == LBM_MIXED_TC && batch >= 2 && batch <= 64) {
        // tensor-core BEM products: padded B / B^T per mesh, split/partial scratch per instance
        const size_t pad = sizeof(float) * (size_t)M->nb * tc_ld(M->nb);
        if (!M->tcA) {
            if (cudaMalloc(&M->tcA, pad) != cudaSuccess || cudaMalloc(&M->tcAT, pad) != cudaSuccess) {
                if (M->tcA) cudaFree(M->tcA);
                M->tcA = M->tcAT = nullptr;
                free_inst(I);
                return fail(LBM_E_OOM, "tensor-core copies of the BEM matrix");
            }
            Launch L = ctx->launch();
            tc_prepare(L, M->B32, M->nb, M->tcA, M->tcAT);
            M->bytes += 2 * pad;
        }
        if (cudaMalloc(&I->tc_scratch, sizeof(float) * tc_scratch_floats(M->nb, batch, ctx->num_sms)) != cudaSuccess) {
            free_inst(I);
            return fail(LBM_E_OOM, "tensor-core scratch");
        }
        I->use_tc = true;
    }
    if (int rc = hm_reserve(ctx, M, batch)) {
        free_inst(I);
        return rc;
    }
    if (batch > 1 && !M->B32lo) {
        // the low FP32 part of the FP64 matrix, for the FP64-accurate batched
        // products of FP64 batches (the FP64 phase of mixed runs included)
        const size_t nb2 = (size_t)M->nb * M->nb;
        if (cudaMalloc(&M->B32lo, sizeof(float) * nb2) != cudaSuccess) {
            M->B32lo = nullptr;
            free_inst(I);
            return fail(LBM_E_OOM, "low part of the boundary matrix");
        }
        launch_bem_lo(M->B64, M->B32, M->B32lo, nb2, ctx->stream);
        ctx->launches += 1;
        M->bytes += sizeof(float) * nb2;
    }
    lbm_material nd = {1.61, 7.7e-12, 4.3e6, {0.0, 0.0, 1.0}};
    I->mats.assign(batch, nd);
    I->h.assign(3 * batch, 0.0);
    const int64_t id = ctx->next_id++;
    ctx->insts[id] = I;
    int rc = upload_consts(ctx, I, *M);
    if (rc) return rc;
    // m = +z everywhere
    std::vector<double> m0((size_t)batch * N * 3, 0.0);
    for (size_t k = 0; k < (size_t)batch * N; ++k) m0[3 * k + 2] = 1.0;
    rc = lbm_set_m(ctx, id, m0.data());
    if (rc) return rc;
    *out = id;
    return LBM_OK;
    LBM_CATCH
}

int lbm_instance_destroy(lbm_ctx* ctx, lbm_inst inst) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I) return fail(LBM_E_INVALID, "unknown instance");
    cudaStreamSynchronize(ctx->stream);
    free_inst(I);
    ctx->insts.erase(inst);
    return LBM_OK;
    LBM_CATCH
}

int lbm_set_material(lbm_ctx* ctx, lbm_inst inst, const lbm_material* mats) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !mats) return fail(LBM_E_INVALID, "bad argument");
    for (int b = 0; b < I->B; ++b)
        if (!(mats[b].Js > 0) || !(mats[b].A >= 0) || !isfinite(mats[b].K1))
            return fail(LBM_E_INVALID, "material %d: need Js > 0, A >= 0, finite K1", b);
    I->mats.assign(mats, mats + I->B);
    return upload_consts(ctx, I, *ctx->meshes[I->mesh]);
    LBM_CATCH
}

int lbm_set_field(lbm_ctx* ctx, lbm_inst inst, const double* h) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !h) return fail(LBM_E_INVALID, "bad argument");
    I->h.assign(h, h + 3 * I->B);
    return upload_consts(ctx, I, *ctx->meshes[I->mesh]);
    LBM_CATCH
}

int lbm_set_m(lbm_ctx* ctx, lbm_inst inst, const double* m) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !m) return fail(LBM_E_INVALID, "bad argument");
    Mesh& M = *ctx->meshes[I->mesh];
    Launch L = ctx->launch();
    StepOpts so{};
    reset_states(L, I->st, I->B, so, 1);
    if (int rc = zero_potentials(ctx, M, *I)) return rc;
    CK(cudaMemcpyAsync(I->staged, m, sizeof(double) * I->B * M.N * 3, cudaMemcpyHostToDevice, ctx->stream));
    if (I->tsize == 8) pack_m<double>(L, M.view(), batch_view<double>(ctx, M, *I, false), I->staged);
    else pack_m<float>(L, M.view(), batch_view<float>(ctx, M, *I, false), I->staged);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    return LBM_OK;
    LBM_CATCH
}

int lbm_set_m_device(lbm_ctx* ctx, lbm_inst inst, const double* d_m) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !d_m) return fail(LBM_E_INVALID, "bad argument");
    Mesh& M = *ctx->meshes[I->mesh];
    Launch L = ctx->launch();
    StepOpts so{};
    reset_states(L, I->st, I->B, so, 1);
    if (int rc = zero_potentials(ctx, M, *I)) return rc;
    if (I->tsize == 8) pack_m<double>(L, M.view(), batch_view<double>(ctx, M, *I, false), d_m);
    else pack_m<float>(L, M.view(), batch_view<float>(ctx, M, *I, false), d_m);
    CK(cudaGetLastError());
    return LBM_OK;
    LBM_CATCH
}

int lbm_profile_enable(lbm_ctx* ctx, int32_t on) {
    LBM_TRY
    if (!ctx) return fail(LBM_E_INVALID, "null context");
    ctx->prof = on != 0;
    return LBM_OK;
    LBM_CATCH
}

int lbm_profile_read(lbm_ctx* ctx, lbm_profile_stats* out, int32_t reset) {
    LBM_TRY
    if (!ctx || !out) return fail(LBM_E_INVALID, "null argument");
    CK(cudaStreamSynchronize(ctx->stream));
    prof_harvest(ctx);
    for (int k = 0; k < LBM_PROF_KINDS; ++k) {
        out->launches[k] = ctx->prof_launches[k];
        out->ms[k] = ctx->prof_ms[k];
    }
    out->cg_iters[0] = ctx->prof_cg[0];
    out->cg_iters[1] = ctx->prof_cg[1];
    unsigned long long sw[4];
    CK(cudaMemcpy(sw, ctx->sweeps, sizeof sw, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 4; ++k) out->cg_sweeps[k] = (int64_t)sw[k];
    if (reset) {
        CK(cudaMemsetAsync(ctx->sweeps, 0, sizeof sw, ctx->stream));
        for (int k = 0; k < LBM_PROF_KINDS; ++k) {
            ctx->prof_launches[k] = 0;
            ctx->prof_ms[k] = 0;
        }
        ctx->prof_cg[0] = ctx->prof_cg[1] = 0;
    }
    return LBM_OK;
    LBM_CATCH
}

int lbm_get_m(lbm_ctx* ctx, lbm_inst inst, double* m) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !m) return fail(LBM_E_INVALID, "bad argument");
    Mesh& M = *ctx->meshes[I->mesh];
    Launch L = ctx->launch();
    if (I->tsize == 8) unpack_m<double>(L, M.view(), batch_view<double>(ctx, M, *I, false), I->staged);
    else unpack_m<float>(L, M.view(), batch_view<float>(ctx, M, *I, false), I->staged);
    CK(cudaMemcpyAsync(m, I->staged, sizeof(double) * I->B * M.N * 3, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    return LBM_OK;
    LBM_CATCH
}

// ---- full instance state (checkpoint / resume) --------------------------------------
namespace {
constexpr int64_t STATE_MAGIC = 0x4554415453424c4cLL;   // "LLBSTATE"
constexpr int64_t STATE_VERSION = 1;
struct StateParts {
    size_t st, ic, mg, pot, shx, mats, hh, total;
};
StateParts state_parts(const Mesh& M, const Inst& I) {
    StateParts p;
    const size_t B = I.B, N = M.N;
    size_t o = 8 * sizeof(int64_t);
    auto take = [&o](size_t b) { const size_t at = o; o += (b + 7) & ~(size_t)7; return at; };
    p.st = take(sizeof(InstState) * B);
    p.ic = take(sizeof(InstConst) * B);
    p.mg = take(sizeof(double) * 2 * 2 * N * 3 * B);             // m[2] and grad phi[2]
    p.pot = take((size_t)I.tsize * 2 * N * 2 * B);                // U1, U2
    p.shx = take(M.shell ? sizeof(double) * M.shell->Ng * B : 0);  // grid potential
    p.mats = take(sizeof(lbm_material) * B);
    p.hh = take(sizeof(double) * 3 * B);
    p.total = o;
    return p;
}
}  // namespace

int lbm_get_state(lbm_ctx* ctx, lbm_inst inst, void* buf, int64_t* bytes) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !bytes) return fail(LBM_E_INVALID, "lbm_get_state: bad argument");
    const Mesh& M = *ctx->meshes[I->mesh];
    const StateParts p = state_parts(M, *I);
    if (!buf) {
        *bytes = (int64_t)p.total;
        return LBM_OK;
    }
    if (*bytes < (int64_t)p.total) return fail(LBM_E_INVALID, "lbm_get_state: buffer of %lld bytes, need %zu",
                                               (long long)*bytes, p.total);
    CK(cudaSetDevice(ctx->device));
    char* b = (char*)buf;
    const int64_t hdr[8] = {STATE_MAGIC, STATE_VERSION, M.N, I->B, I->tsize, M.shell ? M.shell->Ng : 0,
                            (int64_t)p.total, 0};
    memcpy(b, hdr, sizeof hdr);
    const VecLayout L = vec_layout(M, I->B, I->tsize);
    const size_t B = I->B, N = M.N;
    CK(cudaMemcpyAsync(b + p.st, I->st, sizeof(InstState) * B, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b + p.ic, I->ic, sizeof(InstConst) * B, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b + p.mg, (char*)I->vec + L.m, sizeof(double) * 2 * N * 3 * B, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(b + p.mg + sizeof(double) * 2 * N * 3 * B, (char*)I->vec + L.g, sizeof(double) * 2 * N * 3 * B,
                       cudaMemcpyDeviceToHost, ctx->stream));
    const size_t pb = (size_t)I->tsize * N * 2 * B;
    CK(cudaMemcpyAsync(b + p.pot, (char*)I->vec + L.U1, pb, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b + p.pot + pb, (char*)I->vec + L.U2, pb, cudaMemcpyDeviceToHost, ctx->stream));
    if (M.shell)
        CK(cudaMemcpyAsync(b + p.shx, (char*)I->vec + L.shx, sizeof(double) * M.shell->Ng * B, cudaMemcpyDeviceToHost,
                           ctx->stream));
    memcpy(b + p.mats, I->mats.data(), sizeof(lbm_material) * B);
    memcpy(b + p.hh, I->h.data(), sizeof(double) * 3 * B);
    CK(cudaStreamSynchronize(ctx->stream));
    *bytes = (int64_t)p.total;
    return LBM_OK;
    LBM_CATCH
}

int lbm_set_state(lbm_ctx* ctx, lbm_inst inst, const void* buf, int64_t bytes) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !buf) return fail(LBM_E_INVALID, "lbm_set_state: bad argument");
    const Mesh& M = *ctx->meshes[I->mesh];
    const StateParts p = state_parts(M, *I);
    const char* b = (const char*)buf;
    int64_t hdr[8];
    if (bytes < (int64_t)sizeof hdr) return fail(LBM_E_INVALID, "lbm_set_state: buffer too short");
    memcpy(hdr, b, sizeof hdr);
    if (hdr[0] != STATE_MAGIC || hdr[1] != STATE_VERSION)
        return fail(LBM_E_INVALID, "lbm_set_state: not a state written by lbm_get_state of this version");
    if (hdr[2] != M.N || hdr[3] != I->B || hdr[4] != I->tsize || hdr[5] != (M.shell ? M.shell->Ng : 0) ||
        hdr[6] != (int64_t)p.total || bytes < (int64_t)p.total)
        return fail(LBM_E_INVALID, "lbm_set_state: the state is of another mesh size, batch, precision or boundary");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    const VecLayout L = vec_layout(M, I->B, I->tsize);
    const size_t B = I->B, N = M.N;
    CK(cudaMemcpyAsync(I->st, b + p.st, sizeof(InstState) * B, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(I->ic, b + p.ic, sizeof(InstConst) * B, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync((char*)I->vec + L.m, b + p.mg, sizeof(double) * 2 * N * 3 * B, cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync((char*)I->vec + L.g, b + p.mg + sizeof(double) * 2 * N * 3 * B, sizeof(double) * 2 * N * 3 * B,
                       cudaMemcpyHostToDevice, ctx->stream));
    const size_t pb = (size_t)I->tsize * N * 2 * B;
    CK(cudaMemcpyAsync((char*)I->vec + L.U1, b + p.pot, pb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync((char*)I->vec + L.U2, b + p.pot + pb, pb, cudaMemcpyHostToDevice, ctx->stream));
    if (M.shell)
        CK(cudaMemcpyAsync((char*)I->vec + L.shx, b + p.shx, sizeof(double) * M.shell->Ng * B, cudaMemcpyHostToDevice,
                           ctx->stream));
    I->mats.assign((const lbm_material*)(b + p.mats), (const lbm_material*)(b + p.mats) + B);
    I->h.assign((const double*)(b + p.hh), (const double*)(b + p.hh) + 3 * B);
    CK(cudaStreamSynchronize(ctx->stream));   // the caller's buffer may go away
    return LBM_OK;
    LBM_CATCH
}

int lbm_evaluate(lbm_ctx* ctx, lbm_inst inst, const lbm_solve_opts* opt, double* h, double* u, lbm_result* res) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I) return fail(LBM_E_INVALID, "unknown instance");
    lbm_solve_opts o;
    if (opt) o = *opt; else lbm_default_opts(&o, I->precision);
    int rc = check_opts(o);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    return I->tsize == 8 ? run_minimise<double>(ctx, I, o, res, true, h, u)
                         : run_minimise<float>(ctx, I, o, res, true, h, u);
    LBM_CATCH
}

int lbm_energy(lbm_ctx* ctx, lbm_inst inst, double* e_terms) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !e_terms) return fail(LBM_E_INVALID, "lbm_energy: unknown instance or null output");
    lbm_solve_opts o;
    lbm_default_opts(&o, I->precision);
    std::vector<lbm_result> r(I->B);
    const int rc = lbm_evaluate(ctx, inst, &o, nullptr, nullptr, r.data());
    if (rc != LBM_OK) return rc;
    for (int b = 0; b < I->B; ++b)
        for (int k = 0; k < 5; ++k) e_terms[5 * b + k] = r[b].energy[k];
    return LBM_OK;
    LBM_CATCH
}

int lbm_minimise(lbm_ctx* ctx, lbm_inst inst, const lbm_solve_opts* opt, lbm_result* res) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I) return fail(LBM_E_INVALID, "unknown instance");
    lbm_solve_opts o;
    if (opt) o = *opt; else lbm_default_opts(&o, I->precision);
    int rc = check_opts(o);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    if (I->tsize == 8) return run_minimise<double>(ctx, I, o, res, false, nullptr, nullptr);
    if (o.resume) return fail(LBM_E_INVALID, "resume applies to LBM_FP64 instances (a mixed run has two batches)");
    return minimise_mixed(ctx, I, o, res);
    LBM_CATCH
}

int lbm_hysteresis(lbm_ctx* ctx, lbm_inst inst, const double dir[3], const double* fields, int32_t n_pts,
                   const lbm_solve_opts* opt, double* m_par, double* energy, lbm_result* res) {
    LBM_TRY
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !dir || !fields || n_pts < 0) return fail(LBM_E_INVALID, "bad argument");
    const double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(dn > 0)) return fail(LBM_E_INVALID, "zero field direction");
    const double d[3] = {dir[0] / dn, dir[1] / dn, dir[2] / dn};
    std::vector<double> h(3 * I->B);
    std::vector<lbm_result> r(I->B);
    for (int k = 0; k < n_pts; ++k) {
        for (int b = 0; b < I->B; ++b)
            for (int c = 0; c < 3; ++c) h[3 * b + c] = fields[k] * d[c];
        int rc = lbm_set_field(ctx, inst, h.data());
        if (rc) return rc;
        rc = lbm_minimise(ctx, inst, opt, r.data());
        if (rc) return rc;
        for (int b = 0; b < I->B; ++b) {
            if (m_par) m_par[(size_t)k * I->B + b] = r[b].mean_m[0] * d[0] + r[b].mean_m[1] * d[1] + r[b].mean_m[2] * d[2];
            if (energy) energy[(size_t)k * I->B + b] = r[b].energy[4];
            if (res) res[(size_t)k * I->B + b] = r[b];
        }
    }
    return LBM_OK;
    LBM_CATCH
}

}  // extern "C"

// ============================================================================
// Field evaluation without device allocation.
// ============================================================================
// Callers that cannot allocate device memory once they are running -- a host
// application that hands the library a fixed memory budget at start-up, code
// that runs while the CUDA allocator must not be touched (real-time loops, or a
// process whose allocations are all made up front) -- get one entry point that
// evaluates the energy, effective field and potentials of one magnetisation
// using only a fixed device array compiled into this library.
namespace {

constexpr size_t NOALLOC_MAX_NODES = 16384;     // cubes up to 24^3 cells (15 625 nodes)
constexpr size_t NOALLOC_MAX_SURFACE = 4096;    // surface nodes (24^3 cells: 3 458)
constexpr size_t NOALLOC_PART = 16384;          // per-block partial sums (doubles)
constexpr size_t NOALLOC_FIN = 4096;            // grid-reduction results (doubles)
// doubles: m, grad phi (2 x 3N each), field (3N), U1, U2, r, z, p, q (2N each),
// the divergence right-hand side (N), surface in/out (2 nb each), column-split
// partials (32 nb), partials, fin, plus state, constants and the barrier/error
// words (a few hundred bytes)
constexpr size_t NOALLOC_DOUBLES = 28 * NOALLOC_MAX_NODES + 36 * NOALLOC_MAX_SURFACE + NOALLOC_PART + NOALLOC_FIN + 1024;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};   // device address of the array, per device

__global__ void k_noalloc_setup(InstState* st, InstConst* ic, InstConst c) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    memset(st, 0, sizeof(InstState));
    st->phase = PH_INIT;
    st->status = 3;
    st->cur = 0;
    *ic = c;
}

// Energies of the evaluated point; a failed evaluation (a device wait that ran
// out: the error word; a non-finite field: status LBM_E_NAN) is made visible
// without a host round trip: NaN in every energy and in the first field value.
__global__ void k_noalloc_finish(const InstState* st, const InstConst* ic, const int* err, double* e, double* h0) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const bool bad = err[0] != 0 || st->status == 4;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (e) {
        for (int k = 0; k < 4; ++k) e[k] = bad ? nan : st->terms[k] * ic->Eunit;
        e[4] = bad ? nan : st->E * ic->Eunit;
    }
    if (h0 && bad) h0[0] = nan;
}

}  // namespace

extern "C" int lbm_evaluate_noalloc(lbm_ctx* ctx, lbm_mesh mesh, const lbm_material* mat, const double h_ext[3],
                                    const lbm_solve_opts* opt, const double* d_m, double* d_h, double* d_u,
                                    double* d_energy) {
    LBM_TRY
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M || !mat || !h_ext || !d_m) return fail(LBM_E_INVALID, "lbm_evaluate_noalloc: bad argument");
    if (M->shell)
        return fail(LBM_E_INVALID, "lbm_evaluate_noalloc: the mesh has a space-transformation boundary (its grid "
                    "vectors are not part of the static scratch)");
    if ((size_t)M->N > NOALLOC_MAX_NODES || (size_t)M->nb > NOALLOC_MAX_SURFACE)
        return fail(LBM_E_INVALID, "lbm_evaluate_noalloc: mesh of %d nodes / %d surface nodes exceeds the "
                    "static scratch (%zu nodes / %zu surface nodes)", M->N, M->nb, NOALLOC_MAX_NODES,
                    NOALLOC_MAX_SURFACE);
    if (!(mat->Js > 0)) return fail(LBM_E_INVALID, "lbm_evaluate_noalloc: Js must be positive");
    lbm_solve_opts o;
    if (opt) o = *opt; else lbm_default_opts(&o, LBM_FP64);
    int rc = check_opts(o);
    if (o.resume) return fail(LBM_E_INVALID, "lbm_hysteresis: resume is not supported (every field point starts anew)");
    if (rc) return rc;
    if (ctx->device < 0 || ctx->device >= 64) return fail(LBM_E_INVALID, "device index out of range");
    CK(cudaSetDevice(ctx->device));
    double* base;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[ctx->device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(LBM_E_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            g_noalloc_ptr[ctx->device] = (double*)p;
        }
        base = g_noalloc_ptr[ctx->device];
    }
    const size_t N = M->N, nb = M->nb;
    // carve the array (offsets in doubles, each region 256-byte aligned)
    size_t off = 0;
    auto take = [&](size_t n) { double* p = base + off; off += (n + 31) & ~(size_t)31; return p; };
    double* m = take(6 * N);
    double* g = take(6 * N);
    double* hout = take(3 * N);
    double* U1 = take(2 * N);
    double* U2 = take(2 * N);
    double* r = take(2 * N);
    double* z = take(2 * N);
    double* p = take(2 * N);
    double* q = take(2 * N);
    double* bv = take(N);
    double* ubi = take(2 * nb);
    double* ubo = take(2 * nb);
    double* bpart = take(32 * nb);
    double* part = take(NOALLOC_PART);
    double* fin = take(NOALLOC_FIN);
    InstState* st = (InstState*)take((sizeof(InstState) + 7) / 8);
    InstConst* ic = (InstConst*)take((sizeof(InstConst) + 7) / 8);
    unsigned* bar = (unsigned*)take(2);
    int* err = (int*)take(2);   // error word, wait limit, test hook (as the context's)
    unsigned long long* sweeps = (unsigned long long*)take(4);
    if (off > NOALLOC_DOUBLES) return fail(LBM_E_INVALID, "lbm_evaluate_noalloc: static scratch too small");
    const size_t need_part = (size_t)4 * ctx->num_sms * NQ > pcg_part_elems(ctx->num_sms, 1)
                                 ? (size_t)4 * ctx->num_sms * NQ : pcg_part_elems(ctx->num_sms, 1);
    if (need_part > NOALLOC_PART) return fail(LBM_E_INVALID, "lbm_evaluate_noalloc: too many SMs for the static scratch");
    cudaStream_t s = ctx->stream;
    // what must start at zero: the potentials (cold start), barrier, error word, counters
    CK(cudaMemsetAsync(U1, 0, sizeof(double) * 2 * N, s));
    CK(cudaMemsetAsync(U2, 0, sizeof(double) * 2 * N, s));
    CK(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
    CK(cudaMemsetAsync(err, 0, 4 * sizeof(int), s));
    CK(cudaMemcpyAsync(err + 1, ctx->err + 1, 2 * sizeof(int), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(sweeps, 0, 4 * sizeof(unsigned long long), s));
    CK(cudaMemcpyAsync(m, d_m, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
    const double Kd = mat->Js * mat->Js / (2.0 * MU0);
    double an = sqrt(mat->axis[0] * mat->axis[0] + mat->axis[1] * mat->axis[1] + mat->axis[2] * mat->axis[2]);
    if (!(an > 0)) an = 1.0;
    InstConst c;
    c.lam = mat->A / (Kd * M->cell * M->cell);
    c.Q = mat->K1 / Kd;
    for (int d = 0; d < 3; ++d) {
        c.a[d] = mat->axis[d] / an;
        c.hz[d] = h_ext[d] / mat->Js;
    }
    c.Eunit = Kd * M->cell * M->cell * M->cell;
    c.Js = mat->Js;
    k_noalloc_setup<<<1, 1, 0, s>>>(st, ic, c);
    ctx->launches += 1;
    BatchView<double> V;
    V.B = 1;
    V.m = m;
    V.H = g;
    V.hout = hout;
    V.U1 = U1;
    V.U2 = U2;
    V.r = r;
    V.z = z;
    V.p = p;
    V.q = q;
    V.ub_in = ubi;
    V.ub_out = ubo;
    V.bem_part = bpart;
    V.part = part;
    V.st = st;
    V.ic = ic;
    V.m32 = nullptr;   // FP64 evaluation: no FP32 copy of the trial point
    V.bvec = bv;
    Launch L{s, ctx->num_sms, bar, err, &ctx->launches, sweeps, fin, 0};
    L.tune = false;   // no waiting inside this call (and it may be captured)
    const MeshView mv = M->view();
    lbm_solve_opts oo = o;
    oo.max_iter = 0;
    const StepOpts so = step_opts(oo);
    trial_update<double>(L, mv, V);
    if (o.demag) {
        rhs_eval<double>(L, mv, V);
        int e = pcg_solve<double>(L, mv, V, 0, o.cg_tol, o.cg_max_iter, false);
        if (e) return fail(LBM_E_CUDA, "cooperative launch failed: %s", cudaGetErrorString((cudaError_t)e));
        bem_product<double>(L, mv, V);
        e = pcg_solve<double>(L, mv, V, 1, o.cg_tol, o.cg_max_iter, false);
        if (e) return fail(LBM_E_CUDA, "cooperative launch failed: %s", cudaGetErrorString((cudaError_t)e));
    }
    field_eval<double>(L, mv, V, o.demag);
    decide<double>(L, mv, V, so, field_blocks(L, mv, 1));
    if (d_h || d_u) unpack_field<double>(L, mv, V, d_h, d_u);
    if (d_energy || d_h) {
        k_noalloc_finish<<<1, 1, 0, s>>>(st, ic, err, d_energy, d_h);
        ctx->launches += 1;
    }
    CK(cudaGetLastError());
    return LBM_OK;
    LBM_CATCH
}

extern "C" int lbm_set_wait_limit(lbm_ctx* ctx, double seconds, int32_t unreachable) {
    LBM_TRY
    if (!ctx || !(seconds >= 0.0) || seconds > 60.0) return fail(LBM_E_INVALID, "lbm_set_wait_limit: bad argument");
    CK(cudaSetDevice(ctx->device));
    const int cfg[2] = {(int)llround(seconds * 1e3), unreachable ? 1 : 0};
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->err + 1, cfg, sizeof cfg, cudaMemcpyHostToDevice));
    return LBM_OK;
    LBM_CATCH
}



// ============================================================================
// Serving: continuous batching of minimisation requests.
// ============================================================================
namespace {

__global__ void k_slot_reset(InstState* st, int b, int phase) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    InstState& s = st[b];
    s.phase = phase;
    s.status = phase == PH_DONE ? 0 : 3;
    s.cur = 0;
    s.iters = s.evals = s.line_searches = s.backtracks = 0;
    s.nhist = s.hpos = s.ntau2 = 0;
    s.warm = 0;
    s.next_phase = PH_DONE;
    s.cg1 = s.cg2 = 0;
}

// slot d of the FP64 batch continues the step state (BB step, kappa, tau^2
// memory) of slot b of the FP32 batch after its first FP64 evaluation
__global__ void k_slot_warm(InstState* dst, int d, const InstState* src, int b) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    InstState& t = dst[d];
    const InstState& f = src[b];
    t.tau = f.tau;
    t.kappa = f.kappa;
    t.ntau2 = f.ntau2;
    for (int k = 0; k < MALPHA_MAX; ++k) t.tau2[k] = f.tau2[k];
    t.warm = 1;
}

__global__ void k_slots_done(InstState* st, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) { st[b].phase = PH_DONE; st[b].status = 0; st[b].cur = 0; }
}

// m of slot b (buffer 0) from a node-major [N][3] array
__global__ void k_slot_pack_m(const double* __restrict__ src, double* __restrict__ m, int N, int B, int b) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * N; t += gridDim.x * blockDim.x)
        m[(size_t)t * B + b] = src[t];
}

__global__ void k_slot_unpack_m(const double* __restrict__ m, const InstState* st, int N, int B, int b,
                                double* __restrict__ out) {
    const size_t off = (size_t)st[b].cur * N * 3 * B;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * N; t += gridDim.x * blockDim.x)
        out[t] = m[off + (size_t)t * B + b];
}

// zero the forward and adjoint potential columns of slot b (cold start)
template <typename T>
__global__ void k_slot_zero_pot(T* U1, T* U2, int N, int B, int b) {
    const int C = 2 * B;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        U1[(size_t)i * C + b] = T(0);
        U1[(size_t)i * C + B + b] = T(0);
        U2[(size_t)i * C + b] = T(0);
        U2[(size_t)i * C + B + b] = T(0);
    }
}

// column bd of a batch's space-transformation grid potential [Ng][Bd]: column
// bs of src ([Ng][Bs], the FP32 phase's potential: the FP64 phase's warm start),
// or zero (src null: a new magnetisation starts from zero)
__global__ void k_slot_shell(const double* __restrict__ src, int Bs, int bs, double* __restrict__ dst, int Bd, int bd,
                             int Ng) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Ng; i += gridDim.x * blockDim.x)
        dst[(size_t)i * Bd + bd] = src ? src[(size_t)i * Bs + bs] : 0.0;
}

// move slot bs of an FP32 batch to slot bd of an FP64 batch: m (base point)
// and the forward/adjoint potentials (widened), the FP64 phase's warm start
__global__ void k_slot_move(const double* __restrict__ ms, const InstState* sts, int Bs, int bs,
                            const float* __restrict__ U1s, const float* __restrict__ U2s, double* __restrict__ md,
                            int Bd, int bd, double* __restrict__ U1d, double* __restrict__ U2d, int N) {
    const size_t off = (size_t)sts[bs].cur * N * 3 * Bs;
    const int Cs = 2 * Bs, Cd = 2 * Bd;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * N; t += gridDim.x * blockDim.x)
        md[(size_t)t * Bd + bd] = ms[off + (size_t)t * Bs + bs];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        U1d[(size_t)i * Cd + bd] = (double)U1s[(size_t)i * Cs + bs];
        U1d[(size_t)i * Cd + Bd + bd] = (double)U1s[(size_t)i * Cs + Bs + bs];
        U2d[(size_t)i * Cd + bd] = (double)U2s[(size_t)i * Cs + bs];
        U2d[(size_t)i * Cd + Bd + bd] = (double)U2s[(size_t)i * Cs + Bs + bs];
    }
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Ticket {
    lbm_request req{};
    std::vector<double> m0, m_out;
    lbm_result res{};
    InstState s32{};
    bool has32 = false;
    int state = 0;            // 0 pending, 1 active, 2 done
    double t_submit = 0, t_done = 0;
};

struct Group {
    int n = 0;
    double cell = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // the current chunk's start and end on the group's stream
    InstState* pin = nullptr;          // page-locked staging of both batches' states (asynchronous copies)
    int64_t mesh_id = 0, i32_id = 0, i64_id = 0;
    Inst *I32 = nullptr, *I64 = nullptr;
    cudaStream_t stream = nullptr;
    unsigned* bar = nullptr;
    int* err = nullptr;
    double* fin = nullptr;
    unsigned long long* sweeps = nullptr;
    double* staged = nullptr;          // [N*3] device staging of one slot
    std::vector<int64_t> t32, t64;     // ticket of each slot (-1: free)
    std::vector<InstState> h32, h64;   // states read back each poll
    std::vector<char> fresh32, fresh64;
    bool ran32 = false, ran64 = false;  // a chunk of the batch ran (its set-up is done)
    double last_used = 0;
    size_t bytes = 0;
    int occupied() const {
        int k = 0;
        for (auto t : t32) k += t >= 0;
        for (auto t : t64) k += t >= 0;
        return k;
    }
};

struct Server {
    lbm_ctx* ctx = nullptr;
    lbm_serve_opts opt{};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    int worker_rc = LBM_OK;
    std::string worker_err;
    std::deque<int64_t> pending;
    std::map<int64_t, std::unique_ptr<Ticket>> tickets;   // stable storage; map guarded by mu
    int64_t next_ticket = 1;
    std::map<int, Group*> groups;
    int64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_stalls = 0, n_evicted = 0;
    std::vector<double> pinned_m;      // host staging
    cudaEvent_t t_ref = nullptr;       // device-time origin of the trace
    std::deque<std::array<double, 3>> trace;   // per chunk: cube size, start, end (ms)
};

Launch group_launch(lbm_ctx* ctx, Group& G, int max_blocks) {
    return Launch{G.stream, ctx->num_sms, G.bar, G.err, &ctx->launches, G.sweeps, G.fin, max_blocks};
}

void group_free(lbm_ctx* ctx, Group* G) {
    if (G->stream) cudaStreamSynchronize(G->stream);
    if (G->i32_id) lbm_instance_destroy(ctx, G->i32_id);
    if (G->i64_id) lbm_instance_destroy(ctx, G->i64_id);
    if (G->mesh_id) lbm_mesh_destroy(ctx, G->mesh_id);
    void* ptrs[] = {G->bar, G->err, G->fin, G->sweeps, G->staged};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (G->ev0) cudaEventDestroy(G->ev0);
    if (G->ev1) cudaEventDestroy(G->ev1);
    if (G->pin) cudaFreeHost(G->pin);
    if (G->stream) cudaStreamDestroy(G->stream);
    delete G;
}

size_t group_estimate(int n, int slots, int shell_a, int shell_s) {
    const size_t N = (size_t)(n + 1) * (n + 1) * (n + 1);
    const size_t nb = N - (size_t)(n > 1 ? (n - 1) * (n - 1) * (n - 1) : 0);
    size_t mesh = 12 * nb * nb + 100 * N;
    size_t per_slot = 8 * (2 * N * 3 * 2 + 3 * N) * 2 + (4 + 8) * (12 * N + 4 * nb) + 40 * N;
    if (shell_a > 0) {   // the grid's stencil records and, per slot, its six FP64 vectors in both batches
        const size_t g1 = (size_t)n + 2 * ((size_t)shell_a + shell_s) + 1, Ng = g1 * g1 * g1;
        mesh += (16 * 12 + 9) * Ng;
        per_slot += 2 * 6 * 8 * Ng;
    }
    return mesh + per_slot * slots + ((size_t)64 << 20);
}

// Create (or reuse) the group of cube size n, evicting idle groups when the
// device lacks memory.  Returns nullptr when the request must wait.
Group* group_get(Server& S, int n, double cell) {
    auto it = S.groups.find(n);
    if (it != S.groups.end()) return it->second;
    lbm_ctx* ctx = S.ctx;
    const size_t need = group_estimate(n, S.opt.slots, S.opt.shell_a, S.opt.shell_s);
    for (;;) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        if (fr > need + (size_t)(S.opt.mem_reserve * (double)tot)) break;
        Group* victim = nullptr;
        for (auto& kv : S.groups)
            if (kv.second->occupied() == 0 && (!victim || kv.second->last_used < victim->last_used)) victim = kv.second;
        if (!victim) return nullptr;
        S.groups.erase(victim->n);
        group_free(ctx, victim);
        S.n_evicted += 1;
    }
    Group* G = new Group();
    G->n = n;
    G->cell = cell;
    const int B = S.opt.slots;
    auto bad = [&](int rc) {
        (void)rc;
        group_free(ctx, G);
        return (Group*)nullptr;
    };
    if (cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking) != cudaSuccess) return bad(0);
    if (cudaEventCreate(&G->ev0) != cudaSuccess || cudaEventCreate(&G->ev1) != cudaSuccess) return bad(0);
    if (cudaMallocHost(&G->pin, sizeof(InstState) * 2 * (size_t)B) != cudaSuccess) return bad(0);
    if (cudaMalloc(&G->bar, 64) != cudaSuccess || cudaMalloc(&G->err, 64) != cudaSuccess ||
        cudaMalloc(&G->fin, sizeof(double) * 4096) != cudaSuccess || cudaMalloc(&G->sweeps, 64) != cudaSuccess)
        return bad(0);
    cudaMemset(G->bar, 0, 64);
    cudaMemset(G->err, 0, 64);
    cudaMemset(G->sweeps, 0, 64);
    if (lbm_mesh_cube(ctx, cell, n, &G->mesh_id) != LBM_OK) return bad(0);
    if (S.opt.shell_a > 0 && lbm_mesh_shell(ctx, G->mesh_id, S.opt.shell_a, S.opt.shell_s, nullptr) != LBM_OK)
        return bad(0);
    if (lbm_instance_create(ctx, G->mesh_id, B, LBM_MIXED, &G->i32_id) != LBM_OK) return bad(0);
    if (lbm_instance_create(ctx, G->mesh_id, B, LBM_FP64, &G->i64_id) != LBM_OK) return bad(0);
    G->I32 = ctx->insts[G->i32_id];
    G->I64 = ctx->insts[G->i64_id];
    const int N = ctx->meshes[G->mesh_id]->N;
    if (cudaMalloc(&G->staged, sizeof(double) * 3 * N) != cudaSuccess) return bad(0);
    k_slots_done<<<(B + 127) / 128, 128, 0, ctx->stream>>>(G->I32->st, B);
    k_slots_done<<<(B + 127) / 128, 128, 0, ctx->stream>>>(G->I64->st, B);
    ctx->launches += 2;
    cudaStreamSynchronize(ctx->stream);
    G->t32.assign(B, -1);
    G->t64.assign(B, -1);
    G->h32.assign(B, InstState{});
    G->h64.assign(B, InstState{});
    G->fresh32.assign(B, 0);
    G->fresh64.assign(B, 0);
    G->bytes = need;
    S.groups[n] = G;
    return G;
}

void set_slot_consts(Inst* I, int b, const lbm_material& mat, const double h[3], double cell, cudaStream_t st) {
    I->mats[b] = mat;
    for (int d = 0; d < 3; ++d) I->h[3 * b + d] = h[d];
    const double Kd = mat.Js * mat.Js / (2.0 * MU0);
    double an = sqrt(mat.axis[0] * mat.axis[0] + mat.axis[1] * mat.axis[1] + mat.axis[2] * mat.axis[2]);
    if (!(an > 0)) an = 1.0;
    InstConst c;
    c.lam = mat.A / (Kd * cell * cell);
    c.Q = mat.K1 / Kd;
    for (int d = 0; d < 3; ++d) {
        c.a[d] = mat.axis[d] / an;
        c.hz[d] = h[d] / mat.Js;
    }
    c.Eunit = Kd * cell * cell * cell;
    c.Js = mat.Js;
    cudaMemcpyAsync(I->ic + b, &c, sizeof c, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);   // c is a stack value
}

// Put ticket t into a free slot of the FP32 (mixed) or FP64 batch of G.
bool admit(Server& S, Group& G, int64_t t, Ticket& T) {
    lbm_ctx* ctx = S.ctx;
    const bool fp64 = T.req.precision == LBM_FP64;
    std::vector<int64_t>& slots = fp64 ? G.t64 : G.t32;
    int b = -1;
    for (int k = 0; k < (int)slots.size(); ++k)
        if (slots[k] < 0) { b = k; break; }
    if (b < 0) return false;
    Inst* I = fp64 ? G.I64 : G.I32;
    Mesh& M = *ctx->meshes[G.mesh_id];
    const int N = M.N, B = I->B;
    cudaMemcpyAsync(G.staged, T.m0.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice, G.stream);
    k_slot_reset<<<1, 1, 0, G.stream>>>(I->st, b, PH_INIT);
    k_slot_pack_m<<<64, 256, 0, G.stream>>>(G.staged, (double*)I->vec, N, B, b);
    if (fp64) {
        const VecLayout L = vec_layout(M, B, 8);
        k_slot_zero_pot<double><<<64, 256, 0, G.stream>>>((double*)((char*)I->vec + L.U1),
                                                          (double*)((char*)I->vec + L.U2), N, B, b);
    } else {
        const VecLayout L = vec_layout(M, B, 4);
        k_slot_zero_pot<float><<<64, 256, 0, G.stream>>>((float*)((char*)I->vec + L.U1),
                                                         (float*)((char*)I->vec + L.U2), N, B, b);
    }
    ctx->launches += 3;
    if (M.shell) {
        const VecLayout L = vec_layout(M, B, fp64 ? 8 : 4);
        k_slot_shell<<<64, 256, 0, G.stream>>>(nullptr, 0, 0, (double*)((char*)I->vec + L.shx), B, b, M.shell->Ng);
        ctx->launches += 1;
    }
    set_slot_consts(I, b, T.req.mat, T.req.h, G.cell, G.stream);
    slots[b] = t;
    (fp64 ? G.fresh64 : G.fresh32)[b] = 1;
    return true;
}

void complete(Server& S, Group& G, int b, const InstState& s, Ticket& T) {
    lbm_ctx* ctx = S.ctx;
    Mesh& M = *ctx->meshes[G.mesh_id];
    const int N = M.N;
    T.m_out.resize(3 * (size_t)N);
    double* d_out = G.staged;
    k_slot_unpack_m<<<64, 256, 0, G.stream>>>((const double*)G.I64->vec, G.I64->st, N, G.I64->B, b, d_out);
    ctx->launches += 1;
    cudaMemcpyAsync(T.m_out.data(), d_out, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, G.stream);
    cudaStreamSynchronize(G.stream);
    InstConst c;
    cudaMemcpy(&c, G.I64->ic + b, sizeof c, cudaMemcpyDeviceToHost);
    T.t_done = now_s();
    fill_result(s, c, T.res, 1e3 * (T.t_done - T.t_submit));
    if (T.has32) {
        T.res.iterations += T.s32.iters;
        T.res.evaluations += T.s32.evals;
        T.res.line_searches += T.s32.line_searches;
        T.res.cg_iters1 += T.s32.cg1;
        T.res.cg_iters2 += T.s32.cg2;
    }
    T.state = 2;
    S.n_completed += 1;
}

void fail_ticket(Server& S, Ticket& T, int status) {
    T.t_done = now_s();
    memset(&T.res, 0, sizeof T.res);
    T.res.status = status;
    T.res.wall_ms = 1e3 * (T.t_done - T.t_submit);
    T.state = 2;
    S.n_completed += 1;
}

void serve_loop(Server* Sp) {
    Server& S = *Sp;
    lbm_ctx* ctx = S.ctx;
    cudaSetDevice(ctx->device);
    const lbm_solve_opts o = S.opt.opt;
    lbm_solve_opts o1 = o;
    if (o.cg_tol_fp32 > 0) o1.cg_tol = o.cg_tol_fp32;
    o1.tol = o.tol > o.switch_tol ? o.tol : o.switch_tol;
    lbm_solve_opts o2 = o;
    o2.cg_tol = o.cg_tol_polish;
    o2.stall_iters = 0;
    o2.tol = POLISH_MARGIN * o.tol;   // as lbm_minimise's FP64 phase
    const StepOpts so1 = step_opts(o1), so2 = step_opts(o2);
    lbm_solve_opts o64 = o;        // plain FP64 requests
    for (;;) {
        // ---- admission (the queue lock is not held while meshes are built) ---
        std::vector<std::pair<int64_t, Ticket*>> todo;
        {
            std::unique_lock<std::mutex> lk(S.mu);
            if (S.stop) break;
            bool busy = false;
            for (auto& kv : S.groups) busy |= kv.second->occupied() > 0;
            if (!busy && S.pending.empty())
                S.cv_work.wait_for(lk, std::chrono::milliseconds(20));
            if (S.stop) break;
            for (int64_t t : S.pending) todo.emplace_back(t, S.tickets[t].get());
            S.pending.clear();
        }
        std::vector<int64_t> keep, admitted;
        int64_t stalls = 0;
        for (auto& it : todo) {
            Group* G = group_get(S, it.second->req.n, it.second->req.cell_m);
            if (!G) { stalls += 1; keep.push_back(it.first); continue; }
            if (admit(S, *G, it.first, *it.second)) admitted.push_back(it.first);
            else keep.push_back(it.first);
        }
        {
            std::lock_guard<std::mutex> lk(S.mu);
            for (auto it = keep.rbegin(); it != keep.rend(); ++it) S.pending.push_front(*it);
            for (int64_t t : admitted) S.tickets[t]->state = 1;
            S.n_admitted += (int64_t)admitted.size();
            S.n_stalls += stalls;
        }
        // ---- issue a chunk of iterations per group (each on its stream) ------
        std::vector<Group*> active;
        for (auto& kv : S.groups)
            if (kv.second->occupied() > 0) active.push_back(kv.second);
        const int maxb = S.opt.max_pcg_blocks;
        for (Group* G : active) {
            Launch L = group_launch(ctx, *G, maxb);
            L.pcg_kernel = o.pcg_kernel;
            Mesh& M = *ctx->meshes[G->mesh_id];
            G->last_used = now_s();
            bool any32 = false, any64 = false;
            for (int b = 0; b < (int)G->t32.size(); ++b) any32 |= G->t32[b] >= 0 && (G->fresh32[b] || G->h32[b].phase != PH_DONE);
            for (int b = 0; b < (int)G->t64.size(); ++b) any64 |= G->t64[b] >= 0 && (G->fresh64[b] || G->h64[b].phase != PH_DONE);
            // each batch's chunk is captured once as a graph (on the group's own
            // stream) and replayed; the first chunk of a batch runs uncaptured
            bool rep = false;
            cudaEventRecord(G->ev0, G->stream);
            if (any32) {
                BatchView<float> V = batch_view<float>(ctx, M, *G->I32, false);
                run_chunk<float>(ctx, L, M, G->I32, V, o1, so1, field_blocks(L, M.view(), G->I32->B), S.opt.chunk,
                                 !G->ran32, G->stream, &rep);
                G->ran32 = true;
            }
            if (any64) {
                BatchView<double> V = batch_view<double>(ctx, M, *G->I64, false);
                // FP64 batch: mixed requests finish with the polish options,
                // plain FP64 requests share them except for the BEM matrix
                run_chunk<double>(ctx, L, M, G->I64, V, o2, so2, field_blocks(L, M.view(), G->I64->B), S.opt.chunk,
                                  !G->ran64, G->stream, &rep);
                G->ran64 = true;
            }
            cudaEventRecord(G->ev1, G->stream);
            // page-locked staging: the copies stay asynchronous, so the next
            // group's chunk is queued while this one runs
            cudaMemcpyAsync(G->pin, G->I32->st, sizeof(InstState) * G->t32.size(), cudaMemcpyDeviceToHost, G->stream);
            cudaMemcpyAsync(G->pin + G->t32.size(), G->I64->st, sizeof(InstState) * G->t64.size(),
                            cudaMemcpyDeviceToHost, G->stream);
        }
        // ---- retire and move -----------------------------------------------
        std::lock_guard<std::mutex> lk(S.mu);
        for (Group* G : active) {
            cudaError_t e = cudaStreamSynchronize(G->stream);
            std::copy(G->pin, G->pin + G->t32.size(), G->h32.begin());
            std::copy(G->pin + G->t32.size(), G->pin + G->t32.size() + G->t64.size(), G->h64.begin());
            {   // the chunk's device-time interval, relative to the server's start
                float a = 0.f, b = 0.f;
                if (S.t_ref && cudaEventElapsedTime(&a, S.t_ref, G->ev0) == cudaSuccess &&
                    cudaEventElapsedTime(&b, S.t_ref, G->ev1) == cudaSuccess) {
                    S.trace.push_back({(double)G->n, (double)a, (double)b});
                    if (S.trace.size() > 100000) S.trace.pop_front();
                }
            }
            int errw = 0;
            cudaMemcpy(&errw, G->err, sizeof errw, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess || errw) {
                S.worker_rc = e != cudaSuccess ? LBM_E_CUDA : LBM_E_TIMEOUT;
                S.worker_err = e != cudaSuccess ? cudaGetErrorString(e) : "device wait ran out of time";
                cudaMemset(G->err, 0, sizeof(int));
            }
            std::fill(G->fresh32.begin(), G->fresh32.end(), 0);
            std::fill(G->fresh64.begin(), G->fresh64.end(), 0);
            Mesh& M = *ctx->meshes[G->mesh_id];
            for (int b = 0; b < (int)G->t64.size(); ++b) {
                const int64_t t = G->t64[b];
                if (t < 0 || G->h64[b].phase != PH_DONE) continue;
                complete(S, *G, b, G->h64[b], *S.tickets[t]);
                G->t64[b] = -1;
            }
            for (int b = 0; b < (int)G->t32.size(); ++b) {
                const int64_t t = G->t32[b];
                if (t < 0 || G->h32[b].phase != PH_DONE) continue;
                Ticket& T = *S.tickets[t];
                if (G->h32[b].status == 4) {   // non-finite: no FP64 phase
                    fail_ticket(S, T, LBM_E_NAN);
                    G->t32[b] = -1;
                    continue;
                }
                int d = -1;
                for (int k = 0; k < (int)G->t64.size(); ++k)
                    if (G->t64[k] < 0) { d = k; break; }
                if (d < 0) continue;      // parked until an FP64 slot frees up
                const VecLayout L32 = vec_layout(M, G->I32->B, 4), L64 = vec_layout(M, G->I64->B, 8);
                k_slot_reset<<<1, 1, 0, G->stream>>>(G->I64->st, d, PH_INIT);
                k_slot_move<<<64, 256, 0, G->stream>>>(
                    (const double*)G->I32->vec, G->I32->st, G->I32->B, b,
                    (const float*)((const char*)G->I32->vec + L32.U1), (const float*)((const char*)G->I32->vec + L32.U2),
                    (double*)G->I64->vec, G->I64->B, d, (double*)((char*)G->I64->vec + L64.U1),
                    (double*)((char*)G->I64->vec + L64.U2), M.N);
                k_slot_warm<<<1, 1, 0, G->stream>>>(G->I64->st, d, G->I32->st, b);
                ctx->launches += 3;
                if (M.shell) {
                    k_slot_shell<<<64, 256, 0, G->stream>>>((const double*)((const char*)G->I32->vec + L32.shx),
                                                            G->I32->B, b, (double*)((char*)G->I64->vec + L64.shx),
                                                            G->I64->B, d, M.shell->Ng);
                    ctx->launches += 1;
                }
                set_slot_consts(G->I64, d, G->I32->mats[b], &G->I32->h[3 * b], G->cell, G->stream);
                T.s32 = G->h32[b];
                T.has32 = true;
                G->t64[d] = t;
                G->fresh64[d] = 1;
                G->t32[b] = -1;
                k_slot_reset<<<1, 1, 0, G->stream>>>(G->I32->st, b, PH_DONE);
                ctx->launches += 1;
            }
            cudaStreamSynchronize(G->stream);
        }
        (void)o64;
        S.cv_done.notify_all();
    }
    S.cv_done.notify_all();
}

}  // namespace

extern "C" {

void lbm_default_serve_opts(lbm_serve_opts* o) {
    memset(o, 0, sizeof *o);
    o->slots = 16;
    o->chunk = 8;
    o->max_pcg_blocks = 0;
    o->mem_reserve = 0.05;
    lbm_default_opts(&o->opt, LBM_MIXED);
}

int lbm_serve_start(lbm_ctx* ctx, const lbm_serve_opts* opt) {
    LBM_TRY
    if (!ctx) return fail(LBM_E_INVALID, "null context");
    if (ctx->server) return fail(LBM_E_INVALID, "already serving");
    Server* S = new Server();
    S->ctx = ctx;
    if (opt) S->opt = *opt; else lbm_default_serve_opts(&S->opt);
    const bool shell_ok = (S->opt.shell_a == 0 && S->opt.shell_s == 0) || (S->opt.shell_a >= 1 && S->opt.shell_s >= 1);
    if (S->opt.slots < 1 || S->opt.slots > 256 || S->opt.chunk < 1 || !shell_ok) {
        delete S;
        return fail(LBM_E_INVALID, "invalid serve options");
    }
    if (S->opt.max_pcg_blocks <= 0) S->opt.max_pcg_blocks = ctx->num_sms / 4 > 0 ? ctx->num_sms / 4 : 1;
    int rc = check_opts(S->opt.opt);
    if (rc) { delete S; return rc; }
    CK(cudaSetDevice(ctx->device));
    if (cudaEventCreate(&S->t_ref) != cudaSuccess || cudaEventRecord(S->t_ref, ctx->stream) != cudaSuccess) {
        if (S->t_ref) cudaEventDestroy(S->t_ref);
        delete S;
        return fail(LBM_E_CUDA, "serving trace event");
    }
    ctx->server = S;
    S->worker = std::thread(serve_loop, S);
    return LBM_OK;
    LBM_CATCH
}

int lbm_submit(lbm_ctx* ctx, const lbm_request* req, lbm_ticket* out) {
    LBM_TRY
    if (!ctx || !ctx->server || !req || !out || !req->m0) return fail(LBM_E_INVALID, "bad argument or not serving");
    if (req->n < 1 || req->n > 96 || !(req->cell_m > 0) || !(req->mat.Js > 0) ||
        (req->precision != LBM_FP64 && req->precision != LBM_MIXED))
        return fail(LBM_E_INVALID, "invalid request");
    Server& S = *ctx->server;
    const size_t N = (size_t)(req->n + 1) * (req->n + 1) * (req->n + 1);
    const double t0 = now_s();
    std::unique_ptr<Ticket> T(new Ticket());
    T->req = *req;
    T->m0.assign(req->m0, req->m0 + 3 * N);
    T->req.m0 = nullptr;
    T->t_submit = t0;
    std::lock_guard<std::mutex> lk(S.mu);
    const int64_t t = S.next_ticket++;
    S.tickets[t] = std::move(T);
    S.pending.push_back(t);
    S.n_submitted += 1;
    *out = t;
    S.cv_work.notify_one();
    return LBM_OK;
    LBM_CATCH
}

int lbm_poll(lbm_ctx* ctx, lbm_ticket t, lbm_result* res, double* m_out) {
    LBM_TRY
    if (!ctx || !ctx->server) return fail(LBM_E_INVALID, "not serving");
    Server& S = *ctx->server;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.tickets.find(t);
    if (it == S.tickets.end()) return fail(LBM_E_INVALID, "unknown ticket");
    if (S.worker_rc != LBM_OK) return fail(S.worker_rc, "serving failed: %s", S.worker_err.c_str());
    const Ticket& T = *it->second;
    if (T.state != 2) return LBM_E_PENDING;
    if (res) *res = T.res;
    if (m_out && !T.m_out.empty()) memcpy(m_out, T.m_out.data(), sizeof(double) * T.m_out.size());
    return LBM_OK;
    LBM_CATCH
}

int lbm_wait(lbm_ctx* ctx, lbm_ticket t, double timeout_s, lbm_result* res, double* m_out) {
    LBM_TRY
    if (!ctx || !ctx->server) return fail(LBM_E_INVALID, "not serving");
    Server& S = *ctx->server;
    const double t_end = now_s() + timeout_s;
    for (;;) {
        int rc = lbm_poll(ctx, t, res, m_out);
        if (rc != LBM_E_PENDING) return rc;
        if (now_s() > t_end) return fail(LBM_E_TIMEOUT, "request %lld not finished", (long long)t);
        std::unique_lock<std::mutex> lk(S.mu);
        S.cv_done.wait_for(lk, std::chrono::milliseconds(5));
    }
    LBM_CATCH
}

int lbm_serve_stats(lbm_ctx* ctx, int64_t stats[8]) {
    LBM_TRY
    if (!ctx || !ctx->server || !stats) return fail(LBM_E_INVALID, "not serving");
    Server& S = *ctx->server;
    std::lock_guard<std::mutex> lk(S.mu);
    int64_t act = 0;
    for (auto& kv : S.groups) act += kv.second->occupied();
    stats[0] = S.n_submitted;
    stats[1] = S.n_admitted;
    stats[2] = S.n_completed;
    stats[3] = (int64_t)S.pending.size();
    stats[4] = act;
    stats[5] = (int64_t)S.groups.size();
    stats[6] = S.n_stalls;
    stats[7] = S.n_evicted;
    return LBM_OK;
    LBM_CATCH
}

int lbm_serve_stop(lbm_ctx* ctx) {
    LBM_TRY
    if (!ctx || !ctx->server) return fail(LBM_E_INVALID, "not serving");
    Server* S = ctx->server;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->groups) group_free(ctx, kv.second);
    S->groups.clear();
    if (S->t_ref) cudaEventDestroy(S->t_ref);
    ctx->server = nullptr;
    delete S;
    return LBM_OK;
    LBM_CATCH
}

int lbm_serve_trace(lbm_ctx* ctx, double* out, int64_t max, int64_t* n) {
    LBM_TRY
    if (!ctx || !ctx->server || !n || max < 0 || (max > 0 && !out)) return fail(LBM_E_INVALID, "bad argument or not serving");
    Server* S = ctx->server;
    std::lock_guard<std::mutex> lk(S->mu);
    const int64_t have = (int64_t)S->trace.size();
    const int64_t k = have < max ? have : max;
    for (int64_t i = 0; i < k; ++i)
        for (int c = 0; c < 3; ++c) out[3 * i + c] = S->trace[(size_t)(have - k + i)][c];
    *n = k;
    return LBM_OK;
    LBM_CATCH
}

}  // extern "C"
