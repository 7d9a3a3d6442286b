// C ABI of liblbm: contexts, meshes, instance batches, and the host loop that
// drives the device-resident minimiser (Sec. 2.2-2.3) and the hysteresis
// continuation (Sec. 1.1, 3.1).  Every decision of the iteration (step length,
// acceptance, line search, stop test) is taken on the device; the host only
// enqueues kernels and polls the instance phases every `check_every` steps.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <map>
#include <string>
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

struct Mesh {
    int n = 0, N = 0, nb = 0, nnz = 0, F = 0, T = 0;
    double cell = 0;
    int *rowptr = nullptr, *col = nullptr, *pkA = nullptr, *pkB = nullptr, *node = nullptr, *bidx = nullptr;
    int *tris = nullptr, *inc_ptr = nullptr, *inc_slot = nullptr;
    int *kptr = nullptr, *kent = nullptr;
    int nnzK = 0;
    double* B64 = nullptr;
    float* B32 = nullptr;
    size_t bytes = 0;
    MeshView view() const {
        MeshView v;
        v.n = n; v.N = N; v.nb = nb; v.nnz = nnz; v.F = F;
        v.rowptr = rowptr; v.col = col; v.pkA = pkA; v.pkB = pkB; v.node = node; v.bidx = bidx;
        v.kptr = kptr; v.kent = kent;
        v.B64 = B64; v.B32 = B32;
        v.vsum = 24.0 * (double)n * n * n;
        v.cell = cell;
        return v;
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
    bool bem32 = false;            // BEM product with the FP32 matrix (FP64 phase of mixed runs)
    std::vector<lbm_material> mats;
    std::vector<double> h;         // B*3 tesla
    size_t bytes = 0;
};

}  // namespace

struct ProfEvent {
    int kind;
    cudaEvent_t a, b;
};

struct lbm_ctx {
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
    Launch launch() { return Launch{stream, num_sms, bar, err, &launches, sweeps, fin}; }
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

// Brackets one launch of `kind` with events on the context's stream.
struct ProfScope {
    lbm_ctx* ctx;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(lbm_ctx* c, int k) : ctx(c), kind(k) {
        if (ctx->prof) {
            a = pool_get(ctx);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~ProfScope() {
        if (a) {
            cudaEvent_t b = pool_get(ctx);
            cudaEventRecord(b, ctx->stream);
            ctx->ev_live.push_back(ProfEvent{kind, a, b});
        }
    }
};

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
    size_t m, g, hout, U1, U2, r, z, p, q, ub_in, ub_out, bem_part, total;
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
    L.bem_part = take(8 * 32 * nb);
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
    v.part = I.part;
    v.st = I.st;
    v.ic = I.ic;
    return v;
}

size_t vec_bytes(const Mesh& M, int B, int tsize) { return vec_layout(M, B, tsize).total; }

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

void free_mesh(Mesh* m) {
    void* ptrs[] = {m->rowptr, m->col, m->pkA, m->pkB, m->node, m->bidx, m->tris, m->inc_ptr, m->inc_slot,
                    m->kptr, m->kent, m->B64, m->B32};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

void free_inst(Inst* I) {
    if (I->polish) free_inst(I->polish);
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
    return s;
}

int check_opts(const lbm_solve_opts& o) {
    if (!(o.tol >= 0) || o.max_iter < 0 || o.memory < 1 || o.memory > HIST_MAX || o.m_alpha < 1 ||
        o.m_alpha > MALPHA_MAX || o.max_backtracks < 0 || o.cg_max_iter < 1 || !(o.cg_tol > 0) ||
        o.check_every < 1 || !(o.tau_min > 0) || !(o.tau_max >= o.tau_min) || !(o.switch_tol >= 0) ||
        !(o.cg_tol_polish > 0))
        return fail(LBM_E_INVALID, "invalid solve options");
    return LBM_OK;
}

// One field evaluation of every active instance at its trial point.
template <typename T>
int eval_trial(lbm_ctx* ctx, const Mesh& M, const Inst& I, const BatchView<T>& V, const lbm_solve_opts& o) {
    Launch L = ctx->launch();
    MeshView mv = M.view();
    if (o.demag) {
        int e;
        const int k64 = sizeof(T) == 8 ? 5 : 0;
        {
            ProfScope ps(ctx, 1 + k64);
            e = pcg_solve<T>(L, mv, V, 0, o.cg_tol, o.cg_max_iter, nullptr);
        }
        if (e) return fail(LBM_E_CUDA, "cooperative launch failed: %s", cudaGetErrorString((cudaError_t)e));
        {
            ProfScope ps(ctx, 2);
            bem_product<T>(L, mv, V, I.bem32);
        }
        {
            ProfScope ps(ctx, 3 + (k64 ? 4 : 0));
            e = pcg_solve<T>(L, mv, V, 1, o.cg_tol, o.cg_max_iter, nullptr);
        }
        if (e) return fail(LBM_E_CUDA, "cooperative launch failed: %s", cudaGetErrorString((cudaError_t)e));
    }
    {
        ProfScope ps(ctx, 4);
        field_eval<T>(L, mv, V, o.demag);
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
                 double* hout, double* uout, std::vector<InstState>* states_out = nullptr) {
    Mesh& M = *ctx->meshes[I->mesh];
    const auto t0 = std::chrono::steady_clock::now();
    BatchView<T> V = batch_view<T>(ctx, M, *I, evaluate_only && hout);
    Launch L = ctx->launch();
    MeshView mv = M.view();
    lbm_solve_opts oo = o;
    if (evaluate_only) oo.max_iter = 0;
    const StepOpts so = step_opts(oo);
    reset_states(L, I->st, I->B, so, 0);
    const int nblk_field = field_blocks(L, mv, I->B);
    std::vector<InstState> hs(I->B);
    const int64_t max_loops = (int64_t)(oo.max_iter + 1) * (oo.max_backtracks + 2) + 2;
    int64_t loops = 0;
    int rc = LBM_OK;
    while (true) {
        const int chunk = evaluate_only ? 1 : oo.check_every;
        for (int k = 0; k < chunk; ++k) {
            {
                ProfScope ps(ctx, 0);
                trial_update<T>(L, mv, V);
            }
            int e = eval_trial<T>(ctx, M, *I, V, oo);
            if (e) return e;
            ProfScope ps(ctx, 5);
            decide<T>(L, mv, V, so, nblk_field);
        }
        loops += chunk;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hs.data(), I->st, sizeof(InstState) * I->B, cudaMemcpyDeviceToHost, ctx->stream));
        int errw = 0;
        CK(cudaMemcpyAsync(&errw, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        prof_harvest(ctx);
        if (errw) {
            cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream);
            return fail(LBM_E_TIMEOUT, "a device-side wait ran out of time (error word %d)", errw);
        }
        bool all = true;
        for (int b = 0; b < I->B; ++b) all &= hs[b].phase == PH_DONE;
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
    o1.tol = o.tol > o.switch_tol ? o.tol : o.switch_tol;
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
            P->bem32 = true;
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
        lbm_solve_opts o2 = o;
        o2.cg_tol = o.cg_tol_polish;
        rc = run_minimise<double>(ctx, P, o2, nullptr, false, nullptr, nullptr, &s2);
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
    if (precision != LBM_FP64) o->cg_tol = 1e-6;
}

const char* lbm_last_error(void) { return g_err.c_str(); }

int lbm_create(lbm_ctx** out, int32_t device, void* stream) {
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
}

int lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return LBM_OK;
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
    delete ctx;
    return LBM_OK;
}

int lbm_launch_count(lbm_ctx* ctx, int64_t* count) {
    if (!ctx || !count) return fail(LBM_E_INVALID, "null argument");
    *count = ctx->launches;
    return LBM_OK;
}

int lbm_mesh_cube(lbm_ctx* ctx, double cell_m, int32_t n, lbm_mesh* out) {
    if (!ctx || !out || n < 1 || n > 96 || !(cell_m > 0)) return fail(LBM_E_INVALID, "lbm_mesh_cube: bad argument");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    Mesh* M = new Mesh();
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
    launch_bem_assemble(n, M->nb, M->F, M->bidx, M->tris, M->inc_ptr, M->inc_slot, scratch, nblocks, M->B64,
                        M->B32, st);
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
}

int lbm_mesh_destroy(lbm_ctx* ctx, lbm_mesh mesh) {
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M) return fail(LBM_E_INVALID, "unknown mesh");
    for (auto& kv : ctx->insts)
        if (kv.second->mesh == mesh) return fail(LBM_E_INVALID, "mesh still has instances");
    cudaStreamSynchronize(ctx->stream);
    free_mesh(M);
    ctx->meshes.erase(mesh);
    return LBM_OK;
}

int lbm_mesh_info(lbm_ctx* ctx, lbm_mesh mesh, int64_t info[8]) {
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
}

int lbm_mesh_export(lbm_ctx* ctx, lbm_mesh mesh, int32_t* tets, int32_t* rowptr, int32_t* col, int32_t* kval,
                    int32_t* gval, int32_t* gtval, int32_t* vol, int32_t* bnd, int32_t* tris) {
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M) return fail(LBM_E_INVALID, "unknown mesh");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    if (tets) {
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
    CK(cudaMemcpyAsync(a.data(), M->pkA, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(b.data(), M->pkB, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost, st));
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
}

int lbm_bem_rows(lbm_ctx* ctx, lbm_mesh mesh, int64_t row0, int64_t nrows, double* out) {
    Mesh* M = ctx ? get_mesh(ctx, mesh) : nullptr;
    if (!M || !out || row0 < 0 || nrows < 0 || row0 + nrows > M->nb) return fail(LBM_E_INVALID, "bad rows");
    CK(cudaMemcpyAsync(out, M->B64 + (size_t)row0 * M->nb, sizeof(double) * nrows * M->nb,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

int lbm_instance_create(lbm_ctx* ctx, lbm_mesh mesh, int32_t batch, int32_t precision, lbm_inst* out) {
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
}

int lbm_instance_destroy(lbm_ctx* ctx, lbm_inst inst) {
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I) return fail(LBM_E_INVALID, "unknown instance");
    cudaStreamSynchronize(ctx->stream);
    free_inst(I);
    ctx->insts.erase(inst);
    return LBM_OK;
}

int lbm_set_material(lbm_ctx* ctx, lbm_inst inst, const lbm_material* mats) {
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !mats) return fail(LBM_E_INVALID, "bad argument");
    for (int b = 0; b < I->B; ++b)
        if (!(mats[b].Js > 0) || !(mats[b].A >= 0) || !isfinite(mats[b].K1))
            return fail(LBM_E_INVALID, "material %d: need Js > 0, A >= 0, finite K1", b);
    I->mats.assign(mats, mats + I->B);
    return upload_consts(ctx, I, *ctx->meshes[I->mesh]);
}

int lbm_set_field(lbm_ctx* ctx, lbm_inst inst, const double* h) {
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !h) return fail(LBM_E_INVALID, "bad argument");
    I->h.assign(h, h + 3 * I->B);
    return upload_consts(ctx, I, *ctx->meshes[I->mesh]);
}

int lbm_set_m(lbm_ctx* ctx, lbm_inst inst, const double* m) {
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !m) return fail(LBM_E_INVALID, "bad argument");
    Mesh& M = *ctx->meshes[I->mesh];
    Launch L = ctx->launch();
    StepOpts so{};
    reset_states(L, I->st, I->B, so, 1);
    CK(cudaMemcpyAsync(I->staged, m, sizeof(double) * I->B * M.N * 3, cudaMemcpyHostToDevice, ctx->stream));
    if (I->tsize == 8) pack_m<double>(L, M.view(), batch_view<double>(ctx, M, *I, false), I->staged);
    else pack_m<float>(L, M.view(), batch_view<float>(ctx, M, *I, false), I->staged);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    return LBM_OK;
}

int lbm_set_m_device(lbm_ctx* ctx, lbm_inst inst, const double* d_m) {
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I || !d_m) return fail(LBM_E_INVALID, "bad argument");
    Mesh& M = *ctx->meshes[I->mesh];
    Launch L = ctx->launch();
    StepOpts so{};
    reset_states(L, I->st, I->B, so, 1);
    if (I->tsize == 8) pack_m<double>(L, M.view(), batch_view<double>(ctx, M, *I, false), d_m);
    else pack_m<float>(L, M.view(), batch_view<float>(ctx, M, *I, false), d_m);
    CK(cudaGetLastError());
    return LBM_OK;
}

int lbm_profile_enable(lbm_ctx* ctx, int32_t on) {
    if (!ctx) return fail(LBM_E_INVALID, "null context");
    ctx->prof = on != 0;
    return LBM_OK;
}

int lbm_profile_read(lbm_ctx* ctx, lbm_profile_stats* out, int32_t reset) {
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
}

int lbm_get_m(lbm_ctx* ctx, lbm_inst inst, double* m) {
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
}

int lbm_evaluate(lbm_ctx* ctx, lbm_inst inst, const lbm_solve_opts* opt, double* h, double* u, lbm_result* res) {
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I) return fail(LBM_E_INVALID, "unknown instance");
    lbm_solve_opts o;
    if (opt) o = *opt; else lbm_default_opts(&o, I->precision);
    int rc = check_opts(o);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    return I->tsize == 8 ? run_minimise<double>(ctx, I, o, res, true, h, u)
                         : run_minimise<float>(ctx, I, o, res, true, h, u);
}

int lbm_minimise(lbm_ctx* ctx, lbm_inst inst, const lbm_solve_opts* opt, lbm_result* res) {
    Inst* I = ctx ? get_inst(ctx, inst) : nullptr;
    if (!I) return fail(LBM_E_INVALID, "unknown instance");
    lbm_solve_opts o;
    if (opt) o = *opt; else lbm_default_opts(&o, I->precision);
    int rc = check_opts(o);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    if (I->tsize == 8) return run_minimise<double>(ctx, I, o, res, false, nullptr, nullptr);
    return minimise_mixed(ctx, I, o, res);
}

int lbm_hysteresis(lbm_ctx* ctx, lbm_inst inst, const double dir[3], const double* fields, int32_t n_pts,
                   const lbm_solve_opts* opt, double* m_par, double* energy, lbm_result* res) {
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
}

}  // extern "C"
