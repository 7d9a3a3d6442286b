/*
 * lbm.h -- C ABI of the GB300 curvilinear steepest-descent micromagnetic minimiser.
 *
 * Method: Exl, Bance, Reichel, Schrefl, Stimming, Mauser, "LaBonte's method
 * revisited: An effective steepest descent method for micromagnetic energy
 * minimization" (arXiv:1309.5796).  Every entry point below names the passage
 * of the paper that defines what it computes.
 *
 * Conventions for every call:
 *   - The return value is a status code (LBM_OK = 0 or one of LBM_E_*).  No C++
 *     exception crosses this interface.  lbm_last_error() returns a
 *     thread-local message describing the last failure of this thread.
 *   - Host pointers are owned by the caller; the library copies what it needs
 *     and never keeps them.  Device memory is owned by the library (allocated
 *     at mesh/instance creation and freed by the matching destroy call or by
 *     lbm_destroy).
 *   - Units are SI.  Applied and effective fields are mu0*H in tesla; energies
 *     are in joule; lengths in metre.  Magnetisation arrays are unit vectors,
 *     node-major: m[(b*N + i)*3 + c] for instance b, node i, component c.
 *   - A context is bound to one CUDA device and one stream.  Calls on one
 *     context must not be made concurrently from several threads.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define LBM_OK               0
#define LBM_E_INVALID        1   /* bad argument or handle */
#define LBM_E_OOM            2   /* device or host allocation failed */
#define LBM_E_NOT_CONVERGED  3   /* iteration limit reached before the stop test */
#define LBM_E_NAN            4   /* non-finite energy or field */
#define LBM_E_TIMEOUT        5   /* a device-side wait ran out of time (kernel returned) */
#define LBM_E_LINESEARCH     6   /* the step-halving line search gave up */
#define LBM_E_CUDA           7   /* CUDA runtime error */
#define LBM_E_PENDING        8   /* lbm_poll: the request has not finished yet */

/* ---- precision modes ---------------------------------------------------------- */
#define LBM_FP64      0  /* every vector, field and reduction in FP64 */
#define LBM_MIXED     1  /* FP64 state m; FP32 potential solves and BEM
                            product (FP32 matrix) until max|m x h|/Js <
                            switch_tol, then an FP64 phase (FP64 BEM matrix and
                            arithmetic; FP64 solves, see cg_mixed_iter) to tol;
                            FP64 reductions (dots, energy differences, stop
                            test, CG residual norms) throughout */
#define LBM_MIXED_TC  2  /* as LBM_MIXED, with the FP32 phase's BEM products
                            on the tensor cores (3xTF32 split, FP32
                            accumulation) when batch > 1; the FP64 phase as in
                            LBM_MIXED */
#define LBM_MIXED_TF32 LBM_MIXED_TC   /* the same mode under its arithmetic's name */

typedef struct lbm_ctx lbm_ctx;
typedef int64_t lbm_mesh;   /* mesh handle (> 0) */
typedef int64_t lbm_inst;   /* instance-batch handle (> 0) */

/* Material of one instance (Sec. 3.1 uses Nd2Fe14B). */
typedef struct {
    double Js;        /* saturation polarisation mu0*Ms (T) */
    double A;         /* exchange constant (J/m) */
    double K1;        /* uniaxial anisotropy constant (J/m^3) */
    double axis[3];   /* easy axis (normalised by the library) */
} lbm_material;

/* Options of the minimiser (Sec. 2.3 step rules; Sec. 3.1 stop test). */
typedef struct {
    double  tol;            /* stop when max_i |m_i x h_i| / Js < tol */
    double  grad_tol;       /* > 0: stop when sum_i |g_i|^2 < grad_tol instead
                               (the paper's grad h^T grad h test, Sec. 3.1) */
    int32_t max_iter;       /* accepted steps per minimisation */
    double  cg_tol;         /* relative residual |r|/|b| of both potential solves */
    int32_t cg_max_iter;    /* iteration cap of each potential solve */
    double  c1;             /* Armijo constant of the line search */
    int32_t max_backtracks; /* step halvings before LBM_E_LINESEARCH */
    int32_t memory;         /* nonmonotone memory (20 in Sec. 2.3) */
    double  kappa0;         /* initial threshold of the adaptive BB1/BB2 rule */
    int32_t m_alpha;        /* memory of the BB2 values in that rule */
    double  tau_min, tau_max;
    int32_t demag;          /* 1: stray field on (default), 0: off */
    int32_t check_every;    /* host polls convergence every this many steps */
    double  switch_tol;     /* mixed precision: the FP32 phase runs until
                               max|m x h|/Js < switch_tol (or it stalls: its line
                               search gives up, or see stall_iters), then an FP64
                               phase finishes to tol */
    double  cg_tol_polish;  /* relative residual of the potential solves in the
                               FP64 phase of a mixed-precision run */
    int32_t cg_mixed_iter;  /* FP64 potential solves (LBM_FP64 runs and the FP64
                               phase of mixed runs): 1 = CG iterations in FP32 with
                               the FP64 residual recomputed whenever they have
                               reduced it 1e4-fold (restarted CG), the solve ending
                               on the FP64 residual test; 0 = plain FP64 PCG.
                               Default 1 for LBM_MIXED / LBM_MIXED_TC, 0 for
                               LBM_FP64 */
    int32_t bb_rule;        /* step length after the first step (Sec. 2.3): 0 the
                               adaptive BB rule (default), 1 BB1 = s.s/s.y,
                               2 BB2 = s.y/y.y, 3 BB1 and BB2 on alternate steps;
                               every rule restarts from 1/max|H| when s.y <= 0 */
    int32_t method;         /* 0 curvilinear steepest descent with BB steps and the
                               nonmonotone line search (Sec. 2, default); 1 LaBonte's
                               method (Sec. 1.2), all nodes at once: m_i <-
                               normalize((1 - omega) m_i + omega h_i/|h_i|), every
                               step accepted; omega < 1 under-, > 1 over-relaxation.
                               Not guaranteed to converge (exchange-coupled nodes
                               moved together oscillate unless omega is small) */
    double  omega;          /* LaBonte relaxation factor, 0 < omega <= 2 (default 1) */
    int32_t stall_iters;    /* a phase gives up (status LBM_E_NOT_CONVERGED) after this
                               many accepted steps without halving its smallest torque; the
                               FP32 phase of a mixed run then hands the instance to the
                               FP64 phase (which ignores it).  0 = never.  Default 200
                               for the mixed precisions, 0 for LBM_FP64 */
    int32_t pcg_kernel;     /* potential-solve kernel: 0 (default) chooses; 1 the
                               grid-wide kernel (one CTA for small work, else a
                               cooperative grid); 2 prefers one thread-block cluster
                               per group of systems (taken when the batch has a
                               multiple of 4, at least 16 instances, FP32 work vectors
                               and z of a cluster's systems fits its shared memory;
                               otherwise as 1).  0 takes 2 where it qualifies.
                               Results agree to rounding, not bit for bit */
    int32_t use_graphs;     /* 1 (default): each chunk of check_every iterations is
                               captured once as a CUDA graph (per batch, options and
                               mesh operators) and replayed; the first chunk of a solve
                               runs uncaptured.  0: kernels launched one by one.  The
                               same kernels run in the same order: the same bits */
    double  cg_tol_fp32;    /* relative residual of the potential solves in the FP32
                               phase of a mixed-precision minimisation (lbm_minimise,
                               lbm_hysteresis, served requests); 0: cg_tol.  The FP32
                               phase only brings the state to switch_tol, and the FP64
                               phase's solves (cg_tol_polish) fix the final accuracy,
                               so it can take a looser tolerance than an evaluation
                               (lbm_evaluate of a mixed instance uses cg_tol).
                               Default 3e-5 mixed, 0 FP64 */
    int32_t resume;         /* lbm_minimise of an LBM_FP64 instance: 1 continues from
                               the instance's current state (lbm_set_state, or an
                               earlier run) instead of starting anew: instances that
                               the iteration limit (or a stall) stopped continue
                               with the step they had prepared, counters and the
                               nonmonotone memory carry on, converged or failed
                               instances stay done; max_iter counts the iterations
                               of both runs.  A run stopped by max_iter = k and
                               resumed gives the same bits as one uninterrupted run.
                               0 (default): start anew.  LBM_E_INVALID for mixed
                               instances and lbm_hysteresis */
} lbm_solve_opts;

/* Per-instance outcome of a minimisation or an evaluation. */
typedef struct {
    int32_t status;         /* LBM_OK, LBM_E_NOT_CONVERGED, LBM_E_LINESEARCH, LBM_E_NAN */
    int32_t iterations;     /* accepted steps */
    int32_t evaluations;    /* energy-gradient evaluations (incl. the initial one) */
    int32_t line_searches;  /* times the line search was entered */
    int64_t cg_iters1;      /* total iterations of the Neumann (u1) solves */
    int64_t cg_iters2;      /* total iterations of the Dirichlet (u2) solves */
    double  energy[5];      /* exchange, anisotropy, Zeeman, stray field, total (J) */
    double  torque;         /* max_i |m_i x h_i| / Js at the final state */
    double  gg;             /* sum_i |g_i|^2 (units of Kd h^3) */
    double  mean_m[3];      /* volume-weighted mean magnetisation */
    double  wall_ms;        /* host wall time of the call (whole batch) */
} lbm_result;

/* Fill `o` with the defaults for `precision` (tol 1e-6, memory 20, c1 1e-4,
 * 30 halvings, kappa0 0.5, m_alpha 3, cg_tol 1e-13 FP64 / 1e-6 mixed,
 * switch_tol 1e-4, cg_tol_polish 1e-10, cg_mixed_iter 1 mixed / 0 FP64,
 * cg_tol_fp32 3e-5 mixed / 0 FP64, resume 0). */
void lbm_default_opts(lbm_solve_opts* o, int32_t precision);

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t
 * (NULL: the library creates its own non-blocking stream). */
int lbm_create(lbm_ctx** out, int32_t device, void* stream);
int lbm_destroy(lbm_ctx* ctx);
const char* lbm_last_error(void);

/* ---- meshes (Sec. 2.1: standard linear tetrahedral finite elements) ---------- */

/* Canonical Kuhn-split cube: n^3 cubic cells of edge `cell_m`, 6 tetrahedra per
 * cell, node (i,j,k) -> id i + (n+1)(j + (n+1)k).  Builds on the device the
 * CSR pattern, the integer stiffness/divergence/volume tables, the boundary
 * lists and the dense double-layer BEM matrix (FP64 and FP32).
 * 1 <= n <= 96.  Device memory: about 12*nb^2 + 17*nnz + 40*N bytes. */
int lbm_mesh_cube(lbm_ctx* ctx, double cell_m, int32_t n, lbm_mesh* out);

#define LBM_UPLOAD_MAX_NODES 8000000
#define LBM_UPLOAD_MAX_TETS  16000000

/* Any conforming tetrahedral mesh (Sec. 2.1 linear tetrahedral elements; the
 * paper's grain is such a mesh of a sphere, Sec. 3.1).
 *   xyz   HOST [n_nodes*3] node coordinates in metres (copied; caller keeps it)
 *   tets  HOST [n_tets*4]  node ids of each tetrahedron, any orientation (copied)
 * The library checks the ids, rejects degenerate tetrahedra, unused nodes and
 * faces shared by more than two tetrahedra (LBM_E_INVALID with a message), and
 * builds: the CSR pattern of the element adjacency (columns ascending), the
 * surface (faces of one tetrahedron, oriented outward), the surface node list
 * (ascending ids), the P1 stiffness, divergence coupling and lumped volumes in
 * FP64 on the device (each row summing its tetrahedra in ascending order), and
 * the dense double-layer BEM matrix (FP64 and FP32).  Reduced units use the
 * length unit L = (mean |6 x volume|)^(1/3) (the cell edge of a 6-tetrahedra
 * cube split).  4 <= n_nodes <= LBM_UPLOAD_MAX_NODES, n_tets <=
 * LBM_UPLOAD_MAX_TETS, at most 65534 surface nodes.  Device memory: about
 * 12*nb^2 + 100*nnz + 80*N + 16*T bytes. */
int lbm_mesh_upload(lbm_ctx* ctx, const double* xyz, int64_t n_nodes, const int32_t* tets,
                    int64_t n_tets, lbm_mesh* out);
int lbm_mesh_destroy(lbm_ctx* ctx, lbm_mesh mesh);

/* FP64 copies of the assembled P1 operators of any mesh (Sec. 2.1 finite element
 * discretisation), in SI units, on the CSR pattern of lbm_mesh_export (any
 * pointer may be NULL):
 *   K[nnz] int grad phi_i . grad phi_j (m), G[nnz*3] sum_e (vol_e/4) grad phi_i|_e
 *   (m^2), Gt[nnz*3] G_ji, V[N] lumped volumes (m^3), unit_m the length unit
 *   (the cell edge of a cube mesh, L of an uploaded one). */
int lbm_mesh_values(lbm_ctx* ctx, lbm_mesh mesh, double* K, double* G, double* Gt, double* V,
                    double* unit_m);

/* info[0..7] = N, nb, nnz, tets, boundary triangles, device bytes, n (0 for an
 * uploaded mesh), 0. */
int lbm_mesh_info(lbm_ctx* ctx, lbm_mesh mesh, int64_t info[8]);

/* Host copies of the assembled tables (any pointer may be NULL; the integer
 * tables kval, gval, gtval, vol exist for cube meshes only -- an uploaded mesh
 * rejects them with LBM_E_INVALID, use lbm_mesh_values):
 *   tets[T*4], rowptr[N+1], col[nnz] (node ids, boundary flag removed),
 *   kval[nnz] (K in units h/6), gval[nnz*3] (G_ij in units h^2/24),
 *   gtval[nnz*3] (G_ji), vol[N] (V in units h^3/24), bnd[nb] (ascending ids),
 *   tris[F*3] (outward surface triangles, node ids). */
int lbm_mesh_export(lbm_ctx* ctx, lbm_mesh mesh, int32_t* tets, int32_t* rowptr, int32_t* col,
                    int32_t* kval, int32_t* gval, int32_t* gtval, int32_t* vol, int32_t* bnd,
                    int32_t* tris);

/* Rows row0..row0+nrows-1 of the FP64 double-layer matrix B (nb columns each),
 * u2|S = B u1|S of the hybrid FEM/BEM open boundary (Sec. 3.1). */
int lbm_bem_rows(lbm_ctx* ctx, lbm_mesh mesh, int64_t row0, int64_t nrows, double* out);

/* Storage of the hierarchical (H-matrix) form of a mesh's double-layer matrix B
 * (Sec. 3.1 names hierarchical matrices for the boundary element method of the
 * comparison solver), built on the host without a GPU: the surface of the mesh
 * as lbm_mesh_upload finds it, its boundary nodes split by geometric bisection
 * into clusters of at most n_min, a block (rows tau, columns sigma) kept in low
 * rank when min(diam tau, diam sigma) <= eta dist(tau, sigma) (boxes of the
 * collocation points and of the hat functions' supports), each such block
 * approximated by adaptive cross approximation to the relative Frobenius
 * tolerance eps, checked at sampled entries and recompressed; the others keep
 * their exact entries.
 *   xyz, n_nodes, tets, n_tets  HOST, as for lbm_mesh_upload (copied; same checks)
 *   eps      0 < eps < 1;  eta > 0 (2 is a common choice);  n_min >= 1 (e.g. 16)
 *   threads  host threads (>= 1; the result does not depend on their number)
 *   out      HOST [4]: stored values, nb*nb (the dense matrix's), leaves, low-rank leaves
 * Returns LBM_OK, or LBM_E_INVALID with a message (bad mesh or parameters). */
int lbm_hmatrix_plan(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets, double eps,
                     double eta, int32_t n_min, int32_t threads, int64_t out[4]);

/* ---- instances (Eq. 1: min phi_t(m) s.t. |m| = 1) ----------------------------- */

/* A batch of `batch` independent problems on one mesh, solved together
 * (1 <= batch <= 256).  m starts at +z, fields at zero, potentials at zero. */
int lbm_instance_create(lbm_ctx* ctx, lbm_mesh mesh, int32_t batch, int32_t precision,
                        lbm_inst* out);
int lbm_instance_destroy(lbm_ctx* ctx, lbm_inst inst);
int lbm_set_material(lbm_ctx* ctx, lbm_inst inst, const lbm_material* mats /* [batch] */);
int lbm_set_field(lbm_ctx* ctx, lbm_inst inst, const double* h /* [batch*3], tesla */);
/* lbm_set_m / lbm_set_m_device also reset the instances' step state and set
 * their potentials to zero, so that the next solve depends only on its inputs
 * (a repeated solve gives the same bits). */
int lbm_set_m(lbm_ctx* ctx, lbm_inst inst, const double* m /* [batch*N*3] host */);
int lbm_get_m(lbm_ctx* ctx, lbm_inst inst, double* m /* [batch*N*3] host */);

/* Energy and effective field at the current m (Eq. 1 terms; h_eff of Sec. 2.2).
 * h (nullable): [batch*N*3] mu0*h_eff in tesla; u (nullable): [batch*2*N]
 * potentials u1, u2 in metres (U = Ms u).  res (nullable): [batch]. */
int lbm_evaluate(lbm_ctx* ctx, lbm_inst inst, const lbm_solve_opts* opt, double* h, double* u,
                 lbm_result* res);

/* The Eq. (1) energy terms of every instance at its current m, with the
 * instance precision's default solver options:
 *   e_terms HOST [batch*5] exchange, anisotropy, Zeeman, stray field, total (J). */
int lbm_energy(lbm_ctx* ctx, lbm_inst inst, double* e_terms);

/* Minimise every instance of the batch from its current m (Sec. 2.2-2.3).
 * res: [batch].  Returns LBM_OK when the call ran; per-instance outcomes are
 * in res[b].status. */
int lbm_minimise(lbm_ctx* ctx, lbm_inst inst, const lbm_solve_opts* opt, lbm_result* res);

/* Hysteresis branch (Sec. 1.1, 3.1): for k = 0..n_pts-1 set the applied field
 * of every instance to fields[k]*dir (tesla) and minimise, warm-started from
 * the previous point.  m_par[k*batch+b] = volume-weighted mean of m.dir,
 * energy[k*batch+b] = total energy (J); res (nullable): [n_pts*batch]. */
int lbm_hysteresis(lbm_ctx* ctx, lbm_inst inst, const double dir[3], const double* fields,
                   int32_t n_pts, const lbm_solve_opts* opt, double* m_par, double* energy,
                   lbm_result* res);

/* Same as lbm_set_m with a DEVICE pointer d_m (batch*N*3 doubles on the
 * context's device, same layout); no host copy.  The read is stream-ordered on
 * the context's stream. */
int lbm_set_m_device(lbm_ctx* ctx, lbm_inst inst, const double* d_m);

/* Number of kernels this context has launched so far. */
int lbm_launch_count(lbm_ctx* ctx, int64_t* count);

/* Per-kind device time of the minimiser's kernels, measured with CUDA events
 * recorded on the context's stream around every launch while enabled.
 * Kinds: 0 trial update (Eq. 8), 1 potential solves stage 1 (FP32),
 * 2 BEM products, 3 potential solves stage 2 (FP32), 4 field/energy/dot
 * products, 5 step decision, 6 and 7 stages 1 and 2 in FP64. */
#define LBM_PROF_KINDS 8
typedef struct {
    int64_t launches[LBM_PROF_KINDS];
    double  ms[LBM_PROF_KINDS];
    int64_t cg_iters[2];       /* potential-solve iterations summed over all systems
                                  (forward and adjoint of every instance): FP32, FP64 */
    int64_t cg_sweeps[4];      /* potential-solve iterations of the whole batch (each
                                  sweep advances every unconverged system): stage 1
                                  FP32, stage 2 FP32, stage 1 FP64, stage 2 FP64 */
} lbm_profile_stats;
int lbm_profile_enable(lbm_ctx* ctx, int32_t on);
int lbm_profile_read(lbm_ctx* ctx, lbm_profile_stats* out, int32_t reset);

/* ---- evaluation without device allocation ---------------------------------------
 * The paper has no counterpart to this call; it exists for callers that must not
 * allocate device memory while they run -- for example a host application that
 * reserves all of its GPU memory at start-up, or a time-critical loop in which
 * touching the CUDA allocator is not allowed.  It computes what lbm_evaluate
 * computes for one instance in FP64 (energy terms, effective field, forward
 * potentials at the given m) but keeps every intermediate vector in one
 * fixed device array built into the library (about 5.0 MB on every device that
 * loads it, held until the process exits).  It calls no cudaMalloc or cudaFree.
 *
 *   mesh      a mesh (lbm_mesh_cube or lbm_mesh_upload) with at most 16384
 *             nodes and 4096 surface nodes (cubes: n <= 24); larger meshes are
 *             rejected with LBM_E_INVALID and a message
 *   mat, h_ext, opt   as for an instance (opt may be NULL: FP64 defaults)
 *   d_m       DEVICE pointer, [N*3] unit vectors (node-major)
 *   d_h       DEVICE pointer or NULL, [N*3] mu0*h_eff in tesla
 *   d_u       DEVICE pointer or NULL, [2*N] potentials u1, u2 in metres
 *   d_energy  DEVICE pointer or NULL, [5] exchange, anisotropy, Zeeman,
 *             stray field, total (J)
 * The work is queued on the context's stream and the call returns without
 * waiting for it.  The first call on a device looks up the device address of
 * the fixed array (cudaGetSymbolAddress); make that first call before any
 * stream capture.  All calls share the array, and each call overwrites it
 * (the parts that must start from zero -- the potentials, counters and the
 * barrier word -- are cleared by every call): calls whose work overlaps on the
 * GPU, e.g. from two streams or two contexts on one device, race.
 * Failures inside the queued work cannot be returned by this call (it does
 * not wait): when a device wait ran out (LBM_E_TIMEOUT in the other calls) or
 * the field is not finite (LBM_E_NAN), all five energies in d_energy and
 * d_h[0] are set to NaN, so a caller that reads either sees the failure.  The
 * BEM product uses its default launch shape (never an autotuned one), so the
 * result does not depend on earlier calls. */
int lbm_evaluate_noalloc(lbm_ctx* ctx, lbm_mesh mesh, const lbm_material* mat, const double h_ext[3],
                         const lbm_solve_opts* opt, const double* d_m, double* d_h, double* d_u,
                         double* d_energy);

/* ---- hierarchical (H-matrix) boundary operator ------------------------------------
 * Sec. 3.1: the hybrid FEM/BEM boundary operator of the paper's LLG comparison
 * solver is accelerated by hierarchical matrices.  Builds B_H for the mesh's
 * surface on `threads` host threads (cluster tree by geometric bisection,
 * admissibility min(diam) <= eta * dist, leaves of at most n_min positions;
 * inadmissible leaves exact, admissible ones by adaptive cross approximation
 * to |A - U V|_F <= eps |A|_F, then recompressed), and its transpose; uploads
 * both (FP32 and FP64 values) and makes every BEM product of the mesh's
 * instances use them, u2_S = B_H u1_S and c_S = B_H^T t_S, in place of the
 * dense matrix (which stays allocated).  eps <= 0 returns the mesh to the
 * dense matrix.  info (nullable): [stored values, nb^2, leaves, low-rank
 * leaves].  Waits for the context's queued work.  Returns LBM_E_INVALID for a
 * bad argument (eps >= 1, eta <= 0, n_min or threads < 1), LBM_E_OOM when
 * device memory runs out. */
int lbm_mesh_hmatrix(lbm_ctx* ctx, lbm_mesh mesh, double eps, double eta, int32_t n_min, int32_t threads,
                     int64_t info[4]);

/* Open boundary by space transformation (Sec. 3.1: the paper's own
 * steepest-descent solver maps a shell onto the exterior instead of coupling
 * FEM with BEM).  Attaches to a Kuhn-cube mesh (lbm_mesh_create) one Kuhn grid
 * of spacing h over the magnet [0, n]^3, an air layer a cells deep and a shell
 * s cells deep (max-norm radii R1 = n/2 + a, R2 = R1 + s about the magnet's
 * centre); the shell is mapped onto everything outside R1 by
 * x' - c = g(rho)/rho (x - c), g = R1 (R2 - R1)/(R2 - rho), its tetrahedra carry
 * the tensor M = |det J| J^-1 J^-T of the map at their centroids, and the
 * potential vanishes on the outer face (the image of infinity).  From then on
 * every stray-field evaluation of the mesh's instances (minimise, evaluate,
 * serving; every precision) solves the one symmetric system K_grid u = b on
 * the grid (FP64 Jacobi-PCG on the device, cg_tol / cg_max_iter of the solve
 * options, warm-started from the instance's previous grid potential) instead
 * of the two Poisson solves and the boundary product; its iterations count as
 * cg_iters1 and its time as the first potential solve.  The field at the
 * magnet's nodes is the exact gradient field of the discrete stray-field
 * energy (b^T K_grid^-1 b)/2 of this truncated, transformed problem.
 * a = s = 0 detaches it (back to FEM/BEM).  Must be called while the mesh has
 * no instances (their vectors are sized by it).  lbm_evaluate_noalloc refuses
 * such a mesh.
 * info (nullable, int64[3]): grid nodes, stiffness entries, shell tetrahedra.
 * Builds the grid and its stiffness on the host (seconds for n + 2(a + s)
 * near 100), uploads it and waits.  Returns LBM_E_INVALID for a general mesh,
 * a mesh with instances, a or s < 1 (unless both 0), or n + 2(a + s) > 200;
 * LBM_E_OOM when device memory runs out. */
int lbm_mesh_shell(lbm_ctx* ctx, lbm_mesh mesh, int32_t a, int32_t s, int64_t info[3]);

/* The boundary operator of the mesh (dense, or the hierarchical form when
 * built) applied to `batch` host vectors, as the solver applies it (Sec. 3.1,
 * the a3 step): y = B x and yt = B^T x.  precision: LBM_FP64 (FP64 vectors and
 * matrix) or LBM_MIXED (FP32 vectors, the FP32 matrix or values).
 * x: [nb][batch] host, position-major (position = index into the ascending
 * surface node ids); y, yt (nullable): [nb][batch] host.  Allocates and frees
 * its device buffers; waits for the result.  The paper has no counterpart: it
 * serves tests and diagnostics of the product. */
int lbm_bem_apply(lbm_ctx* ctx, lbm_mesh mesh, int32_t precision, int32_t batch, const double* x, double* y,
                  double* yt);

/* CUDA-graph use of the context's solves: out[0] replays of captured chunks,
 * out[1] chunks captured, out[2] captures the driver refused (those chunks run
 * their kernels one by one).  The paper has no counterpart. */
int lbm_graph_stats(lbm_ctx* ctx, int64_t out[3]);

/* ---- checkpoint / resume ----------------------------------------------------
 * The full state of an instance batch (checkpoint and resume of a solve;
 * the paper has no counterpart): per instance the step state (phase, step
 * length, kappa, the tau^2 and energy memories, counters), constants, the
 * magnetisation and energy gradient at the base and trial points, the forward
 * and adjoint potentials (the warm starts of the next solves) and, with the
 * space-transformation boundary, the grid potential; materials and fields.
 * lbm_get_state: buf NULL -> *bytes = the size needed; else buf of *bytes
 * bytes (host, caller-owned) receives it.  lbm_set_state: a state of an
 * instance with the same mesh size, batch, precision and boundary; then
 * lbm_minimise with resume = 1 continues it bit for bit.  Both wait for the
 * context's queued work.  LBM_E_INVALID for a short buffer or a mismatched
 * state. */
int lbm_get_state(lbm_ctx* ctx, lbm_inst inst, void* buf, int64_t* bytes);
int lbm_set_state(lbm_ctx* ctx, lbm_inst inst, const void* buf, int64_t bytes);

/* ---- device waits ------------------------------------------------------------
 * Every device-side wait of this context's kernels (the grid barrier of the
 * cooperative potential solves) gives up after a time limit, sets the
 * context's error word and returns; the call that queued the work then
 * returns LBM_E_TIMEOUT and the context stays usable.  The paper has no
 * counterpart.  seconds: the limit (0 restores the default of 2 s; at most
 * 60).  unreachable != 0 is a test hook: every grid barrier then waits for one
 * arrival more than the grid makes, so each wait runs out after `seconds`
 * (no fault, no trap) -- it exercises the error path; pass 0 to clear it.
 * Waits for the queued work first.  Returns LBM_E_INVALID for a bad argument. */
int lbm_set_wait_limit(lbm_ctx* ctx, double seconds, int32_t unreachable);

/* ---- serving: continuous batching of minimisation requests ---------------------
 * A worker thread of the context owns the device while serving.  Requests
 * (a cube size, material, applied field and initial m) are admitted into free
 * slots of a per-cube-size group when device memory allows (groups are created
 * on demand and idle groups are evicted under memory pressure); every group
 * advances its active slots `chunk` iterations at a time on its own stream, so
 * the work of different groups overlaps on the device; finished slots are
 * retired and refilled from the queue.  Mixed-precision requests run their FP32
 * phase in an FP32 batch and move, on reaching switch_tol, to the group's FP64
 * batch (Sec. 2.2-2.3 iteration, same results as lbm_minimise).  Between
 * lbm_serve_start and lbm_serve_stop no other call may use the context except
 * lbm_submit, lbm_poll, lbm_wait, lbm_serve_stats and lbm_last_error. */
typedef int64_t lbm_ticket;

typedef struct {
    int32_t      n;          /* cells per side of the cube (1..96) */
    double       cell_m;     /* cell edge (m) */
    lbm_material mat;
    double       h[3];       /* applied field mu0*H (T) */
    const double* m0;        /* [N*3] initial m, host; copied by lbm_submit */
    int32_t      precision;  /* LBM_FP64 or LBM_MIXED */
} lbm_request;

typedef struct {
    int32_t slots;           /* batch width of each group (default 16) */
    int32_t chunk;           /* iterations issued per group between polls (default 8) */
    int32_t max_pcg_blocks;  /* cooperative grid cap per group (default 0: a quarter of the SMs) */
    double  mem_reserve;     /* fraction of device memory kept free (default 0.05) */
    lbm_solve_opts opt;      /* solve options of every request */
    int32_t shell_a;         /* > 0: every group's cube gets the space-transformation */
    int32_t shell_s;         /*   boundary with air shell_a and shell shell_s cells
                                (lbm_mesh_shell); default 0, 0: FEM/BEM */
} lbm_serve_opts;

void lbm_default_serve_opts(lbm_serve_opts* o);
int lbm_serve_start(lbm_ctx* ctx, const lbm_serve_opts* opt /* NULL: defaults */);
/* Device-time trace of the serving loop (the paper has no counterpart): per
 * chunk of iterations of a size group, its cube size and the chunk's start and
 * end in milliseconds since lbm_serve_start, from CUDA events on the group's
 * stream (so intervals of different groups that intersect ran concurrently on
 * the device).  out: [max][3] host; *n: entries written (the latest ones). */
int lbm_serve_trace(lbm_ctx* ctx, double* out, int64_t max, int64_t* n);
/* Queue a request; returns immediately with its ticket. */
int lbm_submit(lbm_ctx* ctx, const lbm_request* req, lbm_ticket* out);
/* LBM_OK and the result (res->wall_ms = submit-to-completion latency) when the
 * request finished, LBM_E_PENDING otherwise.  m_out (nullable): [N*3]. */
int lbm_poll(lbm_ctx* ctx, lbm_ticket t, lbm_result* res, double* m_out);
/* Block until the request finished (bounded by timeout_s; LBM_E_TIMEOUT after). */
int lbm_wait(lbm_ctx* ctx, lbm_ticket t, double timeout_s, lbm_result* res, double* m_out);
/* stats[0..7] = submitted, admitted, completed, pending, active slots, groups,
 * admission stalls (memory), groups evicted. */
int lbm_serve_stats(lbm_ctx* ctx, int64_t stats[8]);
int lbm_serve_stop(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
