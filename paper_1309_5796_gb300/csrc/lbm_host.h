// Host-side declarations of the kernel launchers of liblbm (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm {

// ---- mesh set-up (mesh.cu) -------------------------------------------------------
void host_boundary_topology(int n, std::vector<int>& tris, const std::vector<int>& bidx,
                            std::vector<int>& inc_ptr, std::vector<int>& inc_slot);
void launch_row_counts(int n, int* cnt, int* bflag, cudaStream_t st);
void launch_scan(const int* in, int* out, int count, cudaStream_t st);
void launch_assemble(int n, const int* rowptr, const int* bpos, int* col, int* pkA, int* pkB, int* node,
                     cudaStream_t st);
void launch_boundary_ids(int N, const int* bflag, const int* bpos, int* bidx, cudaStream_t st);
void launch_kcsr_count(int N, const int* rowptr, const int* pkA, int* cnt, cudaStream_t st);
void launch_kcsr_fill(int N, const int* rowptr, const int* col, const int* pkA, const int* kptr, int* kent,
                      cudaStream_t st);
void launch_tets(int n, int* tets, cudaStream_t st);
void launch_bem_assemble(int n, int nb, int F, const int* bidx, const int* tris, const int* inc_ptr,
                         const int* inc_slot, const double* xyz, double* scratch, int nblocks, double* B64,
                         float* B32, cudaStream_t st);
void host_incidence(int N, const std::vector<int>& tris, const std::vector<int>& bidx, std::vector<int>& inc_ptr,
                    std::vector<int>& inc_slot);

// general tetrahedral meshes
struct GeneralTopology {
    std::vector<int> nt_ptr, nt_idx;   // node -> tetrahedra (ascending)
    std::vector<int> rowptr, col;      // CSR pattern (columns ascending, no flags)
    std::vector<int> tris, bidx;       // outward surface triangles, surface node ids (ascending)
    std::vector<double> det;           // 6 x signed volume of every tetrahedron (input units)
    double L = 0.0;                    // length unit (mean |det|)^(1/3)
};
std::string host_general_topology(int N, int T, const int* tets, const double* xyz, GeneralTopology& g);
void launch_assemble_gen(int N, const double* xyz, const int* tets, const int* nt_ptr, const int* nt_idx,
                         const int* rowptr, const int* col, Dbl4* A64, float4* A32, Dbl4* Bt64,
                         float4* Bt32, double* Vn, double* d64, float* d32, cudaStream_t st);
void launch_kcsr_count_gen(int N, const int* rowptr, const Dbl4* A64, int* cnt, cudaStream_t st);
void launch_kcsr_fill_gen(int N, const int* rowptr, const int* col, const Dbl4* A64, const int* kptr, int* kent,
                          double* k64, float* k32, cudaStream_t st);

// ---- hierarchical form of the boundary matrix: host set-up (csrc/hpartition.cu) --------
struct HCluster {
    int begin = 0, size = 0;           // boundary positions HPartition::idx[begin, begin + size), ascending
    int child[2] = {-1, -1};           // cluster ids; -1 for a leaf cluster
    double lo_r[3], hi_r[3];           // bounding box of the collocation points
    double lo_c[3], hi_c[3];           // bounding box of the supports of the hat functions
};
struct HLeaf {
    int row, col;                      // cluster ids of the block (row cluster, column cluster)
    int low_rank;                      // 1: admissible (low-rank) leaf, 0: dense leaf
};
struct HPartition {
    std::vector<int> idx;              // the clusters' positions, concatenated
    std::vector<HCluster> clusters;    // [0] is the root; breadth-first, the two children together
    std::vector<HLeaf> leaves;         // leaves of the block tree, depth-first
};
// lo/hi (nb x 3): bounding box of the surface triangles around each boundary node.
void host_support_boxes(int N, const double* xyz, int nb, const int* bidx, int F, const int* tris, double* lo,
                        double* hi);
// Cluster tree and block-tree leaves; returns an empty string, or why the input was refused.
std::string host_hmatrix_partition(int nb, const double* pts, const double* slo, const double* shi, double eta,
                                   int n_min, HPartition& P);

// The leaves filled in (csrc/hbuild.cu): dense leaves hold their m x n entries
// (row-major); low-rank leaves U (m x k, row-major) followed by V (k x n, row-major).
struct HMatrixHost {
    HPartition P;
    std::vector<int> kind;             // per leaf: 0 dense, 1 low rank
    std::vector<int> rank;             // per leaf: k of a low-rank leaf, 0 otherwise
    std::vector<size_t> off;           // per leaf: offset of its values in data
    std::vector<double> data;
    int fallbacks = 0;                 // admissible leaves assembled exactly after failing the sampled check
};
// B_H of the surface (xyz: node coordinates, any length unit; bidx: surface nodes,
// ascending; tris: outward surface triangles) for tolerance eps, filled by `threads`
// host threads (the result does not depend on their number); an empty string, or
// why the input was refused.
std::string host_hmatrix_build(int N, const double* xyz, int nb, const int* bidx, int F, const int* tris, double eta,
                               int n_min, double eps, int threads, HMatrixHost& H);

// The operator packed for a device product (csrc/hpack.cu).
struct HPackedLeaf {
    int row_begin, m;                  // row cluster: idx[row_begin, row_begin + m)
    int col_begin, n;                  // column cluster: idx[col_begin, col_begin + n)
    int kind, rank;                    // 0 dense, 1 low rank (rank k)
    size_t val;                        // offset in values: m*n dense, or V (k x n) then U (m x k)
    size_t t_off;                      // low rank: offset of t = V x (k x B) in the first pass's output
};
struct HPackedEntry {
    int leaf;                          // packed leaf
    size_t rows;                       // offset in row_map of the owner's rows within the leaf's rows
};
struct HPacked {
    int nb = 0;
    std::vector<HPackedLeaf> leaves;   // dense first, then low rank, each by (rows, columns)
    std::vector<int> idx;              // cluster positions (as HPartition::idx)
    std::vector<float> values;
    std::vector<double> values64;      // the same values in FP64 (for FP64 products)
    size_t n_t = 0;                    // sum of the ranks (rows of the first pass's output)
    std::vector<int> owner_begin, owner_size;   // row owners (cluster-tree leaves): idx ranges
    std::vector<size_t> owner_ptr;     // [owners + 1]: their entries, in block-tree order
    std::vector<HPackedEntry> entries;
    std::vector<int> row_map;
};
std::string host_hmatrix_pack(const HMatrixHost& H, int nb, HPacked& P);
// The transpose of a built operator on the same cluster tree: every leaf's row
// and column clusters swapped, dense entries transposed, U V -> V^T U^T.
void host_hmatrix_transpose(const HMatrixHost& H, HMatrixHost& T);

// ---- device form of a packed hierarchical operator (uploaded by lbm_mesh_hmatrix) ----
struct HLeafDev {
    int row_begin, m, col_begin, n, kind, rank;
    long long val, t_off;
};
struct HMView {
    int nb = 0, nleaf = 0, n_t = 0;
    const HLeafDev* leaves = nullptr;
    const int* idx = nullptr;          // cluster positions -> boundary positions
    const float* v32 = nullptr;        // values (FP32 products)
    const double* v64 = nullptr;       // values (FP64 products)
    const int* trow_leaf = nullptr;    // per row of t: its low-rank leaf
    const int* trow_l = nullptr;       //   and its index within the leaf's rank
    const int* slot_owner = nullptr;   // per output row k in [0, nb), owners in order: its row owner
    const int* slot_a = nullptr;       //   and its index within the owner
    const int* owner_begin = nullptr;  // per owner: offset of its positions in idx
    const long long* owner_ptr = nullptr;   // [owners + 1] entries of each owner
    const int* ent_leaf = nullptr;     // per entry: packed leaf
    const long long* ent_rows = nullptr;    //   offset of the owner's local rows in row_map
    const int* row_map = nullptr;
};
// Both products of a mesh's BEM matrix in hierarchical form, y = B_H x (forward)
// and y = B_H^T x (adjoint), and the scratch of their first passes.
struct HMDevice {
    HMView fwd, adj;
    double* t = nullptr;               // first-pass outputs: [2][n_t][B] values of the vector type
    size_t t_bytes = 0;
};


// ---- open boundary by space transformation: host set-up (csrc/shell.cu) -------------
struct ShellGrid {
    int nt = 0;                        // cells a side of the grid (magnet + air + shell)
    double R1 = 0.0, R2 = 0.0;         // max-norm radii of the air box and the outer face (lattice units)
    std::vector<int> rowptr, col;      // CSR of the element adjacency, columns ascending
    std::vector<double> K;             // sum_e c_i^T M_e c_j / (6 |det_e|), SI (m)
    std::vector<int> outer;            // grid nodes on the outer face (Dirichlet u = 0), ascending
    std::vector<int> magnet;           // grid node of every magnet node (magnet's own numbering)
    size_t shell_tets = 0;             // tetrahedra whose centroid lies in the shell
};
std::string host_shell_setup(int n, int a, int s, double cell, ShellGrid& G);

// The grid's operator on the device (uploaded by lbm_mesh_shell), in the
// magnet's reduced units: 6 K / h (the magnet's integer stiffness where M = I),
// so that K_grid u = (1/4) Gint m gives u in units of h.  Every row off the
// outer face is an interior grid node, coupled only along the 14 Kuhn
// directions: per row a 16-value record {K_ii, the couplings along +x, -x, +y,
// -y, +z, -z, +(x+y), -(x+y), +(x+z), -(x+z), +(y+z), -(y+z), +(x+y+z),
// -(x+y+z), 1/K_ii} (zeros on the outer face).
struct ShellDev {
    int Ng = 0, n1 = 0;                // grid nodes, grid nodes a side
    const float* coef32 = nullptr;     // [Ng][16], rounded to FP32
    const double* coef64 = nullptr;    // [Ng][16]
    const unsigned char* kind = nullptr;   // Ng: 0 outer face, 1 seven-point row (M = I), 2 fifteen-point row
    const int* gnode = nullptr;        // Ng: -1, or the magnet's node at this grid node
    const int* magnet = nullptr;       // N: grid node of every magnet node
};

// ---- device view of one mesh --------------------------------------------------------
struct MeshView {
    int n, N, nb, nnz, F;
    const int* rowptr;   // N+1
    const int* col;      // nnz; bit 31 set when the column node lies on the surface
    const int* pkA;      // nnz; int8 x4 {Kint, Gint_x, Gint_y, Gint_z}
    const int* pkB;      // nnz; int8 x4 {Gint^T_x, Gint^T_y, Gint^T_z, 0}
    const int* node;     // N;   Vint | Kint_ii << 8 | (boundary position + 1) << 16
    const int* kptr;     // N+1; stiffness-only CSR (nonzero Kint entries)
    const int* kent;     // nnzK; (column << 8) | (Kint & 0xff)
    const int* bidx;     // nb;  boundary node ids, ascending
    const double* B64;   // nb x nb row-major
    const float* B32;    // nb x nb row-major
    const float* B32lo;  // nb x nb: fp32(B64 - B32), for the FP64-accurate batched product (null: not built)
    const HMDevice* hm = nullptr;   // host pointer: the hierarchical form, when built (lbm_mesh_hmatrix)
    const ShellDev* shell = nullptr;   // host pointer: the space-transformation boundary, when attached
    double vsum;         // sum_i Vint_i = 24 n^3 (general meshes: sum of gV)
    double cell;         // cell edge h (m); general meshes: the length unit L
    // General meshes (gen != 0): the same tables as FP64/FP32 values in the same
    // units (K: L/6, G: L^2/24, V: L^3/24); node[] then holds only the surface
    // position, and kent's low byte only marks an entry.
    int gen;
    const Dbl4* gA64; const float4* gA32;   // nnz  {K, G_x, G_y, G_z}
    const Dbl4* gB64; const float4* gB32;   // nnz  {G^T_x, G^T_y, G^T_z, 0}
    const double* gk64; const float* gk32;     // nnzK values of the stiffness-only CSR
    const double* gV;                          // N    lumped volumes
    const double* gd64; const float* gd32;     // N    K_ii (Jacobi preconditioner)
};

// ---- device view of one instance batch (node-major, instance-minor) ------------------
template <typename T>
struct BatchView {
    int B;
    double* m;   // [2][N][3][B]   m[cur] = base point, m[1-cur] = trial (FP64 in every mode)
    double* H;   // [2][N][3][B]   grad phi at the same points (FP64)
    // Potentials of the forward FEM/BEM chain (u = X b) and of its adjoint
    // (uT = X^T b), solved side by side: column c < B belongs to instance c
    // (forward), column B + b to instance b (adjoint).
    T* U1;       // [N][2B]  stage 1: u1 (Neumann) | w (Dirichlet, zero surface values)
    T* U2;       // [N][2B]  stage 2: u2 (Dirichlet, surface values B u1) | uT (Neumann)
    T* r; T* z; T* p; T* q;    // [N][2B] PCG work vectors
    T* ub_in;    // [nb][2B] BEM input:  u1 on the surface | t = b_S - K_SI w
    T* ub_out;   // [nb][2B] BEM output: B u1_S | B^T t
    T* bem_part; // column-split partial sums of the transposed product (scratch)
    double* part;              // partial sums, >= maxblocks * B * NQ
    InstState* st;             // [B]
    const InstConst* ic;       // [B]
    double* hout;              // optional [N][3][B] effective field (nullable)
    float* m32 = nullptr;      // FP32 batches: [N][3][B] FP32 copy of the trial point (else null)
    double* bvec = nullptr;    // [N][B] divergence right-hand side b = G m at the trial point (rhs_eval)
    double* shx = nullptr;     // [6][Ng][B] FP64 grid potential and five CG work vectors (space-transformation boundary)
};

struct Launch {
    cudaStream_t stream;
    int num_sms;
    unsigned* bar;     // grid-barrier counter (device)
    int* err;          // device error word
    int64_t* launches; // host counter of kernel launches
    unsigned long long* sweeps;  // device counters [4]: batched PCG iterations per stage and precision
    double* fin;                 // device scratch for grid reductions (>= 4 * 512 doubles)
    int max_blocks;              // cap on the cooperative PCG grid (0: one block per SM)
    bool tune = true;            // launch-shape autotuning allowed (it waits on events)
    int pcg_kernel = 0;          // 0 choose, 1 grid-wide kernel, 2 prefer clusters (lbm_solve_opts)
    // host flags [B]: the instances iterating at the start of the chunk (null: all);
    // the cluster potential solves size their launch to the groups still active
    const unsigned char* active = nullptr;
};
// The shape the cluster potential solves take for this launch (CPC * 100 + CL;
// 0: the grid-wide kernel), from the active flags of L.
int pcg_cluster_shape(const Launch& L, const MeshView& M, int B, bool fp64, bool mixed_iter);

// u2_S = B_H u1_S and c_S = B_H^T t_S on the [nb][2B] surface arrays (forward
// columns [0, B), adjoint columns [B, 2B)) with the hierarchical form of B
template <typename T>
void hm_product(const Launch& L, const HMDevice& H, const T* x, T* y, int B);
// The potential by the space-transformation boundary (shell_solve.cu): K_grid u
// = b on the grid for every active instance (Jacobi-PCG on the FP64 grid
// potential, warm-started from V.shx; CG iterations in FP32 for FP32 batches and
// with mixed_iter, plain FP64 otherwise), then U1 = u, U2 = (0 | u) at the
// magnet's nodes; 0 or a CUDA error.
template <typename T>
int shell_solve(const Launch& L, const MeshView& M, const BatchView<T>& V, double tol, int max_iter,
                bool mixed_iter);
// Thread-block-cluster variant of the potential solves (pcg_cluster.cu): 1 when
// launched (*err its status), 0 when the batch does not qualify.
template <typename T>
int pcg_solve_cluster(const Launch& L, const MeshView& M, const BatchView<T>& V, int mode, double tol, int max_iter,
                      bool mixed_iter, cudaError_t* err);
template <typename T>
int pcg_solve(const Launch& L, const MeshView& M, const BatchView<T>& V, int mode, double tol, int max_iter,
              bool mixed_iter);
template <typename T>
void bem_product(const Launch& L, const MeshView& M, const BatchView<T>& V);
// b = G m at every active instance's trial point into V.bvec (before the potential solves)
template <typename T>
void rhs_eval(const Launch& L, const MeshView& M, const BatchView<T>& V);
template <typename T>
void field_eval(const Launch& L, const MeshView& M, const BatchView<T>& V, int demag);
template <typename T>
void trial_update(const Launch& L, const MeshView& M, const BatchView<T>& V);
template <typename T>
void decide(const Launch& L, const MeshView& M, const BatchView<T>& V, const StepOpts& so, int nblk_field);
template <typename T>
void pack_m(const Launch& L, const MeshView& M, const BatchView<T>& V, const double* staged);
template <typename T>
void unpack_m(const Launch& L, const MeshView& M, const BatchView<T>& V, double* staged);
template <typename T>
void unpack_field(const Launch& L, const MeshView& M, const BatchView<T>& V, double* staged_h,
                  double* staged_u);
// warm: keep each instance's step state (tau, kappa, tau^2 memory) for the
// first step after the first evaluation (a new precision phase at the same point)
void reset_states(const Launch& L, InstState* st, int B, const StepOpts& so, int set_cur0, int warm = 0);
// continue the instances stopped by the iteration limit or a stall (resume)
void resume_states(const Launch& L, InstState* st, int B);

// ---- tensor-core BEM products (tc_gemm.cu) ------------------------------------------
int tc_ld(int nb);
size_t tc_scratch_floats(int nb, int B, int num_sms);
void tc_prepare(const Launch& L, const float* B32, int nb, float* A, float* AT);
template <typename T>
int bem_product_tc(const Launch& L, int nb, const float* A32, const float* A32T, const T* ub_in, T* ub_out, int B,
                   float* scratch);
int field_blocks(const Launch& L, const MeshView& M, int B);
// FP64-accurate batched BEM product on the FP32 units: K-split count and the
// doubles of its partial-sum scratch (S * nb * 2B)
int bem_df_splits(int nb, int B, int num_sms);
// B_lo = fp32(B64 - B32) (nb x nb)
void launch_bem_lo(const double* B64, const float* B32, float* B32lo, size_t n, cudaStream_t st);
size_t pcg_part_elems(int num_sms, int B);

// Kernel attributes are per device: set a kernel's dynamic shared-memory limit
// once per (kernel, current device), under a lock (several host threads may
// launch); with `blocks_per_sm` also return the kernel's occupancy at `threads`
// threads and `smem` bytes, cached the same way.
cudaError_t kernel_smem_attr(const void* fn, int smem_limit, int threads = 0, size_t smem = 0,
                             int* blocks_per_sm = nullptr);

}  // namespace lbm
