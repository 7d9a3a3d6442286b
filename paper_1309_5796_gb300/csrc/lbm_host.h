// Host-side declarations of the kernel launchers of liblbm (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
void launch_tets(int n, int* tets, cudaStream_t st);
void launch_bem_assemble(int n, int nb, int F, const int* bidx, const int* tris, const int* inc_ptr,
                         const int* inc_slot, double* scratch, int nblocks, double* B64, float* B32,
                         cudaStream_t st);

// ---- device view of one mesh --------------------------------------------------------
struct MeshView {
    int n, N, nb, nnz, F;
    const int* rowptr;   // N+1
    const int* col;      // nnz; bit 31 set when the column node lies on the surface
    const int* pkA;      // nnz; int8 x4 {Kint, Gint_x, Gint_y, Gint_z}
    const int* pkB;      // nnz; int8 x4 {Gint^T_x, Gint^T_y, Gint^T_z, 0}
    const int* node;     // N;   Vint | Kint_ii << 8 | (boundary position + 1) << 16
    const int* bidx;     // nb;  boundary node ids, ascending
    const double* B64;   // nb x nb row-major
    const float* B32;    // nb x nb row-major
    double vsum;         // sum_i Vint_i = 24 n^3
    double cell;         // cell edge h (m)
};

// ---- device view of one instance batch (node-major, instance-minor) ------------------
template <typename T>
struct BatchView {
    int B;
    double* m;   // [2][N][3][B]   m[cur] = base point, m[1-cur] = trial (FP64 in every mode)
    double* H;   // [2][N][3][B]   H = -m x grad phi at the same points (FP64)
    T* u1;       // [N][B]
    T* u2;       // [N][B]
    T* r; T* z; T* p; T* q;    // [N][B] PCG work vectors
    T* ub1;      // [nb][B]  u1 on the surface (BEM input)
    T* ub2;      // [nb][B]  u2 on the surface (BEM output)
    double* part;              // partial sums, >= maxblocks * B * NQ
    InstState* st;             // [B]
    const InstConst* ic;       // [B]
    double* hout;              // optional [N][3][B] effective field (nullable)
};

struct Launch {
    cudaStream_t stream;
    int num_sms;
    unsigned* bar;     // grid-barrier counter (device)
    int* err;          // device error word
    int64_t* launches; // host counter of kernel launches
    unsigned long long* sweeps;  // device counters [2]: batched PCG iterations (Neumann, Dirichlet)
};

template <typename T>
int pcg_solve(const Launch& L, const MeshView& M, const BatchView<T>& V, int mode, double tol, int max_iter,
              int* iters_dev);
template <typename T>
void bem_product(const Launch& L, const MeshView& M, const BatchView<T>& V);
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
void reset_states(const Launch& L, InstState* st, int B, const StepOpts& so, int set_cur0);
int field_blocks(const Launch& L, const MeshView& M, int B);
size_t pcg_part_elems(int num_sms, int B);

}  // namespace lbm
