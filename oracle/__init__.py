"""Plain FP64 CPU oracle for the curvilinear steepest-descent micromagnetic minimiser.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link or
execute anything in this package: only the tests, the package-level smoke check
and the benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
library (no kernels, headers, tables or constant generators); the two meet only
in the seeded input generators of `synth`.

The oracle follows Exl et al., "LaBonte's method revisited" (arXiv:1309.5796):
  * Eq. (1)   the constrained problem min phi_t(m) s.t. |m| = 1,
  * Eq. (2-4) the projected gradient  m x (-m x grad phi),
  * Sec. 2.1  H(m) := -m x grad phi_t(m),
  * Eq. (8)   the curvilinear (Cayley / Crank-Nicolson) update and its norm
              preservation,
  * Sec. 2.3  first step by inexact line search, Barzilai-Borwein steps, the
              adaptive BB1/BB2 choice, nonmonotone globalisation over the
              previous 20 energies,
  * Sec. 3.1  hysteresis as a continuation of local minima in the applied field,
  * Table 2   gradient = sparse matrix-vector products, scalar potential =
              linear solve.
Readings where the paper is silent are stated in each module.
Modules:
  mesh      Kuhn-split cube, boundary, integer-scaled P1 assembly
  bem       double-layer (Fredkin-Koehler) boundary matrix, whole or by sub-block
  hmatrix   hierarchical (H-matrix) form of that matrix: cluster tree, block
            tree, low-rank leaves (Sec. 3.1 names H-matrices for the BEM)
  micromag  energies, effective fields, magnetostatic potential
  spacetrans the open boundary by space transformation (air box and a shell
            mapped onto the exterior; Sec. 3.1: the paper's own solver's scheme)
  minimise  Cayley update, step rules, minimiser, hysteresis sweep
"""
