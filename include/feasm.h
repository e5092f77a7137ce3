/*
 * feasm.h -- C ABI of the GB300 cell-integration and global-assembly library
 * (libfeasm.so) for grad-conforming Lagrangian Q_p hexahedra, p = 1..3,
 * Poisson and linear elasticity, after the FEMPAR paper (arXiv 1708.01773).
 *
 * Conventions shared by every entry point
 *   - All functions return 0 (FE_OK) or a negative FE_ERR_* code; no C++
 *     exception crosses the ABI. fe_last_error() returns a thread-local message
 *     for the last failure of the calling thread.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *     memory of the current device (for instance torch tensors' data_ptr()).
 *   - Device buffers passed in or out are owned by the caller; the library owns
 *     only what an fe_space / fe_batch holds (tables, DOF map, sparsity
 *     pattern, assembly permutation, cell-matrix scratch), allocated at create
 *     time and freed by the matching destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Compute calls
 *     are asynchronous on it and allocate nothing (the exceptions say so: the
 *     first fe_assemble_host call of a space and the first fe_batch_assemble
 *     of each precision allocate, and fe_assemble_host returns when its
 *     results are in host memory).
 *   - Compute calls on one space (fe_assemble*, fe_assemble_dirichlet on its
 *     constrained systems, fe_batch_assemble of a batch holding it) must not
 *     overlap on the GPU: they share the
 *     space's cell-matrix scratch and the scatter's work counters (which the
 *     scatter leaves at zero when it completes). Issue them on one stream, or
 *     order them with events.
 *   - Errors found on the device (a non-positive Jacobian determinant, a
 *     persistent-kernel wait that gave up) are recorded in a device error word
 *     and reported by fe_status(); kernels never trap.
 *   - Local DOF order in a cell: component-major, index i*nb + a, with the
 *     scalar nodes a in x-fastest lexicographic order (nb = (p+1)^3).
 *   - Mesh vertex order in a cell: x-fastest lexicographic, local vertex v at
 *     reference corner (v&1, (v>>1)&1, (v>>2)&1) of [0,1]^3.
 */
#ifndef FEASM_H
#define FEASM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_space fe_space; /* opaque, library-owned */
typedef struct fe_batch fe_batch; /* opaque, library-owned */

/* FE_STOKES: the Taylor-Hood pair of the paper's Stokes driver (Example
 * "Stokes problem", Sect. "Driver example for the Stokes problem"): velocity
 * Q_p (3 components, p = order = 2 or 3) and pressure Q_{p-1}, with the
 * (p+1)^3 Gauss rule; coefficients are the cell viscosities mu_K; the cell
 * matrix is
 *   velocity-velocity  mu int eps(u) : eps(v)
 *   velocity-pressure  - int (div v) p,  pressure-velocity  - int q (div u)
 *   pressure-pressure  0 (stored: every field pair is coupled, as by default
 *                      in the paper's block layout)
 * and the right-hand side int f . v on the velocity rows, 0 on the pressure
 * rows. Local DOFs: the 3 nb velocity ones (i*nb + a), then the p^3 pressure
 * ones. Global numbering: all velocity DOFs (list_dofs), then all pressure
 * DOFs (list_dofs), so the matrix has the 2x2 block layout velocity/pressure
 * with the split at fe_space_block_offset. FP64 and FP32 forms (BF16:
 * FE_ERR_UNSUPPORTED); the adjoint, the compliance and the batch take
 * Poisson and elasticity spaces only. */
typedef enum { FE_POISSON = 0, FE_ELASTICITY = 1, FE_STOKES = 2 } fe_problem;

/* Arithmetic of the cell-matrix contraction. The geometry (Jacobian,
 * determinant, cofactors) and the global CSR accumulation are always FP64.
 *   FE_PREC_FP64: all FP64 (the plain FP64 GPU assembler).
 *   FE_PREC_FP32: FP32 operands and FP32 accumulation of the contraction.
 *   FE_PREC_BF16: BF16 operands, FP32 accumulation. */
typedef enum { FE_PREC_FP64 = 0, FE_PREC_FP32 = 1, FE_PREC_BF16 = 2 } fe_precision;

enum {
  FE_OK = 0,
  FE_ERR_INVALID_ARG = -1,
  FE_ERR_CUDA = -2,
  FE_ERR_OOM = -3,
  FE_ERR_NEG_JACOBIAN = -4,
  FE_ERR_TIMEOUT = -5,
  FE_ERR_UNSUPPORTED = -6,
  FE_ERR_NOT_CONVERGED = -7
};

typedef struct {
  int64_t n_vertices;
  const double* coords;         /* host [n_vertices*3], copied at create */
  int64_t n_cells;
  const int32_t* cell_vertices; /* host [n_cells*8], x-fastest local order, copied */
} fe_mesh_desc;

/* Builds an FE space on a conforming hexahedral mesh: reference tables of the
 * Q_p Lagrangian element at a tensor Gauss-Legendre rule (paper, Sect.
 * "Numerical integration", Eq. lagbas / Eq. lagbasmd), the global DOF
 * numbering by the list_dofs algorithm (Sect. "Global DOF numbering
 * generation"), the CSR sparsity pattern (every DOF pair sharing a cell, columns
 * ascending; Sect. "Linear algebra": pattern built once and reused) and the
 * cell-to-nonzero assembly permutation used by fe_assemble.
 *   order           p in 1..3 (Stokes: the velocity order, 2 or 3).
 *   quad_points_1d  Gauss points per direction, 0 = p+1 (exact mass matrix on
 *                   affine cells), else 1..6.
 *   problem         FE_POISSON (1 component), FE_ELASTICITY (3 components) or
 *                   FE_STOKES (Taylor-Hood, see fe_problem; quad_points_1d 0
 *                   or p+1).
 *   nu              Poisson ratio (elasticity only, 0 <= nu < 0.5).
 *   out             receives the new space; destroy with fe_space_destroy.
 * Uses the current CUDA device. Host work is multi-threaded. Errors:
 * FE_ERR_INVALID_ARG (bad sizes, vertex ids out of range, a cell that repeats
 * a vertex), FE_ERR_UNSUPPORTED
 * (index widths exceeded, more than 127 cells around one DOF), FE_ERR_OOM,
 * FE_ERR_CUDA. */
int fe_space_create(const fe_mesh_desc* mesh, int order, int quad_points_1d, fe_problem problem,
                    double nu, fe_space** out);

/* Same host-side setup as fe_space_create without touching any GPU (for
 * inspection of the numbering and the pattern on machines without one). The
 * result supports fe_space_sizes, fe_space_cell_dofs_host,
 * fe_space_csr_pattern_host and fe_space_destroy only. */
int fe_space_create_host(const fe_mesh_desc* mesh, int order, int quad_points_1d, fe_problem problem,
                         double nu, fe_space** out);

/* Cell order for memory locality (host only, touches no GPU): order[i] = the
 * input cell placed at position i, the cells sorted by the Morton (Z-order)
 * code of their vertex centroids, quantised to 21 bits per axis over the
 * bounding box of the centroids; equal codes keep the input order. list_dofs
 * numbers DOFs in cell order (Sect. "Global DOF numbering generation"), so a
 * mesh whose cells are given in this order (cell_vertices and any per-cell
 * coefficients permuted alike) gets a numbering and assembly maps in which the
 * cells around a node, and the rows of neighbouring nodes, lie close in
 * memory. The paper leaves the cell order to the mesh generator (its
 * structured generator numbers cells lexicographically); this serves meshes
 * that arrive in arbitrary order. `order` is host [n_cells], caller-owned.
 * Errors: FE_ERR_INVALID_ARG (NULL pointers with n_cells > 0, vertex ids out
 * of range, non-finite coordinates). */
int fe_mesh_locality_order(const fe_mesh_desc* mesh, int64_t* order);

/* Sizes of the space: number of global DOFs, CSR nonzeros, cells, and
 * per-contribution counts (n_cells * n_loc^2). Any pointer may be NULL. */
int fe_space_sizes(const fe_space* s, int64_t* n_dofs, int64_t* nnz, int64_t* n_cells,
                   int64_t* n_contrib);

/* Number of DOFs of the first field: the velocity block of a Stokes space
 * (pressure DOFs are n_first .. n_dofs-1); n_dofs for the other problems. */
int fe_space_block_offset(const fe_space* s, int64_t* n_first);

/* Copies the cell-to-DOF map [n_cells * n_loc] (host, int32, local order
 * i*nb + a, then the pressure DOFs for Stokes) into caller memory (Sect.
 * "Global DOF numbering generation"). */
int fe_space_cell_dofs_host(const fe_space* s, int32_t* cell_dofs);

/* Copies the CSR pattern into caller memory: row_ptr [n_dofs+1] int64 and
 * col_idx [nnz] int32. _host: host pointers; plain: device pointers, copied
 * asynchronously on `stream`. */
int fe_space_csr_pattern_host(const fe_space* s, int64_t* row_ptr, int32_t* col_idx);
int fe_space_csr_pattern(const fe_space* s, int64_t* row_ptr, int32_t* col_idx, void* stream);

/* Copies the assembly permutation of a host-only space into caller memory
 * (host): cnt [nnz] uint8 contributions per nonzero; code_ptr [n_dofs+1] int64
 * first code of each row; codes [code_ptr[n_dofs]] uint16 (may be NULL: call
 * once without it to learn the length); slot_ptr [n_dofs+1] int64; slots
 * [n_cells * n_loc] int32. Row r has the cells ("slots", ascending) given by
 * slots[slot_ptr[r] .. slot_ptr[r+1]), each entry e * n_loc + (local index of
 * DOF r in cell e). The row's ns * n_loc codes start at code_ptr[r] (a
 * multiple of 8; the block is padded to a multiple of 8 codes); code bits are
 * head << 15 | s << 8 | m. Nonzero k of the row (columns ascending) sums, in
 * code order, the cell-matrix entries K^{e_s}[local row][m] of one run of codes
 * that starts with head = 1, i.e. its cells in ascending order. This is the
 * deterministic gather form of Eq. assembly. Only spaces made by
 * fe_space_create_host keep these arrays on the host (FE_ERR_INVALID_ARG
 * otherwise). */
int fe_space_permutation_host(const fe_space* s, uint8_t* cnt, int64_t* code_ptr, uint16_t* codes,
                              int64_t* slot_ptr, int32_t* slots);

/* Integrates every cell and assembles the global matrix and right-hand side
 * (paper Eq. linear_system, Eq. assembly, Eq. fematrix, Eq. shape_grad; the
 * element loop of the Listing "element_matrix_entries_computation").
 *   coefficients  device [n_cells] FP64: conductivity kappa_K (Poisson) or
 *                 Young's modulus E_K (elasticity), constant per cell.
 *   body_force    host [ncomp] FP64: constant source f (Poisson) or body
 *                 force (elasticity).
 *   csr_values    device [nnz] FP64, overwritten (pattern of fe_space_csr_pattern).
 *   rhs           device [n_dofs] FP64, overwritten; may be NULL.
 *   prec          arithmetic of the cell-matrix contraction (see fe_precision).
 * The result is deterministic: every CSR value is the sum of its cell
 * contributions in ascending cell order, in FP64, without atomics. No
 * boundary conditions are applied (the unconstrained, singular operator). */
int fe_assemble(fe_space* s, const double* coefficients, const double* body_force, double* csr_values,
                double* rhs, fe_precision prec, void* stream);

/* fe_assemble that also records `event_mid` (a cudaEvent_t, or NULL) on
 * `stream` between the cell-integration kernel and the scatter kernel, so that
 * a caller can time the two kernels separately with CUDA events. */
int fe_assemble_ex(fe_space* s, const double* coefficients, const double* body_force, double* csr_values,
                   double* rhs, fe_precision prec, void* stream, void* event_mid);

/* fe_assemble with HOST buffers: coefficients [n_cells], csr_values [nnz] and
 * rhs [n_dofs] (may be NULL) are host memory (pinned memory gives full copy
 * speed). The results pass through device staging buffers that the space
 * allocates on its first host-buffer call. The scatter runs in row ranges;
 * each range's values and RHS are copied to the host on a second stream (also
 * created on the first call) as soon as its scatter launch completes, so that
 * the device-to-host copy overlaps the rest of the assembly. The call returns
 * after the results are in host memory. */
int fe_assemble_host(fe_space* s, const double* coefficients, const double* body_force,
                     double* csr_values, double* rhs, fe_precision prec, void* stream);

/* Compliance sensitivity. For a fixed nodal field u, c(coef) = u^T A(coef) u
 * is linear in the cell coefficients (Eq. assembly), so
 *   dc/dcoef_K = u_K^T (A^K / coef_K) u_K,
 * computed per quadrature point from the strain of u without forming A^K:
 * elasticity lambda^ (div u)^2 + 2 mu^ eps(u):eps(u), Poisson |grad u|^2,
 * times w_q det J_q (Eq. fematrix), with lambda^, mu^ the Lame parameters per
 * unit Young's modulus.
 *   u             device [n_dofs] FP64 nodal values.
 *   coefficients  device [n_cells] FP64; needed only for `compliance`.
 *   grad_scale    multiplies dc_dcoef (the incoming gradient of a backward pass).
 *   dc_dcoef      device [n_cells] FP64, overwritten with grad_scale * dc/dcoef.
 *   compliance    device scalar FP64 or NULL: receives c = sum_K coef_K dc/dcoef_K
 *                 (unscaled), reduced in a fixed order (deterministic).
 *   prec          FE_PREC_FP64 or FE_PREC_FP32 (FP32 strain arithmetic, FP64
 *                 geometry and FP64 sums). */
int fe_assemble_adjoint(fe_space* s, const double* u, const double* coefficients, double grad_scale,
                        double* dc_dcoef, double* compliance, fe_precision prec, void* stream);

/* Selects the cell-integration kernel of later fe_assemble calls:
 * FE_KERNEL_AUTO (default: the tensor-core kernel for Q2 elasticity and for
 * the BF16 forms of Q3 Poisson and Q3 elasticity, the warp-role CUDA-core
 * kernel for Q1 elasticity, else the general CUDA-core kernel),
 * FE_KERNEL_CUDA_CORE, or FE_KERNEL_TENSOR_CORE (fe_assemble then fails with
 * FE_ERR_UNSUPPORTED where none exists; tensor-core kernels exist for Q2 / Q3
 * elasticity and Q2 / Q3 Poisson with the (p+1)^3 rule, FP32 or BF16).
 * The kernels of FE_KERNEL_AUTO keep the FP32 form within 1e-6 (row-scaled
 * entry error against FP64) on every mesh tested, single cells included. The
 * Q3 tensor-core kernels' FP32 forms (3xTF32), chosen only on request, are
 * faster but not within 1e-6 everywhere, because the tensor cores' FP32
 * accumulation does not round to nearest: Poisson Q3 reached 1.2e-6 on one
 * distorted cell (within 1e-6 on multi-cell meshes), elasticity Q3 1.9e-6. */
enum { FE_KERNEL_AUTO = 0, FE_KERNEL_CUDA_CORE = 1, FE_KERNEL_TENSOR_CORE = 2 };
int fe_space_set_kernel(fe_space* s, int cell_kernel);

/* fe_assemble_adjoint without any memory allocation (the paper has no
 * counterpart; this is a service for callers that cannot allocate). Same
 * arguments, results and determinism as fe_assemble_adjoint.
 *
 * For applications that own all device memory through their own pool and do
 * not allow a library to call cudaMalloc, and for loops that must not enter
 * the CUDA allocator while they run (cudaMalloc / cudaFree can synchronise the
 * device). The call itself allocates nothing: the reduction scratch of the
 * compliance is a fixed 512 KB array in the library's device image (held by
 * every GPU that loads the library until the process exits).
 * Limits and rules:
 *   - with `compliance` non-NULL the space may have at most 8,388,608 cells
 *     (FE_ERR_UNSUPPORTED with a message otherwise); without it, any size;
 *   - the current device must be the space's device;
 *   - every call looks up the array's device address in the current context
 *     (cudaGetSymbolAddress, which allocates nothing), so the call stays
 *     correct after the application resets the device (cudaDeviceReset); the
 *     first call on a device may also load the library's device code there,
 *     so make that first call before any stream capture of your own;
 *   - all calls share the one array, so calls that overlap on the GPU (on
 *     different streams, or from different threads) race and may return a
 *     wrong compliance: serialise them. Nothing in the array needs clearing:
 *     each call writes every entry it reads. */
int fe_assemble_adjoint_noalloc(fe_space* s, const double* u, const double* coefficients, double grad_scale,
                                double* dc_dcoef, double* compliance, fe_precision prec, void* stream);

/* Synchronises `stream`, returns and clears the device error word:
 * FE_OK, FE_ERR_NEG_JACOBIAN (some det J <= 0 at a quadrature point) or
 * FE_ERR_TIMEOUT (a bounded persistent-kernel wait gave up). */
int fe_status(fe_space* s, void* stream);

void fe_space_destroy(fe_space* s);

/* Thread-local description of the last error of the calling thread. */
const char* fe_last_error(void);

/* Batched assembly: several independent spaces (any order, problem and size)
 * assembled by one persistent launch over a shared work list of (space, cell
 * block) and (space, row block) items, replayed from a CUDA graph. A row item
 * waits (bounded, about one second; FE_ERR_TIMEOUT in the spaces' error
 * words after that) until its space's cells are integrated. Cell items use
 * the CUDA-core cell kernel. A space whose cells fe_assemble would integrate
 * on the tensor cores in the requested precision (its fe_space_set_kernel
 * selection; by default Q2 elasticity and the BF16 forms of Q3 Poisson and
 * Q3 elasticity) has no cell items: its tensor-core cell kernel is launched on
 * the caller's stream before the persistent launch. Results are
 * deterministic and match fe_assemble space by space, with the tensor-core
 * kernel for those spaces and the CUDA-core kernel for the others. The batch
 * reads each space's kernel selection at every call. The batch keeps pointers to the spaces, which must
 * outlive it; spaces must be on the current device with at most 32 cells
 * around any DOF.
 *   cells_per_item  cells per cell item, 0 = autotuned: the first
 *                   fe_batch_assemble of each precision times the candidate
 *                   item sizes on the caller's buffers (running the assembly
 *                   a few times), keeps the fastest, allocates its work list
 *                   and captures its CUDA graph; make that first call before
 *                   any stream capture of your own. */
int fe_batch_create(fe_space* const* spaces, int n, int cells_per_item, fe_batch** out);

/* coefficients[i], csr_values[i], rhs[i] are the device buffers of space i
 * (rhs may be NULL, or rhs[i] NULL); body_force is host [n*3] (force of
 * space i at 3*i). Same semantics as fe_assemble for every space; errors found
 * on the device surface through fe_status of the spaces. */
int fe_batch_assemble(fe_batch* b, const double* const* coefficients, const double* body_force,
                      double* const* csr_values, double* const* rhs, fe_precision prec, void* stream);

/* Test hook of the batch's bounded wait (a check of the failure path, not
 * part of the method): later fe_batch_assemble calls limit each row item's
 * wait to `wait_cycles` clock cycles (0 restores the default, about one
 * second) and make it wait for `extra_cells` more integrated cells than its
 * space has (0 restores the normal target). With extra_cells > 0 no row item
 * can start: each gives up after its limit, its block leaves the launch, the
 * launch ends, and fe_status of every space of the batch returns
 * FE_ERR_TIMEOUT; the CSR values of that call are then incomplete. Takes
 * effect at the next fe_batch_assemble (no recapture). FE_ERR_INVALID_ARG
 * for negative arguments. */
int fe_batch_set_wait(fe_batch* b, long long wait_cycles, int extra_cells);

void fe_batch_destroy(fe_batch* b);

/* Self-test of the library's integer-bit conversions against the hardware
 * conversions (a check of its arithmetic; the paper has no counterpart). For
 * each device FP64 input x[i], i < n, writes (device buffers):
 *   out32[8 i + 0..7] = hardware FP32 rounding h of x; the general integer-bit
 *     rounding; the branch-free one; its out-of-range flags (1: the branch-free
 *     rounding, 2: the remainder); the branch-free remainder x - h rounded to
 *     FP32; the hardware remainder; the TF32 split hi, lo of h;
 *   out64[5 i + 0..4] = the pair (h, hardware remainder) rounded once to FP64 by
 *     the integer path, by the fixed-point sum, and by one hardware FP64
 *     addition; h converted to FP64 on the integer bits and by the hardware.
 * Asynchronous on `stream`; FE_ERR_INVALID_ARG for NULL buffers with n > 0. */
int fe_selftest_conversions(const double* x, int64_t n, float* out32, double* out64, void* stream);

/* ------------------------------------------------------------------------
 * Strong Dirichlet conditions (paper, Sect. "Strong imposition of boundary
 * conditions", Eq. dirichlet_bc_discrete_problem). The DOFs of a space split
 * into free and fixed ones; the constrained system keeps the rows and columns
 * of the free DOFs only,
 *   sum_{b free} A_ab u_b = f_a - sum_{c fixed} A_ac u^D_c   (a free),
 * and its right-hand side carries the prescribed values u^D of the fixed DOFs.
 * Free DOFs are numbered 0 .. n_free-1 and fixed DOFs 0 .. n_fixed-1, each in
 * ascending global DOF id (the paper's labels 1..n_free and -1..-n_fixed).
 * ------------------------------------------------------------------------ */
typedef struct fe_dirichlet fe_dirichlet; /* opaque, library-owned */

/* Physical position of every DOF's node (host [n_dofs*3]): the node's
 * reference point alpha/p mapped by the cell's trilinear map (the DOFs of the
 * ncomp components of one node share it). `mesh` must be the mesh the space
 * was created from (same sizes; host pointers). Serves the choice of fixed
 * DOFs by position. Works on host-only spaces. Errors: FE_ERR_INVALID_ARG. */
int fe_space_dof_points_host(const fe_space* s, const fe_mesh_desc* mesh, double* points);

/* Builds the constrained system of space `s`: the free/fixed labels, the
 * sparsity pattern of the free x free block (columns ascending) and its
 * assembly permutation, and the list of cells that carry both fixed and free
 * DOFs (where the right-hand side is lifted).
 *   fixed  host [n_dofs] uint8 in the space's global numbering: nonzero marks a
 *          fixed DOF; copied.
 * Works on host-only spaces (inspection only). The space must outlive the
 * object and is shared with it: fe_assemble and fe_assemble_dirichlet on one
 * space must not overlap on the GPU. Errors: FE_ERR_INVALID_ARG,
 * FE_ERR_UNSUPPORTED, FE_ERR_OOM, FE_ERR_CUDA. */
int fe_dirichlet_create(fe_space* s, const uint8_t* fixed, fe_dirichlet** out);

/* Numbers of free and fixed DOFs and nonzeros of the constrained matrix. Any
 * pointer may be NULL. */
int fe_dirichlet_sizes(const fe_dirichlet* d, int64_t* n_free, int64_t* n_fixed, int64_t* nnz);

/* Host [n_dofs] int32 labels: the free id (>= 0) of a free DOF, or -1 - its
 * fixed id for a fixed DOF. */
int fe_dirichlet_labels_host(const fe_dirichlet* d, int32_t* labels);

/* CSR pattern of the constrained matrix: row_ptr [n_free+1] int64, col_idx
 * [nnz] int32 (free ids). _host: host pointers; plain: device pointers, copied
 * asynchronously on `stream`. */
int fe_dirichlet_csr_pattern_host(const fe_dirichlet* d, int64_t* row_ptr, int32_t* col_idx);
int fe_dirichlet_csr_pattern(const fe_dirichlet* d, int64_t* row_ptr, int32_t* col_idx, void* stream);

/* Assembly permutation of the constrained system of a host-only space (host
 * pointers), in the layout of fe_space_permutation_host with rows = free DOFs:
 * cnt [nnz]; code_ptr [n_free+1]; codes (may be NULL) hold ncode[r] codes per
 * row, those of fixed columns left out; ncode [n_free] int32; pos (may be
 * NULL) [code_ptr[n_free]] the slot-major positions, where an entry (s, m) of
 * a fixed column holds the index of the reading lane's private dummy
 * accumulator, acc_stride + (m mod 32), acc_stride being the largest row
 * length rounded up to a multiple of 4; slot_ptr [n_free+1]; slots. */
int fe_dirichlet_permutation_host(const fe_dirichlet* d, uint8_t* cnt, int64_t* code_ptr, uint16_t* codes,
                                  int32_t* ncode, uint16_t* pos, int64_t* slot_ptr, int32_t* slots);

/* Lifting lists (host): n_cells cells carrying fixed and free DOFs, ascending
 * (cells [n_cells]); the fixed local columns of cells[i] are m[ptr[i] ..
 * ptr[i+1]) (ascending) with fixed ids fix[...]. Array pointers may be NULL
 * (call once with them NULL to learn n_cells and n_entries). */
int fe_dirichlet_lift_host(const fe_dirichlet* d, int64_t* n_cells, int64_t* n_entries, int32_t* cells,
                           int32_t* ptr, uint8_t* m, int32_t* fix);

/* Integrates every cell and assembles the constrained system (Eq.
 * dirichlet_bc_discrete_problem): the cell matrices and vectors as in
 * fe_assemble, then for each listed cell the lifting
 *   f^K_a -= sum_{fixed local columns m} A^K_am u^D_m  (every local row a;
 *   FP64 products of the stored cell-matrix entries, summed in a fixed order),
 * then the scatter of the free rows and columns.
 *   coefficients, body_force, prec  as for fe_assemble.
 *   u_fixed     device [n_fixed] FP64 prescribed values, or NULL for u^D = 0.
 *   csr_values  device [nnz] FP64, overwritten (fe_dirichlet_csr_pattern).
 *   rhs         device [n_free] FP64, overwritten; may be NULL.
 * Deterministic like fe_assemble. */
int fe_assemble_dirichlet(fe_dirichlet* d, const double* coefficients, const double* body_force,
                          const double* u_fixed, double* csr_values, double* rhs, fe_precision prec, void* stream);

/* ------------------------------------------------------------------------
 * Self-adjoint compliance of a clamped structure (not in the paper; built on
 * the constrained assembly above). With the fixed DOFs of `d` held at zero and
 * the body force f, K(E) u = f on the free DOFs and
 *   c(E) = f^T u,   dc/dE_K = -u_K^T (A^K / E_K) u_K
 * (c = f^T K^-1 f, and K is linear in the cell coefficients, Eq. assembly).
 * ------------------------------------------------------------------------ */

/* Number of doubles of device workspace fe_compliance needs: the constrained
 * matrix and right-hand side plus the solver's vectors and partial sums. */
int fe_compliance_work_size(const fe_dirichlet* d, int64_t* n_doubles);

/* Assembles the constrained system in precision `prec` (fe_assemble_dirichlet
 * with u^D = 0), solves it by the conjugate gradient method with the Jacobi
 * preconditioner in FP64 until ||r|| <= rtol ||f|| (checked every 8
 * iterations) or max_iter iterations, and evaluates c and its gradient (the
 * adjoint kernel of fe_assemble_adjoint with grad_scale -1; FP32 strain
 * arithmetic for the FP32/BF16 forms, FP64 otherwise). Every reduction runs in
 * a fixed order: the results are deterministic on any GPU.
 *   coefficients  device [n_cells] E_K (or kappa_K).
 *   body_force    host [ncomp].
 *   work          device [fe_compliance_work_size] doubles, caller-owned.
 *   u             device [n_dofs] FP64: the displacement over all DOFs (zero
 *                 at the fixed ones).
 *   compliance    device scalar FP64: c.
 *   dc_dcoef      device [n_cells] FP64: dc/dE_K (may be NULL: no gradient).
 *   iterations, rel_residual  host outputs (may be NULL).
 * Synchronises `stream` (the host checks convergence). Errors:
 * FE_ERR_NOT_CONVERGED (max_iter reached; u holds the last iterate),
 * FE_ERR_INVALID_ARG (also: the constrained matrix is not positive definite,
 * e.g. too few DOFs fixed), FE_ERR_CUDA. */
int fe_compliance(fe_dirichlet* d, const double* coefficients, const double* body_force, fe_precision prec,
                  double rtol, int max_iter, double* work, double* u, double* compliance, double* dc_dcoef,
                  int* iterations, double* rel_residual, void* stream);

/* Frees the constrained system (before its space). */
void fe_dirichlet_destroy(fe_dirichlet* d);

/* ------------------------------------------------------------------------
 * Interior penalty discontinuous Galerkin for the Poisson problem (paper,
 * Sect. "Non-conforming methods", Eq. ip_dg_formulations, Eq.
 * mean_and_jump_ops, Eq. local_to_face_matrix). The space is discontinuous
 * Q_p on the mesh: DOF a of cell K is K*(p+1)^3 + a (a lexicographic). The
 * operator is
 *   sum_K int_K grad u . grad v
 *   + sum_{interior F} ( - int [v].{grad u} - tau int [u].{grad v} + gamma/|F| int [u].[v] )
 *   + sum_{boundary F} ( - int v grad u.n - tau int u grad v.n + gamma/|F| int u v ),
 * the right-hand side int f v (homogeneous weak Dirichlet data, u_D = 0).
 * Interior facets take K+ = the lower cell id; each contributes the four
 * blocks (K+K+, K+K-, K-K+, K-K-), row = test function, column = trial
 * function. Facet integrals use (p+1)^2 Gauss points and FP64 geometry; their
 * products are FP64 in the FP64 form and FP32 in the FP32 and BF16 forms.
 * ------------------------------------------------------------------------ */
typedef struct fe_dg fe_dg; /* opaque, library-owned */

/* Builds the DG space on a conforming hexahedral mesh (any local vertex
 * orientation): the cell integration of the Poisson Q_p element, the facets
 * (neighbours matched by their 4 vertex ids) and the CSR pattern (each row of
 * cell K: the DOFs of K and of its face neighbours, columns ascending).
 * _host: no GPU use (inspection: sizes, pattern, facets). Errors as for
 * fe_space_create, and FE_ERR_INVALID_ARG when two cells share a face's four
 * vertices but their corners do not correspond by a symmetry of the square
 * (a twisted face: the facet integrals read the neighbour's reference point
 * off that symmetry). */
int fe_dg_create(const fe_mesh_desc* mesh, int order, fe_dg** out);
int fe_dg_create_host(const fe_mesh_desc* mesh, int order, fe_dg** out);

/* Numbers of DOFs, CSR nonzeros, interior and boundary facets (any may be NULL). */
int fe_dg_sizes(const fe_dg* g, int64_t* n_dofs, int64_t* nnz, int64_t* n_interior, int64_t* n_boundary);

/* CSR pattern: row_ptr [n_dofs+1] int64, col_idx [nnz] int32. _host: host
 * pointers; plain: device pointers, copied asynchronously on `stream`. */
int fe_dg_csr_pattern_host(const fe_dg* g, int64_t* row_ptr, int32_t* col_idx);
int fe_dg_csr_pattern(const fe_dg* g, int64_t* row_ptr, int32_t* col_idx, void* stream);

/* Facets (host): interior facet i joins cells plus[i] < minus[i] through local
 * faces plus_face[i], minus_face[i] (face f lies on xhat_{f/2} = f%2);
 * boundary facet j is face bnd_face[j] of cell bnd_cell[j]. Arrays may be NULL. */
int fe_dg_facets_host(const fe_dg* g, int32_t* plus, int32_t* minus, uint8_t* plus_face, uint8_t* minus_face,
                      int32_t* bnd_cell, uint8_t* bnd_face);

/* Assembles the DG system: tau (the method: 1 symmetric, -1 non-symmetric, 0
 * incomplete IP), gamma > 0 (penalty), source f (constant). prec selects the
 * arithmetic of the cell integrals (as in fe_assemble) and of the facet
 * products; each CSR value is formed in a fixed order (deterministic), the
 * diagonal blocks' sums exactly rounded to FP64 in the FP32 forms.
 *   csr_values  device [nnz] FP64, overwritten.
 *   rhs         device [n_dofs] FP64, overwritten; may be NULL.
 * The facet blocks go to device scratch allocated by fe_dg_create
 * (4 (p+1)^6 doubles per interior and (p+1)^6 per boundary facet; the FP32
 * forms use half of it). */
int fe_dg_assemble(fe_dg* g, double tau, double gamma, double source, double* csr_values, double* rhs,
                   fe_precision prec, void* stream);

void fe_dg_destroy(fe_dg* g);

#ifdef __cplusplus
}
#endif

#endif /* FEASM_H */
