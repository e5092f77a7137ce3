// Internal data structures of libfeasm: the FE space (host setup products and
// their device copies) and the host-side setup routines.
#pragma once

#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/feasm.h"

namespace feasm {

constexpr int kMaxOrder = 3;
constexpr int kMaxQ1d = 6;
constexpr int kMaxSlots = 127;  // cells around one DOF (7 bits of a code)

// Records the message returned by fe_last_error and returns `code`.
int set_error(int code, const char* msg);

// Runs f() and turns a C++ exception into a status code (std::bad_alloc:
// FE_ERR_OOM, any other: FE_ERR_UNSUPPORTED), so that no exception leaves an
// entry point of the C ABI.
template <typename F>
int no_throw(const char* what, F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return set_error(FE_ERR_OOM, (std::string(what) + ": host allocation failed").c_str());
  } catch (const std::exception& x) {
    return set_error(FE_ERR_UNSUPPORTED, (std::string(what) + ": " + x.what()).c_str());
  } catch (...) {
    return set_error(FE_ERR_UNSUPPORTED, (std::string(what) + ": unexpected exception").c_str());
  }
}

// Reference tables of the Q_p element at a tensor Gauss-Legendre rule on
// [0,1]^3. Point q = q0 + n q1 + n^2 q2, node a = a0 + (p+1) a1 + (p+1)^2 a2.
struct RefTables {
  int p = 0, nq1d = 0, nb = 0, nq = 0;
  std::vector<double> w;      // [nq]
  std::vector<double> xq;     // [nq][3]
  std::vector<double> phi;    // [nq][nb]
  std::vector<double> dphi;   // [nq][nb][3]
};

// Products of the host setup of one space.
struct HostSetup {
  int64_t n_dofs = 0, nnz = 0, n_contrib = 0, n_codes = 0;
  int64_t n_first = 0;              // DOFs of the first field (Stokes: the velocity block)
  int max_slots = 0;
  int64_t max_row_nnz = 0;
  bool node_rows = false;           // the ncomp rows of each node share cells and positions
  std::vector<int32_t> cell_dofs;   // [n_cells][nl]
  std::vector<int64_t> row_ptr;     // [n_dofs+1]
  std::vector<int32_t> col;         // [nnz]
  std::vector<uint8_t> cnt;         // [nnz] contributions per nonzero
  std::vector<int64_t> code_ptr;    // [n_dofs+1] first code of each row
  std::vector<uint16_t> codes;      // (head << 15) | (slot << 8) | local column, rows padded to 8 codes
  std::vector<uint16_t> pos;        // same blocks, slot-major: nonzero index within the row of (slot, column),
                                    // bit 15 set on the first contribution of each nonzero
  std::vector<int64_t> slot_ptr;    // [n_dofs+1]
  std::vector<int32_t> slots;       // [n_cells*nl] e*nl + local row, cells ascending
  std::vector<int32_t> ncode;       // [n_dofs] codes of each row (constrained patterns only; empty: ns * nl)
  bool pos_ok = true;               // the positions of dropped columns fit the 15-bit dummy index
};

void build_ref_tables(int p, int nq1d, RefTables* t);
// n-point Gauss-Legendre rule on [0,1].
void gauss_rule(int n, double* x, double* w);
// 1D Lagrange basis of order p (equidistant nodes) and its derivative at the
// nq1d Gauss points: val[q][a], der[q][a], q < nq1d, a <= p.
void lagrange_1d_table(int p, int nq1d, double* val, double* der);
// Numbering, pattern and permutation of a space of order p for `problem`
// (FE_POISSON, FE_ELASTICITY, FE_STOKES). Returns 0 or an FE_ERR_* code
// (message in *err).
int build_host_setup(int p, int problem, int64_t n_cells, int64_t n_vertices, const int32_t* cell_vertices,
                     HostSetup* hs, std::string* err);
// Sparsity pattern and assembly permutation from a cell-to-DOF map with nl
// local DOFs per cell. With label == nullptr the rows and columns are the DOFs
// themselves (n_rows = n_dofs); otherwise DOF d is row/column label[d] if
// label[d] >= 0 and is dropped if label[d] < 0 (a fixed DOF), n_rows being the
// number of kept DOFs. ncomp > 1 checks whether the ncomp rows of each node
// (local rows i * nb + a) can be scattered together. Fills everything in *hs
// except cell_dofs and n_first.
int build_pattern(int nl, int nb, int ncomp, int64_t n_cells, const int32_t* cell_dofs, const int32_t* label,
                  int64_t n_rows, HostSetup* hs, std::string* err);

}  // namespace feasm

struct fe_space {
  int order = 0, nq1d = 0, problem = 0, ncomp = 1, nb = 0, nq = 0, nl = 0;
  int nbp = 0;  // Stokes: pressure nodes per cell (Q_{p-1}); local pressure DOFs follow the 3 nb velocity ones
  int nlp = 0;  // row stride of a cell matrix: nl rounded up to a multiple of 4 (16-byte rows)
  double nu = 0.0;
  int64_t n_cells = 0, n_vertices = 0;
  bool host_only = false;
  int device = 0;
  feasm::RefTables tab;
  feasm::HostSetup hs;  // host arrays (pattern arrays are released after upload)
  int cell_kernel = 0;  // FE_KERNEL_AUTO / _CUDA_CORE / _TENSOR_CORE
  // device data
  double* d_xv = nullptr;        // [n_cells][8][3] cell vertex coordinates
  double* d_w = nullptr;         // [nq]
  double* d_xq = nullptr;        // [nq][3]
  double* d_phi = nullptr;       // [nq][nb]
  double* d_dphi = nullptr;      // [nq][nb][3]
  float* d_dphi32 = nullptr;     // [nq][nb][3]
  float* d_phi2 = nullptr;       // [nq][nb][2] phihat as FP32 hi + lo
  double* d_psi = nullptr;       // Stokes: [nq][nbp] pressure basis at the quadrature points
  int32_t* d_cell_dofs = nullptr;
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  uint8_t* d_cnt = nullptr;
  int64_t* d_code_ptr = nullptr;
  uint16_t* d_codes = nullptr;
  uint16_t* d_pos = nullptr;
  int64_t* d_slot_ptr = nullptr;
  int32_t* d_slots = nullptr;
  void* d_ke = nullptr;          // cell matrices, [n_cells][nl][nlp] FP64 or FP32
  double* d_fe = nullptr;        // cell vectors [n_cells][nl]
  int* d_err = nullptr;          // device error word
  unsigned long long* d_sched = nullptr;  // [2] scatter schedule counters (zero between launches)
  double* d_partials = nullptr;  // reduction scratch for the compliance
  int n_partials = 0;
  // staging buffers of fe_assemble_host, its copy stream and one event per row range
  double* d_stage_coef = nullptr;
  double* d_stage_vals = nullptr;
  double* d_stage_rhs = nullptr;
  void* copy_stream = nullptr;           // cudaStream_t
  void* range_done[16] = {nullptr};     // cudaEvent_t
};
