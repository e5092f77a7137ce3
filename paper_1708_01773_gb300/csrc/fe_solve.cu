// Self-adjoint compliance of a clamped structure (not in the paper; it uses
// the paper's assembly with strong Dirichlet conditions, Sect. "Strong
// imposition of boundary conditions"): K(E) u = f on the free DOFs, c = f^T u
// and dc/dE_K = -u_K^T (A^K / E_K) u_K. The free system is solved by the
// conjugate gradient method with the Jacobi preconditioner, in FP64, with
// every reduction in a fixed order (the result is deterministic on any GPU).
//
// One PCG iteration is three kernels:
//   k_spmv_dot  q = A p (G lanes per row), block partials of p.q
//   k_update    alpha = rz / sum(p.q partials), summed by every block in the
//               same fixed order; x += alpha p, r -= alpha q, z = D^-1 r;
//               block partials of r.z and r.r
//   k_pupdate   beta = rz_new / rz (partials summed likewise); p = z + beta p
// Every kernel with partial sums runs on a fixed grid of kGridBlocks blocks,
// so the partial sums (and with them every result) do not depend on the SM
// count.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fe_device.cuh"
#include "fe_launch.h"

namespace feasm {
namespace solve {

constexpr int kBlock = 256;
constexpr int kGridBlocks = 1216;  // elementwise grid (152 SMs x 8), fixed
constexpr int kCheckEvery = 8;     // iterations between host convergence checks

// device scalars
enum { S_RZ0 = 0, S_RZ1 = 1, S_RR = 2, S_BB = 3, S_FLAG = 4, S_C = 5, kScalars = 8 };
// S_FLAG bits
constexpr int kFlagNotSpd = 1;

struct CgParams {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double* b;
  double* x;
  double* r;
  double* z;
  double* p;
  double* q;
  double* dinv;
  double* part_a;  // [kGridBlocks] p.q, or r.z at init
  double* part_b;  // [kGridBlocks] r.z
  double* part_c;  // [kGridBlocks] r.r, or b.b at init
  double* s;       // [kScalars]
};

// Fixed-order block reduction of one value per thread; the result is valid in
// thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kBlock / 32; ++w) t += sh[w];
  __syncthreads();
  return t;
}

// Sum of the kGridBlocks partials in a fixed order, by one warp (every lane
// ends with the same value).
__device__ __forceinline__ double sum_partials(const double* part) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < kGridBlocks; i += 32) v += part[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// x = 0, r = b, z = D^-1 b, p = z; partials of r.z and b.b. The diagonal of
// each row is found by binary search (columns ascending).
__global__ void __launch_bounds__(kBlock) k_cg_init(CgParams p) {
  __shared__ double sh[kBlock / 32];
  double rz = 0.0, bb = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * kBlock + threadIdx.x; i < p.n; i += int64_t(gridDim.x) * kBlock) {
    int64_t lo = p.row_ptr[i], hi = p.row_ptr[i + 1] - 1;
    double d = 0.0;
    while (lo <= hi) {
      const int64_t mid = (lo + hi) >> 1;
      const int64_t c = p.col[mid];
      if (c == i) { d = p.val[mid]; break; }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    if (!(d > 0.0)) atomicOr(reinterpret_cast<unsigned long long*>(p.s + S_FLAG), 0ull | kFlagNotSpd);
    const double di = d > 0.0 ? 1.0 / d : 0.0;
    const double bi = p.b[i];
    p.dinv[i] = di;
    p.x[i] = 0.0;
    p.r[i] = bi;
    p.z[i] = di * bi;
    p.p[i] = di * bi;
    rz += bi * (di * bi);
    bb += bi * bi;
  }
  const double a = block_sum(rz, sh);
  const double c = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    p.part_a[blockIdx.x] = a;
    p.part_c[blockIdx.x] = c;
  }
}

// rz (buffer 0) and b.b from the init partials; one warp.
__global__ void k_cg_init_sums(CgParams p) {
  const double rz = sum_partials(p.part_a);
  const double bb = sum_partials(p.part_c);
  if (threadIdx.x == 0) {
    p.s[S_RZ0] = rz;
    p.s[S_BB] = bb;
    p.s[S_RR] = bb;
  }
}

// q = A p and the block partials of p.q. GB300 issues FP64 at 2 lanes per
// clock per SM and charges a warp instruction in full whatever its active
// lanes, so the kernel packs its FP64 work: a group of G lanes takes one row
// (a warp 32/G consecutive rows), each lane summing every G-th nonzero of the
// row (loads of 4 nonzeros in flight per lane), then a log2(G)-step xor
// butterfly within the group. One warp per row would spend 3 multiply-add
// rounds, 5 butterfly adds and a multiply per 81-entry row; G = 4 spends 21
// rounds, 2 adds and one multiply per 8 rows. Fixed summation order
// (deterministic).
template <int G>
__global__ void __launch_bounds__(kBlock) k_spmv_dot(CgParams p) {
  __shared__ double sh[kBlock / 32];
  constexpr int RPW = 32 / G;  // rows per warp pass
  constexpr int U = 4;         // loads in flight per lane
  const int lane = threadIdx.x & 31, j = lane % G, slot = lane / G;
  const int64_t w0 = (int64_t(blockIdx.x) * kBlock + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * kBlock) >> 5;
  double pq = 0.0;
  for (int64_t base = w0 * RPW; base < p.n; base += nw * RPW) {
    const int64_t i = base + slot;
    int64_t k0 = 0, k1 = 0;
    if (i < p.n) {
      k0 = p.row_ptr[i];
      k1 = p.row_ptr[i + 1];
    }
    double acc = 0.0;
    for (int64_t k = k0 + j; k < k1; k += G * U) {
      double v[U];
      int c[U];
#pragma unroll
      for (int t = 0; t < U; ++t) {
        const int64_t kk = k + int64_t(t) * G;
        v[t] = kk < k1 ? __ldg(p.val + kk) : 0.0;
        c[t] = kk < k1 ? __ldg(p.col + kk) : 0;
      }
      // past the row's end v = 0 and c = 0: the multiply-add adds an exact zero
#pragma unroll
      for (int t = 0; t < U; ++t) acc = fma(v[t], __ldg(p.p + c[t]), acc);
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (j == 0 && i < p.n) {
      p.q[i] = acc;
      pq += p.p[i] * acc;
    }
  }
  const double t = block_sum(pq, sh);
  if (threadIdx.x == 0) p.part_a[blockIdx.x] = t;
}

// alpha = rz / p.q; x += alpha p; r -= alpha q; z = D^-1 r; partials of r.z, r.r.
__global__ void __launch_bounds__(kBlock) k_update(CgParams p, int parity) {
  __shared__ double sh[kBlock / 32];
  __shared__ double s_alpha;
  if (threadIdx.x < 32) {
    const double pq = sum_partials(p.part_a);
    if (threadIdx.x == 0) {
      const double rz = p.s[parity ? S_RZ1 : S_RZ0];
      if (!(pq > 0.0) && blockIdx.x == 0 && rz > 0.0)
        atomicOr(reinterpret_cast<unsigned long long*>(p.s + S_FLAG), 0ull | kFlagNotSpd);
      s_alpha = pq > 0.0 ? rz / pq : 0.0;
    }
  }
  __syncthreads();
  const double alpha = s_alpha;
  double rz = 0.0, rr = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * kBlock + threadIdx.x; i < p.n; i += int64_t(gridDim.x) * kBlock) {
    p.x[i] = fma(alpha, p.p[i], p.x[i]);
    const double ri = fma(-alpha, p.q[i], p.r[i]);
    const double zi = p.dinv[i] * ri;
    p.r[i] = ri;
    p.z[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
  }
  const double a = block_sum(rz, sh);
  const double c = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    p.part_b[blockIdx.x] = a;
    p.part_c[blockIdx.x] = c;
  }
}

// beta = rz_new / rz; p = z + beta p. Block 0 records rz_new (in the other
// buffer, so that no block reads a value being replaced) and r.r.
__global__ void __launch_bounds__(kBlock) k_pupdate(CgParams p, int parity) {
  __shared__ double s_beta;
  if (threadIdx.x < 32) {
    const double rz_new = sum_partials(p.part_b);
    if (threadIdx.x == 0) {
      const double rz = p.s[parity ? S_RZ1 : S_RZ0];
      s_beta = rz > 0.0 ? rz_new / rz : 0.0;
      if (blockIdx.x == 0) p.s[parity ? S_RZ0 : S_RZ1] = rz_new;
    }
    const double rr = sum_partials(p.part_c);
    if (threadIdx.x == 0 && blockIdx.x == 0) p.s[S_RR] = rr;
  }
  __syncthreads();
  const double beta = s_beta;
  for (int64_t i = int64_t(blockIdx.x) * kBlock + threadIdx.x; i < p.n; i += int64_t(gridDim.x) * kBlock)
    p.p[i] = fma(beta, p.p[i], p.z[i]);
}

// u[g] = x[label[g]] for free DOFs, 0 for fixed ones.
__global__ void __launch_bounds__(kBlock) k_expand(const int32_t* label, int64_t n_dofs, const double* x, double* u) {
  for (int64_t g = int64_t(blockIdx.x) * kBlock + threadIdx.x; g < n_dofs; g += int64_t(gridDim.x) * kBlock) {
    const int32_t l = label[g];
    u[g] = l >= 0 ? x[l] : 0.0;
  }
}

__global__ void __launch_bounds__(kBlock) k_dot(const double* a, const double* b, int64_t n, double* part) {
  __shared__ double sh[kBlock / 32];
  double v = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * kBlock + threadIdx.x; i < n; i += int64_t(gridDim.x) * kBlock)
    v += a[i] * b[i];
  const double t = block_sum(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_dot_final(const double* part, double* out) {
  const double v = sum_partials(part);
  if (threadIdx.x == 0) *out = v;
}

}  // namespace solve

int64_t compliance_work_doubles(int64_t n_free, int64_t nnz) {
  // values [nnz] | b [n] | x, r, z, p, q, D^-1 [6n] | partials [3 G] | scalars
  return nnz + 7 * n_free + 3 * solve::kGridBlocks + solve::kScalars;
}

int compliance_solve(const ComplianceArgs& a, cudaStream_t st) {
  using namespace solve;
  const int64_t n = a.n_free;
  double* w = a.work;
  double* val = w;
  double* b = val + a.nnz;
  CgParams p;
  p.n = n;
  p.row_ptr = a.row_ptr;
  p.col = a.col;
  p.val = val;
  p.b = b;
  p.x = b + n;
  p.r = p.x + n;
  p.z = p.r + n;
  p.p = p.z + n;
  p.q = p.p + n;
  p.dinv = p.q + n;
  p.part_a = p.dinv + n;
  p.part_b = p.part_a + kGridBlocks;
  p.part_c = p.part_b + kGridBlocks;
  p.s = p.part_c + kGridBlocks;
  *a.iterations = 0;
  *a.rel_residual = 0.0;
  cudaError_t e = cudaMemsetAsync(p.s, 0, kScalars * sizeof(double), st);
  if (e != cudaSuccess) return set_error(FE_ERR_CUDA, "compliance: memset");
  std::vector<double> hs(kScalars);
  if (n > 0) {
    k_cg_init<<<kGridBlocks, kBlock, 0, st>>>(p);
    k_cg_init_sums<<<1, 32, 0, st>>>(p);
    e = cudaMemcpyAsync(hs.data(), p.s, kScalars * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(FE_ERR_CUDA, "compliance: PCG start");
    const double bb = hs[S_BB];
    uint64_t flag = 0;
    std::memcpy(&flag, &hs[S_FLAG], sizeof(flag));
    if (flag & kFlagNotSpd) return set_error(FE_ERR_INVALID_ARG, "compliance: a diagonal entry is not positive");
    int it = 0;
    double rel = 0.0;
    const int64_t avg_row = a.nnz / n;  // lanes per row of the SpMV: 4 up to 128 nonzeros per row, else 8
    if (bb > 0.0) {
      rel = 1.0;
      while (it < a.max_iter && rel > a.rtol) {
        for (int j = 0; j < kCheckEvery && it < a.max_iter; ++j, ++it) {
          if (avg_row <= 128)
            k_spmv_dot<4><<<kGridBlocks, kBlock, 0, st>>>(p);
          else
            k_spmv_dot<8><<<kGridBlocks, kBlock, 0, st>>>(p);
          k_update<<<kGridBlocks, kBlock, 0, st>>>(p, it & 1);
          k_pupdate<<<kGridBlocks, kBlock, 0, st>>>(p, it & 1);
        }
        e = cudaMemcpyAsync(hs.data(), p.s, kScalars * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_error(FE_ERR_CUDA, "compliance: PCG iteration");
        std::memcpy(&flag, &hs[S_FLAG], sizeof(flag));
        if (flag & kFlagNotSpd) return set_error(FE_ERR_INVALID_ARG, "compliance: the constrained matrix is not positive definite");
        rel = std::sqrt(std::max(0.0, hs[S_RR]) / bb);
        if (!std::isfinite(rel)) return set_error(FE_ERR_INVALID_ARG, "compliance: PCG diverged");
      }
    }  // else b = 0: the initial x = 0 is the solution
    *a.iterations = it;
    *a.rel_residual = rel;
    if (rel > a.rtol) {
      return set_error(FE_ERR_NOT_CONVERGED, "compliance: PCG reached max_iter before rtol");
    }
  }
  // u over all DOFs, c = f . x over the free DOFs
  const int eb = int(std::min<int64_t>(std::max<int64_t>(1, (a.n_dofs + kBlock - 1) / kBlock), kGridBlocks));
  k_expand<<<eb, kBlock, 0, st>>>(a.label, a.n_dofs, p.x, a.u);
  k_dot<<<kGridBlocks, kBlock, 0, st>>>(b, p.x, n, p.part_a);
  k_dot_final<<<1, 32, 0, st>>>(p.part_a, a.compliance);
  e = cudaGetLastError();
  return e == cudaSuccess ? FE_OK : set_error(FE_ERR_CUDA, "compliance: kernels");
}

}  // namespace feasm
