// Self-test of the conversions that the kernels of this library do on the
// integer bits instead of the FP64 pipe (a check of the library's arithmetic
// against the hardware conversions; the paper has no counterpart). For each
// FP64 input the kernel writes the integer-bit results next to the hardware
// results, and the caller compares them bit for bit.
#include "fe_device.cuh"

namespace feasm {
namespace {

__global__ void k_selftest_conversions(const double* x, int64_t n, float* out32, double* out64) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool in = i < n;
  const double v = in ? x[i] : 0.0;
  // FP64 -> FP32: hardware, the general integer-bit conversion, the
  // branch-free one (with its out-of-range flag) and the remainder below it
  const float hw = __double2float_rn(v);
  const float a = d2f_rn(v);
  bool odd = false, odd_rest = false;
  const float b = d2f_fast(v, odd);
  const float r = d2f_rest(v, odd_rest);
  const float r_hw = __double2float_rn(v - double(hw));
  // FP32 pair -> FP64 rounded once: the warp-collective integer path and the
  // fixed-point sum, against one hardware FP64 addition of the exact operands
  const double p_int = df_to_double(hw, r_hw);
  const float pair[2] = {hw, r_hw};
  const double p_fx = fx_sum_regs_f32(pair);
  const double p_hw = __dadd_rn(double(hw), double(r_hw));
  // FP32 -> FP64 (exact), integer bits against the hardware
  const double f_int = f32_to_f64_exact(hw);
  const double f_hw = double(hw);
  // TF32 split of the FP32 value (hi = tf32(x), lo = tf32(x - hi))
  const float th = to_tf32(hw), tl = to_tf32(hw - th);
  if (in) {
    float* o = out32 + i * 8;
    o[0] = hw;
    o[1] = a;
    o[2] = b;
    o[3] = float(int(odd) + 2 * int(odd_rest));
    o[4] = r;
    o[5] = r_hw;
    o[6] = th;
    o[7] = tl;
    double* d = out64 + i * 5;
    d[0] = p_int;
    d[1] = p_fx;
    d[2] = p_hw;
    d[3] = f_int;
    d[4] = f_hw;
  }
}

}  // namespace
}  // namespace feasm

extern "C" int fe_selftest_conversions(const double* x, int64_t n, float* out32, double* out64, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out32 || !out64)))
    return feasm::set_error(FE_ERR_INVALID_ARG, "invalid self-test buffers");
  if (n == 0) return FE_OK;
  const int64_t blocks = (n + 255) / 256;
  feasm::k_selftest_conversions<<<unsigned(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, out32, out64);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FE_OK : feasm::set_error(FE_ERR_CUDA, cudaGetErrorString(e));
}
