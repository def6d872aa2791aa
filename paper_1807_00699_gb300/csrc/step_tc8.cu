// FP8 coupling operands: E4M3 instantiation of the tensor-core step kernel
// (step_tc.cuh) and the conversions that produce its operands.
//
// J0 is stored row-scaled, J8_ij = e4m3(J0_ij / s_i) with s_i = max_j |J0_ij|
// / 448 (448 is E4M3's largest finite value), and the amplitudes at the fixed
// scale sigma = 1/64, X8 = e4m3(psi / sigma).  The accumulator then holds
// sum_j (J0_ij / s_i)(psi_j / sigma) and the epilogue multiplies by s_i sigma.
// All conversions round to nearest even and saturate (satfinite).
#include <cuda_fp8.h>

#include "step_tc.cuh"

namespace gda {

namespace {

// One block of 256 threads per row of J0 (FP32, diagonal removed).
__global__ void k_prepare_J8(const float* J32, int Np, unsigned char* J8, float* scale) {
  const int i = blockIdx.x;
  const float* row = J32 + size_t(i) * Np;
  float m = 0.0f;
  for (int j = threadIdx.x; j < Np; j += blockDim.x) m = fmaxf(m, fabsf(row[j]));
  __shared__ float red[8];
  for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
    for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  m = red[0];
  const float s = m > 0.0f ? __fdiv_rn(m, 448.0f) : 1.0f;
  if (threadIdx.x == 0) scale[i] = s;
  unsigned char* out = J8 + size_t(i) * Np;
  for (int j = threadIdx.x; j < Np; j += blockDim.x)
    out[j] = __nv_cvt_float_to_fp8(__fdiv_rn(row[j], s), __NV_SATFINITE, __NV_E4M3);
}

__global__ void k_to_e4m3(const float* x, unsigned char* y, size_t n, float inv) {
  for (size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x; k < n; k += size_t(gridDim.x) * blockDim.x)
    y[k] = __nv_cvt_float_to_fp8(__fmul_rn(x[k], inv), __NV_SATFINITE, __NV_E4M3);
}

}  // namespace

cudaError_t launch_prepare_J8(const float* J32, int Np, unsigned char* J8, float* scale, cudaStream_t s) {
  k_prepare_J8<<<Np, 256, 0, s>>>(J32, Np, J8, scale);
  return cudaGetLastError();
}

cudaError_t launch_to_e4m3(const float* x, unsigned char* y, size_t n, cudaStream_t s) {
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks == 0) blocks = 1;
  k_to_e4m3<<<unsigned(blocks), 256, 0, s>>>(x, y, n, 1.0f / kFp8PsiScale);
  return cudaGetLastError();
}

cudaError_t tc_plan8_create(TcPlan** plan, const unsigned char* J8, int Np, const unsigned char* ops8, int n_op_bufs,
                            int Cp) {
  TcPlan* p = new TcPlan();
  if (!plan_maps<true>(p, J8, Np, ops8, n_op_bufs, Cp)) {
    delete p;
    return cudaErrorInvalidValue;
  }
  *plan = p;
  return cudaSuccess;
}

cudaError_t launch_step_tcs8(const TcPlan* plan, const StepArgs& a, const SegArgs& g, cudaStream_t s, bool pair) {
  return launch_seg_plan<true>(plan, a, g, pair, s);
}

cudaError_t launch_step_tc8(const TcPlan* plan, const StepArgs& a, int op_buf, cudaStream_t s, bool pair) {
  if (!a.row_scale) return cudaErrorInvalidValue;
  return launch_plan<true>(plan, a, op_buf, pair, s);
}

}  // namespace gda
