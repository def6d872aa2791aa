// FP32 CUDA-core GD step: a tiled SGEMM Y = J0 X over one 64x64 tile of
// (spins i) x (columns c), fused with the step epilogue (Eqs. 2, 5, 6).  This
// is the plain FP32 path the tensor-core path is measured against, and the
// path whose amplitudes are compared with the FP64 oracle.
#include "epilogue.cuh"

namespace gda {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, PAD = 4;

template <bool CPLX>
__global__ void __launch_bounds__(256) step_simt_kernel(StepArgs a, const float* __restrict__ J,
                                                        const float* __restrict__ X) {
  __shared__ __align__(16) float As[BK][BM + PAD];
  __shared__ __align__(16) float Bs[BK][BN + PAD];
  __shared__ float s_beta[BN], s_dsc[BN];
  __shared__ int s_bad;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int Np = a.Np;
  constexpr int RPT = CPLX ? BN / 2 : BN;  // restarts per tile
  const int rbase = CPLX ? n0 / 2 : n0;

  if (tid == 0) s_bad = 0;
  if (tid < RPT) {
    const int r = rbase + tid;
    const float b = r < a.R ? a.beta_in[r] : 1.0f;
    s_beta[tid] = stage_beta(a, b);
    s_dsc[tid] = r < a.R ? noise_scale(a, r) : 0.0f;
  }

  float acc[4][4] = {};
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const float* Jp = J + size_t(m0 + lr) * Np + lk;
  const float* Xp = X + size_t(n0 + lr) * Np + lk;
  for (int k0 = 0; k0 < Np; k0 += BK) {
    const float4 av = *reinterpret_cast<const float4*>(Jp + k0);
    const float4 bv = *reinterpret_cast<const float4*>(Xp + k0);
    __syncthreads();
    As[lk + 0][lr] = av.x; As[lk + 1][lr] = av.y; As[lk + 2][lr] = av.z; As[lk + 3][lr] = av.w;
    Bs[lk + 0][lr] = bv.x; Bs[lk + 1][lr] = bv.y; Bs[lk + 2][lr] = bv.z; Bs[lk + 3][lr] = bv.w;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[k][4 * ty]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float av2 = As[k][tx + 16 * q];
        acc[q][0] += av2 * b4.x; acc[q][1] += av2 * b4.y;
        acc[q][2] += av2 * b4.z; acc[q][3] += av2 * b4.w;
      }
    }
  }
  __syncthreads();

  // Epilogue: rows m0 + tx + 16 q, columns c0 .. c0 + 3.
  const int c0 = n0 + 4 * ty;
  constexpr int U = CPLX ? 2 : 4;
  const int lr0 = CPLX ? 2 * ty : 4 * ty;  // first local restart of the quad
  float rsum[4] = {0.f, 0.f, 0.f, 0.f};
  int bad = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = m0 + tx + 16 * q;
    if (i >= a.N) continue;
    float red[4];
    epi_quad<CPLX>(a, i, c0, acc[q], &s_beta[lr0], &s_dsc[lr0], red, bad);
#pragma unroll
    for (int u = 0; u < U; ++u) rsum[u] += red[u];
  }
  // Sum over the 16 row groups (lanes with the same ty are one half-warp).
#pragma unroll
  for (int u = 0; u < U; ++u) {
#pragma unroll
    for (int off = 8; off; off >>= 1) rsum[u] += __shfl_xor_sync(0xffffffffu, rsum[u], off);
  }
  float* out = (a.mode == M_ENERGY) ? a.e_part : (step_completes(a.mode) ? a.rho_out : nullptr);
  if (tx == 0 && out) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = rbase + lr0 + u;
      if (r < a.R) out[size_t(blockIdx.y) * a.Rp + r] = rsum[u];
    }
  }
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (tid == 0 && s_bad) atomicOr(a.err, E_DIVERGED);
  if (blockIdx.y == 0 && step_completes(a.mode) && tid < RPT) {
    const int r = rbase + tid;
    if (r < a.R) a.beta_out[r] = next_beta(a, a.beta_in[r]);
  }
}

}  // namespace

int simt_mtiles(int N) { return (N + BM - 1) / BM; }

cudaError_t launch_step_simt(const StepArgs& a, const float* J32, const float* operand, cudaStream_t s) {
  dim3 grid((a.C + BN - 1) / BN, simt_mtiles(a.N));
  if (a.cplx)
    step_simt_kernel<true><<<grid, 256, 0, s>>>(a, J32, operand);
  else
    step_simt_kernel<false><<<grid, 256, 0, s>>>(a, J32, operand);
  return cudaGetLastError();
}

}  // namespace gda
