// GD-mod step (Sec. 2; Eqs. 2, 5, 6 with Delta_ij = gamma_i^inj + gamma_j^inj):
// every restart r carries its own coupling matrix K_r, so the coupling sum is
// a per-restart matrix-vector product and K_r is rewritten every step.  The
// step streams K (read + write, 8 bytes per element) from HBM; J (shared by
// all restarts) stays in L2.  FP32 throughout.
//
// One CTA (8 warps) handles 32 rows of one restart (CTA index = restart x
// row blocks + row block): the restart's gains
// gamma^inj_j = gamma_j + gamma_c and amplitudes are staged in shared memory,
// each warp walks whole rows with 16-byte loads (K with streaming hints), and
// lane 0 applies the amplitude / gain update of the row after a shuffle
// reduction.  Gains are double-buffered (other CTAs read gamma_j during the
// step); K_rij is read and written by one thread only, so it is updated in
// place.
#include "epilogue.cuh"
#include "gda_internal.h"

namespace gda {

namespace {

constexpr int kModThreads = 256;
constexpr int kModRows = 32;  // rows per CTA (4 per warp)

struct ModArgs {
  StepArgs a;         // N, Np, R, Rp, cplx, step parameters, psi_n -> psi_out, h1, err
  const float* J;     // [Np][Np] J with the diagonal removed
  float* K;           // [R][N][Np]
  const float* gin;   // gamma^n   [Rp][Np]
  float* gout;        // gamma^n+1 [Rp][Np]
  float gamma_c;
  float ceh;          // dt * eps_hat
};

template <bool CPLX>
__global__ void __launch_bounds__(kModThreads) k_gdmod_step(ModArgs m) {
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const StepArgs& a = m.a;
  const int Np = a.Np, N = a.N;
  const int nrb = (N + kModRows - 1) / kModRows;
  const int r = blockIdx.x / nrb, rb = blockIdx.x % nrb;
  const int c = CPLX ? 2 * r : r;
  float* s_g = sm;             // gamma^inj_j (0 beyond N)
  float* s_pr = sm + Np;       // Re psi_j
  float* s_pi = sm + 2 * Np;   // Im psi_j (XY)
  const float* pr = a.psi_n + size_t(c) * Np;
  const float* gr = m.gin + size_t(r) * Np;
  for (int j = threadIdx.x; j < Np; j += kModThreads) {
    s_g[j] = j < N ? __fadd_rn(gr[j], m.gamma_c) : 0.0f;
    s_pr[j] = pr[j];
    if (CPLX) s_pi[j] = pr[Np + j];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float dsc = noise_scale(a, r);
  int bad = 0;
  for (int k = 0; k < kModRows / 8; ++k) {
    const int i = rb * kModRows + k * 8 + warp;
    if (i >= N) break;  // warp-uniform
    const float gi = s_g[i];
    float4* Krow = reinterpret_cast<float4*>(m.K + (size_t(r) * N + i) * Np);
    const float4* Jrow = reinterpret_cast<const float4*>(m.J + size_t(i) * Np);
    float yr = 0.0f, yi = 0.0f;
#pragma unroll 4
    for (int q = lane; q < Np / 4; q += 32) {
      float4 kv = __ldcs(Krow + q);
      const float4 jv = __ldg(Jrow + q);
      const float4 gv = reinterpret_cast<const float4*>(s_g)[q];
      const float4 pv = reinterpret_cast<const float4*>(s_pr)[q];
      float4 iv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (CPLX) iv = reinterpret_cast<const float4*>(s_pi)[q];
      float* kp = &kv.x;
      const float* jp = &jv.x;
      const float* gp = &gv.x;
      const float* pp = &pv.x;
      const float* ip = &iv.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float dk = __fmul_rn(__fadd_rn(gi, gp[e]), kp[e]);  // Delta_ij K_ij
        yr = __fmaf_rn(dk, pp[e], yr);
        if (CPLX) yi = __fmaf_rn(dk, ip[e], yi);
        kp[e] = __fmaf_rn(m.ceh, __fsub_rn(jp[e], dk), kp[e]);  // Eq. (6), Euler
      }
      __stcs(Krow + q, kv);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      yr += __shfl_xor_sync(0xffffffffu, yr, off);
      if (CPLX) yi += __shfl_xor_sync(0xffffffffu, yi, off);
    }
    if (lane == 0) {
      const float xr = s_pr[i], xi = CPLX ? s_pi[i] : 0.0f;
      const float gs = gr[i];
      float kr, ki, kg;
      gd_rhs(xr, xi, gs, yr, yi, 1.0f, a.h1[i], a.eps, a.rho_th, kr, ki, kg);
      float nr = axpy(a.dt, kr, xr);
      float ni = axpy(a.dt, ki, xi);
      if (dsc != 0.0f) {
        float z[4];
        philox_normal4(uint32_t(i), uint32_t(c >> 2), a.step, 0u, a.seed, z);
        nr = axpy(dsc, z[c & 3], nr);
        if (CPLX) ni = axpy(dsc, z[(c & 3) + 1], ni);
      }
      const size_t o0 = size_t(c) * Np + i;
      a.psi_out[o0] = nr;
      if (CPLX) a.psi_out[o0 + Np] = ni;
      m.gout[size_t(r) * Np + i] = axpy(a.dt, kg, gs);
      bad |= !(density(nr, ni) < 1e30f);
    }
  }
  if (bad) atomicOr(a.err, E_DIVERGED);
}

__global__ void k_gdmod_init(float* K, const float* J, float beta0, int N, int Np, int R) {
  const size_t per = size_t(N) * Np / 4;
  const size_t total = per * R;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < total; q += size_t(gridDim.x) * blockDim.x) {
    const float4 jv = reinterpret_cast<const float4*>(J)[q % per];
    reinterpret_cast<float4*>(K)[q] = make_float4(beta0 * jv.x, beta0 * jv.y, beta0 * jv.z, beta0 * jv.w);
  }
}

}  // namespace

size_t gdmod_smem_bytes(int Np, bool cplx) { return size_t(cplx ? 3 : 2) * Np * sizeof(float); }

cudaError_t launch_gdmod_init(float* K, const float* J, float beta0, int N, int Np, int R, cudaStream_t s) {
  k_gdmod_init<<<152 * 8, 256, 0, s>>>(K, J, beta0, N, Np, R);
  return cudaGetLastError();
}

cudaError_t launch_gdmod_step(const StepArgs& a, const float* J, float* K, const float* gin, float* gout,
                              float gamma_c, float ceh, cudaStream_t s) {
  ModArgs m{a, J, K, gin, gout, gamma_c, ceh};
  m.a.mode = M_EULER;
  m.a.noise_decay = 0;
  const size_t smem = gdmod_smem_bytes(a.Np, a.cplx);
  const unsigned grid = unsigned((a.N + kModRows - 1) / kModRows) * unsigned(a.R);
  if (a.cplx) {
    static bool set = false;
    if (!set && smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_gdmod_step<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      if (e != cudaSuccess) return e;
      set = true;
    }
    k_gdmod_step<true><<<grid, kModThreads, smem, s>>>(m);
  } else {
    static bool set = false;
    if (!set && smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_gdmod_step<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      if (e != cudaSuccess) return e;
      set = true;
    }
    k_gdmod_step<false><<<grid, kModThreads, smem, s>>>(m);
  }
  return cudaGetLastError();
}

}  // namespace gda
