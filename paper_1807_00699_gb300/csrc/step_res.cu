// Resident persistent GD kernel (forward Euler, BF16 coupling product).
//
// One cooperative launch runs many steps.  Each CTA owns one 128 x 128 tile
// (spins i x columns c) for the whole launch and keeps that tile's FP32 state
// in tensor memory: the accumulator (columns 0..127), the amplitudes psi
// (128..255) and the gains gamma (256..), so per step the only global traffic
// is the BF16 operand X = bf16(psi) that every CTA reads and writes.  Steps are
// separated by a grid-wide barrier (an arrival counter with bounded waits):
// the epilogue of step n writes its slice of X^{n+1}, arrives, and the TMA
// producer of every CTA waits for all arrivals before loading X^{n+1}.
//
// Roles: warp 0 TMA producer; warp 1 TMEM allocator + MMA issuer; warps 2..9
// epilogue (warp w reads TMEM lane quarter w % 4, half of the columns).
// Per-element arithmetic is the Euler update of Eqs. (2), (5), (6) with the
// same FP32 expression sequence as the per-step kernels.
#include "tc_epilogue.cuh"
#include "tc_ptx.cuh"
#include "res.h"

namespace gda {
namespace {

using namespace ptx;
constexpr int RES_THREADS = 320;
constexpr int BN = 128;
constexpr int STAGES = 6;
constexpr uint32_t A_BYTES = BM * BK * 2;
constexpr uint32_t B_BYTES = BN * BK * 2;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t T_PSI = 128;  // tensor-memory column of psi
constexpr uint32_t T_GAM = 256;  // tensor-memory column of gamma
constexpr uint32_t TAIL = (2 * STAGES + 2) * 8 + 8 * BN * 4 + 16;
constexpr uint32_t SMEM = 1024 + STAGES * STAGE_BYTES + TAIL;

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Bounded wait until the grid barrier counter reaches target.
__device__ __forceinline__ bool grid_wait(const unsigned* gbar, unsigned target) {
  if (ld_acquire_gpu(gbar) >= target) return true;
  const long long t0 = clock64();
  while (ld_acquire_gpu(gbar) < target) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

template <bool CPLX>
__global__ void __launch_bounds__(RES_THREADS, 1)
    step_res_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, ResArgs ra,
                    StepArgs a) {
  constexpr int W = CPLX ? 2 : 1;
  constexpr int RPT = BN / W;
  constexpr int CW = 16;
  constexpr int NCH = (BN / 2) / CW;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  const uint32_t sA = base;
  const uint32_t sB = base + STAGES * A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  float* s_beta = reinterpret_cast<float*>(bars + 2 * STAGES + 2);  // beta^n per local restart
  float* s_bstage = s_beta + BN;                                    // beta used in this step
  float* s_dsc = s_bstage + BN;
  float* s_red = s_dsc + BN;  // [4][BN]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_red + 4 * BN);
  int* s_flag = reinterpret_cast<int*>(s_tmem + 1);  // [0] abort, [1] diverged

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int KB = (a.N + BK - 1) / BK;
  const unsigned G = gridDim.x * gridDim.y;
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  const uint32_t acc_full = smem_u32(bars + 2 * STAGES);
  const uint32_t acc_free = smem_u32(bars + 2 * STAGES + 1);

  if (threadIdx.x == 0) {
    stamp(a, 0);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_free, 1);
    s_flag[0] = 0;
    s_flag[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(s_tmem), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  if (threadIdx.x == 0) stamp(a, 1);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int it = 0;
      for (int n = 0; n < ra.steps; ++n) {
        if (n > 0) {
          if (!grid_wait(ra.gbar, unsigned(n) * G)) {
            atomicOr(&s_flag[0], 1);
            break;
          }
          fence_proxy_async_global();
        }
        if (*(volatile int*)&s_flag[0]) break;
        const int brow = ((ra.buf0 + n) & 1) * ra.Cp + n0;
        bool stop = false;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!mbar_wait(empty_bar(s), ph ^ 1u) || *(volatile int*)&s_flag[0]) {
            atomicOr(&s_flag[0], 1);
            stop = true;
            break;
          }
          mbar_arrive_expect_tx(full_bar(s), STAGE_BYTES);
          tma_load_2d(sA + s * A_BYTES, &tmA, kb * BK, m0, full_bar(s));
          tma_load_2d(sB + s * B_BYTES, &tmB, kb * BK, brow, full_bar(s));
        }
        if (stop) break;
      }
      if (*(volatile int*)&s_flag[0]) {
        for (int k = it - 1; k >= 0 && k >= it - STAGES; --k) (void)mbar_wait(full_bar(k % STAGES), (k / STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16<BN>();
      int it = 0;
      for (int n = 0; n < ra.steps; ++n) {
        if (n > 0 && (!mbar_wait(acc_free, (n - 1) & 1) || *(volatile int*)&s_flag[0])) {
          atomicOr(&s_flag[0], 1);
          break;
        }
        tc_fence_after();
        bool stop = false;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!mbar_wait(full_bar(s), ph) || *(volatile int*)&s_flag[0]) {
            atomicOr(&s_flag[0], 1);
            stop = true;
            break;
          }
          tc_fence_after();
          if (n == 0 && kb == 0) stamp(a, 2);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            mma_bf16(tmem, sdesc_sw128(sA + s * A_BYTES + k * 32), sdesc_sw128(sB + s * B_BYTES + k * 32), idesc,
                     (kb | k) != 0);
          mma_commit(empty_bar(s));
        }
        if (n == 0) stamp(a, 3);
        mma_commit(acc_full);  // also after an abort: tracks every MMA issued
        if (stop) break;
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int e = threadIdx.x - 64;
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int i = m0 + 32 * q + lane;
    const bool row_ok = i < a.N;
    const int rbase = n0 / W;
    const size_t Np = a.Np;
    const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
    const int cb = half * (BN / 2);  // first local column of this thread
    const float h = row_ok ? a.h1[i] : 0.0f;
    const bool need_red = a.noise_decay && a.noise_D != 0.0f;

    // state -> tensor memory
#pragma unroll 1
    for (int ch = 0; ch < NCH; ++ch) {
      float v[CW];
#pragma unroll
      for (int k = 0; k < CW; ++k) v[k] = a.psi_n[size_t(n0 + cb + ch * CW + k) * Np + i];
      tmem_st16(tmem + lane_base + T_PSI + cb + ch * CW, v);
    }
#pragma unroll 1
    for (int ch = 0; ch < NCH / W; ++ch) {
      float v[CW];
#pragma unroll
      for (int k = 0; k < CW; ++k) v[k] = a.gam[size_t(rbase + cb / W + ch * CW + k) * Np + i];
      tmem_st16(tmem + lane_base + T_GAM + cb / W + ch * CW, v);
    }
    tmem_st_wait();
    if (e < RPT) {
      const int r = rbase + e;
      s_beta[e] = r < a.R ? a.beta_in[r] : 1.0f;
    }

    StepArgs sa = a;
    sa.mode = M_EULER;
    int bad = 0;
#pragma unroll 1
    for (int n = 0; n < ra.steps; ++n) {
      sa.step = a.step + unsigned(n);
      sa.rho_in = (n & 1) ? ra.rho[1] : ra.rho[0];
      if (e < RPT) {
        const int r = rbase + e;
        s_bstage[e] = s_beta[e];
        if (need_red && n > 0) (void)grid_wait(ra.gbar, unsigned(n) * G);  // partial sums of step n-1
        s_dsc[e] = r < a.R ? noise_scale(sa, r) : 0.0f;
      }
      epi_sync();
      const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_full, n & 1) && !*(volatile int*)&s_flag[0]);
      tc_fence_after();
      if (!ok) {
        if (lane == 0) atomicOr(a.err, E_TIMEOUT);
        atomicOr(&s_flag[0], 1);
        break;
      }
      if (n == 0 && e == 0) stamp(a, 4);
      __nv_bfloat16* op = ra.ops + size_t((ra.buf0 + n + 1) & 1) * ra.Cp * Np;
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) {
        const int lc0 = cb + ch * CW;       // local column of the chunk
        const int lr0 = lc0 / W;            // local restart
        uint32_t ry[CW], rp[CW], rg[CW];
        tmem_ld16_nowait(tmem + lane_base + lc0, ry);
        tmem_ld16_nowait(tmem + lane_base + T_PSI + lc0, rp);
        if (CPLX) {
          tmem_ld8_nowait(tmem + lane_base + T_GAM + lr0, rg);
        } else {
          tmem_ld16_nowait(tmem + lane_base + T_GAM + lr0, rg);
        }
        tmem_ld_wait();
        const int c0 = n0 + lc0;
        float z[CW];
        bool any = false;
#pragma unroll
        for (int u = 0; u < CW / W; ++u) any |= s_dsc[lr0 + u] != 0.0f;
#pragma unroll
        for (int qd = 0; qd < CW / 4; ++qd) {
          if (any) {
            philox_normal4(uint32_t(i), uint32_t((c0 >> 2) + qd), sa.step, 0u, a.seed, &z[4 * qd]);
          } else {
            z[4 * qd] = z[4 * qd + 1] = z[4 * qd + 2] = z[4 * qd + 3] = 0.0f;
          }
        }
        float npsi[CW], ngam[CW];
        float red[CW];
#pragma unroll
        for (int u = 0; u < CW / W; ++u) {
          const int k0 = u * W;
          const float xr = __uint_as_float(rp[k0]), xi = CPLX ? __uint_as_float(rp[k0 + 1]) : 0.0f;
          const float yr = __uint_as_float(ry[k0]), yi = CPLX ? __uint_as_float(ry[k0 + 1]) : 0.0f;
          const float gs = __uint_as_float(rg[u]);
          const float bs = s_bstage[lr0 + u];
          float kr, ki, kg;
          gd_rhs(xr, xi, gs, yr, yi, bs, h, a.eps, a.rho_th, kr, ki, kg);
          float nr = axpy(a.dt, kr, xr);
          float ni = axpy(a.dt, ki, xi);
          const float ng = axpy(a.dt, kg, gs);
          nr = axpy(s_dsc[lr0 + u], z[k0], nr);
          if (CPLX) ni = axpy(s_dsc[lr0 + u], z[k0 + 1], ni);
          const bool live = row_ok && (rbase + lr0 + u) < a.R;
          npsi[k0] = live ? nr : 0.0f;
          if (CPLX) npsi[k0 + 1] = live ? ni : 0.0f;
          ngam[u] = live ? ng : gs;
          const float rn = density(nr, ni);
          red[u] = live ? rn : 0.0f;
          bad |= live && !(rn < 1e30f);
          if (live) {
            op[size_t(c0 + k0) * Np + i] = __float2bfloat16_rn(nr);
            if (CPLX) op[size_t(c0 + k0 + 1) * Np + i] = __float2bfloat16_rn(ni);
          }
        }
        tmem_st16(tmem + lane_base + T_PSI + lc0, npsi);
        if (CPLX) {
          tmem_st8(tmem + lane_base + T_GAM + lr0, ngam);
        } else {
          tmem_st16(tmem + lane_base + T_GAM + lr0, ngam);
        }
        if (need_red) {
#pragma unroll
          for (int u = 0; u < CW / W; ++u) {
            float x = red[u];
#pragma unroll
            for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) s_red[q * BN + lr0 + u] = x;
          }
        }
      }
      tmem_st_wait();
      tc_fence_before();
      fence_proxy_async_global();
      epi_sync();
      if (e == 0) {
        mbar_arrive(acc_free);
        if (n == 0) stamp(a, 5);
      }
      if (e < RPT) {
        const int r = rbase + e;
        if (need_red && r < a.R)
          ((n & 1) ? ra.rho[0] : ra.rho[1])[size_t(blockIdx.y) * a.Rp + r] =
              s_red[e] + s_red[BN + e] + s_red[2 * BN + e] + s_red[3 * BN + e];
        s_beta[e] = next_beta(sa, s_beta[e]);
      }
      epi_sync();
      if (e == 0 && n + 1 < ra.steps) {
        __threadfence();
        red_release_gpu_add(ra.gbar, 1u);
      }
    }
    // tensor memory -> state
    if (!*(volatile int*)&s_flag[0]) {
#pragma unroll 1
      for (int ch = 0; ch < NCH; ++ch) {
        uint32_t rp[CW];
        tmem_ld16_nowait(tmem + lane_base + T_PSI + cb + ch * CW, rp);
        tmem_ld_wait();
        if (row_ok)
#pragma unroll
          for (int k = 0; k < CW; ++k) {
            const int c = n0 + cb + ch * CW + k;
            if (c < a.C) ra.psi_final[size_t(c) * Np + i] = __uint_as_float(rp[k]);
          }
      }
#pragma unroll 1
      for (int ch = 0; ch < NCH / W; ++ch) {
        uint32_t rg[CW];
        tmem_ld16_nowait(tmem + lane_base + T_GAM + cb / W + ch * CW, rg);
        tmem_ld_wait();
        if (row_ok)
#pragma unroll
          for (int k = 0; k < CW; ++k) {
            const int r = rbase + cb / W + ch * CW + k;
            if (r < a.R) a.gam[size_t(r) * Np + i] = __uint_as_float(rg[k]);
          }
      }
      if (blockIdx.y == 0 && e < RPT && rbase + e < a.R) ra.beta_final[rbase + e] = s_beta[e];
    }
    if (bad) s_flag[1] = 1;
    epi_sync();
    if (e == 0 && s_flag[1]) atomicOr(a.err, E_DIVERGED);
    if (e == 0) stamp(a, 6);
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && s_flag[0]) atomicOr(a.err, E_TIMEOUT);
  if (threadIdx.x == 0) stamp(a, 7);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

template <bool CPLX>
cudaError_t launch_res_impl(const CUtensorMap& A, const CUtensorMap& B, const ResArgs& ra, const StepArgs& a,
                            cudaStream_t s) {
  static bool attr_set = false;
  auto kern = step_res_kernel<CPLX>;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((a.C + BN - 1) / BN, (a.N + BM - 1) / BM);
  cfg.blockDim = dim3(RES_THREADS);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, A, B, ra, a);
}

}  // namespace

bool res_fits(int N, int C, int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return false;
  int per_sm = 0;
  auto kern = step_res_kernel<true>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess) return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RES_THREADS, SMEM) != cudaSuccess) return false;
  const long long grid = (long long)((C + BN - 1) / BN) * ((N + BM - 1) / BM);
  return per_sm >= 1 && grid <= (long long)per_sm * sms;
}

cudaError_t launch_step_res(const TcPlan* plan, const ResArgs& ra, const StepArgs& a, cudaStream_t s) {
  const CUtensorMap* A = tc_plan_A(plan);
  const CUtensorMap* B = tc_plan_B(plan);
  return a.cplx ? launch_res_impl<true>(*A, *B, ra, a, s) : launch_res_impl<false>(*A, *B, ra, a, s);
}

}  // namespace gda
