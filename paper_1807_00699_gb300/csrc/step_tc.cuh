// Tensor-core GD step kernel for sm_103a, shared by the BF16 (step_tc.cu) and
// FP8 (step_tc8.cu) instantiations: Y = J0 X with tcgen05.mma (BF16 or E4M3
// operands, FP32 accumulator in tensor memory), both operands staged in shared
// memory by TMA (cp.async.bulk.tensor, 128-byte swizzle, no multicast), fused
// with the step epilogue of Eqs. (2), (5), (6).
//
// One CTA computes one 128 x BN tile of Y (spins x columns).  Warp roles:
//   warp 0        TMA producer (one elected lane), STAGES-deep ring
//   warp 1        TMEM allocator and MMA issuer (one elected lane)
//   warps 2..      epilogue (16 warps, 8 for RK stages 2-4): warp w reads
//                 TMEM lane quarter (w % 4) and one of 4 (2) column parts,
//                 and runs the per-element update.
// A pipeline stage holds 128 bytes of K per row in either precision (64 BF16
// or 128 E4M3 values), so stage sizes, swizzle and descriptors are shared.
// Every mbarrier wait is bounded by a clock budget; on expiry the CTA records
// E_TIMEOUT, stops issuing work, drains what it issued and frees its TMEM.
#pragma once
#include <cuda.h>

#include <cstdio>

#include "tc_epilogue.cuh"
#include "tc_ptx.cuh"

namespace gda {

namespace {

using namespace ptx;
// Epilogue warps per CTA: 16 in every mode.  The epilogue streams the FP32
// state, and more warps keep more loads and stores in flight: for RK stages
// 2-4 this outweighs the few registers their extra stage values spill at the
// 96-register budget of a 576-thread block (measured 14-30 % faster per RK4
// step than 8 warps without spills).
template <int MODE>
struct TcThreads {
  static constexpr int EPI = 16;
  static constexpr int N = 64 + 32 * EPI;
};

// PAIR: two-SM tiles (cta_group::2); each CTA of the pair stages its own 128
// rows of A and half (BN / 2) of B's columns.
template <int BN, int STAGES, bool PAIR = false>
struct TcCfg {
  static constexpr int BH = PAIR ? BN / 2 : BN;  // B columns staged per CTA
  static constexpr uint32_t A_BYTES = BM * BK * 2;
  static constexpr uint32_t B_BYTES = BH * BK * 2;
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr uint32_t TAIL = (2 * STAGES + 4) * 8 + 6 * BN * 4 + 16;
  static constexpr uint32_t SMEM = 1024 + STAGES * STAGE_BYTES + TAIL;
};

// Persistent over output tiles: CTA b processes tiles b, b + gridDim.x, ...
// (column block fastest), with two tensor-memory accumulators so that the
// epilogue of one tile overlaps the MMAs of the next.
//
// PAIR: launched in clusters of two CTAs; cluster c processes pair tiles c,
// c + clusters, ... of 256 x BN (row blocks 2p and 2p + 1, one per CTA).
// Both CTAs load their A rows and their half of B with completion counted on
// the even CTA's full barrier; the even CTA's MMA warp issues M = 256 MMAs and
// commits to the empty / accumulator barriers of both CTAs; each CTA's
// epilogue reads its own 128 accumulator rows and arrives on the even CTA's
// accumulator-empty barrier.
template <int BN, int STAGES, bool CPLX, int MODE, bool F8, bool PAIR>
__global__ void __launch_bounds__(TcThreads<MODE>::N, 1)
    step_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int b_row0,
                   StepArgs a) {
  using Cfg = TcCfg<BN, STAGES, PAIR>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  const uint32_t sA = base;
  const uint32_t sB = base + STAGES * Cfg::A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  float* s_beta = reinterpret_cast<float*>(bars + 2 * STAGES + 4);
  float* s_dsc = s_beta + BN;
  float* s_red = s_dsc + BN;  // [4][BN]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_red + 4 * BN);
  int* s_flag = reinterpret_cast<int*>(s_tmem + 1);  // [0] abort, [1] diverged

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long lim = a.wait_cycles;
  constexpr int BKE = F8 ? 2 * BK : BK;  // elements per 128-byte K slice
  const int KB = (a.N + BKE - 1) / BKE;
  const int NT = (a.C + BN - 1) / BN;
  const int MT = (a.N + BM - 1) / BM;  // even when PAIR (the host checks)
  const int T = NT * (PAIR ? MT / 2 : MT);
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  const int unit0 = PAIR ? int(cluster_id_x()) : int(blockIdx.x);
  const int nunit = PAIR ? int(ncluster_x()) : int(gridDim.x);
  auto tile_m0 = [&](int t) { return (PAIR ? 2 * (t / NT) + int(rank) : t / NT) * BM; };
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto acc_full = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto acc_empty = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };

  if (threadIdx.x == 0) {
    stamp(a, 0);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), PAIR ? 2 : 1);
    }
    s_flag[0] = 0;
    s_flag[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr uint32_t TCOLS = 2 * BN <= 256 ? 256 : 512;  // power of two
  if (warp == 1) {
    if (PAIR)
      tmem_alloc_pair(smem_u32(s_tmem), TCOLS);
    else
      tmem_alloc(smem_u32(s_tmem), TCOLS);
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // barriers of both CTAs initialised before any remote arrival
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  if (threadIdx.x == 0) stamp(a, 1);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const uint64_t keep = policy_evict_last();  // J and the operand are re-read by every tile row / column
      int it = 0;
      bool stop = false;
      for (int t = unit0; t < T && !stop; t += nunit) {
        const int m0 = tile_m0(t), n0 = (t % NT) * BN + int(rank) * Cfg::BH;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!mbar_wait(empty_bar(s), ph ^ 1u, lim) || *(volatile int*)&s_flag[0]) {
            stop = true;
            break;
          }
          if (PAIR) {
            const uint32_t fb = mapa_shared(full_bar(s), 0);  // the even CTA counts both CTAs' bytes
            if (leader) mbar_arrive_expect_tx(full_bar(s), 2 * Cfg::STAGE_BYTES);
            tma_load_2d_pair_hint(sA + s * Cfg::A_BYTES, &tmA, kb * BKE, m0, fb, keep);
            tma_load_2d_pair_hint(sB + s * Cfg::B_BYTES, &tmB, kb * BKE, b_row0 + n0, fb, keep);
          } else {
            mbar_arrive_expect_tx(full_bar(s), Cfg::STAGE_BYTES);
            tma_load_2d_hint(sA + s * Cfg::A_BYTES, &tmA, kb * BKE, m0, full_bar(s), keep);
            tma_load_2d_hint(sB + s * Cfg::B_BYTES, &tmB, kb * BKE, b_row0 + n0, full_bar(s), keep);
          }
        }
      }
      if (stop) {
        atomicOr(&s_flag[0], 1);
        // copies still in flight: the even CTA waits for its full barriers (they
        // count both CTAs' bytes); the odd CTA for the MMAs that consume its
        // stages to release them (bounded: the even CTA may have stopped)
        for (int k = it - 1; k >= 0 && k >= it - STAGES; --k) {
          if (!PAIR || leader)
            (void)mbar_wait(full_bar(k % STAGES), (k / STAGES) & 1, lim);
          else
            (void)mbar_wait(empty_bar(k % STAGES), (k / STAGES) & 1, lim);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && leader) {
      constexpr uint32_t idesc = PAIR ? (F8 ? idesc_e4m3_m256<BN>() : idesc_bf16_m256<BN>())
                                      : (F8 ? idesc_e4m3<BN>() : idesc_bf16<BN>());
      int it = 0, lt = 0;
      bool stop = false;
      for (int t = unit0; t < T && !stop; t += nunit, ++lt) {
        const int b = lt & 1;
        const uint32_t use = lt >> 1;
        const bool free_ok = PAIR ? mbar_wait_cluster(acc_empty(b), (use & 1) ^ 1u, lim)
                                  : mbar_wait(acc_empty(b), (use & 1) ^ 1u, lim);
        if (!free_ok || *(volatile int*)&s_flag[0]) {
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t dacc = tmem + b * BN;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!mbar_wait(full_bar(s), ph, lim) || *(volatile int*)&s_flag[0]) {
            stop = true;
            break;
          }
          tc_fence_after();
          if (lt == 0 && kb == 0) stamp(a, 2);
#pragma unroll
          for (int k = 0; k < 4; ++k) {  // 32 bytes of K per instruction
            const uint64_t da = sdesc_sw128(sA + s * Cfg::A_BYTES + k * 32);
            const uint64_t db = sdesc_sw128(sB + s * Cfg::B_BYTES + k * 32);
            if (PAIR) {
              if (F8)
                mma_e4m3_pair(dacc, da, db, idesc, (kb | k) != 0);
              else
                mma_bf16_pair(dacc, da, db, idesc, (kb | k) != 0);
            } else {
              if (F8)
                mma_e4m3(dacc, da, db, idesc, (kb | k) != 0);
              else
                mma_bf16(dacc, da, db, idesc, (kb | k) != 0);
            }
          }
          if (PAIR)
            mma_commit_pair(empty_bar(s));
          else
            mma_commit(empty_bar(s));
        }
        if (lt == 0) stamp(a, 3);
        if (PAIR)
          mma_commit_pair(acc_full(b));  // also after an abort: tracks every MMA issued into b
        else
          mma_commit(acc_full(b));
        if (stop) {
          (void)mbar_wait(acc_full(b), use & 1, lim);  // those MMAs finish before the CTA frees TMEM
          break;
        }
      }
      if (stop) atomicOr(&s_flag[0], 1);
    }
  } else {
    // ---------------- epilogue warps ----------------
    constexpr int W = CPLX ? 2 : 1;
    constexpr int RPT = BN / W;
    constexpr int NEPI = TcThreads<MODE>::EPI;
    constexpr int NPART = NEPI / 4;  // column parts
    constexpr int PW = BN / NPART;   // columns per part
    constexpr int CW = (ModeTraits<MODE>::rk_mid || !CPLX || NPART > 2) ? 8 : 16;
    constexpr int NCH = PW / CW;
    static_assert(PW % CW == 0, "column part must hold whole chunks");
    const int e = threadIdx.x - 64;
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;
    const bool need_red = MODE == M_ENERGY || ((MODE == M_EULER || MODE == M_RK4) && a.rho_out != nullptr);
    float* out = (MODE == M_ENERGY) ? a.e_part : ((MODE == M_EULER || MODE == M_RK4) ? a.rho_out : nullptr);
    constexpr int PD = ModeTraits<MODE>::prefetch;  // chunks loaded ahead of the one computed
    constexpr int NB = PD + 1;
    constexpr int PF = ModeTraits<MODE>::l2_ahead;  // chunks pulled into L2 ahead of their loads
    int bad = 0;
    int lt = 0;
    EpiRegs<MODE, CPLX, CW> R[NB];
    for (int t = unit0; t < T; t += nunit, ++lt) {
      const int m0 = tile_m0(t), n0 = (t % NT) * BN;
      const int mt = m0 / BM;
      const int b = lt & 1;
      const uint32_t use = lt >> 1;
      const int rbase = n0 / W;
      const int i = m0 + 32 * q + lane;
      const int cbeg = n0 + part * PW;
      // FP8: the accumulator holds (J0_ij / s_i)(psi_j / sigma); one product
      // with s_i sigma restores Y (sigma a power of two: exact).
      const float rs = F8 ? __fmul_rn(a.row_scale[i], kFp8PsiScale) : 1.0f;
      if (lt == 0) {  // later tiles had theirs pulled in during the previous tile
#pragma unroll
        for (int p = 0; p < PF && p < NCH; ++p) epi_prefetch_l2<MODE, CPLX, CW>(a, i, cbeg + p * CW, lane);
      }
#pragma unroll
      for (int p = 0; p < PD && p < NCH; ++p) epi_load<MODE, CPLX, CW>(a, i, cbeg + p * CW, R[p]);  // overlaps the MMAs
      if (e < RPT) {
        const int r = rbase + e;
        const float bt = r < a.R ? a.beta_in[r] : 1.0f;
        s_beta[e] = stage_beta(a, bt);
        s_dsc[e] = r < a.R ? noise_scale(a, r) : 0.0f;
      }
      // one decision for all epilogue warps (the vote is also the barrier that
      // publishes s_beta / s_dsc)
      const bool ok = epi_vote_all<32 * NEPI>(mbar_wait(acc_full(b), use & 1, lim) && !*(volatile int*)&s_flag[0]);
      tc_fence_after();
      if (!ok) {
        if (lane == 0) atomicOr(a.err, E_TIMEOUT);
        atomicOr(&s_flag[0], 1);
        break;
      }
      if (lt == 0 && e == 0) stamp(a, 4);
      const uint32_t taddr = tmem + b * BN + (static_cast<uint32_t>(32 * q) << 16) + part * PW;
      auto body = [&](int ch, const EpiRegs<MODE, CPLX, CW>& cur) {
        float v[CW];
        tmem_ld<CW>(taddr + ch * CW, v);
        if (F8) {
#pragma unroll
          for (int k = 0; k < CW; ++k) v[k] = __fmul_rn(v[k], rs);
        }
        const int lr0 = (part * PW + ch * CW) / W;
        float red[CW / W];
        epi_chunk<MODE, CPLX, CW>(a, i, cbeg + ch * CW, v, cur, &s_beta[lr0], &s_dsc[lr0], red, bad);
        if (need_red) {
#pragma unroll
          for (int u = 0; u < CW / W; ++u) {
            float x = red[u];
#pragma unroll
            for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) s_red[q * BN + lr0 + u] = x;
          }
        }
      };
      // fully unrolled, so every register buffer index is a constant
      // the next tile of this CTA: its first chunks are pulled into L2 during
      // the last chunks of this one
      const int tn = t + nunit;
      const int i_next = tile_m0(tn) + 32 * q + lane;
      const int cbeg_next = (tn % NT) * BN + part * PW;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        if (PF > 0) {
          if (ch + PF < NCH)
            epi_prefetch_l2<MODE, CPLX, CW>(a, i, cbeg + (ch + PF) * CW, lane);
          else if (tn < T && ch + PF - NCH < NCH)
            epi_prefetch_l2<MODE, CPLX, CW>(a, i_next, cbeg_next + (ch + PF - NCH) * CW, lane);
        }
        if (ch + PD < NCH) epi_load<MODE, CPLX, CW>(a, i, cbeg + (ch + PD) * CW, R[(ch + PD) % NB]);
        body(ch, R[ch % NB]);
      }
      tc_fence_before();
      epi_bar_sync_n<32 * NEPI>();
      if (e == 0) {  // accumulator b may be overwritten
        if (PAIR && !leader)
          mbar_arrive_cluster(mapa_shared(acc_empty(b), 0));
        else
          mbar_arrive(acc_empty(b));
      }
      if (lt == 0 && e == 0) stamp(a, 5);
      if (e < RPT) {
        const int r = rbase + e;
        if (r < a.R) {
          if (out)
            out[size_t(mt) * a.Rp + r] = s_red[e] + s_red[BN + e] + s_red[2 * BN + e] + s_red[3 * BN + e];
          if (mt == 0 && (MODE == M_EULER || MODE == M_RK4)) a.beta_out[r] = next_beta(a, a.beta_in[r]);
        }
      }
    }
    if (bad) s_flag[1] = 1;
    epi_bar_sync_n<32 * NEPI>();
    if (e == 0 && s_flag[1]) atomicOr(a.err, E_DIVERGED);
    if (e == 0) stamp(a, 6);
  }

  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // no CTA leaves while its peer may still signal or read it
  if (threadIdx.x == 0 && s_flag[0]) atomicOr(a.err, E_TIMEOUT);
  if (threadIdx.x == 0) stamp(a, 7);
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem, TCOLS);
    else
      tmem_dealloc(tmem, TCOLS);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D tensor [rows][Np] of BF16 (f8 false) or E4M3 bytes (f8 true) with a
// box of 128 bytes x box_rows and 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* ptr, int Np, int rows, int box_rows, bool f8 = false) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  const cuuint64_t esz = f8 ? 1 : 2;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(Np), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(Np) * esz};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / esz), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr),
             dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int STAGES, bool CPLX, int MODE, bool F8, bool PAIR>
cudaError_t launch_cfg(const CUtensorMap& A, const CUtensorMap& B, int b_row0, const StepArgs& a, cudaStream_t s) {
  using Cfg = TcCfg<BN, STAGES, PAIR>;
  static bool attr_set = false;
  auto kern = step_tc_kernel<BN, STAGES, CPLX, MODE, F8, PAIR>;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaErrorUnknown;
  }
  const int NT = (a.C + BN - 1) / BN, MT = (a.N + BM - 1) / BM;
  if (!PAIR) {
    const int tiles = NT * MT;
    kern<<<tiles < sms ? tiles : sms, TcThreads<MODE>::N, Cfg::SMEM, s>>>(A, B, b_row0, a);
    return cudaGetLastError();
  }
  if (MT % 2) return cudaErrorInvalidValue;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(TcThreads<MODE>::N);
  cfg.dynamicSmemBytes = Cfg::SMEM;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  static int max_clusters = 0;
  if (!max_clusters) {
    cfg.gridDim = dim3(2 * (sms / 2));
    cudaError_t e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (max_clusters < 1) return cudaErrorLaunchOutOfResources;
  }
  const int ptiles = NT * (MT / 2);
  cfg.gridDim = dim3(2 * (ptiles < max_clusters ? ptiles : max_clusters));
  return cudaLaunchKernelEx(&cfg, kern, A, B, b_row0, a);
}

template <int BN, int STAGES, bool CPLX, bool F8, bool PAIR>
cudaError_t dispatch_cplx(const CUtensorMap& A, const CUtensorMap& B, int b_row0, const StepArgs& a, cudaStream_t s) {
  switch (a.mode) {
    case M_EULER: return launch_cfg<BN, STAGES, CPLX, M_EULER, F8, PAIR>(A, B, b_row0, a, s);
    case M_RK1: return launch_cfg<BN, STAGES, CPLX, M_RK1, F8, PAIR>(A, B, b_row0, a, s);
    case M_RK2: return launch_cfg<BN, STAGES, CPLX, M_RK2, F8, PAIR>(A, B, b_row0, a, s);
    case M_RK3: return launch_cfg<BN, STAGES, CPLX, M_RK3, F8, PAIR>(A, B, b_row0, a, s);
    case M_RK4: return launch_cfg<BN, STAGES, CPLX, M_RK4, F8, PAIR>(A, B, b_row0, a, s);
    case M_ENERGY: return launch_cfg<BN, STAGES, CPLX, M_ENERGY, F8, PAIR>(A, B, b_row0, a, s);
    case M_RAW: return launch_cfg<BN, STAGES, CPLX, M_RAW, F8, PAIR>(A, B, b_row0, a, s);
  }
  return cudaErrorInvalidValue;
}

template <int BN, int STAGES, bool F8, bool PAIR = false>
cudaError_t dispatch_mode(const CUtensorMap& A, const CUtensorMap& B, int b_row0, const StepArgs& a, cudaStream_t s) {
  return a.cplx ? dispatch_cplx<BN, STAGES, true, F8, PAIR>(A, B, b_row0, a, s)
                : dispatch_cplx<BN, STAGES, false, F8, PAIR>(A, B, b_row0, a, s);
}

}  // namespace

struct TcPlan {  // tensor maps of one operand set (BF16 or FP8)
  CUtensorMap A;
  CUtensorMap B128;
  CUtensorMap B224;
  CUtensorMap B256;
  CUtensorMap B64;   // halves of 128- and 224-wide tiles for two-SM pairs
  CUtensorMap B112;
  int Cp;
};

// Shared by both precisions: the tensor maps of an operand set, then the
// launch for the tile width the chooser picks.
template <bool F8>
bool plan_maps(TcPlan* p, const void* Jop, int Np, const void* ops, int n_op_bufs, int Cp) {
  p->Cp = Cp;
  const int rows = n_op_bufs * Cp;
  return make_map(&p->A, Jop, Np, Np, BM, F8) && make_map(&p->B128, ops, Np, rows, 128, F8) &&
         make_map(&p->B224, ops, Np, rows, 224, F8) && make_map(&p->B256, ops, Np, rows, 256, F8) &&
         make_map(&p->B64, ops, Np, rows, 64, F8) && make_map(&p->B112, ops, Np, rows, 112, F8);
}

template <bool F8>
cudaError_t launch_plan(const TcPlan* plan, const StepArgs& a, int op_buf, bool pair, cudaStream_t s) {
  const int b_row0 = op_buf * plan->Cp;
  if (pair) {
    const int bn = tc_pick_bn_pair(a.N, a.C);
    if (bn == 256) return dispatch_mode<256, 6, F8, true>(plan->A, plan->B128, b_row0, a, s);
    if (bn == 224) return dispatch_mode<224, 6, F8, true>(plan->A, plan->B112, b_row0, a, s);
    return dispatch_mode<128, 8, F8, true>(plan->A, plan->B64, b_row0, a, s);
  }
  const int bn = tc_pick_bn(a.N, a.C);
  if (bn == 256) return dispatch_mode<256, 4, F8>(plan->A, plan->B256, b_row0, a, s);
  if (bn == 224) return dispatch_mode<224, 4, F8>(plan->A, plan->B224, b_row0, a, s);
  return dispatch_mode<128, 6, F8>(plan->A, plan->B128, b_row0, a, s);
}

}  // namespace gda

#include "step_tcs.cuh"
