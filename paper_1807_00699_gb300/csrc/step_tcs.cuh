// Persistent multi-step form of the tensor-core step kernel (forward Euler,
// Eqs. 2, 5, 6), for instances whose FP32 state does not fit in tensor
// memory: one launch runs a segment of steps, the state streams from HBM
// every step as in the per-step kernel, and steps are ordered by dataflow
// flags instead of kernel boundaries.
//
// Every CTA (or CTA pair) keeps the same tiles for the whole segment, taken in
// column-major order (tile t covers column block t / MTU and row block / pair
// t % MTU), so the tiles of the first column blocks finish first in every
// step.  After its epilogue a CTA publishes flag[column block][row block] =
// step + 1 (its rows of the next operand, and of beta and the density partial
// sums for row block 0 / every row block, are written).  The producer of step
// s waits, before loading K-block kb of column block c, until flag[c][kb / 2]
// reaches s; the epilogue waits on flag[c][0] before it reads beta (and on
// every row block's flag before the density sums, with noise decay).  So the
// first tiles of step s + 1 run on the tensor cores while the last epilogues
// of step s are still streaming their state, instead of after a kernel
// boundary.  Epilogue arguments of the current step live in shared memory.
// Every wait is bounded; on expiry the launch aborts as the per-step kernel's.
#pragma once

namespace gda {

namespace {

// Bounded wait until a tile flag reaches target (acquire).
__device__ __forceinline__ bool seg_flag_wait(const unsigned* f, unsigned target, long long limit) {
  if (ld_acquire_gpu(f) >= target) return true;
  const long long t0 = clock64();
  while (ld_acquire_gpu(f) < target) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

template <int BN, int STAGES, bool CPLX, bool F8, bool PAIR>
__global__ void __launch_bounds__(TcThreads<M_EULER>::N, 1)
    step_tcs_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ StepArgs a0, const __grid_constant__ SegArgs g) {
  constexpr int MODE = M_EULER;
  using Cfg = TcCfg<BN, STAGES, PAIR>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ StepArgs s_args;  // the epilogue's arguments of the current step
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
  const long long lim = a0.wait_cycles;
  constexpr int BKE = F8 ? 2 * BK : BK;  // elements per 128-byte K slice
  const int KB = (a0.N + BKE - 1) / BKE;
  const int NT = (a0.C + BN - 1) / BN;
  const int MT = (a0.N + BM - 1) / BM;  // even when PAIR (the host checks)
  const int MTU = PAIR ? MT / 2 : MT;   // row units (blocks or pairs)
  const int T = NT * MTU;
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  const int unit0 = PAIR ? int(cluster_id_x()) : int(blockIdx.x);
  const int nunit = PAIR ? int(ncluster_x()) : int(gridDim.x);
  // column-major tiles: column block t / MTU, row unit t % MTU
  auto tile_m0 = [&](int t) { return (PAIR ? 2 * (t % MTU) + int(rank) : t % MTU) * BM; };
  auto tile_c = [&](int t) { return t / MTU; };
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto acc_full = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto acc_empty = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };

  if (threadIdx.x == 0) {
    stamp(a0, 0);
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
  if (threadIdx.x == 0) stamp(a0, 1);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const uint64_t keep = policy_evict_last();  // J and the operand are re-read by every tile row / column
      int it = 0;
      bool stop = false;
      for (int n = 0; n < g.steps && !stop; ++n) {
        const int b_row0 = ((g.buf0 + n) & 1) * g.Cp;
        for (int t = unit0; t < T && !stop; t += nunit) {
          const int c = tile_c(t);
          const int m0 = tile_m0(t), n0 = c * BN + int(rank) * Cfg::BH;
          const unsigned* fl = g.flags + size_t(c) * MT;
          int ready_m = -1;
          for (int kb = 0; kb < KB; ++kb, ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            const int mb = (kb * BKE) / BM;  // row block that produced these spins
            if (n > 0 && mb != ready_m) {
              if (!seg_flag_wait(fl + mb, unsigned(n), lim)) {
                stop = true;
                break;
              }
              fence_proxy_async_global();
              ready_m = mb;
            }
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
      for (int n = 0; n < g.steps && !stop; ++n) {
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
            if (lt == 0 && kb == 0) stamp(a0, 2);
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
          if (lt == 0) stamp(a0, 3);
          if (PAIR)
            mma_commit_pair(acc_full(b));  // also after an abort: tracks every MMA issued into b
          else
            mma_commit(acc_full(b));
          if (stop) {
            (void)mbar_wait(acc_full(b), use & 1, lim);  // those MMAs finish before the CTA frees TMEM
            break;
          }
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
    constexpr int CW = 8;
    constexpr int NCH = PW / CW;
    static_assert(PW % CW == 0, "column part must hold whole chunks");
    constexpr int PF = ModeTraits<MODE>::l2_ahead;  // chunks pulled into L2 ahead of their loads
    const int e = threadIdx.x - 64;
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;
    const size_t cn = size_t(g.Cp) * a0.Np;
    int bad = 0;
    int lt = 0;
    bool run = true;
    EpiRegs<MODE, CPLX, CW> R[2];
    for (int n = 0; n < g.steps && run; ++n) {
      // this step's arguments: buffers alternate with the step's parity
      epi_bar_sync_n<32 * NEPI>();  // every thread is done with the previous step's
      if (e == 0) {
        StepArgs sa = a0;
        sa.step = a0.step + unsigned(n);
        sa.psi_n = g.psi[n & 1];
        sa.xs = g.psi[n & 1];
        sa.psi_out = g.psi[(n + 1) & 1];
        sa.beta_in = g.beta[n & 1];
        sa.beta_out = g.beta[(n + 1) & 1];
        sa.rho_in = g.rho[n & 1];
        sa.rho_out = a0.rho_out ? g.rho[(n + 1) & 1] : nullptr;
        const int ob = (g.buf0 + n + 1) & 1;
        sa.op_out = g.ops ? g.ops + ob * cn : nullptr;
        sa.op8_out = g.ops8 ? g.ops8 + ob * cn : nullptr;
        s_args = sa;
      }
      epi_bar_sync_n<32 * NEPI>();
      const StepArgs& a = s_args;
      const bool need_red = a.rho_out != nullptr;
      for (int t = unit0; t < T; t += nunit, ++lt) {
        const int c = tile_c(t);
        const int m0 = tile_m0(t), n0 = c * BN;
        const int mt = m0 / BM;
        const int b = lt & 1;
        const uint32_t use = lt >> 1;
        const int rbase = n0 / W;
        const int i = m0 + 32 * q + lane;
        const int cbeg = n0 + part * PW;
        const unsigned* fl = g.flags + size_t(c) * MT;
        const float rs = F8 ? __fmul_rn(a.row_scale[i], kFp8PsiScale) : 1.0f;
#pragma unroll
        for (int p = 0; p < PF && p < NCH; ++p) epi_prefetch_l2<MODE, CPLX, CW>(a, i, cbeg + p * CW, lane);
        epi_load<MODE, CPLX, CW>(a, i, cbeg, R[0]);  // own rows of psi and gamma: written by this thread
        bool fok = true;
        if (e < RPT) {
          if (n > 0) {  // beta (row block 0) and, with noise decay, every row block's density sums of step n - 1
            fok = seg_flag_wait(fl, unsigned(n), lim);
            if (a.noise_decay)
              for (int mb = 1; mb < MT && fok; ++mb) fok = seg_flag_wait(fl + mb, unsigned(n), lim);
          }
          const int r = rbase + e;
          const float bt = r < a.R ? a.beta_in[r] : 1.0f;
          s_beta[e] = stage_beta(a, bt);
          s_dsc[e] = r < a.R ? noise_scale(a, r) : 0.0f;
        }
        // one decision for all epilogue warps (the vote is also the barrier that
        // publishes s_beta / s_dsc)
        const bool ok = epi_vote_all<32 * NEPI>(fok && mbar_wait(acc_full(b), use & 1, lim) &&
                                                !*(volatile int*)&s_flag[0]);
        tc_fence_after();
        if (!ok) {
          if (lane == 0) atomicOr(a.err, E_TIMEOUT);
          atomicOr(&s_flag[0], 1);
          run = false;
          break;
        }
        if (lt == 0 && e == 0) stamp(a0, 4);
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
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
          if (PF > 0 && ch + PF < NCH) epi_prefetch_l2<MODE, CPLX, CW>(a, i, cbeg + (ch + PF) * CW, lane);
          if (ch + 1 < NCH) epi_load<MODE, CPLX, CW>(a, i, cbeg + (ch + 1) * CW, R[(ch + 1) & 1]);
          body(ch, R[ch & 1]);
        }
        tc_fence_before();
        fence_proxy_async_global();  // the next operand rows are read by other CTAs' TMA loads
        epi_bar_sync_n<32 * NEPI>();
        if (e == 0) {  // accumulator b may be overwritten
          if (PAIR && !leader)
            mbar_arrive_cluster(mapa_shared(acc_empty(b), 0));
          else
            mbar_arrive(acc_empty(b));
        }
        if (lt == 0 && e == 0) stamp(a0, 5);
        if (e < RPT) {
          const int r = rbase + e;
          if (r < a.R) {
            if (need_red)
              a.rho_out[size_t(mt) * a.Rp + r] = s_red[e] + s_red[BN + e] + s_red[2 * BN + e] + s_red[3 * BN + e];
            if (mt == 0) a.beta_out[r] = next_beta(a, a.beta_in[r]);
          }
        }
        epi_bar_sync_n<32 * NEPI>();
        if (e == 0)  // a release store: ordered after every epilogue thread's writes (seen through the barrier)
          st_release_gpu(g.flags + size_t(c) * MT + mt, unsigned(n + 1));
      }
    }
    if (bad) s_flag[1] = 1;
    epi_bar_sync_n<32 * NEPI>();
    if (e == 0 && s_flag[1]) atomicOr(a0.err, E_DIVERGED);
    if (e == 0) stamp(a0, 6);
  }

  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // no CTA leaves while its peer may still signal or read it
  if (threadIdx.x == 0 && s_flag[0]) atomicOr(a0.err, E_TIMEOUT);
  if (threadIdx.x == 0) stamp(a0, 7);
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem, TCOLS);
    else
      tmem_dealloc(tmem, TCOLS);
  }
}

template <int BN, int STAGES, bool CPLX, bool F8, bool PAIR>
cudaError_t launch_seg_cfg(const CUtensorMap& A, const CUtensorMap& B, const StepArgs& a, const SegArgs& g,
                           cudaStream_t s) {
  using Cfg = TcCfg<BN, STAGES, PAIR>;
  auto kern = step_tcs_kernel<BN, STAGES, CPLX, F8, PAIR>;
  static bool attr_set = false;
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
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(TcThreads<M_EULER>::N);
  cfg.dynamicSmemBytes = Cfg::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (!PAIR) {
    // every CTA resident at once: the step flags need it
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    const int tiles = NT * MT;
    cfg.gridDim = dim3(tiles < sms ? tiles : sms);
    return cudaLaunchKernelEx(&cfg, kern, A, B, a, g);
  }
  if (MT % 2) return cudaErrorInvalidValue;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  // as many clusters as the device holds at once (one CTA per SM), so that
  // every cluster is resident for the flags
  static int max_clusters = 0;
  if (!max_clusters) {
    cfg.gridDim = dim3(2 * (sms / 2));
    cudaError_t e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (max_clusters < 1) return cudaErrorLaunchOutOfResources;
  }
  const int ptiles = NT * (MT / 2);
  cfg.gridDim = dim3(2 * (ptiles < max_clusters ? ptiles : max_clusters));
  return cudaLaunchKernelEx(&cfg, kern, A, B, a, g);
}

template <int BN, int STAGES, bool F8, bool PAIR>
cudaError_t seg_dispatch(const CUtensorMap& A, const CUtensorMap& B, const StepArgs& a, const SegArgs& g,
                         cudaStream_t s) {
  return a.cplx ? launch_seg_cfg<BN, STAGES, true, F8, PAIR>(A, B, a, g, s)
                : launch_seg_cfg<BN, STAGES, false, F8, PAIR>(A, B, a, g, s);
}

}  // namespace

// Tile width as for the per-step kernel; one launch of g.steps steps.
template <bool F8>
cudaError_t launch_seg_plan(const TcPlan* plan, const StepArgs& a, const SegArgs& g, bool pair, cudaStream_t s) {
  if (pair) {
    const int bn = tc_pick_bn_pair(a.N, a.C);
    if (bn == 256) return seg_dispatch<256, 6, F8, true>(plan->A, plan->B128, a, g, s);
    if (bn == 224) return seg_dispatch<224, 6, F8, true>(plan->A, plan->B112, a, g, s);
    return seg_dispatch<128, 8, F8, true>(plan->A, plan->B64, a, g, s);
  }
  const int bn = tc_pick_bn(a.N, a.C);
  if (bn == 256) return seg_dispatch<256, 4, F8, false>(plan->A, plan->B256, a, g, s);
  if (bn == 224) return seg_dispatch<224, 4, F8, false>(plan->A, plan->B224, a, g, s);
  return seg_dispatch<128, 6, F8, false>(plan->A, plan->B128, a, g, s);
}

}  // namespace gda
