// Resident persistent GD kernel (forward Euler, BF16 coupling product).
//
// One cooperative launch runs many steps.  Each CTA owns one 128 x 128 tile
// (spins i x columns c) for the whole launch and keeps that tile's FP32 state
// in tensor memory: the accumulator (columns 0..127), the amplitudes psi
// (128..255) and the gains gamma (256..), so per step the only global traffic
// is the BF16 operand X = bf16(psi) that every CTA reads and writes.  Steps are
// ordered by dataflow flags, one per tile: the epilogue of tile (m, n) writes
// its slice of X^{n+1} (spins of row block m, columns of block n) and then
// releases flag[n][m] = step + 1; the producer of every tile in column block n
// acquires flag[n][kb / 2] before loading K-block kb of X^{n+1}.  Column
// blocks never wait on each other, and the A (coupling) tiles of the next step
// are prefetched while the epilogue runs.  Every wait is bounded.
//
// Roles: warp 0 TMA producer; warp 1 TMEM allocator + MMA issuer; warps 2..17
// epilogue (warp w reads TMEM lane quarter w % 4 and a quarter of the columns).
//
// PAIR form: the CTAs of row blocks 2p and 2p + 1 of a column block run as a
// cluster of two, and the even CTA issues M = 256 tcgen05.mma.cta_group::2
// instructions over both CTAs' shared memory.  Each CTA loads its own 128 rows
// of the coupling tile and half (64 columns) of the operand tile, and receives
// its own rows of the accumulator in its tensor memory, where its state stays;
// the K loop moves a quarter fewer bytes through each SM's shared memory.
// Per-element arithmetic is the Euler update of Eqs. (2), (5), (6) with the
// same FP32 expression sequence as the per-step kernels.
#include "tc_epilogue.cuh"
#include "tc_ptx.cuh"
#include "res.h"

namespace gda {
namespace {

using namespace ptx;
constexpr int EPI_WARPS = 16;                 // 4 per tensor-memory lane quarter
constexpr int RES_THREADS = 64 + 32 * EPI_WARPS;
constexpr int CPT = 128 / (EPI_WARPS / 4);    // columns per epilogue thread
constexpr int BN = 128;
constexpr uint32_t A_BYTES = BM * BK * 2;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t T_PSI = 128;  // tensor-memory column of psi
constexpr uint32_t T_GAM = 256;  // tensor-memory column of gamma
// The ring of one CTA: a one-SM tile loads the whole 128-column operand slice
// of a K-block, a CTA of a pair its 64-column half, so its stages are smaller
// and its ring deeper.
template <bool PAIR>
struct ResCfg {
  static constexpr int STAGES = PAIR ? 8 : 6;
  static constexpr int BH = PAIR ? BN / 2 : BN;  // operand columns loaded by this CTA
  static constexpr uint32_t B_BYTES = BH * BK * 2;
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr uint32_t TAIL = (2 * STAGES + 2) * 8 + 8 * BN * 4 + 16;
  static constexpr uint32_t SMEM = 1024 + STAGES * STAGE_BYTES + TAIL;
};

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS) : "memory"); }

// Bounded wait until a tile flag reaches target (acquire).
__device__ __forceinline__ bool flag_wait(const unsigned* f, unsigned target, long long limit) {
  if (ld_acquire_gpu(f) >= target) return true;
  const long long t0 = clock64();
  while (ld_acquire_gpu(f) < target) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

template <bool CPLX, bool PAIR>
__global__ void __launch_bounds__(RES_THREADS, 1)
    step_res_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, ResArgs ra,
                    StepArgs a) {
  using Cfg = ResCfg<PAIR>;
  constexpr int STAGES = Cfg::STAGES;
  constexpr uint32_t B_BYTES = Cfg::B_BYTES;
  constexpr uint32_t STAGE_BYTES = Cfg::STAGE_BYTES;
  constexpr int W = CPLX ? 2 : 1;
  constexpr int RPT = BN / W;
  constexpr int CW = 8;                 // columns per epilogue chunk
  constexpr int GR = CW / W;            // restarts per chunk
  constexpr int NCH = CPT / CW;
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
  const long long lim = a.wait_cycles;
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;  // the odd row block of a pair: 1
  const bool leader = rank == 0;
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
    mbar_init(acc_free, PAIR ? 2 : 1);  // both CTAs' epilogues free a pair's accumulator
    s_flag[0] = 0;
    s_flag[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if (PAIR)
      tmem_alloc_pair(smem_u32(s_tmem), TMEM_COLS);
    else
      tmem_alloc(smem_u32(s_tmem), TMEM_COLS);
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
      int it = 0;
      const int pre = KB < STAGES ? KB : STAGES;
      const unsigned* col_flags = ra.flags + size_t(blockIdx.x) * gridDim.y;
      // ring slots [a_lo, a_hi) have their A tile issued but not yet their B tile
      int a_lo = 0, a_hi = 0, brow = 0;
      // a stage's copies: the A tile arms the stage (a pair's even CTA counts
      // both CTAs' bytes on its own barrier), the B tile follows
      auto issue_a = [&](int s, int kb) {
        if (PAIR) {
          if (leader) mbar_arrive_expect_tx(full_bar(s), 2 * STAGE_BYTES);
          tma_load_2d_pair(sA + s * A_BYTES, &tmA, kb * BK, m0, mapa_shared(full_bar(s), 0));
        } else {
          mbar_arrive_expect_tx(full_bar(s), STAGE_BYTES);
          tma_load_2d(sA + s * A_BYTES, &tmA, kb * BK, m0, full_bar(s));
        }
      };
      auto issue_b = [&](int s, int kb) {
        if (PAIR)
          tma_load_2d_pair(sB + s * B_BYTES, &tmB, kb * BK, brow, mapa_shared(full_bar(s), 0));
        else
          tma_load_2d(sB + s * B_BYTES, &tmB, kb * BK, brow, full_bar(s));
      };
      bool stop = false;
      for (int n = 0; n < ra.steps && !stop; ++n) {
        brow = ((ra.buf0 + n) & 1) * ra.Cp + n0 + int(rank) * Cfg::BH;
        a_lo = a_hi = it;
        // A tiles of the first `pre` K-blocks do not depend on the previous step
        for (int kb = 0; kb < pre; ++kb) {
          const int s = (it + kb) % STAGES;
          const uint32_t ph = ((it + kb) / STAGES) & 1;
          if (!mbar_wait(empty_bar(s), ph ^ 1u, lim) || *(volatile int*)&s_flag[0]) {
            stop = true;
            break;
          }
          issue_a(s, kb);
          a_hi = it + kb + 1;
        }
        if (stop) break;
        int ready_m = -1;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          if (kb >= pre) {
            const uint32_t ph = (it / STAGES) & 1;
            if (!mbar_wait(empty_bar(s), ph ^ 1u, lim) || *(volatile int*)&s_flag[0]) {
              stop = true;
              break;
            }
            issue_a(s, kb);
            a_hi = it + 1;
          }
          const int mb = (kb * BK) / BM;  // row block that produced these spins
          if (n > 0 && mb != ready_m) {
            if (!flag_wait(col_flags + mb, unsigned(n), lim)) {
              stop = true;
              break;
            }
            fence_proxy_async_global();
            ready_m = mb;
          }
          issue_b(s, kb);
          a_lo = it + 1;
        }
      }
      if (stop) {
        atomicOr(&s_flag[0], 1);
        // complete every armed slot (the B data is irrelevant now), then wait for
        // all copies this CTA may still have in flight
        for (int k = a_lo; k < a_hi; ++k) issue_b(k % STAGES, 0);
        // a pair's odd CTA waits for the MMAs that consume its stages to release
        // them (bounded: the even CTA may have stopped)
        for (int k = a_hi - 1; k >= 0 && k >= a_hi - STAGES; --k) {
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
      constexpr uint32_t idesc = PAIR ? idesc_bf16_m256<BN>() : idesc_bf16<BN>();
      int it = 0;
      int committed = -1;  // last step whose MMAs were committed to acc_full
      for (int n = 0; n < ra.steps; ++n) {
        const bool freed = n == 0 || (PAIR ? mbar_wait_cluster(acc_free, (n - 1) & 1, lim)
                                           : mbar_wait(acc_free, (n - 1) & 1, lim));
        if (!freed || *(volatile int*)&s_flag[0]) {
          atomicOr(&s_flag[0], 1);
          break;
        }
        tc_fence_after();
        bool stop = false;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!mbar_wait(full_bar(s), ph, lim) || *(volatile int*)&s_flag[0]) {
            atomicOr(&s_flag[0], 1);
            stop = true;
            break;
          }
          tc_fence_after();
          if (n == 0 && kb == 0) stamp(a, 2);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t da = sdesc_sw128(sA + s * A_BYTES + k * 32);
            const uint64_t db = sdesc_sw128(sB + s * B_BYTES + k * 32);
            if (PAIR)
              mma_bf16_pair(tmem, da, db, idesc, (kb | k) != 0);
            else
              mma_bf16(tmem, da, db, idesc, (kb | k) != 0);
          }
          if (PAIR)
            mma_commit_pair(empty_bar(s));  // both CTAs' stages
          else
            mma_commit(empty_bar(s));
        }
        if (n == 0) stamp(a, 3);
        if (PAIR)  // also after an abort: tracks every MMA issued
          mma_commit_pair(acc_full);
        else
          mma_commit(acc_full);
        committed = n;
        if (stop) break;
      }
      // after an abort, the MMAs still in flight finish before the CTA frees
      // its tensor memory (the epilogue may have stopped waiting for them)
      if (*(volatile int*)&s_flag[0] && committed >= 0) (void)mbar_wait(acc_full, committed & 1, lim);
    }
  } else {
    // ---------------- epilogue ----------------
    const int e = threadIdx.x - 64;
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;
    const int i = m0 + 32 * q + lane;
    const bool row_ok = i < a.N;
    const int rbase = n0 / W;
    const size_t Np = a.Np;
    const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
    const int cb = part * CPT;  // first local column of this thread
    const float h = row_ok ? a.h1[i] : 0.0f;
    const bool need_red = a.noise_decay && a.noise_D != 0.0f;

    // state -> tensor memory
#pragma unroll 1
    for (int ch = 0; ch < CPT / 16; ++ch) {
      float v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = a.psi_n[size_t(n0 + cb + ch * 16 + k) * Np + i];
      tmem_st16(tmem + lane_base + T_PSI + cb + ch * 16, v);
    }
#pragma unroll 1
    for (int ch = 0; ch < CPT / 16 / W; ++ch) {
      float v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = a.gam[size_t(rbase + cb / W + ch * 16 + k) * Np + i];
      tmem_st16(tmem + lane_base + T_GAM + cb / W + ch * 16, v);
    }
    tmem_st_wait();
    if (e < RPT) {
      const int r = rbase + e;
      s_beta[e] = r < a.R ? a.beta_in[r] : 1.0f;
    }

    StepArgs sa = a;
    sa.mode = M_EULER;
    int bad = 0;
    const unsigned* col_flags = ra.flags + size_t(blockIdx.x) * gridDim.y;

    const uint32_t tb = tmem + lane_base;

    // one chunk of CW columns: accumulator, amplitudes, gains (8 restarts)
    struct Chunk {
      uint32_t y[CW], p[CW], g[GR];
    };
    auto issue = [&](int ch, Chunk& t) {
      const int lc0 = cb + ch * CW;
      if (CW == 16) {
        tmem_ld16_nowait(tb + lc0, t.y);
        tmem_ld16_nowait(tb + T_PSI + lc0, t.p);
      } else {
        tmem_ld8_nowait(tb + lc0, t.y);
        tmem_ld8_nowait(tb + T_PSI + lc0, t.p);
      }
      if (GR == 8)
        tmem_ld8_nowait(tb + T_GAM + lc0 / W, t.g);
      else
        tmem_ld4_nowait(tb + T_GAM + lc0 / W, t.g);
    };
    auto settle = [&](Chunk& t) {  // wait, then pin every register of t after it
      if (GR == 8)
        tmem_wait_ld8(t.g);
      else
        tmem_wait_ld4(t.g);
      if (CW == 16) {
        tmem_regs_after_wait16(t.y);
        tmem_regs_after_wait16(t.p);
      } else {
        tmem_regs_after_wait8(t.y);
        tmem_regs_after_wait8(t.p);
      }
    };

#pragma unroll 1
    for (int n = 0; n < ra.steps; ++n) {
      sa.step = a.step + unsigned(n);
      sa.rho_in = (n & 1) ? ra.rho[1] : ra.rho[0];
      bool flags_ok = true;
      if (e < RPT) {
        const int r = rbase + e;
        s_bstage[e] = s_beta[e];
        if (need_red && n > 0)  // partial sums of step n-1 from every row block of this column block
          for (unsigned mb = 0; mb < gridDim.y && flags_ok; ++mb) flags_ok = flag_wait(col_flags + mb, unsigned(n), lim);
        s_dsc[e] = r < a.R ? noise_scale(sa, r) : 0.0f;
      }
      // one decision for all epilogue warps (the vote is also the barrier that
      // publishes s_bstage / s_dsc)
      const bool ok =
          epi_vote_all<32 * EPI_WARPS>(flags_ok && mbar_wait(acc_full, n & 1, lim) && !*(volatile int*)&s_flag[0]);
      tc_fence_after();
      if (!ok) {
        if (lane == 0) atomicOr(a.err, E_TIMEOUT);
        atomicOr(&s_flag[0], 1);
        break;
      }
      if (n == 0 && e == 0) stamp(a, 4);
      __nv_bfloat16* op = ra.ops + size_t((ra.buf0 + n + 1) & 1) * ra.Cp * Np;

      auto body = [&](int ch, Chunk& t, Chunk& nxt) {
        if (ch + 1 < NCH) issue(ch + 1, nxt);  // next chunk's loads overlap this chunk's arithmetic
        const int lc0 = cb + ch * CW;
        const int lr0 = lc0 / W;
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
        float npsi[CW], ngam[GR], red[GR];
#pragma unroll
        for (int u = 0; u < CW / W; ++u) {
          const int k0 = u * W;
          const float xr = __uint_as_float(t.p[k0]), xi = CPLX ? __uint_as_float(t.p[k0 + 1]) : 0.0f;
          const float yr = __uint_as_float(t.y[k0]), yi = CPLX ? __uint_as_float(t.y[k0 + 1]) : 0.0f;
          const float gs = __uint_as_float(t.g[u]);
          float kr, ki, kg;
          gd_rhs(xr, xi, gs, yr, yi, s_bstage[lr0 + u], h, a.eps, a.rho_th, kr, ki, kg);
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
        if (CW == 16)
          tmem_st16(tb + T_PSI + lc0, npsi);
        else
          tmem_st8(tb + T_PSI + lc0, npsi);
        if (GR == 8)
          tmem_st8(tb + T_GAM + lr0, ngam);
        else
          tmem_st4(tb + T_GAM + lr0, ngam);
        if (need_red) {
#pragma unroll
          for (int u = 0; u < GR; ++u) {
            float x = red[u];
#pragma unroll
            for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) s_red[q * BN + lr0 + u] = x;
          }
        }
        if (ch + 1 < NCH) settle(nxt);
      };
      Chunk c0buf, c1buf;
      issue(0, c0buf);
      settle(c0buf);
      static_assert(NCH % 2 == 0, "chunks are processed in pairs");
#pragma unroll 1
      for (int ch = 0; ch < NCH; ch += 2) {
        body(ch, c0buf, c1buf);
        body(ch + 1, c1buf, c0buf);
      }
      tmem_st_wait();
      tc_fence_before();
      fence_proxy_async_global();
      epi_sync();
      if (e == 0) {
        if (PAIR && !leader)
          mbar_arrive_cluster(mapa_shared(acc_free, 0));
        else
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
      const int tile = int(blockIdx.x * gridDim.y + blockIdx.y);
      if (e == 0 && n + 1 < ra.steps && !(tile == ra.withhold_tile && n + 1 == ra.withhold_step)) {
        __threadfence();
        st_release_gpu(ra.flags + tile, unsigned(n + 1));
      }
    }
    // tensor memory -> state
    if (!*(volatile int*)&s_flag[0]) {
#pragma unroll 1
      for (int ch = 0; ch < CPT / 16; ++ch) {
        float v[16];
        tmem_ld16(tb + T_PSI + cb + ch * 16, v);
        if (row_ok)
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int c = n0 + cb + ch * 16 + k;
            if (c < a.C) ra.psi_final[size_t(c) * Np + i] = v[k];
          }
      }
#pragma unroll 1
      for (int ch = 0; ch < CPT / 16 / W; ++ch) {
        float v[16];
        tmem_ld16(tb + T_GAM + cb / W + ch * 16, v);
        if (row_ok)
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int r = rbase + cb / W + ch * 16 + k;
            if (r < a.R) a.gam[size_t(r) * Np + i] = v[k];
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
  if (PAIR) cluster_sync();  // no CTA leaves while its peer may still signal or read it
  if (threadIdx.x == 0 && s_flag[0]) atomicOr(a.err, E_TIMEOUT);
  if (threadIdx.x == 0) stamp(a, 7);
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem, TMEM_COLS);
    else
      tmem_dealloc(tmem, TMEM_COLS);
  }
}

template <bool CPLX, bool PAIR>
cudaError_t launch_res_impl(const CUtensorMap& A, const CUtensorMap& B, const ResArgs& ra, const StepArgs& a,
                            cudaStream_t s) {
  constexpr uint32_t SMEM = ResCfg<PAIR>::SMEM;
  static bool attr_set = false;
  auto kern = step_res_kernel<CPLX, PAIR>;
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
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!PAIR) {
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the tile flags need it
    attr[0].val.cooperative = 1;
    return cudaLaunchKernelEx(&cfg, kern, A, B, ra, a);
  }
  // clusters of the two row blocks of a pair; every cluster resident at once
  // (the tile flags need it): at most as many clusters as the device holds
  if (cfg.gridDim.y % 2) return cudaErrorInvalidValue;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 2;
  attr[0].val.clusterDim.z = 1;
  static int max_clusters = 0;
  if (!max_clusters) {
    cudaError_t e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
  }
  if ((long long)cfg.gridDim.x * cfg.gridDim.y / 2 > max_clusters) return cudaErrorInvalidValue;
  return cudaLaunchKernelEx(&cfg, kern, A, B, ra, a);
}

}  // namespace

bool res_fits(int N, int C, int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return false;
  int per_sm = 0;
  auto kern = step_res_kernel<true, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, ResCfg<false>::SMEM) != cudaSuccess)
    return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RES_THREADS, ResCfg<false>::SMEM) != cudaSuccess)
    return false;
  const long long grid = (long long)((C + BN - 1) / BN) * ((N + BM - 1) / BM);
  return per_sm >= 1 && grid <= (long long)per_sm * sms;
}

bool res_pair_fits(int N, int C) {
  const int mt = (N + BM - 1) / BM, nt = (C + BN - 1) / BN;
  if (mt % 2) return false;
  auto kern = step_res_kernel<true, true>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, ResCfg<true>::SMEM) != cudaSuccess)
    return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nt, mt);
  cfg.blockDim = dim3(RES_THREADS);
  cfg.dynamicSmemBytes = ResCfg<true>::SMEM;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 2;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int max_clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg) != cudaSuccess) return false;
  return (long long)nt * mt / 2 <= max_clusters;
}

cudaError_t launch_step_res(const TcPlan* plan, const ResArgs& ra, const StepArgs& a, cudaStream_t s, bool pair) {
  const CUtensorMap* A = tc_plan_A(plan);
  if (pair) {
    const CUtensorMap* B = tc_plan_B64(plan);
    return a.cplx ? launch_res_impl<true, true>(*A, *B, ra, a, s) : launch_res_impl<false, true>(*A, *B, ra, a, s);
  }
  const CUtensorMap* B = tc_plan_B(plan);
  return a.cplx ? launch_res_impl<true, false>(*A, *B, ra, a, s) : launch_res_impl<false, false>(*A, *B, ra, a, s);
}

}  // namespace gda
