// Batched GD: many independent instances of different N and R stepped
// together (not in the paper; the serving form of the method).
//
// Couplings of all instances are packed into one BF16 tensor [sum Np_i][P]
// and their operands into one BF16 tensor [sum 2 Cp_i][P] (common row pitch
// P = max Np_i), so a single TMA tensor map per tensor addresses every tile.
// FP32 state is stored compactly per instance.  A work unit is one 128 x BN
// output tile (instance, row block, column block) of either model type; the
// units of all instances are assigned to CTAs on the host by longest
// processing time first.
//
// One persistent cooperative launch runs a chunk of steps for every instance:
// each CTA walks its unit list once per step, with the double-buffered
// tensor-memory accumulators of the per-step kernel, and steps are ordered by
// dataflow flags, one per unit (as in the resident single-instance kernel):
// after the epilogue of unit (k, m, n) has written its rows of instance k's
// next operand (and, for m = 0, the next coupling scales beta), it publishes
// flag = step + 1; a producer loading K-block kb of instance k's column block
// n for step s waits until the flag of unit (k, kb / 2, n) reaches s, and the
// epilogue reading beta of that column block waits for unit (k, 0, n).  The
// epilogue is specialised per unit for real or complex amplitudes.  The step
// index comes from a device counter, so a captured CUDA graph of chunk
// launches replays correctly.  Euler steps, Eqs. (2), (5), (6), each instance
// with its own gain speed, threshold, ramp and Philox key.  Every wait is
// bounded; a wait that runs out aborts the launch (E_TIMEOUT).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/gda.h"
#include "gda_internal.h"
#include "tc_epilogue.cuh"
#include "tc_ptx.cuh"

namespace gda {
namespace {

using namespace ptx;
constexpr int NEPI = 16;  // epilogue warps: 4 column parts x 4 lane quarters
constexpr int NTHREADS = 64 + 32 * NEPI;

struct BatchInst {
  int N, Np, C, R, Cp, Rp, mt;
  int cplx;
  int rowJ;            // first row of the instance's couplings in the packed tensor
  int rowX;            // first row of operand buffer 0 (buffer 1 follows at rowX + Cp)
  int flag0;           // flag of unit (row block 0, column block 0); unit (m, n) at flag0 + n * mt + m
  int has_base;        // init_mode 3: per-spin base amplitudes at off_base
  long long off_psi;   // psi [2][Cp][Np]
  long long off_gam;   // gamma [Rp][Np]
  long long off_h1;    // h1 [Np]
  long long off_beta;  // beta [2][Rp]
  long long off_base;  // base amplitudes [N][2]
  unsigned long long seed;
  float dt, eps, rho_th, eps_hat, beta0, sq;  // the instance's settings (sq = sqrt(rho_th) in FP32)
};

struct BatchUnit {
  int inst, mt, nt, pad;
};

struct BatchArgs {
  const BatchInst* inst;
  const BatchUnit* units;   // ordered by CTA
  const int* cta_begin;     // [gridDim.x + 1]
  float* psi;
  float* gam;
  const float* h1;
  float* beta;
  __nv_bfloat16* ops;
  int pitch;
  const unsigned* step_base;  // device step counter of the run
  unsigned step_off;          // this launch's offset from it
  int nsteps;                 // steps of this launch
  unsigned* flags;            // per-unit step flags (absolute step + 1)
  float noise_D;
  long long wait_cycles;
  int* err;
};

template <int BN, int STAGES>
struct BCfg {
  static constexpr uint32_t A_BYTES = BM * BK * 2;
  static constexpr uint32_t B_BYTES = BN * BK * 2;
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr uint32_t TAIL = (2 * STAGES + 4) * 8 + 6 * BN * 4 + 16;
  static constexpr uint32_t SMEM = 1024 + STAGES * STAGE_BYTES + TAIL;
};

__device__ __forceinline__ void bar_epi() { asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory"); }

// Bounded wait until a unit flag reaches target (acquire).
__device__ __forceinline__ bool bflag_wait(const unsigned* f, unsigned target, long long limit) {
  if (ld_acquire_gpu(f) >= target) return true;
  const long long t0 = clock64();
  while (ld_acquire_gpu(f) < target) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// StepArgs of one instance for a forward-Euler step with parity cur.
__device__ __forceinline__ StepArgs unit_args(const BatchArgs& b, const BatchInst& I, unsigned step, int cur) {
  StepArgs a{};
  a.N = I.N; a.Np = I.Np; a.C = I.C; a.R = I.R; a.Cp = I.Cp; a.Rp = I.Rp;
  a.mode = M_EULER;
  a.cplx = I.cplx;
  a.mt_count = I.mt;
  a.dt = I.dt; a.eps = I.eps; a.rho_th = I.rho_th; a.eps_hat = I.eps_hat;
  a.noise_D = b.noise_D;
  a.noise_decay = 0;
  a.seed = I.seed;
  a.step = step;
  const size_t cn = size_t(I.Cp) * I.Np;
  a.psi_n = b.psi + I.off_psi + size_t(cur) * cn;
  a.xs = a.psi_n;
  a.psi_out = b.psi + I.off_psi + size_t(cur ^ 1) * cn;
  a.gam = b.gam + I.off_gam;
  a.h1 = b.h1 + I.off_h1;
  a.beta_in = b.beta + I.off_beta + size_t(cur) * I.Rp;
  a.beta_out = b.beta + I.off_beta + size_t(cur ^ 1) * I.Rp;
  a.op_out = b.ops + (size_t(I.rowX) + size_t(cur ^ 1) * I.Cp) * b.pitch;
  a.op_pitch = b.pitch;
  a.err = b.err;
  return a;
}

// Epilogue of one unit at one step (all NEPI epilogue warps): waits for the
// unit's accumulator, runs the Euler update of its 128 x BN tile, frees the
// accumulator and publishes the unit's flag.  Returns false on an abort.
template <int BN, bool CPLX>
__device__ __forceinline__ bool epi_unit(const BatchArgs& b, const BatchInst& I, const BatchUnit& U, unsigned step,
                                         int cur, int n, uint32_t tacc, uint32_t full, uint32_t empty, uint32_t use,
                                         float* s_beta, float* s_dsc, int* s_flag, StepArgs* s_args, int& bad) {
  constexpr int W = CPLX ? 2 : 1;
  constexpr int RPT = BN / W;
  constexpr int PW = BN / (NEPI / 4);  // columns per part
  constexpr int CW = 8;
  constexpr int NCH = PW / CW;
  static_assert(PW % CW == 0, "column part must hold whole chunks");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = threadIdx.x - 64;
  const int q = warp & 3;
  const int part = (warp - 2) >> 2;
  // the unit's arguments live in shared memory (read where used), not in
  // every epilogue thread's registers
  bar_epi();  // every thread is done with the previous unit's arguments
  if (e == 0) *s_args = unit_args(b, I, step, cur);
  bar_epi();
  const StepArgs& a = *s_args;
  const int m0 = U.mt * BM, n0 = U.nt * BN;
  const int rbase = n0 / W;
  const int i = m0 + 32 * q + lane;
  const int cbeg = n0 + part * PW;
  const unsigned* fl = b.flags + I.flag0 + U.nt * I.mt;
  constexpr int PF = ModeTraits<M_EULER>::l2_ahead;  // chunks pulled into L2 ahead of their loads
#pragma unroll
  for (int p = 1; p <= PF && p < NCH; ++p) epi_prefetch_l2<M_EULER, CPLX, CW>(a, i, cbeg + p * CW, lane);
  EpiRegs<M_EULER, CPLX, CW> R[2];
  epi_load<M_EULER, CPLX, CW>(a, i, cbeg, R[0]);  // own rows of psi and gamma: written by this thread
  bool fok = true;
  if (e < RPT) {
    // beta^n of this column block was written by unit (k, 0, n) at the previous step
    if (n > 0) fok = bflag_wait(fl, step, b.wait_cycles);
    const int r = rbase + e;
    s_beta[e] = r < a.R ? a.beta_in[r] : 1.0f;
    s_dsc[e] = r < a.R ? noise_scale(a, r) : 0.0f;
  }
  // one decision for all epilogue warps; the vote also publishes s_beta / s_dsc
  const bool ok = epi_vote_all<32 * NEPI>(fok && mbar_wait(full, use & 1, b.wait_cycles) &&
                                          !*(volatile int*)&s_flag[0]);
  tc_fence_after();
  if (!ok) {
    if (lane == 0) atomicOr(b.err, E_TIMEOUT);
    atomicOr(&s_flag[0], 1);
    return false;
  }
  const uint32_t taddr = tacc + (static_cast<uint32_t>(32 * q) << 16) + part * PW;
  auto body = [&](int ch, const EpiRegs<M_EULER, CPLX, CW>& cr, EpiRegs<M_EULER, CPLX, CW>& nx) {
    if (ch + 1 + PF < NCH) epi_prefetch_l2<M_EULER, CPLX, CW>(a, i, cbeg + (ch + 1 + PF) * CW, lane);
    if (ch + 1 < NCH) epi_load<M_EULER, CPLX, CW>(a, i, cbeg + (ch + 1) * CW, nx);
    float v[CW];
    tmem_ld<CW>(taddr + ch * CW, v);
    const int lr0 = (part * PW + ch * CW) / W;
    float red[CW / W];
    epi_chunk<M_EULER, CPLX, CW>(a, i, cbeg + ch * CW, v, cr, &s_beta[lr0], &s_dsc[lr0], red, bad);
  };
#pragma unroll 1
  for (int ch = 0; ch + 1 < NCH; ch += 2) {
    body(ch, R[0], R[1]);
    body(ch + 1, R[1], R[0]);
  }
  if (NCH & 1) body(NCH - 1, R[0], R[1]);
  const bool publish = b.nsteps > 1;  // later steps of this launch read what this unit wrote
  tc_fence_before();
  if (publish) fence_proxy_async_global();  // the next operand rows are read by other CTAs' TMA loads
  bar_epi();
  if (e == 0) mbar_arrive(empty);
  if (e < RPT && U.mt == 0) {
    const int r = rbase + e;
    if (r < a.R) a.beta_out[r] = next_beta(a, a.beta_in[r]);
  }
  if (publish) {
    bar_epi();
    if (e == 0)  // a release store: ordered after every epilogue thread's writes (seen through the barrier)
      st_release_gpu(b.flags + I.flag0 + U.nt * I.mt + U.mt, step + 1u);
  }
  return true;
}

template <int BN, int STAGES>
__global__ void __launch_bounds__(NTHREADS, 1)
    step_batch_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, BatchArgs b) {
  using Cfg = BCfg<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  const uint32_t sA = base;
  const uint32_t sB = base + STAGES * Cfg::A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  float* s_beta = reinterpret_cast<float*>(bars + 2 * STAGES + 4);
  float* s_dsc = s_beta + BN;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_dsc + 5 * BN);
  int* s_flag = reinterpret_cast<int*>(s_tmem + 1);
  __shared__ StepArgs s_args;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned step0 = *b.step_base + b.step_off;
  const long long lim = b.wait_cycles;
  const int u0 = b.cta_begin[blockIdx.x], u1 = b.cta_begin[blockIdx.x + 1];
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto acc_full = [&](int k) { return smem_u32(bars + 2 * STAGES + k); };
  auto acc_empty = [&](int k) { return smem_u32(bars + 2 * STAGES + 2 + k); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(acc_full(k), 1);
      mbar_init(acc_empty(k), 1);
    }
    s_flag[0] = 0;
    s_flag[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr uint32_t TCOLS = 2 * BN <= 256 ? 256 : 512;
  if (warp == 1) tmem_alloc(smem_u32(s_tmem), TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int it = 0;
      bool stop = false;
      for (int n = 0; n < b.nsteps && !stop; ++n) {
        const unsigned step = step0 + unsigned(n);
        const int cur = int(step & 1u);
        for (int u = u0; u < u1 && !stop; ++u) {
          const BatchUnit U = b.units[u];
          const BatchInst& I = b.inst[U.inst];
          const int KB = (I.N + BK - 1) / BK;
          const int ya = I.rowJ + U.mt * BM;
          const int yb = I.rowX + cur * I.Cp + U.nt * BN;
          const unsigned* fl = b.flags + I.flag0 + U.nt * I.mt;
          int ready_m = -1;
          for (int kb = 0; kb < KB; ++kb, ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            const int mb = (kb * BK) / BM;  // row block that produced these spins
            if (n > 0 && mb != ready_m) {
              if (!bflag_wait(fl + mb, step, lim)) {
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
            mbar_arrive_expect_tx(full_bar(s), Cfg::STAGE_BYTES);
            tma_load_2d(sA + s * Cfg::A_BYTES, &tmA, kb * BK, ya, full_bar(s));
            tma_load_2d(sB + s * Cfg::B_BYTES, &tmB, kb * BK, yb, full_bar(s));
          }
        }
      }
      if (stop) {
        atomicOr(&s_flag[0], 1);
        for (int k = it - 1; k >= 0 && k >= it - STAGES; --k) (void)mbar_wait(full_bar(k % STAGES), (k / STAGES) & 1, lim);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16<BN>();
      int it = 0, lt = 0;
      int committed = -1;  // accumulator of the last commit (lt), -1 before any
      bool stop = false;
      for (int n = 0; n < b.nsteps && !stop; ++n) {
        for (int u = u0; u < u1 && !stop; ++u, ++lt) {
          const int KB = (b.inst[b.units[u].inst].N + BK - 1) / BK;
          const int k2 = lt & 1;
          const uint32_t use = lt >> 1;
          if (!mbar_wait(acc_empty(k2), (use & 1) ^ 1u, lim) || *(volatile int*)&s_flag[0]) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t dacc = tmem + k2 * BN;
          for (int kb = 0; kb < KB; ++kb, ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!mbar_wait(full_bar(s), ph, lim) || *(volatile int*)&s_flag[0]) {
              stop = true;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
              mma_bf16(dacc, sdesc_sw128(sA + s * Cfg::A_BYTES + k * 32), sdesc_sw128(sB + s * Cfg::B_BYTES + k * 32),
                       idesc, (kb | k) != 0);
            mma_commit(empty_bar(s));
          }
          mma_commit(acc_full(k2));  // also after an abort: tracks every MMA issued into k2
          committed = lt;
        }
      }
      if (stop) {
        atomicOr(&s_flag[0], 1);
        // the MMAs in flight finish before the CTA frees its tensor memory
        if (committed >= 0) (void)mbar_wait(acc_full(committed & 1), (committed >> 1) & 1, lim);
      }
    }
  } else {
    // ---------------- epilogue warps ----------------
    const int e = threadIdx.x - 64;
    int bad = 0, lt = 0;
    bool run = true;
    for (int n = 0; n < b.nsteps && run; ++n) {
      const unsigned step = step0 + unsigned(n);
      const int cur = int(step & 1u);
      for (int u = u0; u < u1 && run; ++u, ++lt) {
        const BatchUnit U = b.units[u];
        const BatchInst& I = b.inst[U.inst];
        const int k2 = lt & 1;
        const uint32_t use = lt >> 1;
        const uint32_t tacc = tmem + k2 * BN;
        run = I.cplx ? epi_unit<BN, true>(b, I, U, step, cur, n, tacc, acc_full(k2), acc_empty(k2), use, s_beta,
                                          s_dsc, s_flag, &s_args, bad)
                     : epi_unit<BN, false>(b, I, U, step, cur, n, tacc, acc_full(k2), acc_empty(k2), use, s_beta,
                                           s_dsc, s_flag, &s_args, bad);
      }
    }
    if (bad) s_flag[1] = 1;
    bar_epi();
    if (e == 0 && s_flag[1]) atomicOr(b.err, E_DIVERGED);
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && s_flag[0]) atomicOr(b.err, E_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

// Initial state of every instance: psi (init_mode 0 / 1 / 3, as the
// single-instance init: seeded U(-a, a) per component, plus the instance's
// base amplitudes for mode 3), its gamma0 and beta0, the BF16 operand and h1.
__global__ void k_batch_init(const BatchInst* inst, int n_inst, float* psi, float* gam, float* beta, float* h1,
                             const double* g64, const long long* off_g, const float* base, __nv_bfloat16* ops,
                             int pitch, int mode, float amp, float gamma0) {
  const int b = blockIdx.y;
  if (b >= n_inst) return;
  const BatchInst I = inst[b];
  const size_t total = size_t(I.R) * I.N;
  const bool with_base = mode == 3 && I.has_base;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / I.N), i = int(idx % I.N);
    float re = 0.0f, im = 0.0f;
    if (mode == 1 || mode == 3) {
      const U4 o = philox4x32_10(U4{uint32_t(i), uint32_t(r), 0u, 1u}, uint32_t(I.seed), uint32_t(I.seed >> 32));
      re = amp * (2.0f * philox_u01(o.x) - 1.0f);
      im = amp * (2.0f * philox_u01(o.y) - 1.0f);
      if (with_base) {
        re = __fadd_rn(base[I.off_base + 2 * i], re);
        im = __fadd_rn(base[I.off_base + 2 * i + 1], im);
      }
    }
    const int W = I.cplx ? 2 : 1;
    float* p = psi + I.off_psi;
    __nv_bfloat16* op = ops + size_t(I.rowX) * pitch;
    p[size_t(W * r) * I.Np + i] = re;
    op[size_t(W * r) * pitch + i] = __float2bfloat16_rn(re);
    if (I.cplx) {
      p[size_t(2 * r + 1) * I.Np + i] = im;
      op[size_t(2 * r + 1) * pitch + i] = __float2bfloat16_rn(im);
    }
    gam[I.off_gam + size_t(r) * I.Np + i] = gamma0;
    if (i == 0) beta[I.off_beta + r] = I.beta0;
    if (r == 0) h1[I.off_h1 + i] = float(-g64[off_g[b] + i]) * I.sq;
  }
}

__global__ void k_batch_advance(unsigned* step_base, unsigned by) { *step_base += by; }

// FP64 Eq. (1) energies per instance and restart: one block per
// (instance, 64-row tile, 64-column tile) unit; projection on the fly from
// the FP32 amplitudes of buffer parity cur.
__global__ void __launch_bounds__(256) k_batch_energy(const BatchInst* inst, const int4* units, const double* J64,
                                                      const long long* off_J, const double* g64,
                                                      const long long* off_g, const float* psi, int cur,
                                                      double* part, const long long* off_part) {
  const int4 U = units[blockIdx.x];
  const BatchInst I = inst[U.x];
  const int W = I.cplx ? 2 : 1, N = I.N, C = I.C;
  const float* p = psi + I.off_psi + size_t(cur) * I.Cp * I.Np;
  const double* J = J64 + off_J[U.x];
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = U.y * 64, n0 = U.z * 64;
  auto spin = [&](int c, int j) -> double {  // projected spin, column c = W r + part
    if (W == 1) return p[size_t(c) * I.Np + j] >= 0.0f ? 1.0 : -1.0;
    const int r = c >> 1;
    const double re = p[size_t(2 * r) * I.Np + j], im = p[size_t(2 * r + 1) * I.Np + j];
    const double m = sqrt(re * re + im * im);
    if (!(m > 0.0)) return (c & 1) ? 0.0 : 1.0;
    return ((c & 1) ? im : re) / m;
  };
  double acc[4][4] = {};
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (int k0 = 0; k0 < N; k0 += 16) {
    __syncthreads();
    for (int t = 0; t < 4; ++t) {
      const int row = m0 + lr, col = n0 + lr, k = k0 + lk + t;
      As[lk + t][lr] = (row < N && k < N) ? J[size_t(row) * N + k] : 0.0;
      Bs[lk + t][lr] = (col < C && k < N) ? spin(col, k) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double bv[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) bv[v] = Bs[k][4 * ty + v];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double av = As[k][tx + 16 * a];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[a][v] += av * bv[v];
      }
    }
  }
  double rs[4] = {0.0, 0.0, 0.0, 0.0};
  const int c0 = n0 + 4 * ty;
  for (int a = 0; a < 4; ++a) {
    const int i = m0 + tx + 16 * a;
    if (i >= N) continue;
    const double gi = g64[off_g[U.x] + i];
    for (int u = 0; u < 4 / W; ++u) {
      const int c = c0 + W * u;
      if (c >= C) continue;
      const double sr = spin(c, i);
      double e = -sr * acc[a][W * u] + gi * sr;
      if (W == 2) e -= spin(c + 1, i) * acc[a][W * u + 1];
      rs[u] += e;
    }
  }
  for (int u = 0; u < 4; ++u)
    for (int off = 8; off; off >>= 1) rs[u] += __shfl_xor_sync(0xffffffffu, rs[u], off);
  if (tx == 0)
    for (int u = 0; u < 4 / W; ++u) {
      const int r = c0 / W + u;
      if (r < I.R) part[off_part[U.x] + size_t(U.y) * I.R + r] = rs[u];
    }
}

// Per instance: E_r = sum of its row-tile partials, then the argmin (ties to
// the lowest restart).  One block per instance.
__global__ void k_batch_best(const BatchInst* inst, const double* part, const long long* off_part, double* E_all,
                             const long long* off_E, double* bestE, int* bestR) {
  const int b = blockIdx.x;
  const BatchInst I = inst[b];
  const int tiles = (I.N + 63) / 64;
  __shared__ double sE[32];
  __shared__ int sR[32];
  double best = 1.0 / 0.0;
  int br = 0x7fffffff;
  for (int r = threadIdx.x; r < I.R; r += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < tiles; ++t) s += part[off_part[b] + size_t(t) * I.R + r];
    E_all[off_E[b] + r] = s;
    if (s < best || (s == best && r < br)) { best = s; br = r; }
  }
  for (int off = 16; off; off >>= 1) {
    const double oE = __shfl_xor_sync(0xffffffffu, best, off);
    const int oR = __shfl_xor_sync(0xffffffffu, br, off);
    if (oE < best || (oE == best && oR < br)) { best = oE; br = oR; }
  }
  if ((threadIdx.x & 31) == 0) { sE[threadIdx.x >> 5] = best; sR[threadIdx.x >> 5] = br; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < int(blockDim.x >> 5); ++k)
      if (sE[k] < best || (sE[k] == best && sR[k] < br)) { best = sE[k]; br = sR[k]; }
    bestE[b] = best;
    bestR[b] = br;
  }
}

// Packs instance b's FP64 couplings into the BF16 tensor (diagonal removed).
__global__ void k_batch_pack_J(const double* J64, long long offJ, int N, __nv_bfloat16* J16, int rowJ, int pitch) {
  const size_t total = size_t(N) * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int i = int(idx / N), j = int(idx % N);
    const float v = (i == j) ? 0.0f : float(J64[offJ + idx]);
    J16[size_t(rowJ + i) * pitch + j] = __float2bfloat16_rn(v);
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode(CUtensorMap* m, const void* ptr, int pitch, int rows, int box_rows) {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    fn = reinterpret_cast<EncodeFn>(p);
  }
  const cuuint64_t dims[2] = {cuuint64_t(pitch), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(pitch) * 2};
  const cuuint32_t box[2] = {cuuint32_t(BK), cuuint32_t(box_rows)};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace
}  // namespace gda

using namespace gda;

// One launch list (the instances of one model type) for a tile width.
struct BatchPlan {
  int bn = 0;
  int grid = 0;
  BatchUnit* units = nullptr;
  int* cta_begin = nullptr;
  int n_units = 0;
};

struct gda_batch {
  int n = 0, dev = 0, sms = 148, pitch = 0;
  cudaStream_t stream = nullptr;
  std::vector<BatchInst> host;
  BatchInst* inst = nullptr;
  long long rowsJ = 0, rowsX = 0;
  __nv_bfloat16* J16 = nullptr;
  __nv_bfloat16* ops = nullptr;
  double* J64 = nullptr;
  double* g64 = nullptr;
  long long* off_J = nullptr;
  long long* off_g = nullptr;
  float* psi = nullptr;
  float* gam = nullptr;
  float* h1 = nullptr;
  float* beta = nullptr;
  double* part = nullptr;
  long long* off_part = nullptr;
  double* E_all = nullptr;
  long long* off_E = nullptr;
  double* bestE = nullptr;
  int* bestR = nullptr;
  int4* eunits = nullptr;
  int n_eunits = 0;
  unsigned* step_base = nullptr;
  unsigned* flags = nullptr;  // per-unit step flags [n_flags]
  int n_flags = 0;
  float* base = nullptr;      // per-instance base amplitudes for init_mode 3 [sum N][2]
  int* err = nullptr;
  CUtensorMap tmA{}, tmB128{}, tmB256{};
  BatchPlan plan[2][2];  // [persistent order, longest first][width: 128, 256], units of both model types
  int bn = 128;          // tile width in use (autotuned)
  bool persistent = true;  // one launch per chunk of steps (else one launch per step)
  std::vector<char> own;  // instance k has its own settings (gda_batch_set_params)
  std::vector<BatchInst> uploaded;  // the instance table as last copied to the device
  unsigned long long step = 0;
  bool have_state = false;
  std::string msg;
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;  // capture of the cooperative launch was refused: launch directly
  unsigned graph_key[8] = {};
};

namespace {

gda_status bfail(gda_batch* b, gda_status s, const char* m) {
  if (b) b->msg = m;
  return s;
}

#define BCK(expr)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      cudaGetLastError();                                                           \
      b->msg = std::string(#expr) + ": " + cudaGetErrorString(e_);                  \
      return e_ == cudaErrorMemoryAllocation ? GDA_ERR_OOM : GDA_ERR_CUDA;           \
    }                                                                               \
  } while (0)

template <typename T>
cudaError_t balloc(T** p, size_t n) {
  *p = nullptr;
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
}

// Longest-processing-time assignment of every instance's tiles to CTAs.
// sorted: within a CTA, units in one global order (instance, column block,
// row block), so that a unit of the next step depends on tiles every CTA
// finished early in this step (the persistent schedule); else longest first,
// which leaves the short units for the end of a launch (one launch per step).
gda_status build_plan(gda_batch* b, int bn, bool sorted, BatchPlan* P) {
  std::vector<BatchUnit> units;
  std::vector<double> cost;
  for (int k = 0; k < b->n; ++k) {
    const BatchInst& I = b->host[k];
    const int nt = (I.C + bn - 1) / bn;
    for (int mt = 0; mt < I.mt; ++mt)
      for (int t = 0; t < nt; ++t) {
        units.push_back(BatchUnit{k, mt, t, 0});
        cost.push_back(double((I.N + BK - 1) / BK) * (128 + bn) + 64.0);  // K-blocks x smem cycles + epilogue
      }
  }
  P->bn = bn;
  P->n_units = int(units.size());
  P->grid = std::min<int>(b->sms, std::max<int>(1, P->n_units));
  std::vector<int> order(units.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = int(k);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<std::vector<int>> bins(P->grid);
  std::vector<double> load(P->grid, 0.0);
  for (int u : order) {
    int best = 0;
    for (int c = 1; c < P->grid; ++c)
      if (load[c] < load[best]) best = c;
    bins[best].push_back(u);
    load[best] += cost[u];
  }
  auto key = [&](int u) { return std::make_tuple(units[u].inst, units[u].nt, units[u].mt); };
  if (sorted)
    for (auto& bin : bins) std::sort(bin.begin(), bin.end(), [&](int x, int y) { return key(x) < key(y); });
  std::vector<BatchUnit> flat;
  std::vector<int> begin(P->grid + 1, 0);
  for (int c = 0; c < P->grid; ++c) {
    begin[c] = int(flat.size());
    for (int u : bins[c]) flat.push_back(units[u]);
  }
  begin[P->grid] = int(flat.size());
  BCK(balloc(&P->units, flat.size()));
  BCK(balloc(&P->cta_begin, begin.size()));
  if (!flat.empty())
    BCK(cudaMemcpy(P->units, flat.data(), flat.size() * sizeof(BatchUnit), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(P->cta_begin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice));
  return GDA_OK;
}

template <int BN, int STAGES>
cudaError_t launch_batch(gda_batch* b, const BatchPlan& P, const BatchArgs& a) {
  using Cfg = BCfg<BN, STAGES>;
  const CUtensorMap& B = BN == 256 ? b->tmB256 : b->tmB128;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P.grid);
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = Cfg::SMEM;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the step flags need it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step_batch_kernel<BN, STAGES>, b->tmA, B, a);
}

// Shared-memory limits of both kernel variants, set once (outside any
// stream capture).
cudaError_t set_batch_attrs() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(step_batch_kernel<128, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                BCfg<128, 6>::SMEM)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(step_batch_kernel<256, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              BCfg<256, 4>::SMEM);
}

// One persistent launch of `nsteps` steps of every instance (offset `off`
// from the device step counter).
gda_status launch_chunk(gda_batch* b, const gda_params* p, unsigned off, int nsteps) {
  BatchArgs a{};
  a.inst = b->inst;
  a.psi = b->psi;
  a.gam = b->gam;
  a.h1 = b->h1;
  a.beta = b->beta;
  a.ops = b->ops;
  a.pitch = b->pitch;
  a.step_base = b->step_base;
  a.step_off = off;
  a.nsteps = nsteps;
  a.flags = b->flags;
  a.noise_D = float(p->noise_D);
  a.wait_cycles = p->wait_s > 0 ? (long long)(p->wait_s * kCyclesPerSecond) : kWaitCycles;
  a.err = b->err;
  const int wi = b->bn == 256 ? 1 : 0;
  const BatchPlan& P = b->plan[b->persistent ? 0 : 1][wi];
  if (P.n_units == 0) return GDA_OK;
  a.units = P.units;
  a.cta_begin = P.cta_begin;
  const cudaError_t le = wi ? launch_batch<256, 4>(b, P, a) : launch_batch<128, 6>(b, P, a);
  BCK(le);
  return GDA_OK;
}

// Instance settings of a run: the run's eps, rho_th, beta0 and eps_hat for
// instances without their own; copied to the device when they change.
gda_status upload_settings(gda_batch* b, const gda_params* p) {
  for (int k = 0; k < b->n; ++k) {
    if (b->own[k]) continue;
    BatchInst& I = b->host[k];
    I.dt = float(p->dt);
    I.eps = float(p->eps);
    I.rho_th = float(p->rho_th);
    I.beta0 = float(p->beta0);
    I.eps_hat = float(p->eps_hat);
    I.sq = float(std::sqrt(p->rho_th));
  }
  if (b->uploaded.size() == b->host.size() &&
      std::memcmp(b->uploaded.data(), b->host.data(), b->host.size() * sizeof(BatchInst)) == 0)
    return GDA_OK;
  BCK(cudaMemcpyAsync(b->inst, b->host.data(), b->host.size() * sizeof(BatchInst), cudaMemcpyHostToDevice,
                      b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  b->uploaded = b->host;
  return GDA_OK;
}

}  // namespace

extern "C" {

gda_status gda_batch_create(int32_t n, const int32_t* N, const int32_t* model, const int32_t* R,
                            const double* const* J, const double* const* g, uint64_t seed, gda_batch** out) {
  if (!out) return GDA_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || !N || !model || !R || !J) return GDA_ERR_INVALID;
  for (int k = 0; k < n; ++k) {
    if (N[k] < 1 || N[k] > 65536 || R[k] < 1 || (model[k] != GDA_ISING && model[k] != GDA_XY) || !J[k])
      return GDA_ERR_INVALID;
    const int64_t nn = N[k];
    for (int64_t i = 0; i < nn; ++i)
      for (int64_t j = 0; j < nn; ++j) {
        const double v = J[k][i * nn + j];
        if (!std::isfinite(v) || v != J[k][j * nn + i]) return GDA_ERR_INVALID;
      }
    if (g && g[k])
      for (int64_t i = 0; i < nn; ++i)
        if (!std::isfinite(g[k][i])) return GDA_ERR_INVALID;
  }
  gda_batch* b = new gda_batch();
  gda_status st = GDA_OK;
  auto done = [&](gda_status s) {
    if (s != GDA_OK) {
      gda_batch_destroy(b);
      return s;
    }
    *out = b;
    return GDA_OK;
  };
  if (cudaGetDevice(&b->dev) != cudaSuccess || !tc_supported(b->dev)) {
    cudaGetLastError();
    delete b;
    return GDA_ERR_UNSUPPORTED;
  }
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
  b->n = n;
  b->host.resize(n);
  long long off_psi = 0, off_gam = 0, off_h1 = 0, off_beta = 0, off_J = 0, off_g = 0, off_part = 0, off_E = 0;
  long long off_base = 0, n_flags = 0;
  std::vector<long long> oJ(n), oG(n), oP(n), oE(n);
  int pitch = 64;
  b->own.assign(n, 0);
  for (int k = 0; k < n; ++k) {
    BatchInst& I = b->host[k];
    I.N = N[k];
    I.Np = (N[k] + 127) / 128 * 128;
    I.cplx = model[k] == GDA_XY;
    I.R = R[k];
    I.C = I.cplx ? 2 * R[k] : R[k];
    I.Cp = (I.C + 255) / 256 * 256;
    I.Rp = (I.R + 255) / 256 * 256;
    I.mt = (I.N + 127) / 128;
    I.rowJ = int(b->rowsJ);
    I.rowX = int(b->rowsX);
    b->rowsJ += I.Np;
    b->rowsX += 2 * I.Cp;
    I.off_psi = off_psi;
    off_psi += 2LL * I.Cp * I.Np;
    I.off_gam = off_gam;
    off_gam += (long long)I.Rp * I.Np;
    I.off_h1 = off_h1;
    off_h1 += I.Np;
    I.off_beta = off_beta;
    off_beta += 2LL * I.Rp;
    I.off_base = off_base;
    off_base += 2LL * I.N;
    I.has_base = 0;
    I.flag0 = int(n_flags);
    n_flags += (long long)I.mt * ((I.C + 127) / 128);  // units at the narrowest tile width
    I.dt = 0.01f;
    I.eps = 0.1f;
    I.rho_th = 1.0f;
    I.eps_hat = 0.0f;
    I.beta0 = 1.0f;
    I.sq = 1.0f;
    I.seed = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)k;
    oJ[k] = off_J;
    off_J += (long long)I.N * I.N;
    oG[k] = off_g;
    off_g += I.N;
    oP[k] = off_part;
    off_part += (long long)((I.N + 63) / 64) * I.R;
    oE[k] = off_E;
    off_E += I.R;
    pitch = std::max(pitch, I.Np);
  }
  if (b->rowsJ > INT32_MAX / 2 || b->rowsX > INT32_MAX / 2 || n_flags > INT32_MAX / 2)
    return done(bfail(b, GDA_ERR_INVALID, "batch too large"));
  b->n_flags = int(n_flags);
  b->pitch = pitch;
  st = [&]() -> gda_status {
    BCK(balloc(&b->inst, n));
    BCK(cudaMemcpy(b->inst, b->host.data(), n * sizeof(BatchInst), cudaMemcpyHostToDevice));
    BCK(balloc(&b->J16, size_t(b->rowsJ) * pitch));
    BCK(cudaMemset(b->J16, 0, size_t(b->rowsJ) * pitch * sizeof(__nv_bfloat16)));
    BCK(balloc(&b->ops, size_t(b->rowsX) * pitch));
    BCK(cudaMemset(b->ops, 0, size_t(b->rowsX) * pitch * sizeof(__nv_bfloat16)));
    BCK(balloc(&b->J64, size_t(off_J)));
    BCK(balloc(&b->g64, size_t(off_g)));
    BCK(balloc(&b->off_J, n));
    BCK(balloc(&b->off_g, n));
    BCK(balloc(&b->off_part, n));
    BCK(balloc(&b->off_E, n));
    BCK(cudaMemcpy(b->off_J, oJ.data(), n * sizeof(long long), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->off_g, oG.data(), n * sizeof(long long), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->off_part, oP.data(), n * sizeof(long long), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->off_E, oE.data(), n * sizeof(long long), cudaMemcpyHostToDevice));
    BCK(balloc(&b->psi, size_t(off_psi)));
    BCK(cudaMemset(b->psi, 0, size_t(off_psi) * sizeof(float)));
    BCK(balloc(&b->gam, size_t(off_gam)));
    BCK(cudaMemset(b->gam, 0, size_t(off_gam) * sizeof(float)));
    BCK(balloc(&b->h1, size_t(off_h1)));
    BCK(cudaMemset(b->h1, 0, size_t(off_h1) * sizeof(float)));
    BCK(balloc(&b->beta, size_t(off_beta)));
    BCK(balloc(&b->part, size_t(off_part)));
    BCK(balloc(&b->E_all, size_t(off_E)));
    BCK(balloc(&b->bestE, n));
    BCK(balloc(&b->bestR, n));
    BCK(balloc(&b->step_base, 1));
    BCK(cudaMemset(b->step_base, 0, sizeof(unsigned)));
    BCK(balloc(&b->flags, size_t(b->n_flags)));
    BCK(cudaMemset(b->flags, 0, size_t(b->n_flags) * sizeof(unsigned)));
    BCK(balloc(&b->base, size_t(off_base)));
    BCK(cudaMemset(b->base, 0, size_t(off_base) * sizeof(float)));
    BCK(balloc(&b->err, 1));
    BCK(cudaMemset(b->err, 0, sizeof(int)));
    for (int k = 0; k < n; ++k) {
      BCK(cudaMemcpy(b->J64 + oJ[k], J[k], size_t(N[k]) * N[k] * sizeof(double), cudaMemcpyHostToDevice));
      if (g && g[k])
        BCK(cudaMemcpy(b->g64 + oG[k], g[k], size_t(N[k]) * sizeof(double), cudaMemcpyHostToDevice));
      else
        BCK(cudaMemset(b->g64 + oG[k], 0, size_t(N[k]) * sizeof(double)));
      const size_t tot = size_t(N[k]) * N[k];
      k_batch_pack_J<<<int(std::min<size_t>(4096, (tot + 255) / 256)), 256>>>(b->J64, oJ[k], N[k], b->J16,
                                                                               b->host[k].rowJ, pitch);
      BCK(cudaGetLastError());
    }
    // FP64 energy units: (instance, 64-row tile, 64-column tile)
    std::vector<int4> eu;
    for (int k = 0; k < n; ++k) {
      const BatchInst& I = b->host[k];
      for (int mt = 0; mt < (I.N + 63) / 64; ++mt)
        for (int nt = 0; nt < (I.C + 63) / 64; ++nt) eu.push_back(make_int4(k, mt, nt, 0));
    }
    b->n_eunits = int(eu.size());
    BCK(balloc(&b->eunits, eu.size()));
    BCK(cudaMemcpy(b->eunits, eu.data(), eu.size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (!encode(&b->tmA, b->J16, pitch, int(b->rowsJ), 128) || !encode(&b->tmB128, b->ops, pitch, int(b->rowsX), 128) ||
        !encode(&b->tmB256, b->ops, pitch, int(b->rowsX), 256))
      return bfail(b, GDA_ERR_CUDA, "tensor map encoding failed");
    for (int oi = 0; oi < 2; ++oi)
      for (int wi = 0; wi < 2; ++wi) {
        gda_status s = build_plan(b, wi ? 256 : 128, oi == 0, &b->plan[oi][wi]);
        if (s != GDA_OK) return s;
      }
    BCK(set_batch_attrs());
    BCK(cudaDeviceSynchronize());
    return GDA_OK;
  }();
  return done(st);
}

gda_status gda_batch_set_stream(gda_batch* b, void* stream) {
  if (!b) return GDA_ERR_INVALID;
  b->stream = static_cast<cudaStream_t>(stream);
  return GDA_OK;
}

gda_status gda_batch_set_tile(gda_batch* b, int32_t bn) {
  if (!b || (bn != 128 && bn != 256)) return GDA_ERR_INVALID;
  b->bn = bn;
  return GDA_OK;
}

gda_status gda_batch_set_schedule(gda_batch* b, int32_t schedule) {
  if (!b || (schedule != GDA_SCHEDULE_RESIDENT && schedule != GDA_SCHEDULE_PER_STEP)) return GDA_ERR_INVALID;
  b->persistent = schedule == GDA_SCHEDULE_RESIDENT;
  return GDA_OK;
}

gda_status gda_batch_set_params(gda_batch* b, int32_t k, const gda_params* p) {
  if (!b || k < 0 || k >= b->n) return GDA_ERR_INVALID;
  if (!p) {
    b->own[k] = 0;
    return GDA_OK;
  }
  if (!std::isfinite(p->eps) || !std::isfinite(p->rho_th) || !std::isfinite(p->beta0) || !std::isfinite(p->eps_hat) ||
      !(p->rho_th > 0) || !(p->dt > 0) || !std::isfinite(p->dt))
    return bfail(b, GDA_ERR_INVALID, "non-finite settings, dt <= 0 or rho_th <= 0");
  BatchInst& I = b->host[k];
  I.dt = float(p->dt);
  I.eps = float(p->eps);
  I.rho_th = float(p->rho_th);
  I.beta0 = float(p->beta0);
  I.eps_hat = float(p->eps_hat);
  I.sq = float(std::sqrt(p->rho_th));
  b->own[k] = 1;
  return GDA_OK;
}

gda_status gda_batch_set_init_base(gda_batch* b, int32_t k, const float* base, int32_t on_device) {
  if (!b || k < 0 || k >= b->n) return GDA_ERR_INVALID;
  BatchInst& I = b->host[k];
  if (!base) {
    I.has_base = 0;
    return GDA_OK;
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (I.cplx) {
    BCK(cudaMemcpyAsync(b->base + I.off_base, base, size_t(2) * I.N * sizeof(float), kind, b->stream));
  } else {  // real amplitudes: imaginary parts zero
    BCK(cudaMemsetAsync(b->base + I.off_base, 0, size_t(2) * I.N * sizeof(float), b->stream));
    BCK(cudaMemcpy2DAsync(b->base + I.off_base, 2 * sizeof(float), base, sizeof(float), sizeof(float), I.N, kind,
                          b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  I.has_base = 1;
  return GDA_OK;
}

gda_status gda_batch_run(gda_batch* b, const gda_params* p, int64_t steps) {
  if (!b || !p) return GDA_ERR_INVALID;
  if (steps < 0) return bfail(b, GDA_ERR_INVALID, "steps < 0");
  if (p->integ != GDA_EULER || p->prec != GDA_BF16)
    return bfail(b, GDA_ERR_UNSUPPORTED, "batched runs are BF16 forward Euler");
  if (p->noise_D != 0.0 && p->noise_decay)
    return bfail(b, GDA_ERR_UNSUPPORTED, "batched runs support noise without decay only");
  if (!(p->dt > 0) || !(p->rho_th > 0) || p->init_mode < 0 || p->init_mode > 3 || !std::isfinite(p->wait_s) ||
      p->wait_s < 0 || p->wait_s > 1e3)
    return bfail(b, GDA_ERR_INVALID, "bad parameters");
  if (p->init_mode == 2 && !b->have_state) return bfail(b, GDA_ERR_STATE, "nothing to continue");
  gda_status us = upload_settings(b, p);
  if (us != GDA_OK) return us;
  if (p->init_mode != 2) {
    int maxRN = 1;
    for (auto& I : b->host) maxRN = std::max(maxRN, I.R * I.N);
    dim3 grid(std::min(1024, (maxRN + 255) / 256), b->n);
    k_batch_init<<<grid, 256, 0, b->stream>>>(b->inst, b->n, b->psi, b->gam, b->beta, b->h1, b->g64, b->off_g,
                                              b->base, b->ops, b->pitch, p->init_mode, float(p->init_amp),
                                              float(p->gamma0));
    BCK(cudaGetLastError());
    BCK(cudaMemsetAsync(b->step_base, 0, sizeof(unsigned), b->stream));
    BCK(cudaMemsetAsync(b->flags, 0, size_t(b->n_flags) * sizeof(unsigned), b->stream));
    b->step = 0;
    b->have_state = true;
  }
  // Chunks of `chunk` steps: one persistent launch each, replayed from a
  // captured graph (launch + step counter advance); the kernel reads the step
  // index and buffer parity from the device counter.
  const int chunk = 100;
  float ws = float(p->wait_s);
  unsigned wbits = 0;
  std::memcpy(&wbits, &ws, sizeof(wbits));
  float nd = float(p->noise_D);
  unsigned nbits = 0;
  std::memcpy(&nbits, &nd, sizeof(nbits));
  const unsigned key[8] = {unsigned(b->bn), nbits, wbits, unsigned(chunk), unsigned(b->persistent), 0u, 0u, 0u};
  if (steps >= chunk && !b->graph_failed && (!b->graph || std::memcmp(key, b->graph_key, sizeof(key)) != 0)) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaStream_t cap = nullptr;
    BCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = b->stream;
    b->stream = cap;
    BCK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    gda_status s = GDA_OK;
    if (b->persistent) {
      s = launch_chunk(b, p, 0u, chunk);
    } else {
      for (int k = 0; k < chunk && s == GDA_OK; ++k) s = launch_chunk(b, p, unsigned(k), 1);
    }
    k_batch_advance<<<1, 1, 0, cap>>>(b->step_base, unsigned(chunk));
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cap, &g);
    b->stream = saved;
    cudaStreamDestroy(cap);
    cudaError_t ie = cudaErrorUnknown;
    if (s == GDA_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ie != cudaSuccess) {  // the CUDA runtime declined to capture this launch: chunks launch directly
      cudaGetLastError();
      b->graph = nullptr;
      b->graph_failed = true;
    } else {
      std::memcpy(b->graph_key, key, sizeof(key));
    }
  }
  int64_t done = 0;
  for (; done + chunk <= steps; done += chunk) {
    if (b->graph) {
      BCK(cudaGraphLaunch(b->graph, b->stream));
      continue;
    }
    for (int k = 0; k < (b->persistent ? 1 : chunk); ++k) {
      gda_status s = launch_chunk(b, p, unsigned(k), b->persistent ? chunk : 1);
      if (s != GDA_OK) return s;
    }
    k_batch_advance<<<1, 1, 0, b->stream>>>(b->step_base, unsigned(chunk));
    BCK(cudaGetLastError());
  }
  if (done < steps) {
    const int rest = int(steps - done);
    for (int k = 0; k < (b->persistent ? 1 : rest); ++k) {
      gda_status s = launch_chunk(b, p, unsigned(k), b->persistent ? rest : 1);
      if (s != GDA_OK) return s;
    }
    k_batch_advance<<<1, 1, 0, b->stream>>>(b->step_base, unsigned(rest));
    BCK(cudaGetLastError());
  }
  b->step += steps;
  return GDA_OK;
}

int32_t gda_batch_launch_mode(const gda_batch* b) { return !b ? -1 : (b->graph ? 1 : 0); }

gda_status gda_batch_best(gda_batch* b, double* E, int32_t* r) {
  if (!b) return GDA_ERR_INVALID;
  if (!b->have_state) return bfail(b, GDA_ERR_STATE, "no state");
  const int cur = int(b->step & 1ULL);
  k_batch_energy<<<b->n_eunits, 256, 0, b->stream>>>(b->inst, b->eunits, b->J64, b->off_J, b->g64, b->off_g, b->psi,
                                                      cur, b->part, b->off_part);
  BCK(cudaGetLastError());
  k_batch_best<<<b->n, 256, 0, b->stream>>>(b->inst, b->part, b->off_part, b->E_all, b->off_E, b->bestE, b->bestR);
  BCK(cudaGetLastError());
  if (E) BCK(cudaMemcpyAsync(E, b->bestE, size_t(b->n) * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  if (r) BCK(cudaMemcpyAsync(r, b->bestR, size_t(b->n) * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  int e = 0;
  BCK(cudaMemcpyAsync(&e, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (e) {
    BCK(cudaMemset(b->err, 0, sizeof(int)));
    return bfail(b, (e & E_TIMEOUT) ? GDA_ERR_TIMEOUT : GDA_ERR_DIVERGED, "device error during the batched run");
  }
  return GDA_OK;
}

gda_status gda_batch_get_state(gda_batch* b, int32_t k, float* psi, float* gamma, float* beta) {
  if (!b || k < 0 || k >= b->n) return GDA_ERR_INVALID;
  if (!b->have_state) return bfail(b, GDA_ERR_STATE, "no state");
  BCK(cudaStreamSynchronize(b->stream));
  const BatchInst& I = b->host[k];
  const int cur = int(b->step & 1ULL);
  const int W = I.cplx ? 2 : 1;
  std::vector<float> blk(size_t(I.Cp) * I.Np), gb(size_t(I.Rp) * I.Np);
  BCK(cudaMemcpy(blk.data(), b->psi + I.off_psi + size_t(cur) * I.Cp * I.Np, blk.size() * sizeof(float),
                 cudaMemcpyDeviceToHost));
  BCK(cudaMemcpy(gb.data(), b->gam + I.off_gam, gb.size() * sizeof(float), cudaMemcpyDeviceToHost));
  for (int r = 0; r < I.R; ++r)
    for (int i = 0; i < I.N; ++i) {
      if (psi)
        for (int q = 0; q < W; ++q) psi[(size_t(r) * I.N + i) * W + q] = blk[size_t(W * r + q) * I.Np + i];
      if (gamma) gamma[size_t(r) * I.N + i] = gb[size_t(r) * I.Np + i];
    }
  if (beta) BCK(cudaMemcpy(beta, b->beta + I.off_beta + size_t(cur) * I.Rp, I.R * sizeof(float),
                           cudaMemcpyDeviceToHost));
  return GDA_OK;
}

const char* gda_batch_last_error(const gda_batch* b) { return b ? b->msg.c_str() : "NULL batch"; }

void gda_batch_destroy(gda_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& row : b->plan)
    for (auto& P : row) {
      if (P.units) cudaFree(P.units);
      if (P.cta_begin) cudaFree(P.cta_begin);
    }
  void* ptrs[] = {b->inst, b->J16, b->ops, b->J64, b->g64, b->off_J, b->off_g, b->psi, b->gam, b->h1, b->beta,
                  b->part, b->off_part, b->E_all, b->off_E, b->bestE, b->bestR, b->eunits, b->step_base, b->err,
                  b->flags, b->base};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete b;
}

}  // extern "C"
