// Register-staged epilogue of the tensor-core step kernel.
//
// Each epilogue thread owns one spin row i and walks its columns in chunks of
// CW.  All inputs a chunk needs (amplitudes, gains, RK4 accumulators) are
// loaded into registers one chunk ahead of the arithmetic, and the first chunk
// is loaded while the MMAs are still running, so global-memory latency is
// paid about once per kernel instead of once per element.  The arithmetic is
// the same FP32 expression sequence as epi_quad (epilogue.cuh).
#pragma once
#include <cuda_fp8.h>

#include "epilogue.cuh"

namespace gda {

template <int MODE>
struct ModeTraits {
  static constexpr bool rk_mid = MODE == M_RK2 || MODE == M_RK3 || MODE == M_RK4;
  static constexpr bool has_x = MODE != M_RAW;
  static constexpr bool has_g = MODE != M_RAW && MODE != M_ENERGY;
  // chunks whose inputs are loaded into registers ahead of the one computed
  // (a second chunk in registers spills at the 96 registers of a 576-thread
  // block and measured slower)
  static constexpr int prefetch = 1;
  // chunks whose state lines are pulled into L2 ahead of their register
  // loads (no registers: the loads of a chunk then find their lines in L2)
  static constexpr int l2_ahead = MODE == M_RAW ? 0 : 3;
};

// Loads and stores of the FP32 state.  (An evict-first L2 policy on them
// measured slower: the lines the L2 prefetch brings in were dropped before
// their loads.)
static __device__ __forceinline__ float ld_state(const float* p) { return *p; }
static __device__ __forceinline__ void st_state(float* p, float v) { *p = v; }

template <int MODE, bool CPLX, int CW>
struct EpiRegs {
  static constexpr int W = CPLX ? 2 : 1;
  static constexpr int NR = CW / W;
  using T = ModeTraits<MODE>;
  float x[T::has_x ? CW : 1];
  float pn[T::rk_mid ? CW : 1];
  float ac[T::rk_mid ? CW : 1];
  float gs[T::has_g ? NR : 1];
  float gn[T::rk_mid ? NR : 1];
  float ga[T::rk_mid ? NR : 1];
};

// Loads the inputs of columns c0 .. c0+CW-1 at row i.  Column and restart
// indices are clamped to the padded buffers (columns < Cp, restarts < Rp), so
// every address is valid whatever the tile width; values of columns beyond C
// are discarded by epi_chunk.
template <int MODE, bool CPLX, int CW>
__device__ __forceinline__ void epi_load(const StepArgs& a, int i, int c0, EpiRegs<MODE, CPLX, CW>& R) {
  using Tr = ModeTraits<MODE>;
  constexpr int W = CPLX ? 2 : 1;
  const size_t Np = a.Np;
  const int r0 = CPLX ? c0 / 2 : c0;
#pragma unroll
  for (int k = 0; k < CW; ++k) {
    const size_t o = size_t(min(c0 + k, a.Cp - 1)) * Np + i;
    if (MODE == M_ENERGY) {
      R.x[k] = ld_state(a.psi_n + o);
    } else if (Tr::has_x) {
      R.x[k] = ld_state(a.xs + o);
      if (Tr::rk_mid) {
        R.pn[k] = ld_state(a.psi_n + o);
        R.ac[k] = ld_state(a.acc + o);
      }
    }
  }
  if (Tr::has_g) {
#pragma unroll
    for (int u = 0; u < CW / W; ++u) {
      const size_t og = size_t(min(r0 + u, a.Rp - 1)) * Np + i;
      R.gs[u] = ld_state(((MODE == M_EULER || MODE == M_RK1) ? a.gam : a.gstg) + og);
      if (Tr::rk_mid) {
        R.gn[u] = ld_state(a.gam + og);
        R.ga[u] = ld_state(a.gacc + og);
      }
    }
  }
}

static __device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Pulls into L2 the state lines that epi_load of columns c0 .. c0+CW-1 will
// read for the warp's 32 rows (i - lane .. i - lane + 31: one 128-byte line per
// column): lanes 0 .. CW-1 take the amplitude columns, the next CW / W lanes
// the gain rows.  Addresses are clamped as in epi_load.
template <int MODE, bool CPLX, int CW>
__device__ __forceinline__ void epi_prefetch_l2(const StepArgs& a, int i, int c0, int lane) {
  using Tr = ModeTraits<MODE>;
  constexpr int W = CPLX ? 2 : 1;
  constexpr int NR = CW / W;
  if (MODE == M_RAW) return;
  const size_t Np = a.Np;
  const int ib = i - lane;
  if (lane < CW) {
    const size_t o = size_t(min(c0 + lane, a.Cp - 1)) * Np + ib;
    prefetch_l2((MODE == M_ENERGY ? a.psi_n : a.xs) + o);
    if (Tr::rk_mid) {
      prefetch_l2(a.psi_n + o);
      prefetch_l2(a.acc + o);
    }
  } else if (Tr::has_g && lane < CW + NR) {
    const int r0 = CPLX ? c0 / 2 : c0;
    const size_t og = size_t(min(r0 + lane - CW, a.Rp - 1)) * Np + ib;
    prefetch_l2(((MODE == M_EULER || MODE == M_RK1) ? a.gam : a.gstg) + og);
    if (Tr::rk_mid) {
      prefetch_l2(a.gam + og);
      prefetch_l2(a.gacc + og);
    }
  }
}

// Arithmetic and stores of one chunk.  y: the CW accumulator values of row i.
// beta_s / dsc: per-restart stage scale and noise amplitude, indexed by the
// chunk's local restart.  red[u]: per-restart contribution (density of the
// new amplitude, or Eq. (1) partial energy).  nxt (NXT only): receives the
// chunk's next operand values (the new amplitudes, or the next RK stage
// input), 0 for restarts beyond R.
template <int MODE, bool CPLX, int CW, bool NXT = false>
__device__ __forceinline__ void epi_chunk(const StepArgs& a, int i, int c0, const float* y,
                                          const EpiRegs<MODE, CPLX, CW>& R, const float* beta_s, const float* dsc,
                                          float* red, int& bad, float* nxt = nullptr) {
  constexpr int W = CPLX ? 2 : 1;
  constexpr int NR = CW / W;
  const size_t Np = a.Np;
  const int r0 = CPLX ? c0 / 2 : c0;
  const bool row_ok = i < a.N;
  const float h = row_ok ? a.h1[i] : 0.0f;
  const float gi = (MODE == M_ENERGY && row_ok) ? a.g[i] : 0.0f;
  float z[CW];
  if (MODE == M_EULER || MODE == M_RK4) {
    bool any = false;
#pragma unroll
    for (int u = 0; u < NR; ++u) any |= dsc[u] != 0.0f;
#pragma unroll
    for (int q = 0; q < CW / 4; ++q) {
      if (any) {
        philox_normal4(uint32_t(i), uint32_t((c0 >> 2) + q), a.step, 0u, a.seed, &z[4 * q]);
      } else {
        z[4 * q] = z[4 * q + 1] = z[4 * q + 2] = z[4 * q + 3] = 0.0f;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    red[u] = 0.0f;
    if (NXT) {
      nxt[u * W] = 0.0f;
      if (CPLX) nxt[u * W + 1] = 0.0f;
    }
    const int r = r0 + u;
    if (!row_ok || r >= a.R) continue;
    const int k0 = u * W;
    const size_t o0 = size_t(c0 + k0) * Np + i;
    const size_t o1 = o0 + Np;
    const size_t og = size_t(r) * Np + i;
    const float yr = y[k0], yi = CPLX ? y[k0 + 1] : 0.0f;
    if (MODE == M_RAW) {
      a.psi_out[o0] = yr;
      if (CPLX) a.psi_out[o1] = yi;
      continue;
    }
    if (MODE == M_ENERGY) {
      const float pr = R.x[k0], pi = CPLX ? R.x[k0 + 1] : 0.0f;
      float sr, si = 0.0f;
      if (CPLX && a.q >= 2) {  // Potts: the nearest q-th root, as the operand's projection
        double dr, di;
        potts_project(pr, pi, a.q, dr, di);
        sr = float(dr);
        si = float(di);
      } else if (CPLX) {
        const float m = sqrtf(pr * pr + pi * pi);
        sr = m > 0.0f ? pr / m : 1.0f;
        si = m > 0.0f ? pi / m : 0.0f;
      } else {
        sr = pr >= 0.0f ? 1.0f : -1.0f;
      }
      red[u] = -(sr * yr + si * yi) + gi * sr;
      continue;
    }
    const float xr = R.x[k0], xi = CPLX ? R.x[k0 + 1] : 0.0f;
    const float gs = R.gs[u];
    float kr, ki, kg;
    gd_rhs(xr, xi, gs, yr, yi, beta_s[u], h, a.eps, a.rho_th, kr, ki, kg);
    if (CPLX && a.q) resonant_drive(xr, xi, a.q, a.hq, kr, ki);
    float nr, ni, ng;
    if (MODE == M_EULER) {
      nr = axpy(a.dt, kr, xr);
      ni = axpy(a.dt, ki, xi);
      ng = axpy(a.dt, kg, gs);
    } else {
      const float pr = (MODE == M_RK1) ? xr : R.pn[ModeTraits<MODE>::rk_mid ? k0 : 0];
      const float pi = (MODE == M_RK1) ? xi : (CPLX ? R.pn[ModeTraits<MODE>::rk_mid ? k0 + 1 : 0] : 0.0f);
      const float gn = (MODE == M_RK1) ? gs : R.gn[ModeTraits<MODE>::rk_mid ? u : 0];
      if (MODE == M_RK4) {
        const float d6 = __fdiv_rn(a.dt, 6.0f);
        nr = axpy(d6, __fadd_rn(R.ac[k0], kr), pr);
        ni = CPLX ? axpy(d6, __fadd_rn(R.ac[CPLX ? k0 + 1 : 0], ki), pi) : 0.0f;
        ng = axpy(d6, __fadd_rn(R.ga[u], kg), gn);
      } else {
        const float cf = (MODE == M_RK3) ? a.dt : __fmul_rn(0.5f, a.dt);
        if (MODE == M_RK1) {
          st_state(a.acc + o0, kr);
          if (CPLX) st_state(a.acc + o1, ki);
          st_state(a.gacc + og, kg);
        } else {
          st_state(a.acc + o0, axpy(2.0f, kr, R.ac[ModeTraits<MODE>::rk_mid ? k0 : 0]));
          if (CPLX) st_state(a.acc + o1, axpy(2.0f, ki, R.ac[ModeTraits<MODE>::rk_mid ? k0 + 1 : 0]));
          st_state(a.gacc + og, axpy(2.0f, kg, R.ga[ModeTraits<MODE>::rk_mid ? u : 0]));
        }
        const float sr = axpy(cf, kr, pr), si = axpy(cf, ki, pi);
        if (NXT) {
          nxt[k0] = sr;
          if (CPLX) nxt[k0 + 1] = si;
        }
        st_state(a.xs_next + o0, sr);
        if (CPLX) st_state(a.xs_next + o1, si);
        st_state(a.gstg + og, axpy(cf, kg, gn));
        if (a.op_out) {
          const size_t p0 = size_t(c0 + k0) * a.op_pitch + i;
          a.op_out[p0] = __float2bfloat16_rn(sr);
          if (CPLX) a.op_out[p0 + a.op_pitch] = __float2bfloat16_rn(si);
        }
        if (a.op8_out) {
          a.op8_out[o0] = __nv_cvt_float_to_fp8(sr * a.op8_inv, __NV_SATFINITE, __NV_E4M3);
          if (CPLX) a.op8_out[o1] = __nv_cvt_float_to_fp8(si * a.op8_inv, __NV_SATFINITE, __NV_E4M3);
        }
        continue;
      }
    }
    if (MODE == M_EULER || MODE == M_RK4) {
      nr = axpy(dsc[u], z[k0], nr);
      if (CPLX) ni = axpy(dsc[u], z[k0 + 1], ni);
    }
    if (NXT) {
      nxt[k0] = nr;
      if (CPLX) nxt[k0 + 1] = ni;
    }
    st_state(a.psi_out + o0, nr);
    if (CPLX) st_state(a.psi_out + o1, ni);
    st_state(a.gam + og, ng);
    if (a.op_out) {
      const size_t p0 = size_t(c0 + k0) * a.op_pitch + i;
      a.op_out[p0] = __float2bfloat16_rn(nr);
      if (CPLX) a.op_out[p0 + a.op_pitch] = __float2bfloat16_rn(ni);
    }
    if (a.op8_out) {
      a.op8_out[o0] = __nv_cvt_float_to_fp8(nr * a.op8_inv, __NV_SATFINITE, __NV_E4M3);
      if (CPLX) a.op8_out[o1] = __nv_cvt_float_to_fp8(ni * a.op8_inv, __NV_SATFINITE, __NV_E4M3);
    }
    const float rn = density(nr, ni);
    red[u] = rn;
    bad |= !(rn < 1e30f);
  }
}

}  // namespace gda
