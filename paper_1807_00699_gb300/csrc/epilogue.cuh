// Fused per-element epilogue of one GD step (Eqs. 2, 5, 6; Sec. 2 RK4), shared
// by the FP32 SIMT kernel and the tcgen05 kernel.  It receives the coupling
// sum Y = J Psi of one row i for four consecutive columns c0..c0+3 (c0 a
// multiple of 4) and updates amplitude, gain and RK4 stage state in place.
//
// A column quad holds four Ising restarts, or two XY restarts as (re, im)
// pairs; one Philox call with counter (i, c0/4, step, 0) gives the quad's four
// normals, z_k for column c0+k (scaled by 1/sqrt 2 for complex amplitudes).
#pragma once
#include "gda_internal.h"
#include "philox.cuh"

namespace gda {

// Every rounding below is explicit (fused multiply-add, IEEE add / multiply /
// divide / square root), so each kernel that performs an update computes the
// same bits whatever code surrounds it.

// d beta / dt = eps_hat (1 - beta) (Eq. 6 with Delta = 1, K = beta J).
__device__ __forceinline__ float beta_rate(float eh, float b) { return __fmul_rn(eh, __fsub_rn(1.0f, b)); }

// Stage coupling scale beta_s of a restart for the launch's mode.
__device__ __forceinline__ float stage_beta(const StepArgs& a, float b) {
  const float eh = a.eps_hat, hdt = __fmul_rn(0.5f, a.dt);
  switch (a.mode) {
    case M_RK2: return __fmaf_rn(hdt, beta_rate(eh, b), b);
    case M_RK3: {
      const float b2 = __fmaf_rn(hdt, beta_rate(eh, b), b);
      return __fmaf_rn(hdt, beta_rate(eh, b2), b);
    }
    case M_RK4: {
      const float b2 = __fmaf_rn(hdt, beta_rate(eh, b), b);
      const float b3 = __fmaf_rn(hdt, beta_rate(eh, b2), b);
      return __fmaf_rn(a.dt, beta_rate(eh, b3), b);
    }
    case M_ENERGY: return 1.0f;
    default: return b;
  }
}

// beta^{n+1} from beta^n for a completed Euler or RK4 step.
__device__ __forceinline__ float next_beta(const StepArgs& a, float b) {
  const float eh = a.eps_hat, dt = a.dt, hdt = __fmul_rn(0.5f, a.dt);
  if (a.mode == M_EULER) return __fmaf_rn(dt, beta_rate(eh, b), b);
  const float k1 = beta_rate(eh, b);
  const float k2 = beta_rate(eh, __fmaf_rn(hdt, k1, b));
  const float k3 = beta_rate(eh, __fmaf_rn(hdt, k2, b));
  const float k4 = beta_rate(eh, __fmaf_rn(dt, k3, b));
  const float sum = __fadd_rn(__fadd_rn(__fadd_rn(k1, __fmul_rn(2.0f, k2)), __fmul_rn(2.0f, k3)), k4);
  return __fmaf_rn(__fdiv_rn(dt, 6.0f), sum, b);
}

__device__ __forceinline__ bool step_completes(int mode) { return mode == M_EULER || mode == M_RK4; }

// Noise amplitude sqrt(dt) D_r (times 1/sqrt 2 for complex amplitudes) of
// restart r; D_r = D max(0, 1 - mean_i rho_i / rho_th) under noise decay,
// with the mean over the N spins of psi^n from the per-tile partial sums.
__device__ __forceinline__ float noise_scale(const StepArgs& a, int r) {
  if (!step_completes(a.mode) || a.noise_D == 0.0f) return 0.0f;
  float D = a.noise_D;
  if (a.noise_decay) {
    float s = 0.0f;
    for (int t = 0; t < a.mt_count; ++t) s = __fadd_rn(s, a.rho_in[t * a.Rp + r]);
    const float ratio = __fdiv_rn(__fdiv_rn(s, float(a.N)), a.rho_th);
    D = __fmul_rn(D, fmaxf(0.0f, __fsub_rn(1.0f, ratio)));
  }
  return __fmul_rn(__fmul_rn(__fsqrt_rn(a.dt), D), a.cplx ? 0.70710678118654752f : 1.0f);
}

// Right-hand side of Eqs. (2) and (5) for one restart at one spin:
// k = x (gamma_s - |x|^2) + beta_s y + h,  k_gamma = eps (rho_th - |x|^2).
__device__ __forceinline__ void gd_rhs(float xr, float xi, float gs, float yr, float yi, float bs, float h, float eps,
                                       float rho_th, float& kr, float& ki, float& kg) {
  const float rho = density(xr, xi);
  const float t = __fsub_rn(gs, rho);
  kr = __fmaf_rn(xr, t, __fmaf_rn(bs, yr, h));
  ki = __fmaf_rn(xi, t, __fmul_rn(bs, yi));
  kg = __fmul_rn(eps, __fsub_rn(rho_th, rho));
}

// Resonant q:1 drive of Eq. (2) for complex amplitudes: (kr, ki) += h_q conj(x)^(q-1).
__device__ __forceinline__ void resonant_drive(float xr, float xi, int q, float hq, float& kr, float& ki) {
  float pr = 1.0f, pi = 0.0f;
  for (int k = 1; k < q; ++k) {  // p <- p conj(x)
    const float nr = __fmaf_rn(pr, xr, __fmul_rn(pi, xi));
    const float ni = __fmaf_rn(pi, xr, -__fmul_rn(pr, xi));
    pr = nr;
    pi = ni;
  }
  kr = __fmaf_rn(hq, pr, kr);
  ki = __fmaf_rn(hq, pi, ki);
}

// y + a x with one rounding.
__device__ __forceinline__ float axpy(float a, float x, float y) { return __fmaf_rn(a, x, y); }

// One quad.  beta_s[u], dsc[u]: per-restart stage scale and noise amplitude
// of the quad's restarts (4 Ising, 2 XY).  red[u] receives |psi^{n+1}|^2
// (completed steps) or the restart's Eq. (1) contribution of spin i (energy
// mode); 0 for padded restarts.  bad is set for a non-finite amplitude.
// TSTORE: also write the quad's next operand values to a.opT_out (spin-major).
// MODE: the launch's mode (a compile-time copy of a.mode, so that each mode's
// kernel holds only its own branch).
template <bool CPLX, bool TSTORE, int MODE>
__device__ __forceinline__ void epi_quad(const StepArgs& a, int i, int c0, const float y[4],
                                         const float* beta_s, const float* dsc, float red[4],
                                         int& bad) {
  constexpr int U = CPLX ? 2 : 4;
  constexpr int W = CPLX ? 2 : 1;
  const int Np = a.Np;
  constexpr int mode = MODE;
  const int r0 = CPLX ? (c0 >> 1) : c0;
  float z[4] = {0.f, 0.f, 0.f, 0.f};
  if (step_completes(mode)) {
    bool any = false;
#pragma unroll
    for (int u = 0; u < U; ++u) any |= dsc[u] != 0.0f;
    if (any) philox_normal4(uint32_t(i), uint32_t(c0 >> 2), a.step, 0u, a.seed, z);
  }
  const float h = a.h1[i];
  float t4[4] = {0.f, 0.f, 0.f, 0.f};  // the quad's next operand values (spin-major copy)
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int r = r0 + u;
    const int col = c0 + u * W;
    red[u] = 0.0f;
    if (r >= a.R) continue;
    const size_t o0 = size_t(col) * Np + i;
    const size_t o1 = o0 + Np;  // imaginary part (XY)
    const size_t og = size_t(r) * Np + i;
    const float yr = y[u * W], yi = CPLX ? y[u * W + 1] : 0.0f;

    if (mode == M_RAW) {
      a.psi_out[o0] = yr;
      if (CPLX) a.psi_out[o1] = yi;
      continue;
    }

    if (mode == M_ENERGY) {
      // e_i = -Re(conj(s_i) (J0 s)_i) + g_i Re(s_i), s the projection of psi^n.
      const float pr = a.psi_n[o0], pi = CPLX ? a.psi_n[o1] : 0.0f;
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
      red[u] = -(sr * yr + si * yi) + a.g[i] * sr;
      continue;
    }

    const float xr = a.xs[o0], xi = CPLX ? a.xs[o1] : 0.0f;
    const float gs = (mode == M_EULER || mode == M_RK1) ? a.gam[og] : a.gstg[og];
    float kr, ki, kg;
    gd_rhs(xr, xi, gs, yr, yi, beta_s[u], h, a.eps, a.rho_th, kr, ki, kg);
    if (CPLX && a.q) resonant_drive(xr, xi, a.q, a.hq, kr, ki);
    float nr, ni, ng;
    if (mode == M_EULER) {
      nr = axpy(a.dt, kr, xr);
      ni = axpy(a.dt, ki, xi);
      ng = axpy(a.dt, kg, gs);
    } else {
      const float pr = (mode == M_RK1) ? xr : a.psi_n[o0];
      const float pi = (mode == M_RK1) ? xi : (CPLX ? a.psi_n[o1] : 0.0f);
      const float gn = (mode == M_RK1) ? gs : a.gam[og];
      if (mode == M_RK4) {
        const float d6 = __fdiv_rn(a.dt, 6.0f);
        nr = axpy(d6, __fadd_rn(a.acc[o0], kr), pr);
        ni = CPLX ? axpy(d6, __fadd_rn(a.acc[o1], ki), pi) : 0.0f;
        ng = axpy(d6, __fadd_rn(a.gacc[og], kg), gn);
      } else {
        const float cf = (mode == M_RK3) ? a.dt : __fmul_rn(0.5f, a.dt);
        if (mode == M_RK1) {
          a.acc[o0] = kr;
          if (CPLX) a.acc[o1] = ki;
          a.gacc[og] = kg;
        } else {
          a.acc[o0] = axpy(2.0f, kr, a.acc[o0]);
          if (CPLX) a.acc[o1] = axpy(2.0f, ki, a.acc[o1]);
          a.gacc[og] = axpy(2.0f, kg, a.gacc[og]);
        }
        const float sr = axpy(cf, kr, pr), si = axpy(cf, ki, pi);
        a.xs_next[o0] = sr;
        if (CPLX) a.xs_next[o1] = si;
        if (TSTORE) {
          t4[u * W] = sr;
          if (CPLX) t4[u * W + 1] = si;
        }
        a.gstg[og] = axpy(cf, kg, gn);
        if (a.op_out) {
          a.op_out[o0] = __float2bfloat16_rn(sr);
          if (CPLX) a.op_out[o1] = __float2bfloat16_rn(si);
        }
        continue;
      }
    }
    // completed step: noise, then write psi^{n+1}, gamma^{n+1}
    nr = axpy(dsc[u], z[(col) & 3], nr);
    if (CPLX) ni = axpy(dsc[u], z[(col + 1) & 3], ni);
    a.psi_out[o0] = nr;
    if (CPLX) a.psi_out[o1] = ni;
    a.gam[og] = ng;
    if (TSTORE) {
      t4[u * W] = nr;
      if (CPLX) t4[u * W + 1] = ni;
    }
    if (a.op_out) {
      a.op_out[o0] = __float2bfloat16_rn(nr);
      if (CPLX) a.op_out[o1] = __float2bfloat16_rn(ni);
    }
    const float rn = density(nr, ni);
    red[u] = rn;
    bad |= !(rn < 1e30f);
  }
  if (TSTORE && a.opT_out && mode != M_RAW && mode != M_ENERGY)
    *reinterpret_cast<float4*>(a.opT_out + size_t(i) * a.Cp + c0) = make_float4(t4[0], t4[1], t4[2], t4[3]);
}

}  // namespace gda
