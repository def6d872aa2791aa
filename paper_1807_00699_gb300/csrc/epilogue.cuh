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

// Stage coupling scale beta_s of restart r for the launch's mode.  beta
// obeys d beta/dt = eps_hat (1 - beta) (Eq. 6 with Delta = 1, K = beta J).
__device__ __forceinline__ float stage_beta(const StepArgs& a, float b) {
  const float eh = a.eps_hat, dt = a.dt;
  switch (a.mode) {
    case M_RK2: return b + 0.5f * dt * (eh * (1.0f - b));
    case M_RK3: {
      const float b2 = b + 0.5f * dt * (eh * (1.0f - b));
      return b + 0.5f * dt * (eh * (1.0f - b2));
    }
    case M_RK4: {
      const float b2 = b + 0.5f * dt * (eh * (1.0f - b));
      const float b3 = b + 0.5f * dt * (eh * (1.0f - b2));
      return b + dt * (eh * (1.0f - b3));
    }
    case M_ENERGY: return 1.0f;
    default: return b;
  }
}

// beta^{n+1} from beta^n for a completed Euler or RK4 step.
__device__ __forceinline__ float next_beta(const StepArgs& a, float b) {
  const float eh = a.eps_hat, dt = a.dt;
  if (a.mode == M_EULER) return b + dt * (eh * (1.0f - b));
  const float k1 = eh * (1.0f - b);
  const float k2 = eh * (1.0f - (b + 0.5f * dt * k1));
  const float k3 = eh * (1.0f - (b + 0.5f * dt * k2));
  const float k4 = eh * (1.0f - (b + dt * k3));
  return b + dt / 6.0f * (k1 + 2.0f * k2 + 2.0f * k3 + k4);
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
    for (int t = 0; t < a.mt_count; ++t) s += a.rho_in[t * a.Rp + r];
    D *= fmaxf(0.0f, 1.0f - (s / float(a.N)) / a.rho_th);
  }
  return sqrtf(a.dt) * D * (a.cplx ? 0.70710678118654752f : 1.0f);
}

// One quad.  beta_s[u], dsc[u]: per-restart stage scale and noise amplitude
// of the quad's restarts (4 Ising, 2 XY).  red[u] receives |psi^{n+1}|^2
// (completed steps) or the restart's Eq. (1) contribution of spin i (energy
// mode); 0 for padded restarts.  bad is set for a non-finite amplitude.
template <bool CPLX>
__device__ __forceinline__ void epi_quad(const StepArgs& a, int i, int c0, const float y[4],
                                         const float* beta_s, const float* dsc, float red[4],
                                         int& bad) {
  constexpr int U = CPLX ? 2 : 4;
  constexpr int W = CPLX ? 2 : 1;
  const int Np = a.Np;
  const int mode = a.mode;
  const int r0 = CPLX ? (c0 >> 1) : c0;
  float z[4] = {0.f, 0.f, 0.f, 0.f};
  if (step_completes(mode)) {
    bool any = false;
#pragma unroll
    for (int u = 0; u < U; ++u) any |= dsc[u] != 0.0f;
    if (any) philox_normal4(uint32_t(i), uint32_t(c0 >> 2), a.step, 0u, a.seed, z);
  }
  const float h = a.h1[i];
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
      if (CPLX) {
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
    const float rho = density(xr, xi);
    const float kr = xr * (gs - rho) + beta_s[u] * yr + h;
    const float ki = xi * (gs - rho) + beta_s[u] * yi;
    const float kg = a.eps * (a.rho_th - rho);
    float nr, ni, ng;
    if (mode == M_EULER) {
      nr = xr + a.dt * kr;
      ni = xi + a.dt * ki;
      ng = gs + a.dt * kg;
    } else {
      const float pr = (mode == M_RK1) ? xr : a.psi_n[o0];
      const float pi = (mode == M_RK1) ? xi : (CPLX ? a.psi_n[o1] : 0.0f);
      const float gn = (mode == M_RK1) ? gs : a.gam[og];
      if (mode == M_RK4) {
        nr = pr + a.dt / 6.0f * (a.acc[o0] + kr);
        ni = CPLX ? pi + a.dt / 6.0f * (a.acc[o1] + ki) : 0.0f;
        ng = gn + a.dt / 6.0f * (a.gacc[og] + kg);
      } else {
        const float cf = (mode == M_RK3) ? a.dt : 0.5f * a.dt;
        if (mode == M_RK1) {
          a.acc[o0] = kr;
          if (CPLX) a.acc[o1] = ki;
          a.gacc[og] = kg;
        } else {
          a.acc[o0] += 2.0f * kr;
          if (CPLX) a.acc[o1] += 2.0f * ki;
          a.gacc[og] += 2.0f * kg;
        }
        const float sr = pr + cf * kr, si = pi + cf * ki;
        a.xs_next[o0] = sr;
        if (CPLX) a.xs_next[o1] = si;
        a.gstg[og] = gn + cf * kg;
        if (a.op_out) {
          a.op_out[o0] = __float2bfloat16_rn(sr);
          if (CPLX) a.op_out[o1] = __float2bfloat16_rn(si);
        }
        continue;
      }
    }
    // completed step: noise, then write psi^{n+1}, gamma^{n+1}
    nr += dsc[u] * z[(col) & 3];
    if (CPLX) ni += dsc[u] * z[(col + 1) & 3];
    a.psi_out[o0] = nr;
    if (CPLX) a.psi_out[o1] = ni;
    a.gam[og] = ng;
    if (a.op_out) {
      a.op_out[o0] = __float2bfloat16_rn(nr);
      if (CPLX) a.op_out[o1] = __float2bfloat16_rn(ni);
    }
    const float rn = density(nr, ni);
    red[u] = rn;
    bad |= !(rn < 1e30f);
  }
}

}  // namespace gda
