// Spin projection, Eq. (1) energies and the argmin over restarts.
//
//  * tracking: the projected spins are written as the operand of one more
//    coupling product (FP32 or BF16, the run's path) whose epilogue forms the
//    per-restart partial energies; k_track_reduce sums them, adds -sum_i J_ii
//    and records the best restart;
//  * final: an FP64 (or, for integer-J Ising runs with g = 0, an int32 row /
//    int64 total) tiled product of the full J with the projected spins.
#include <cfloat>

#include "gda_internal.h"
#include "kernels.h"

namespace gda {


// ---------------------------------------------------------------- init
__global__ void k_init_state(float* psi, float* gam, float* beta, int N, int Np, int R, int cplx, int mode,
                             float amp, float gamma0, float beta0, unsigned long long seed, const float* base) {
  const size_t total = size_t(R) * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / N), i = int(idx % N);
    float re = 0.0f, im = 0.0f;
    if (mode == 1 || mode == 3) {
      const U4 o = philox4x32_10(U4{uint32_t(i), uint32_t(r), 0u, 1u}, uint32_t(seed), uint32_t(seed >> 32));
      re = amp * (2.0f * philox_u01(o.x) - 1.0f);
      im = amp * (2.0f * philox_u01(o.y) - 1.0f);
      if (mode == 3) {  // per-spin base amplitude plus the seeded perturbation
        re = __fadd_rn(base[2 * i], re);
        im = __fadd_rn(base[2 * i + 1], im);
      }
    }
    if (cplx) {
      psi[size_t(2 * r) * Np + i] = re;
      psi[size_t(2 * r + 1) * Np + i] = im;
    } else {
      psi[size_t(r) * Np + i] = re;
    }
    gam[size_t(r) * Np + i] = gamma0;
    if (i == 0) beta[r] = beta0;
  }
}

__global__ void k_fill_h1(const double* g, float* h1, int N, float sq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) h1[i] = float(-g[i]) * sq;
}

__global__ void k_to_bf16(const float* x, __nv_bfloat16* y, size_t n) {
  for (size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x; k < n; k += size_t(gridDim.x) * blockDim.x)
    y[k] = __float2bfloat16_rn(x[k]);
}

// Partial sums of |psi|^2 over the spin tiles of one path, in the same order
// as that path's step epilogue, so a resumed run draws the same noise scale.
// TC order: rows of a 128-row tile reduced per 32-row quarter by an xor tree,
// quarters added in order.  SIMT order: rows tx + 16q summed over q, then an
// xor tree over the 16 tx.
__global__ void k_rho_partials_tc(const float* psi, int N, int Np, int R, int Rp, int cplx, float* out) {
  const int t = blockIdx.x, r = blockIdx.y;  // blockDim = 128
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ float part[4];
  const int i = t * 128 + 32 * q + lane;
  float x = 0.0f;
  if (i < N) {
    const float re = psi[size_t(cplx ? 2 * r : r) * Np + i];
    const float im = cplx ? psi[size_t(2 * r + 1) * Np + i] : 0.0f;
    x = density(re, im);
  }
  for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  if (lane == 0) part[q] = x;
  __syncthreads();
  if (threadIdx.x == 0) out[size_t(t) * Rp + r] = part[0] + part[1] + part[2] + part[3];
}

__global__ void k_rho_partials_simt(const float* psi, int N, int Np, int R, int Rp, int cplx, float* out) {
  const int t = blockIdx.x, r = blockIdx.y;  // blockDim = 16
  const int tx = threadIdx.x;
  float s = 0.0f;
  for (int q = 0; q < 4; ++q) {
    const int i = t * 64 + tx + 16 * q;
    if (i >= N) continue;
    const float re = psi[size_t(cplx ? 2 * r : r) * Np + i];
    const float im = cplx ? psi[size_t(2 * r + 1) * Np + i] : 0.0f;
    s += density(re, im);
  }
  for (int off = 8; off; off >>= 1) s += __shfl_xor_sync(0x0000ffffu, s, off);
  if (tx == 0) out[size_t(t) * Rp + r] = s;
}

// ---------------------------------------------------------------- projection
template <typename T>
__device__ __forceinline__ T conv(float v);
template <>
__device__ __forceinline__ float conv<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 conv<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Projected spins s of psi as a coupling-product operand [Cp][Np].
template <typename T>
__global__ void k_project_op(const float* psi, T* S, int N, int Np, int R, int cplx) {
  const size_t total = size_t(R) * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / N), i = int(idx % N);
    if (cplx >= 2) {
      double sr, si;
      potts_project(psi[size_t(2 * r) * Np + i], psi[size_t(2 * r + 1) * Np + i], cplx, sr, si);
      S[size_t(2 * r) * Np + i] = conv<T>(float(sr));
      S[size_t(2 * r + 1) * Np + i] = conv<T>(float(si));
    } else if (cplx) {
      const float re = psi[size_t(2 * r) * Np + i], im = psi[size_t(2 * r + 1) * Np + i];
      const float m = sqrtf(re * re + im * im);
      S[size_t(2 * r) * Np + i] = conv<T>(m > 0.0f ? re / m : 1.0f);
      S[size_t(2 * r + 1) * Np + i] = conv<T>(m > 0.0f ? im / m : 0.0f);
    } else {
      S[size_t(r) * Np + i] = conv<T>(psi[size_t(r) * Np + i] >= 0.0f ? 1.0f : -1.0f);
    }
  }
}

// FP64 projection (XY: s = psi / |psi| evaluated in double).
__global__ void k_project64(const float* psi, double* S, int N, int Np, int R, int cplx) {
  const size_t total = size_t(R) * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / N), i = int(idx % N);
    if (cplx >= 2) {
      potts_project(psi[size_t(2 * r) * Np + i], psi[size_t(2 * r + 1) * Np + i], cplx, S[size_t(2 * r) * Np + i],
                    S[size_t(2 * r + 1) * Np + i]);
    } else if (cplx) {
      const double re = psi[size_t(2 * r) * Np + i], im = psi[size_t(2 * r + 1) * Np + i];
      const double m = sqrt(re * re + im * im);
      S[size_t(2 * r) * Np + i] = m > 0.0 ? re / m : 1.0;
      S[size_t(2 * r + 1) * Np + i] = m > 0.0 ? im / m : 0.0;
    } else {
      S[size_t(r) * Np + i] = psi[size_t(r) * Np + i] >= 0.0f ? 1.0 : -1.0;
    }
  }
}

__global__ void k_project_int(const float* psi, int* S, int N, int Np, int R) {
  const size_t total = size_t(R) * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / N), i = int(idx % N);
    S[size_t(r) * Np + i] = psi[size_t(r) * Np + i] >= 0.0f ? 1 : -1;
  }
}

// ---------------------------------------------------------------- tracking
// One block.  E_r = sum_t e_part[t][r] - sum_i J_ii; records (step, E, r) of
// the lowest E (ties: lowest r) at trace slot *count when it fits.
__global__ void k_track_reduce(const float* e_part, int mt, int R, int Rp, double diag, long long step,
                               long long* t_step, double* t_E, int* t_r, int cap, int* count, double* lastE,
                               int* lastR) {
  __shared__ double sE[32];
  __shared__ int sR[32];
  double best = DBL_MAX;
  int br = 0x7fffffff;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    float s = 0.0f;
    for (int t = 0; t < mt; ++t) s += e_part[size_t(t) * Rp + r];
    const double E = double(s) + diag;
    if (E < best || (E == best && r < br)) { best = E; br = r; }
  }
  for (int off = 16; off; off >>= 1) {
    const double oE = __shfl_xor_sync(0xffffffffu, best, off);
    const int oR = __shfl_xor_sync(0xffffffffu, br, off);
    if (oE < best || (oE == best && oR < br)) { best = oE; br = oR; }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sE[w] = best; sR[w] = br; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < int(blockDim.x >> 5); ++k)
      if (sE[k] < best || (sE[k] == best && sR[k] < br)) { best = sE[k]; br = sR[k]; }
    const int c = *count;
    if (c < cap) { t_step[c] = step; t_E[c] = best; t_r[c] = br; }
    *count = c + 1;
    *lastE = best;
    *lastR = br;
  }
}

// ---------------------------------------------------------------- final energy
// Tiled product T = J S (64 x 64 tiles, 4 x 4 per thread) with an epilogue
// that forms each restart's Eq. (1) partial over the tile's rows:
//   Ising: -s_i T_i + g_i s_i;   XY: -(Re s_i Re T_i + Im s_i Im T_i) + g_i Re s_i.
// J here keeps its diagonal (Eq. 1 sums all ordered pairs).
template <typename T, typename P, bool CPLX>
__global__ void __launch_bounds__(256) k_energy_tile(const T* __restrict__ J, const T* __restrict__ S,
                                                     const double* __restrict__ g, int N, int Np, int R, int Rp,
                                                     P* part) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (int k0 = 0; k0 < Np; k0 += BK) {
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      As[lk + t][lr] = J[size_t(m0 + lr) * Np + k0 + lk + t];
      Bs[lk + t][lr] = S[size_t(n0 + lr) * Np + k0 + lk + t];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T b[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[k][4 * ty + v];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const T av = As[k][tx + 16 * a];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[a][v] += av * b[v];
      }
    }
  }
  constexpr int U = CPLX ? 2 : 4;
  P rs[4] = {P(0), P(0), P(0), P(0)};
  const int c0 = n0 + 4 * ty;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = m0 + tx + 16 * a;
    if (i >= N) continue;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (CPLX) {
        const int c = c0 + 2 * u;
        const double sr = double(S[size_t(c) * Np + i]), si = double(S[size_t(c + 1) * Np + i]);
        rs[u] += P(-(sr * double(acc[a][2 * u]) + si * double(acc[a][2 * u + 1])) + g[i] * sr);
      } else {
        const int c = c0 + u;
        const T s = S[size_t(c) * Np + i];
        rs[u] += -P(s) * P(acc[a][u]);
        if (g) rs[u] += P(g[i] * double(s));
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int off = 8; off; off >>= 1) rs[u] += __shfl_xor_sync(0xffffffffu, rs[u], off);
  if (tx == 0) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = (CPLX ? c0 / 2 : c0) + u;
      if (r < R) part[size_t(blockIdx.y) * Rp + r] = rs[u];
    }
  }
}

template <typename P>
__global__ void k_energy_finish(const P* part, int mt, int R, int Rp, double* E) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    P s = P(0);
    for (int t = 0; t < mt; ++t) s += part[size_t(t) * Rp + r];
    E[r] = double(s);
  }
}

// Lowest energy over restarts (ties: lowest index) -> best[0] = E, best_r.
__global__ void k_argmin(const double* E, int R, double* bestE, int* bestR) {
  __shared__ double sE[32];
  __shared__ int sR[32];
  double best = DBL_MAX;
  int br = 0x7fffffff;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double e = E[r];
    if (e < best || (e == best && r < br)) { best = e; br = r; }
  }
  for (int off = 16; off; off >>= 1) {
    const double oE = __shfl_xor_sync(0xffffffffu, best, off);
    const int oR = __shfl_xor_sync(0xffffffffu, br, off);
    if (oE < best || (oE == best && oR < br)) { best = oE; br = oR; }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sE[w] = best; sR[w] = br; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < int(blockDim.x >> 5); ++k)
      if (sE[k] < best || (sE[k] == best && sR[k] < br)) { best = sE[k]; br = sR[k]; }
    *bestE = best;
    *bestR = br;
  }
}

// Configuration of the best restart: int8 spins (Ising) or theta (XY).
__global__ void k_best_cfg(const float* psi, const int* bestR, int N, int Np, int cplx, signed char* s8, double* th) {
  const int r = *bestR;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (cplx >= 2) {
      double sr, si;
      potts_project(psi[size_t(2 * r) * Np + i], psi[size_t(2 * r + 1) * Np + i], cplx, sr, si);
      th[i] = atan2(si, sr);
    } else if (cplx) {
      const double re = psi[size_t(2 * r) * Np + i], im = psi[size_t(2 * r + 1) * Np + i];
      th[i] = (re == 0.0 && im == 0.0) ? 0.0 : atan2(im, re);
    } else {
      s8[i] = psi[size_t(r) * Np + i] >= 0.0f ? 1 : -1;
    }
  }
}

// ---------------------------------------------------------------- launchers
static int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return int(b > 4096 ? 4096 : (b ? b : 1));
}

cudaError_t launch_init_state(float* psi, float* gam, float* beta, int N, int Np, int R, int cplx, int mode,
                              float amp, float gamma0, float beta0, unsigned long long seed, const float* base,
                              cudaStream_t s) {
  k_init_state<<<grid_for(size_t(R) * N), 256, 0, s>>>(psi, gam, beta, N, Np, R, cplx, mode, amp, gamma0, beta0,
                                                        seed, base);
  return cudaGetLastError();
}

cudaError_t launch_fill_h1(const double* g, float* h1, int N, float sq, cudaStream_t s) {
  k_fill_h1<<<grid_for(N), 256, 0, s>>>(g, h1, N, sq);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* x, __nv_bfloat16* y, size_t n, cudaStream_t s) {
  k_to_bf16<<<grid_for(n), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_rho_partials(bool tc, const float* psi, int N, int Np, int R, int Rp, int cplx, float* out,
                                cudaStream_t s) {
  if (tc) {
    k_rho_partials_tc<<<dim3((N + 127) / 128, R), 128, 0, s>>>(psi, N, Np, R, Rp, cplx, out);
  } else {
    k_rho_partials_simt<<<dim3((N + 63) / 64, R), 16, 0, s>>>(psi, N, Np, R, Rp, cplx, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_project_f32(const float* psi, float* S, int N, int Np, int R, int cplx, cudaStream_t s) {
  k_project_op<float><<<grid_for(size_t(R) * N), 256, 0, s>>>(psi, S, N, Np, R, cplx);
  return cudaGetLastError();
}

cudaError_t launch_project_bf16(const float* psi, __nv_bfloat16* S, int N, int Np, int R, int cplx, cudaStream_t s) {
  k_project_op<__nv_bfloat16><<<grid_for(size_t(R) * N), 256, 0, s>>>(psi, S, N, Np, R, cplx);
  return cudaGetLastError();
}

cudaError_t launch_track_reduce(const float* e_part, int mt, int R, int Rp, double diag, long long step,
                                long long* t_step, double* t_E, int* t_r, int cap, int* count, double* lastE,
                                int* lastR, cudaStream_t s) {
  k_track_reduce<<<1, 1024, 0, s>>>(e_part, mt, R, Rp, diag, step, t_step, t_E, t_r, cap, count, lastE, lastR);
  return cudaGetLastError();
}

namespace {

// Running best of the energy trace: when this evaluation's lowest tracking
// energy (*lastE, restart *lastR) is below the best so far, the restart's
// amplitudes (W columns of Np) are copied to snap and (E, r, step) recorded.
// Also keeps that restart's amplitudes in hist[entry] for the trace entry just
// recorded (entry = *count - 1) when entry < hist_cap.
__global__ void k_snapshot(const float* psi, int Np, int W, const double* lastE, const int* lastR, long long step,
                           double* snapE, int* snapR, long long* snapStep, float* snap, float* hist, int hist_cap,
                           const int* count) {
  __shared__ int take;
  if (threadIdx.x == 0) {
    take = *lastE < *snapE;
    if (take) {
      *snapE = *lastE;
      *snapR = *lastR;
      *snapStep = step;
    }
  }
  __syncthreads();
  const float* src = psi + size_t(*lastR) * W * Np;
  const int entry = *count - 1;
  if (hist && entry >= 0 && entry < hist_cap) {
    float* dst = hist + size_t(entry) * W * Np;
    for (int k = threadIdx.x; k < W * Np; k += blockDim.x) dst[k] = src[k];
  }
  if (!take) return;
  for (int k = threadIdx.x; k < W * Np; k += blockDim.x) snap[k] = src[k];
}

__global__ void k_snapshot_reset(double* snapE, int* snapR, long long* snapStep) {
  *snapE = DBL_MAX;
  *snapR = -1;
  *snapStep = -1;
}

}  // namespace

cudaError_t launch_snapshot(const float* psi, int Np, int W, const double* lastE, const int* lastR, long long step,
                            double* snapE, int* snapR, long long* snapStep, float* snap, float* hist, int hist_cap,
                            const int* count, cudaStream_t s) {
  k_snapshot<<<1, 1024, 0, s>>>(psi, Np, W, lastE, lastR, step, snapE, snapR, snapStep, snap, hist, hist_cap, count);
  return cudaGetLastError();
}

cudaError_t launch_snapshot_reset(double* snapE, int* snapR, long long* snapStep, cudaStream_t s) {
  k_snapshot_reset<<<1, 1, 0, s>>>(snapE, snapR, snapStep);
  return cudaGetLastError();
}

cudaError_t launch_energy64(const float* psi, const double* J64, const double* g, double* S64, double* part,
                            double* E, int N, int Np, int R, int Rp, int C, int cplx, cudaStream_t s) {
  k_project64<<<grid_for(size_t(R) * N), 256, 0, s>>>(psi, S64, N, Np, R, cplx);
  const int mt = (N + 63) / 64;
  dim3 grid((C + 63) / 64, mt);
  if (cplx)
    k_energy_tile<double, double, true><<<grid, 256, 0, s>>>(J64, S64, g, N, Np, R, Rp, part);
  else
    k_energy_tile<double, double, false><<<grid, 256, 0, s>>>(J64, S64, g, N, Np, R, Rp, part);
  k_energy_finish<double><<<grid_for(R), 256, 0, s>>>(part, mt, R, Rp, E);
  return cudaGetLastError();
}

cudaError_t launch_energy_int(const float* psi, const int* Jint, int* Sint, long long* part, double* E, int N,
                              int Np, int R, int Rp, int C, cudaStream_t s) {
  k_project_int<<<grid_for(size_t(R) * N), 256, 0, s>>>(psi, Sint, N, Np, R);
  const int mt = (N + 63) / 64;
  dim3 grid((C + 63) / 64, mt);
  k_energy_tile<int, long long, false><<<grid, 256, 0, s>>>(Jint, Sint, nullptr, N, Np, R, Rp, part);
  k_energy_finish<long long><<<grid_for(R), 256, 0, s>>>(part, mt, R, Rp, E);
  return cudaGetLastError();
}

cudaError_t launch_argmin(const double* E, int R, double* bestE, int* bestR, cudaStream_t s) {
  k_argmin<<<1, 1024, 0, s>>>(E, R, bestE, bestR);
  return cudaGetLastError();
}

cudaError_t launch_best_cfg(const float* psi, const int* bestR, int N, int Np, int cplx, signed char* s8, double* th,
                            cudaStream_t s) {
  k_best_cfg<<<grid_for(N), 256, 0, s>>>(psi, bestR, N, Np, cplx, s8, th);
  return cudaGetLastError();
}

}  // namespace gda

namespace gda {

// Host layout <-> device layout of the state.  Host psi: restart-major,
// (re, im) interleaved for XY; gamma: [R][N]; beta: [R].
__global__ void k_pack_state(const float* psi, const float* gam, const float* beta, int N, int Np, int R, int cplx,
                             float* hpsi, float* hgam, float* hbeta) {
  const size_t total = size_t(R) * N;
  const int W = cplx ? 2 : 1;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / N), i = int(idx % N);
    if (hpsi)
      for (int p = 0; p < W; ++p) hpsi[idx * W + p] = psi[size_t(W * r + p) * Np + i];
    if (hgam) hgam[idx] = gam[size_t(r) * Np + i];
    if (hbeta && i == 0) hbeta[r] = beta[r];
  }
}

__global__ void k_unpack_state(float* psi, float* gam, float* beta, int N, int Np, int R, int cplx, const float* hpsi,
                               const float* hgam, const float* hbeta) {
  const size_t total = size_t(R) * N;
  const int W = cplx ? 2 : 1;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / N), i = int(idx % N);
    for (int p = 0; p < W; ++p) psi[size_t(W * r + p) * Np + i] = hpsi[idx * W + p];
    gam[size_t(r) * Np + i] = hgam ? hgam[idx] : 0.0f;
    if (i == 0) beta[r] = hbeta ? hbeta[r] : 1.0f;
  }
}

// Instance checks and operand preparation.  J64 is [Np][Np] (zero padded,
// diagonal kept).  flags: bit0 non-finite, bit1 asymmetric, bit2 non-integer;
// maxabs: |J| maximum as the bits of a non-negative double.
__global__ void k_check_J(const double* J64, int N, int Np, int* flags, unsigned long long* maxabs) {
  int f = 0;
  double m = 0.0;
  const size_t total = size_t(N) * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int i = int(idx / N), j = int(idx % N);
    const double v = J64[size_t(i) * Np + j];
    if (!isfinite(v)) { f |= 1; continue; }
    if (v != J64[size_t(j) * Np + i]) f |= 2;
    if (v != rint(v)) f |= 4;
    m = fmax(m, fabs(v));
  }
  if (f) atomicOr(flags, f);
  atomicMax(maxabs, __double_as_longlong(m));
}

__global__ void k_check_g(const double* g, int N, int* flags) {
  int f = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (!isfinite(g[i])) f |= 8;
    if (g[i] != 0.0) f |= 16;
  }
  if (f) atomicOr(flags, f);
}

// diag = -sum_i J_ii in a fixed order (one thread).
__global__ void k_diag(const double* J64, int N, int Np, double* diag) {
  double s = 0.0;
  for (int i = 0; i < N; ++i) s += J64[size_t(i) * Np + i];
  *diag = -s;
}

// Coupling operands: J0 (diagonal removed) in FP32 and BF16, and the integer
// copy of J (diagonal kept) for the exact Ising energy.
__global__ void k_prepare_J(const double* J64, int Np, float* J32, __nv_bfloat16* J16, int* Jint) {
  const size_t total = size_t(Np) * Np;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int i = int(idx / Np), j = int(idx % Np);
    const double v = J64[idx];
    const float f = (i == j) ? 0.0f : float(v);
    J32[idx] = f;
    if (J16) J16[idx] = __float2bfloat16_rn(f);
    if (Jint) Jint[idx] = int(v);
  }
}

cudaError_t launch_pack_state(const float* psi, const float* gam, const float* beta, int N, int Np, int R, int cplx,
                              float* hpsi, float* hgam, float* hbeta, cudaStream_t s) {
  k_pack_state<<<grid_for(size_t(R) * N), 256, 0, s>>>(psi, gam, beta, N, Np, R, cplx, hpsi, hgam, hbeta);
  return cudaGetLastError();
}

cudaError_t launch_unpack_state(float* psi, float* gam, float* beta, int N, int Np, int R, int cplx, const float* hpsi,
                                const float* hgam, const float* hbeta, cudaStream_t s) {
  k_unpack_state<<<grid_for(size_t(R) * N), 256, 0, s>>>(psi, gam, beta, N, Np, R, cplx, hpsi, hgam, hbeta);
  return cudaGetLastError();
}

cudaError_t launch_check_instance(const double* J64, const double* g, int N, int Np, int* flags,
                                  unsigned long long* maxabs, double* diag, cudaStream_t s) {
  k_check_J<<<grid_for(size_t(N) * N), 256, 0, s>>>(J64, N, Np, flags, maxabs);
  k_check_g<<<grid_for(N), 256, 0, s>>>(g, N, flags);
  k_diag<<<1, 1, 0, s>>>(J64, N, Np, diag);
  return cudaGetLastError();
}

cudaError_t launch_prepare_J(const double* J64, int Np, float* J32, __nv_bfloat16* J16, int* Jint, cudaStream_t s) {
  k_prepare_J<<<grid_for(size_t(Np) * Np), 256, 0, s>>>(J64, Np, J32, J16, Jint);
  return cudaGetLastError();
}

}  // namespace gda

// ---------------------------------------------------------------- ranking
// Candidate ranking for the argmin of the FP64 energies (gda_best): every
// restart's Eq. (1) energy is first bounded in FP32 with compensated sums,
// then only the restarts within twice the error bound of the lowest such
// value are evaluated in FP64.  The FP64 argmin over those candidates is the
// FP64 argmin over all restarts (ties: lowest index, candidates ascending).
namespace gda {
namespace {

// FP32 projection computed in double, rounded once (|s32 - s| <= 2^-24 |s|).
__global__ void k_project_rank(const float* psi, float* S, int N, int Np, int R, int cplx) {
  const size_t total = size_t(R) * N;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total; idx += size_t(gridDim.x) * blockDim.x) {
    const int r = int(idx / N), i = int(idx % N);
    if (cplx >= 2) {
      double sr, si;
      potts_project(psi[size_t(2 * r) * Np + i], psi[size_t(2 * r + 1) * Np + i], cplx, sr, si);
      S[size_t(2 * r) * Np + i] = float(sr);
      S[size_t(2 * r + 1) * Np + i] = float(si);
    } else if (cplx) {
      const double re = psi[size_t(2 * r) * Np + i], im = psi[size_t(2 * r + 1) * Np + i];
      const double m = sqrt(re * re + im * im);
      S[size_t(2 * r) * Np + i] = float(m > 0.0 ? re / m : 1.0);
      S[size_t(2 * r + 1) * Np + i] = float(m > 0.0 ? im / m : 0.0);
    } else {
      S[size_t(r) * Np + i] = psi[size_t(r) * Np + i] >= 0.0f ? 1.0f : -1.0f;
    }
  }
}

// T = J0 S over 64 x 64 tiles (4 x 4 per thread) in FP32: each 16-deep K
// block is summed with FMAs, then added into a (hi, lo) pair with an exact
// two-sum, so one element's error is at most ~17 u sum_j |J0_ij S_j|.  The
// Eq. (1) partials per tile of 64 rows are formed and summed in double.
template <bool CPLX>
__global__ void __launch_bounds__(256) k_energy32c(const float* __restrict__ J, const float* __restrict__ S,
                                                   const double* __restrict__ g, int N, int Np, int R, int Rp,
                                                   double* part) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.0f;
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (int k0 = 0; k0 < Np; k0 += BK) {
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      As[lk + t][lr] = J[size_t(m0 + lr) * Np + k0 + lk + t];
      Bs[lk + t][lr] = S[size_t(n0 + lr) * Np + k0 + lk + t];
    }
    __syncthreads();
    float blk[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) blk[a][b] = 0.0f;
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float b[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[k][4 * ty + v];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float av = As[k][tx + 16 * a];
#pragma unroll
        for (int v = 0; v < 4; ++v) blk[a][v] = __fmaf_rn(av, b[v], blk[a][v]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int v = 0; v < 4; ++v) {  // two-sum (Knuth): hi + blk = s + e exactly
        const float s = __fadd_rn(hi[a][v], blk[a][v]);
        const float bp = __fsub_rn(s, hi[a][v]);
        const float e = __fadd_rn(__fsub_rn(hi[a][v], __fsub_rn(s, bp)), __fsub_rn(blk[a][v], bp));
        hi[a][v] = s;
        lo[a][v] = __fadd_rn(lo[a][v], e);
      }
  }
  constexpr int U = CPLX ? 2 : 4;
  double rs[4] = {0.0, 0.0, 0.0, 0.0};
  const int c0 = n0 + 4 * ty;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = m0 + tx + 16 * a;
    if (i >= N) continue;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (CPLX) {
        const int c = c0 + 2 * u;
        const double sr = S[size_t(c) * Np + i], si = S[size_t(c + 1) * Np + i];
        const double tr = double(hi[a][2 * u]) + double(lo[a][2 * u]);
        const double ti = double(hi[a][2 * u + 1]) + double(lo[a][2 * u + 1]);
        rs[u] += -(sr * tr + si * ti) + g[i] * sr;
      } else {
        const int c = c0 + u;
        const double sv = S[size_t(c) * Np + i];
        rs[u] += -sv * (double(hi[a][u]) + double(lo[a][u])) + g[i] * sv;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int off = 8; off; off >>= 1) rs[u] += __shfl_xor_sync(0xffffffffu, rs[u], off);
  if (tx == 0) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = (CPLX ? c0 / 2 : c0) + u;
      if (r < R) part[size_t(blockIdx.y) * Rp + r] = rs[u];
    }
  }
}

// sum_ij |J0_ij| + sum_i |g_i| (J0: the FP64 J without its diagonal).
__global__ void k_abs_sum(const double* J64, const double* g, int N, int Np, double* out) {
  double s = 0.0;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < size_t(N) * N;
       idx += size_t(gridDim.x) * blockDim.x) {
    const int i = int(idx / N), j = int(idx % N);
    if (i != j) s += fabs(J64[size_t(i) * Np + j]);
    if (j == 0 && g) s += fabs(g[i]);
  }
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// One block: E32[r] = sum_t part[t][r] + diag; the restarts with E32 <= min + margin,
// ascending, to idx[0 .. *count).
__global__ void k_rank(const double* part, int mt, int R, int Rp, double diag, double margin, double* E32, int* idx,
                       int* count) {
  __shared__ double smin[32];
  __shared__ int spre[1024 / 32 + 1];
  __shared__ int sbase;
  double mn = DBL_MAX;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < mt; ++t) s += part[size_t(t) * Rp + r];
    s += diag;
    E32[r] = s;
    mn = fmin(mn, s);
  }
  for (int off = 16; off; off >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, off));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) smin[w] = mn;
  if (threadIdx.x == 0) sbase = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < nw; ++k) mn = fmin(mn, smin[k]);
    smin[0] = mn;
  }
  __syncthreads();
  const double lim = smin[0] + margin;
  for (int r0 = 0; r0 < R; r0 += blockDim.x) {
    const int r = r0 + threadIdx.x;
    const bool in = r < R && E32[r] <= lim;
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (lane == 0) spre[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = sbase;
      for (int k = 0; k < nw; ++k) {
        const int c = spre[k];
        spre[k] = acc;
        acc += c;
      }
      spre[nw] = acc;
    }
    __syncthreads();
    if (in) idx[spre[w] + __popc(m & ((1u << lane) - 1u))] = r;
    __syncthreads();
    if (threadIdx.x == 0) sbase = spre[nw];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = sbase;
}

// Candidate columns (restart idx[k] -> column block k) of psi into a compact buffer.
__global__ void k_gather_cols(const float* psi, int Np, const int* idx, int count, int cplx, float* out) {
  const int W = cplx ? 2 : 1;
  const size_t total = size_t(count) * W * Np;
  for (size_t q = blockIdx.x * size_t(blockDim.x) + threadIdx.x; q < total; q += size_t(gridDim.x) * blockDim.x) {
    const int col = int(q / Np), i = int(q % Np);
    const int k = col / W, w = col % W;
    out[q] = psi[size_t(idx[k] * W + w) * Np + i];
  }
}

__global__ void k_map_best(const int* idx, int* bestR) { *bestR = idx[*bestR]; }

}  // namespace

cudaError_t launch_abs_sum(const double* J64, const double* g, int N, int Np, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_abs_sum<<<grid_for(size_t(N) * N), 256, 0, s>>>(J64, g, N, Np, out);
  return cudaGetLastError();
}

cudaError_t launch_rank(const float* psi, const float* J32, const double* g, float* S32, double* part, double* E32,
                        int* idx, int* count, int N, int Np, int R, int Rp, int C, int cplx, double diag,
                        double margin, cudaStream_t s) {
  k_project_rank<<<grid_for(size_t(R) * N), 256, 0, s>>>(psi, S32, N, Np, R, cplx);
  const int mt = (N + 63) / 64;
  dim3 grid((C + 63) / 64, mt);
  if (cplx)
    k_energy32c<true><<<grid, 256, 0, s>>>(J32, S32, g, N, Np, R, Rp, part);
  else
    k_energy32c<false><<<grid, 256, 0, s>>>(J32, S32, g, N, Np, R, Rp, part);
  k_rank<<<1, 1024, 0, s>>>(part, mt, R, Rp, diag, margin, E32, idx, count);
  return cudaGetLastError();
}

cudaError_t launch_gather_cols(const float* psi, int Np, const int* idx, int count, int cplx, float* out,
                               cudaStream_t s) {
  k_gather_cols<<<grid_for(size_t(count) * (cplx ? 2 : 1) * Np), 256, 0, s>>>(psi, Np, idx, count, cplx, out);
  return cudaGetLastError();
}

cudaError_t launch_map_best(const int* idx, int* bestR, cudaStream_t s) {
  k_map_best<<<1, 1, 0, s>>>(idx, bestR);
  return cudaGetLastError();
}

}  // namespace gda
