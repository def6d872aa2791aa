// Learned proposal network (not in the paper): per-spin features of J and a
// 3-layer MLP, 8 -> 128 -> 128 -> 5 with ReLU, whose outputs give each spin's
// initial amplitude (outputs 0, 1: real and imaginary part) and, averaged over
// an instance's spins, the instance's run settings (outputs 2, 3, 4).
// Forward, backward, loss and Adam are hand-written FP32 kernels.
//
// Parameter vector layout (P = 18309 floats):
//   W1 [128][8], b1 [128], W2 [128][128], b2 [128], W3 [5][128], b3 [5].
#include "../../include/gda.h"
#include "gda_internal.h"

namespace gda {
namespace {

constexpr int DIN = GDA_MLP_IN, DH = GDA_MLP_HIDDEN, DOUT = GDA_MLP_OUT;
constexpr int O_W1 = 0, O_B1 = O_W1 + DH * DIN, O_W2 = O_B1 + DH, O_B2 = O_W2 + DH * DH, O_W3 = O_B2 + DH,
              O_B3 = O_W3 + DOUT * DH, P_TOTAL = O_B3 + DOUT;
static_assert(P_TOTAL == GDA_MLP_PARAMS, "parameter count");
constexpr int ROWS = 128;  // rows (spins) per block

// Shared memory of the forward / backward kernels: all weights, plus the
// block's hidden activations stored [unit][row] so that thread t (row t)
// reads a column without bank conflicts.
struct MlpSmem {
  float W1[DH * DIN], b1[DH], W2[DH * DH], b2[DH], W3[DOUT * DH], b3[DOUT];
  float H1[DH][ROWS + 1];
  float H2[DH][ROWS + 1];
};

__device__ void load_params(MlpSmem& s, const float* __restrict__ p) {
  for (int k = threadIdx.x; k < DH * DIN; k += blockDim.x) s.W1[k] = p[O_W1 + k];
  for (int k = threadIdx.x; k < DH; k += blockDim.x) s.b1[k] = p[O_B1 + k];
  for (int k = threadIdx.x; k < DH * DH; k += blockDim.x) s.W2[k] = p[O_W2 + k];
  for (int k = threadIdx.x; k < DH; k += blockDim.x) s.b2[k] = p[O_B2 + k];
  for (int k = threadIdx.x; k < DOUT * DH; k += blockDim.x) s.W3[k] = p[O_W3 + k];
  for (int k = threadIdx.x; k < DOUT; k += blockDim.x) s.b3[k] = p[O_B3 + k];
}

// Forward for ROWS rows per block; H (optional) caches h1, h2 for backward as
// [row][2*DH].
__global__ void __launch_bounds__(ROWS) k_mlp_forward(const float* __restrict__ p, const float* __restrict__ X, int M,
                                                      float* __restrict__ O, float* __restrict__ H) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(raw);
  load_params(s, p);
  __syncthreads();
  const int t = threadIdx.x;
  const int m = blockIdx.x * ROWS + t;
  float x[DIN];
#pragma unroll
  for (int k = 0; k < DIN; ++k) x[k] = m < M ? X[size_t(m) * DIN + k] : 0.0f;
  for (int j = 0; j < DH; ++j) {
    float a = s.b1[j];
#pragma unroll
    for (int k = 0; k < DIN; ++k) a = fmaf(s.W1[j * DIN + k], x[k], a);
    s.H1[j][t] = fmaxf(a, 0.0f);
  }
  float o[DOUT];
#pragma unroll
  for (int k = 0; k < DOUT; ++k) o[k] = s.b3[k];
  for (int j = 0; j < DH; ++j) {
    float a = s.b2[j];
    for (int k = 0; k < DH; ++k) a = fmaf(s.W2[j * DH + k], s.H1[k][t], a);
    a = fmaxf(a, 0.0f);
    s.H2[j][t] = a;
#pragma unroll
    for (int k = 0; k < DOUT; ++k) o[k] = fmaf(s.W3[k * DH + j], a, o[k]);
  }
  if (m < M) {
#pragma unroll
    for (int k = 0; k < DOUT; ++k) O[size_t(m) * DOUT + k] = o[k];
    if (H) {
      for (int j = 0; j < DH; ++j) {
        H[size_t(m) * 2 * DH + j] = s.H1[j][t];
        H[size_t(m) * 2 * DH + DH + j] = s.H2[j][t];
      }
    }
  }
}

// Backward for ROWS rows per block: accumulates the parameter gradient of
// sum_m dO[m] . O[m] into G (atomics across blocks).
__global__ void __launch_bounds__(ROWS) k_mlp_backward(const float* __restrict__ p, const float* __restrict__ X,
                                                       const float* __restrict__ H, const float* __restrict__ dO,
                                                       int M, float* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(raw);
  __shared__ float sdO[DOUT][ROWS];
  __shared__ float sX[DIN][ROWS];
  load_params(s, p);
  const int t = threadIdx.x;
  const int m = blockIdx.x * ROWS + t;
  const bool live = m < M;
  for (int j = 0; j < DH; ++j) {
    s.H1[j][t] = live ? H[size_t(m) * 2 * DH + j] : 0.0f;
    s.H2[j][t] = live ? H[size_t(m) * 2 * DH + DH + j] : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < DOUT; ++k) sdO[k][t] = live ? dO[size_t(m) * DOUT + k] : 0.0f;
#pragma unroll
  for (int k = 0; k < DIN; ++k) sX[k][t] = live ? X[size_t(m) * DIN + k] : 0.0f;
  __syncthreads();
  // layer 3: dW3[k][j] = sum_t dO[t][k] h2[t][j], db3[k] = sum_t dO[t][k]
  {
    const int j = t;
    for (int k = 0; k < DOUT; ++k) {
      float a = 0.0f;
      for (int r = 0; r < ROWS; ++r) a = fmaf(sdO[k][r], s.H2[j][r], a);
      atomicAdd(&G[O_W3 + k * DH + j], a);
    }
    if (t < DOUT) {
      float a = 0.0f;
      for (int r = 0; r < ROWS; ++r) a += sdO[t][r];
      atomicAdd(&G[O_B3 + t], a);
    }
  }
  __syncthreads();
  // dh2 = (W3^T dO) * relu'(h2), in place of H2 (the h2 values are no longer needed)
  for (int j = 0; j < DH; ++j) {
    float a = 0.0f;
#pragma unroll
    for (int k = 0; k < DOUT; ++k) a = fmaf(s.W3[k * DH + j], sdO[k][t], a);
    s.H2[j][t] = s.H2[j][t] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  // layer 2: dW2[j][k] = sum_t dh2[t][j] h1[t][k], db2[j] = sum_t dh2[t][j]
  {
    const int j = t;
    float db = 0.0f;
    for (int r = 0; r < ROWS; ++r) db += s.H2[j][r];
    atomicAdd(&G[O_B2 + j], db);
    for (int k0 = 0; k0 < DH; k0 += 32) {
      float acc[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) acc[q] = 0.0f;
      for (int r = 0; r < ROWS; ++r) {
        const float d = s.H2[j][r];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = fmaf(d, s.H1[k0 + q][r], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) atomicAdd(&G[O_W2 + j * DH + k0 + q], acc[q]);
    }
  }
  // dh1 = (W2^T dh2) * relu'(h1), row t, written over h1 (column t only)
  __syncthreads();
  for (int k = 0; k < DH; ++k) {
    float a = 0.0f;
    for (int j = 0; j < DH; ++j) a = fmaf(s.W2[j * DH + k], s.H2[j][t], a);
    s.H1[k][t] = s.H1[k][t] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  // layer 1: dW1[j][k] = sum_t dh1[t][j] x[t][k], db1[j] = sum_t dh1[t][j]
  {
    const int j = t;
    float acc[DIN];
#pragma unroll
    for (int k = 0; k < DIN; ++k) acc[k] = 0.0f;
    float db = 0.0f;
    for (int r = 0; r < ROWS; ++r) {
      const float d = s.H1[j][r];
      db += d;
#pragma unroll
      for (int k = 0; k < DIN; ++k) acc[k] = fmaf(d, sX[k][r], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < DIN; ++k) atomicAdd(&G[O_W1 + j * DIN + k], acc[k]);
    atomicAdd(&G[O_B1 + j], db);
  }
}

// Proposal loss of one instance per block (rows [off[b], off[b+1])):
//   amplitude: min over the global symmetry of mean_i |a_i - u s_i|^2, with u
//   = +-1 (Ising, a real) or the unit complex number aligning s with a (XY);
//   settings: sum_k (mean_i o_{i,2+k} - tgt_k)^2, weighted by wset.
// Writes dO (gradient of the loss) and loss[b].
__global__ void k_proposal_loss(const float* __restrict__ O, const float* __restrict__ S,
                                const float* __restrict__ Tset, const int* __restrict__ off,
                                const int* __restrict__ cplx, float wset, float* __restrict__ dO,
                                float* __restrict__ loss) {
  const int b = blockIdx.x;
  const int i0 = off[b], i1 = off[b + 1], n = i1 - i0;
  const bool cx = cplx[b] != 0;
  __shared__ float red[5][32];
  float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // Re<s,a>, Im<s,a>, sum o2, sum o3, sum o4
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float ar = O[size_t(i) * DOUT], ai = cx ? O[size_t(i) * DOUT + 1] : 0.0f;
    const float sr = S[size_t(i) * 2], si = cx ? S[size_t(i) * 2 + 1] : 0.0f;
    acc[0] += sr * ar + si * ai;  // Re(conj(s) a)
    acc[1] += sr * ai - si * ar;  // Im(conj(s) a)
    acc[2] += O[size_t(i) * DOUT + 2];
    acc[3] += O[size_t(i) * DOUT + 3];
    acc[4] += O[size_t(i) * DOUT + 4];
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float v = acc[k];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][w] = v;
  }
  __syncthreads();
  __shared__ float tot[5];
  if (threadIdx.x < 5) {
    float v = 0.0f;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) v += red[threadIdx.x][q];
    tot[threadIdx.x] = v;
  }
  __syncthreads();
  // u = <s, a> / |<s, a>| (XY) or sign(<s, a>) (Ising; +1 at 0)
  float ur, ui = 0.0f;
  if (cx) {
    const float mag = sqrtf(tot[0] * tot[0] + tot[1] * tot[1]);
    ur = mag > 0.0f ? tot[0] / mag : 1.0f;
    ui = mag > 0.0f ? tot[1] / mag : 0.0f;
  } else {
    ur = tot[0] >= 0.0f ? 1.0f : -1.0f;
  }
  const float inv = 1.0f / float(n);
  float pset[3], dset[3], lset = 0.0f;
  for (int k = 0; k < 3; ++k) {
    pset[k] = tot[2 + k] * inv;
    const float d = pset[k] - Tset[b * 3 + k];
    dset[k] = 2.0f * wset * d * inv;
    lset += wset * d * d;
  }
  float lamp = 0.0f;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float ar = O[size_t(i) * DOUT], ai = cx ? O[size_t(i) * DOUT + 1] : 0.0f;
    const float sr = S[size_t(i) * 2], si = cx ? S[size_t(i) * 2 + 1] : 0.0f;
    const float tr = ur * sr - ui * si, ti = ur * si + ui * sr;  // u s
    const float er = ar - tr, ei = ai - ti;
    lamp += er * er + ei * ei;
    dO[size_t(i) * DOUT] = 2.0f * er * inv;
    dO[size_t(i) * DOUT + 1] = cx ? 2.0f * ei * inv : 0.0f;
    for (int k = 0; k < 3; ++k) dO[size_t(i) * DOUT + 2 + k] = dset[k];
  }
  for (int o = 16; o; o >>= 1) lamp += __shfl_xor_sync(0xffffffffu, lamp, o);
  __syncthreads();
  if (lane == 0) red[0][w] = lamp;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.0f;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) v += red[0][q];
    loss[b] = v * inv + lset;
  }
}

// Adam (Kingma & Ba 2015) with bias correction, step t >= 1.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int P, float lr, float b1, float b2, float eps, int t) {
  const float c1 = 1.0f - powf(b1, float(t)), c2 = 1.0f - powf(b2, float(t));
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float a = b1 * m1[k] + (1.0f - b1) * gk;
    const float v = b2 * m2[k] + (1.0f - b2) * gk * gk;
    m1[k] = a;
    m2[k] = v;
    p[k] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
  }
}

// The proposal's head for one instance (one block): base amplitudes
// amp * O[:, 0] (+ the imaginary part amp * O[:, 1], interleaved, for XY),
// each the float rounding of the double product, and the settings from the
// spin-means of outputs 2..4 (double sums in a fixed tree order):
// eps = 0.02 + 0.48 s(m0), rho_th = 0.5 + 1.5 s(m1), beta0 = 0.1 + 0.9 s(m2),
// s the logistic function.
constexpr int HEAD_THREADS = 256;
__global__ void __launch_bounds__(HEAD_THREADS) k_proposal_head(const float* __restrict__ O, int N, int cplx,
                                                               double amp, float* __restrict__ base,
                                                               double* __restrict__ settings) {
  __shared__ double red[3][HEAD_THREADS];
  const int t = threadIdx.x;
  double m[3] = {0.0, 0.0, 0.0};
  for (int i = t; i < N; i += HEAD_THREADS) {
    const float* o = O + size_t(i) * DOUT;
    if (cplx) {
      base[2 * size_t(i)] = float(amp * double(o[0]));
      base[2 * size_t(i) + 1] = float(amp * double(o[1]));
    } else {
      base[i] = float(amp * double(o[0]));
    }
    for (int k = 0; k < 3; ++k) m[k] += double(o[2 + k]);
  }
  for (int k = 0; k < 3; ++k) red[k][t] = m[k];
  __syncthreads();
  for (int w = HEAD_THREADS / 2; w > 0; w >>= 1) {
    if (t < w)
      for (int k = 0; k < 3; ++k) red[k][t] += red[k][t + w];
    __syncthreads();
  }
  if (t == 0) {
    const double lo[3] = {0.02, 0.5, 0.1}, span[3] = {0.48, 1.5, 0.9};
    for (int k = 0; k < 3; ++k) {
      const double mean = N > 0 ? red[k][0] / double(N) : 0.0;
      settings[k] = lo[k] + span[k] * (1.0 / (1.0 + exp(-mean)));
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- features
// Per-spin features of an instance, J0 = J without its diagonal, row i:
//   f0 = sum_j J0_ij / |J0_i|        f1 = sum_j |J0_ij| / (sqrt(N) |J0_i|)
//   f2 = |J0_i|                       f3 = max_j |J0_ij| / |J0_i|
//   f4 = g_i                          f5 = (J0 v1)_i / rms(J0 v1)
//   f6 = (J0 f5)_i / rms(J0 f5)       f7 = 1 for XY, 0 for Ising
// with v1 = (J0 1) / rms(J0 1) (two power-iteration steps from the all-ones
// vector), |.| the Euclidean norm and rms over the N spins; 0/0 is taken as 0.
__global__ void k_feat_rows(const double* __restrict__ J, const double* __restrict__ g, int N, int Np, int cplx,
                            float* __restrict__ F) {
  const int i = blockIdx.x;
  double sum = 0.0, sabs = 0.0, ssq = 0.0, mx = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    if (j == i) continue;
    const double v = J[size_t(i) * Np + j];
    sum += v;
    sabs += fabs(v);
    ssq += v * v;
    mx = fmax(mx, fabs(v));
  }
  __shared__ double red[4][32];
  double a[4] = {sum, sabs, ssq, mx};
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < 4; ++k) {
    double x = a[k];
    for (int o = 16; o; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = (k == 3) ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int q = 0; q < int(blockDim.x >> 5); ++q)
      for (int k = 0; k < 4; ++k) t[k] = (k == 3) ? fmax(t[k], red[k][q]) : t[k] + red[k][q];
    const double nrm = sqrt(t[2]);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    F[size_t(i) * DIN + 0] = float(t[0] * inv);
    F[size_t(i) * DIN + 1] = float(t[1] * inv / sqrt(double(N)));
    F[size_t(i) * DIN + 2] = float(nrm);
    F[size_t(i) * DIN + 3] = float(t[3] * inv);
    F[size_t(i) * DIN + 4] = float(g ? g[i] : 0.0);
    F[size_t(i) * DIN + 7] = float(cplx);
  }
}

// y = J0 x (x = all ones when null), FP64, one block per row.
__global__ void k_feat_matvec(const double* __restrict__ J, const double* __restrict__ x, int N, int Np,
                              double* __restrict__ y) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x)
    if (j != i) s += J[size_t(i) * Np + j] * (x ? x[j] : 1.0);
  __shared__ double red[32];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) t += red[q];
    y[i] = t;
  }
}

// v = y / rms(y) (one block); optionally also F[i][col] = v_i.
__global__ void k_feat_normalize(const double* __restrict__ y, int N, double* __restrict__ v, float* __restrict__ F,
                                 int col) {
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += y[i] * y[i];
  __shared__ double red[32];
  __shared__ double scale;
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) t += red[q];
    const double rms = sqrt(t / double(N));
    scale = rms > 0.0 ? 1.0 / rms : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double vi = y[i] * scale;
    v[i] = vi;
    if (F) F[size_t(i) * DIN + col] = float(vi);
  }
}

cudaError_t launch_features(const double* J, const double* g, int N, int Np, int cplx, double* w0, double* w1,
                            float* F, cudaStream_t s) {
  k_feat_rows<<<N, 128, 0, s>>>(J, g, N, Np, cplx, F);
  k_feat_matvec<<<N, 128, 0, s>>>(J, nullptr, N, Np, w0);     // J0 1
  k_feat_normalize<<<1, 1024, 0, s>>>(w0, N, w1, nullptr, 0);  // v1
  k_feat_matvec<<<N, 128, 0, s>>>(J, w1, N, Np, w0);          // J0 v1
  k_feat_normalize<<<1, 1024, 0, s>>>(w0, N, w1, F, 5);       // f5
  k_feat_matvec<<<N, 128, 0, s>>>(J, w1, N, Np, w0);          // J0 f5
  k_feat_normalize<<<1, 1024, 0, s>>>(w0, N, w1, F, 6);       // f6
  return cudaGetLastError();
}

}  // namespace gda

using namespace gda;

extern "C" gda_status gda_mlp_forward(const float* params, const float* X, int32_t M, float* O, float* H,
                                      void* stream) {
  if (!params || !X || !O || M < 0) return GDA_ERR_INVALID;
  if (M == 0) return GDA_OK;
  const size_t smem = sizeof(MlpSmem);
  static bool set = false;
  if (!set) {
    if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
      return GDA_ERR_CUDA;
    set = true;
  }
  k_mlp_forward<<<(M + ROWS - 1) / ROWS, ROWS, smem, static_cast<cudaStream_t>(stream)>>>(params, X, M, O, H);
  return cudaGetLastError() == cudaSuccess ? GDA_OK : GDA_ERR_CUDA;
}

extern "C" gda_status gda_mlp_backward(const float* params, const float* X, const float* H, const float* dO,
                                       int32_t M, float* G, void* stream) {
  if (!params || !X || !H || !dO || !G || M < 0) return GDA_ERR_INVALID;
  if (M == 0) return GDA_OK;
  const size_t smem = sizeof(MlpSmem);
  static bool set = false;
  if (!set) {
    if (cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
      return GDA_ERR_CUDA;
    set = true;
  }
  k_mlp_backward<<<(M + ROWS - 1) / ROWS, ROWS, smem, static_cast<cudaStream_t>(stream)>>>(params, X, H, dO, M, G);
  return cudaGetLastError() == cudaSuccess ? GDA_OK : GDA_ERR_CUDA;
}

extern "C" gda_status gda_proposal_loss(const float* O, const float* S, const float* Tset, const int32_t* offsets,
                                        const int32_t* cplx, int32_t n_inst, float wset, float* dO, float* loss,
                                        void* stream) {
  if (!O || !S || !Tset || !offsets || !cplx || !dO || !loss || n_inst < 0) return GDA_ERR_INVALID;
  if (n_inst == 0) return GDA_OK;
  k_proposal_loss<<<n_inst, 256, 0, static_cast<cudaStream_t>(stream)>>>(O, S, Tset, offsets, cplx, wset, dO, loss);
  return cudaGetLastError() == cudaSuccess ? GDA_OK : GDA_ERR_CUDA;
}

extern "C" gda_status gda_adam_step(float* params, const float* grad, float* m1, float* m2, int32_t P, float lr,
                                    float beta1, float beta2, float eps, int32_t t, void* stream) {
  if (!params || !grad || !m1 || !m2 || P < 0 || t < 1) return GDA_ERR_INVALID;
  k_adam<<<(P + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m1, m2, P, lr, beta1, beta2,
                                                                          eps, t);
  return cudaGetLastError() == cudaSuccess ? GDA_OK : GDA_ERR_CUDA;
}

extern "C" gda_status gda_proposal_head(const float* O, int32_t N, int32_t cplx, double amp, float* base,
                                        double* settings, void* stream) {
  if (!O || !base || !settings || N < 1) return GDA_ERR_INVALID;
  k_proposal_head<<<1, HEAD_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(O, N, cplx ? 1 : 0, amp, base,
                                                                             settings);
  return cudaGetLastError() == cudaSuccess ? GDA_OK : GDA_ERR_CUDA;
}
