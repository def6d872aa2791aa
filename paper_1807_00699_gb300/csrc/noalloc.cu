// Allocation-free Eq. (1) energy evaluation: gda_energy_noalloc.
//
// Some callers cannot allocate device memory while they run: a host that has
// pre-reserved all of its GPU memory in its own pool, an inference server
// that forbids allocations once it is serving, or code running where
// cudaMalloc would synchronise the device or is simply unavailable to it.
// This entry point therefore takes only caller-owned device buffers and keeps
// its scratch (the per-tile partial energies) in a fixed-size file-scope
// device array that every GPU loading this library holds until the process
// exits.  It computes the same quantity as gda_energy (FP64 energies of the
// projected spins) with the same tiled product, but projects the spins on the
// fly instead of staging them in a context buffer.
#include <mutex>

#include "../../include/gda.h"
#include "gda_internal.h"

namespace gda {
namespace {

constexpr int kTile = 64;
constexpr int kMaxTiles = (GDA_NOALLOC_MAX_N + kTile - 1) / kTile;

// Partial energies [row tile][restart].  Each call overwrites every entry it
// later reads, so stale contents of an earlier call never leak into a result.
static __device__ __align__(256) double g_noalloc_partial[kMaxTiles * GDA_NOALLOC_MAX_R];

// Spin s of column c (= W r + p) at spin j, projected from psi [R][N][W].
__device__ __forceinline__ double proj_spin(const float* psi, int N, int W, int c, int j) {
  const int r = c / W, p = c - W * r;
  const size_t o = (size_t(r) * N + j) * W;
  if (W == 1) return psi[o] >= 0.0f ? 1.0 : -1.0;
  const double re = psi[o], im = psi[o + 1];
  const double m = sqrt(re * re + im * im);
  if (!(m > 0.0)) return p == 0 ? 1.0 : 0.0;
  return (p == 0 ? re : im) / m;
}

// 64 x 64 tile of T = J S (rows i, columns c) over K = N, then each restart's
// partial of Eq. (1) over the tile's rows.  J is N x N row-major with its
// diagonal (Eq. 1 sums all ordered pairs).
template <int W>
__global__ void __launch_bounds__(256) k_energy_noalloc(const double* __restrict__ J, const double* __restrict__ g,
                                                        const float* __restrict__ psi, int N, int R,
                                                        double* __restrict__ part) {
  __shared__ double As[16][kTile + 1];
  __shared__ double Bs[16][kTile + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  const int C = W * R;
  double acc[4][4] = {};
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (int k0 = 0; k0 < N; k0 += 16) {
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int row = m0 + lr, col = n0 + lr, k = k0 + lk + t;
      As[lk + t][lr] = (row < N && k < N) ? J[size_t(row) * N + k] : 0.0;
      Bs[lk + t][lr] = (col < C && k < N) ? proj_spin(psi, N, W, col, k) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double b[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[k][4 * ty + v];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double av = As[k][tx + 16 * a];
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[a][v] += av * b[v];
      }
    }
  }
  // restarts of this thread's column quad: 4 (Ising) or 2 (XY)
  const int c0 = n0 + 4 * ty;
  constexpr int U = 4 / W;
  double rs[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = m0 + tx + 16 * a;
    if (i >= N) continue;
    const double gi = g ? g[i] : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = c0 + W * u;
      if (c >= C) continue;
      const double sr = proj_spin(psi, N, W, c, i);
      double e = -sr * acc[a][W * u] + gi * sr;
      if (W == 2) e -= proj_spin(psi, N, W, c + 1, i) * acc[a][W * u + 1];
      rs[u] += e;
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int off = 8; off; off >>= 1) rs[u] += __shfl_xor_sync(0xffffffffu, rs[u], off);
  if (tx == 0) {
    for (int u = 0; u < U; ++u) {
      const int r = c0 / W + u;
      if (r < R) part[size_t(blockIdx.y) * GDA_NOALLOC_MAX_R + r] = rs[u];
    }
  }
}

__global__ void k_energy_noalloc_finish(const double* __restrict__ part, int tiles, int R, double* __restrict__ E) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < tiles; ++t) s += part[size_t(t) * GDA_NOALLOC_MAX_R + r];
    E[r] = s;
  }
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace gda

extern "C" gda_status gda_energy_noalloc(const double* J_dev, const double* g_dev, int32_t N, int32_t model,
                                         const float* psi_dev, int32_t R, double* E_dev, void* stream) {
  if (!J_dev || !psi_dev || !E_dev || N < 1 || R < 1) return GDA_ERR_INVALID;
  if (model != GDA_ISING && model != GDA_XY) return GDA_ERR_INVALID;
  if (N > GDA_NOALLOC_MAX_N || R > GDA_NOALLOC_MAX_R) return GDA_ERR_INVALID;
  double* part = nullptr;
  if (gda::scratch_for_current_device(&part) != cudaSuccess) {
    cudaGetLastError();
    return GDA_ERR_CUDA;
  }
  const int W = model == GDA_XY ? 2 : 1;
  const int tiles = (N + gda::kTile - 1) / gda::kTile;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid((W * R + gda::kTile - 1) / gda::kTile, tiles);
  if (W == 2)
    gda::k_energy_noalloc<2><<<grid, 256, 0, s>>>(J_dev, g_dev, psi_dev, N, R, part);
  else
    gda::k_energy_noalloc<1><<<grid, 256, 0, s>>>(J_dev, g_dev, psi_dev, N, R, part);
  gda::k_energy_noalloc_finish<<<(R + 255) / 256, 256, 0, s>>>(part, tiles, R, E_dev);
  if (cudaGetLastError() != cudaSuccess) return GDA_ERR_CUDA;
  return GDA_OK;
}
