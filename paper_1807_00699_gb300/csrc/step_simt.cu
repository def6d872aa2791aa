// FP32 CUDA-core GD step: a tiled SGEMM Y = J0 X over one 64x64 tile of
// (spins i) x (columns c), fused with the step epilogue (Eqs. 2, 5, 6).  This
// is the plain FP32 path the tensor-core path is measured against, and the
// path whose amplitudes are compared with the FP64 oracle.
//
// The sparse variant (SPARSE = true) replaces the SGEMM by a gather over the
// nonzeros of J0 in ELL form (col / val [dmax][Np], deg [Np]): thread (tx, ty)
// sums, for its 4 rows and 4 columns, val_ik X[c][col_ik] in ascending k.  The
// tile shape, the thread-to-element map and the epilogue (with its partial-sum
// order) are the dense kernel's, so density partials, noise decay and the
// energy mode carry over unchanged.
#include "epilogue.cuh"
#include "tc_epilogue.cuh"
#include "tc_ptx.cuh"

namespace gda {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, PAD = 4;
constexpr size_t kPairSmemMax = 200 * 1024;  // the staged sparse kernel: N rounded up to 128 <= 25600

struct Ell {
  const int* col;   // [dmax][Np]
  const float* val; // [dmax][Np]
  const int* deg;   // [Np], 0 beyond N
};

// DW (sparse): the ELL width the loop runs over, a power of two >= the largest
// row count; entries beyond a row's count are (column 0, value 0) and add
// exact zeros, so the sums equal those over the row's nonzeros alone.
template <bool CPLX, bool SPARSE, int DW, int MODE>
__global__ void __launch_bounds__(256) step_simt_kernel(StepArgs a, const float* __restrict__ J,
                                                        const float* __restrict__ X, Ell ell) {
  __shared__ __align__(16) float As[SPARSE ? 1 : BK][BM + PAD];
  __shared__ __align__(16) float Bs[SPARSE ? 1 : BK][BN + PAD];
  __shared__ float s_beta[BN], s_dsc[BN];
  __shared__ int s_bad;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int Np = a.Np;
  constexpr int RPT = CPLX ? BN / 2 : BN;  // restarts per tile
  const int rbase = CPLX ? n0 / 2 : n0;

  if (tid == 0) s_bad = 0;
  if (tid < RPT) {
    const int r = rbase + tid;
    const float b = r < a.R ? a.beta_in[r] : 1.0f;
    s_beta[tid] = stage_beta(a, b);
    s_dsc[tid] = r < a.R ? noise_scale(a, r) : 0.0f;
  }

  float acc[4][4] = {};
  if (SPARSE) {
    // The 4 rows' index loads, then their gathers, are issued together (rows
    // beyond N read the ELL padding: column 0, value 0), so the dependent
    // index -> gather chains of the rows overlap instead of following each other.
    constexpr int KC = DW < 1 ? 1 : (DW < 4 ? DW : 4);  // entries per row whose loads are issued together
    const int cq = n0 + 4 * ty;          // the thread's 4 columns (always < Cp)
#pragma unroll 1
    for (int k0 = 0; k0 < DW; k0 += KC) {
      int jj[4][KC];
      float vv[4][KC];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          const size_t o = size_t(k0 + k) * Np + m0 + tx + 16 * q;
          jj[q][k] = ell.col[o];
          vv[q][k] = ell.val[o];
        }
      if (a.opT_in) {  // spin-major operand: the 4 columns of spin j are one 16-byte load
        float4 x[4][KC];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < KC; ++k)
            x[q][k] = *reinterpret_cast<const float4*>(a.opT_in + size_t(jj[q][k]) * a.Cp + cq);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < KC; ++k) {
            acc[q][0] = __fmaf_rn(vv[q][k], x[q][k].x, acc[q][0]);
            acc[q][1] = __fmaf_rn(vv[q][k], x[q][k].y, acc[q][1]);
            acc[q][2] = __fmaf_rn(vv[q][k], x[q][k].z, acc[q][2]);
            acc[q][3] = __fmaf_rn(vv[q][k], x[q][k].w, acc[q][3]);
          }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < KC; ++k)
#pragma unroll
            for (int u = 0; u < 4; ++u)
              acc[q][u] = __fmaf_rn(vv[q][k], X[size_t(cq + u) * Np + jj[q][k]], acc[q][u]);
      }
    }
  }
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const float* Jp = SPARSE ? nullptr : J + size_t(m0 + lr) * Np + lk;
  const float* Xp = SPARSE ? nullptr : X + size_t(n0 + lr) * Np + lk;
  for (int k0 = 0; !SPARSE && k0 < Np; k0 += BK) {
    const float4 av = *reinterpret_cast<const float4*>(Jp + k0);
    const float4 bv = *reinterpret_cast<const float4*>(Xp + k0);
    __syncthreads();
    As[lk + 0][lr] = av.x; As[lk + 1][lr] = av.y; As[lk + 2][lr] = av.z; As[lk + 3][lr] = av.w;
    Bs[lk + 0][lr] = bv.x; Bs[lk + 1][lr] = bv.y; Bs[lk + 2][lr] = bv.z; Bs[lk + 3][lr] = bv.w;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[k][4 * ty]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float av2 = As[k][tx + 16 * q];
        acc[q][0] += av2 * b4.x; acc[q][1] += av2 * b4.y;
        acc[q][2] += av2 * b4.z; acc[q][3] += av2 * b4.w;
      }
    }
  }
  __syncthreads();

  // Epilogue: rows m0 + tx + 16 q, columns c0 .. c0 + 3.
  const int c0 = n0 + 4 * ty;
  constexpr int U = CPLX ? 2 : 4;
  const int lr0 = CPLX ? 2 * ty : 4 * ty;  // first local restart of the quad
  float rsum[4] = {0.f, 0.f, 0.f, 0.f};
  int bad = 0;
  if (SPARSE) {
    // every input of the 4 rows is loaded before the first store, so that the
    // rows' loads are in flight together (the stores could alias them for the
    // compiler); same arithmetic as epi_quad
    EpiRegs<MODE, CPLX, 4> E[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) epi_load<MODE, CPLX, 4>(a, m0 + tx + 16 * q, c0, E[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = m0 + tx + 16 * q;
      if (i >= a.N) continue;
      float red[4] = {0.f, 0.f, 0.f, 0.f}, t4[4];
      epi_chunk<MODE, CPLX, 4, true>(a, i, c0, acc[q], E[q], &s_beta[lr0], &s_dsc[lr0], red, bad, t4);
      if (a.opT_out && MODE != M_RAW && MODE != M_ENERGY)
        *reinterpret_cast<float4*>(a.opT_out + size_t(i) * a.Cp + c0) = make_float4(t4[0], t4[1], t4[2], t4[3]);
#pragma unroll
      for (int u = 0; u < U; ++u) rsum[u] += red[u];
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = m0 + tx + 16 * q;
      if (i >= a.N) continue;
      float red[4];
      epi_quad<CPLX, SPARSE, MODE>(a, i, c0, acc[q], &s_beta[lr0], &s_dsc[lr0], red, bad);
#pragma unroll
      for (int u = 0; u < U; ++u) rsum[u] += red[u];
    }
  }
  // Sum over the 16 row groups (lanes with the same ty are one half-warp).
#pragma unroll
  for (int u = 0; u < U; ++u) {
#pragma unroll
    for (int off = 8; off; off >>= 1) rsum[u] += __shfl_xor_sync(0xffffffffu, rsum[u], off);
  }
  float* out = (a.mode == M_ENERGY) ? a.e_part : (step_completes(a.mode) ? a.rho_out : nullptr);
  if (tx == 0 && out) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = rbase + lr0 + u;
      if (r < a.R) out[size_t(blockIdx.y) * a.Rp + r] = rsum[u];
    }
  }
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (tid == 0 && s_bad) atomicOr(a.err, E_DIVERGED);
  if (blockIdx.y == 0 && step_completes(a.mode) && tid < RPT) {
    const int r = rbase + tid;
    if (r < a.R) a.beta_out[r] = next_beta(a, a.beta_in[r]);
  }
}

}  // namespace

int simt_mtiles(int N) { return (N + BM - 1) / BM; }

template <bool CPLX, bool SPARSE, int DW>
cudaError_t launch_modes(const StepArgs& a, const float* J32, const float* operand, const Ell& ell, cudaStream_t s) {
  dim3 grid((a.C + BN - 1) / BN, simt_mtiles(a.N));
  switch (a.mode) {
    case M_EULER: step_simt_kernel<CPLX, SPARSE, DW, M_EULER><<<grid, 256, 0, s>>>(a, J32, operand, ell); break;
    case M_RK1: step_simt_kernel<CPLX, SPARSE, DW, M_RK1><<<grid, 256, 0, s>>>(a, J32, operand, ell); break;
    case M_RK2: step_simt_kernel<CPLX, SPARSE, DW, M_RK2><<<grid, 256, 0, s>>>(a, J32, operand, ell); break;
    case M_RK3: step_simt_kernel<CPLX, SPARSE, DW, M_RK3><<<grid, 256, 0, s>>>(a, J32, operand, ell); break;
    case M_RK4: step_simt_kernel<CPLX, SPARSE, DW, M_RK4><<<grid, 256, 0, s>>>(a, J32, operand, ell); break;
    case M_ENERGY: step_simt_kernel<CPLX, SPARSE, DW, M_ENERGY><<<grid, 256, 0, s>>>(a, J32, operand, ell); break;
    case M_RAW: step_simt_kernel<CPLX, SPARSE, DW, M_RAW><<<grid, 256, 0, s>>>(a, J32, operand, ell); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_step_simt(const StepArgs& a, const float* J32, const float* operand, cudaStream_t s) {
  const Ell none{nullptr, nullptr, nullptr};
  return a.cplx ? launch_modes<true, false, 0>(a, J32, operand, none, s)
                : launch_modes<false, false, 0>(a, J32, operand, none, s);
}

namespace {

// Forward-Euler step over a sparse J0, one CTA per column pair (two Ising
// restarts, or the real and imaginary columns of one XY restart): the pair's
// amplitudes psi^n (two contiguous columns of Np floats) are staged in shared
// memory once (bulk asynchronous copies), then the CTA sweeps every row i, gathers sum_k val_ik X[col_ik]
// from shared memory in ascending k (the per-step kernel's order, so Y has the
// same bits) and runs the Euler update of Eqs. (2), (5), (6) on the staged
// psi_i, with the same FP32 expression sequence as the other epilogues.  Each
// amplitude is read from HBM once per step and no spin-major copy is kept.
// Rows go to 16-thread groups by 64-row tile (thread tx of a group takes rows
// tx + 16 q, q = 0..3), so the per-tile density sums are formed in the
// per-step kernel's order and layout.
// PAIR_THREADS threads per CTA: 512 where two CTAs share an SM, 1024 where the
// staged columns take most of an SM's shared memory (more loads in flight).
// Pairs from split_from on are each swept by split_k CTAs, one contiguous
// range of tiles each (every one staging the pair): the pairs that would fill
// only part of the last wave of CTAs are spread over all of it.
template <bool CPLX, int DW, int PAIR_THREADS>
__global__ void __launch_bounds__(PAIR_THREADS) k_sparse_euler_pair(StepArgs a, Ell ell, int split_from,
                                                                   int split_k) {
  extern __shared__ __align__(16) float xs[];  // [2][Np]: the pair's columns of psi^n
  __shared__ float s_beta[2], s_dsc[2];
  __shared__ int s_bad;
  __shared__ __align__(8) uint64_t s_bar;
  constexpr int U = CPLX ? 1 : 2;  // restarts of the pair
  const int tid = threadIdx.x;
  const int Np = a.Np;
  int pair = blockIdx.x, t_begin = 0, t_end = a.mt_count;
  if (int(blockIdx.x) >= split_from) {
    const int idx = int(blockIdx.x) - split_from, ch = idx % split_k;
    pair = split_from + idx / split_k;
    t_begin = int((long long)a.mt_count * ch / split_k);
    t_end = int((long long)a.mt_count * (ch + 1) / split_k);
  }
  const bool owner = int(blockIdx.x) < split_from || (int(blockIdx.x) - split_from) % split_k == 0;
  const int c0 = 2 * pair;                 // first column of the pair (< Cp)
  const int r0 = CPLX ? pair : c0;         // first restart
  // stage psi^n of both columns: bulk copies of <= 32 KB (Np is a multiple
  // of 128, so every piece is a multiple of 16 bytes and 16-byte aligned)
  const uint32_t bar = ptx::smem_u32(&s_bar);
  if (tid == 0) {
    ptx::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint32_t col_bytes = uint32_t(Np) * 4u;
    ptx::mbar_arrive_expect_tx(bar, 2u * col_bytes);
    for (int u = 0; u < 2; ++u)
      for (uint32_t off = 0; off < col_bytes; off += 32768u) {
        const uint32_t len = col_bytes - off < 32768u ? col_bytes - off : 32768u;
        ptx::bulk_load(ptx::smem_u32(xs) + uint32_t(u) * col_bytes + off,
                       reinterpret_cast<const char*>(a.psi_n + size_t(c0 + u) * Np) + off, len, bar);
      }
  }
  if (tid == 0) s_bad = 0;
  if (tid < U) {
    const int r = r0 + tid;
    const float b = r < a.R ? a.beta_in[r] : 1.0f;
    s_beta[tid] = stage_beta(a, b);
    s_dsc[tid] = r < a.R ? noise_scale(a, r) : 0.0f;
  }
  __syncthreads();  // publishes the barrier's initialisation and s_beta / s_dsc
  // every thread waits for the copies (bounded); a CTA whose copies did not
  // land in time reports a timeout and leaves once they have (again bounded)
  if (!__syncthreads_and(ptx::mbar_wait(bar, 0, a.wait_cycles))) {
    if (tid == 0) atomicOr(a.err, E_TIMEOUT);
    (void)ptx::mbar_wait(bar, 0, a.wait_cycles);
    return;
  }
  const float* x0 = xs;
  const float* x1 = xs + Np;
  const bool noise = s_dsc[0] != 0.0f || (U > 1 && s_dsc[1] != 0.0f);
  int bad = 0;
  const int grp = tid >> 4, tx = tid & 15;
  // the two halves of a warp may run different numbers of tiles: shuffles
  // stay within the half
  const unsigned half = (tid & 16) ? 0xffff0000u : 0x0000ffffu;
  for (int t = t_begin + grp; t < t_end; t += PAIR_THREADS / 16) {  // 64-row tiles
   // the tile's four rows of a thread: every load first (the gathers, the
   // gains, the fields), then the updates and stores, so that no store sits
   // between two loads and a thread keeps all of them in flight
   float y[4][2], gv[4][U], hv[4];
   {  // the next tile's gain lines (two 128-byte lines per restart) into L2
     const int tn = t + PAIR_THREADS / 16;
     if (tn < t_end && tx < 2 * U && r0 + (tx >> 1) < a.R)
       prefetch_l2(a.gam + size_t(r0 + (tx >> 1)) * Np + tn * 64 + 32 * (tx & 1));
   }
#pragma unroll
   for (int qq = 0; qq < 4; ++qq) {
    const int i = t * 64 + tx + 16 * qq;
    const bool ok = i < a.N;
    const int ic = ok ? i : 0;
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int k = 0; k < DW; ++k) {
      const size_t o = size_t(k) * Np + ic;
      const int j = ell.col[o];
      const float v = ell.val[o];
      y0 = __fmaf_rn(v, x0[j], y0);
      y1 = __fmaf_rn(v, x1[j], y1);
    }
    y[qq][0] = y0;
    y[qq][1] = y1;
    hv[qq] = a.h1[ic];
#pragma unroll
    for (int u = 0; u < U; ++u)
      gv[qq][u] = ok && r0 + u < a.R ? a.gam[size_t(r0 + u) * Np + i] : 0.0f;
   }
   float red[2] = {0.0f, 0.0f};
#pragma unroll
   for (int qq = 0; qq < 4; ++qq) {
    const int i = t * 64 + tx + 16 * qq;
    if (i >= a.N) continue;
    float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (noise) philox_normal4(uint32_t(i), uint32_t(c0 >> 2), a.step, 0u, a.seed, z);
    // the pair's two normals: elements c0 & 3 and (c0 & 3) + 1 (c0 is even)
    const float zp[2] = {(c0 & 2) ? z[2] : z[0], (c0 & 2) ? z[3] : z[1]};
    const float h = hv[qq];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u;
      if (r >= a.R) continue;
      const int col = c0 + u;  // Ising: the restart's column; XY: the real part's
      const size_t og = size_t(r) * Np + i;
      const float xr = u == 0 ? x0[i] : x1[i];
      const float xi = CPLX ? x1[i] : 0.0f;
      const float yr = y[qq][u];
      const float yi = CPLX ? y[qq][1] : 0.0f;
      const float gs = gv[qq][u];
      float kr, ki, kg;
      gd_rhs(xr, xi, gs, yr, yi, s_beta[u], h, a.eps, a.rho_th, kr, ki, kg);
      if (CPLX && a.q) resonant_drive(xr, xi, a.q, a.hq, kr, ki);
      float nr = axpy(a.dt, kr, xr);
      float ni = axpy(a.dt, ki, xi);
      const float ng = axpy(a.dt, kg, gs);
      nr = axpy(s_dsc[u], zp[u], nr);
      if (CPLX) ni = axpy(s_dsc[u], zp[1], ni);
      a.psi_out[size_t(col) * Np + i] = nr;
      if (CPLX) a.psi_out[size_t(col + 1) * Np + i] = ni;
      a.gam[og] = ng;
      const float rn = density(nr, ni);
      red[u] += rn;
      bad |= !(rn < 1e30f);
    }
   }
   if (a.rho_out) {  // the tile's density sum per restart: an xor tree over the group's 16 threads
#pragma unroll
     for (int u = 0; u < U; ++u) {
       float v = red[u];
#pragma unroll
       for (int off = 8; off; off >>= 1) v += __shfl_xor_sync(half, v, off);
       if (tx == 0 && r0 + u < a.R) a.rho_out[size_t(t) * a.Rp + r0 + u] = v;
     }
   }
  }
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (tid < U && owner) {  // one CTA of a split pair advances its coupling scales
    const int r = r0 + tid;
    if (r < a.R) a.beta_out[r] = next_beta(a, a.beta_in[r]);
  }
  if (tid == 0 && s_bad) atomicOr(a.err, E_DIVERGED);
}

template <bool CPLX, int DW, int NT>
cudaError_t launch_pair_nt(const StepArgs& a, const Ell& ell, size_t smem, cudaStream_t s) {
  auto kern = k_sparse_euler_pair<CPLX, DW, NT>;
  static int slots = 0;  // CTAs of this form resident at once (at the largest staging)
  static size_t slots_smem = 0;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmemMax);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (slots_smem != smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    slots = sms * per_sm;
    slots_smem = smem;
  }
  // pairs beyond the last full wave are split over the whole of it (k >= 2)
  const int npairs = (a.C + 1) / 2;
  const int rem = slots > 0 ? npairs % slots : 0;
  int k = rem > 0 ? slots / rem : 1;
  k = k > 8 ? 8 : k;
  k = k > a.mt_count ? a.mt_count : k;
  const int split_from = k >= 2 ? npairs - rem : npairs;
  const int split_k = k >= 2 ? k : 1;
  const int grid = split_from + (npairs - split_from) * split_k;
  kern<<<grid, NT, smem, s>>>(a, ell, split_from, split_k);
  return cudaGetLastError();
}

template <bool CPLX, int DW>
cudaError_t launch_pair(const StepArgs& a, const Ell& ell, cudaStream_t s) {
  const size_t smem = size_t(2) * a.Np * sizeof(float);
  return smem <= size_t(110) * 1024 ? launch_pair_nt<CPLX, DW, 512>(a, ell, smem, s)
                                    : launch_pair_nt<CPLX, DW, 1024>(a, ell, smem, s);
}

}  // namespace

template <int DW>
cudaError_t launch_sparse_w(const StepArgs& a, const Ell& ell, const float* operand, cudaStream_t s) {
  // Euler steps whose column pair fits in shared memory: the staged kernel
  if (a.mode == M_EULER && size_t(2) * a.Np * sizeof(float) <= kPairSmemMax)
    return a.cplx ? launch_pair<true, DW>(a, ell, s) : launch_pair<false, DW>(a, ell, s);
  return a.cplx ? launch_modes<true, true, DW>(a, nullptr, operand, ell, s)
                : launch_modes<false, true, DW>(a, nullptr, operand, ell, s);
}

cudaError_t launch_step_sparse(const StepArgs& a, const int* col, const float* val, const int* deg,
                               const float* operand, int maxdeg, cudaStream_t s) {
  const Ell ell{col, val, deg};
  // the paper's 3-regular graphs: the staged Euler kernel loops over exactly
  // three entries (a fourth slot would add a zero product and cost a load)
  if (maxdeg <= 3 && a.mode == M_EULER && size_t(2) * a.Np * sizeof(float) <= kPairSmemMax)
    return a.cplx ? launch_pair<true, 3>(a, ell, s) : launch_pair<false, 3>(a, ell, s);
  if (maxdeg <= 4) return launch_sparse_w<4>(a, ell, operand, s);
  if (maxdeg <= 8) return launch_sparse_w<8>(a, ell, operand, s);
  if (maxdeg <= 16) return launch_sparse_w<16>(a, ell, operand, s);
  if (maxdeg <= 32) return launch_sparse_w<32>(a, ell, operand, s);
  if (maxdeg <= 64) return launch_sparse_w<64>(a, ell, operand, s);
  return cudaErrorInvalidValue;
}

namespace {

__global__ void k_transpose_state(const float* __restrict__ x, int Np, int Cp, float* __restrict__ out) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) t[k][threadIdx.x] = x[size_t(c0 + k) * Np + i0 + threadIdx.x];
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) out[size_t(i0 + k) * Cp + c0 + threadIdx.x] = t[threadIdx.x][k];
}

// One warp per row of J0 (FP32, diagonal removed, zero padding): the nonzeros
// of row i in ascending column order go to col / val [k][Np] for k < dmax;
// deg[i] = min(count, dmax) and *maxdeg receives the largest count.
__global__ void k_prepare_ell(const float* __restrict__ J32, int N, int Np, int dmax, int* col, float* val, int* deg,
                              int* maxdeg) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= Np) return;
  const int i = warp;
  int count = 0;
  if (i < N) {
    const float* row = J32 + size_t(i) * Np;
    for (int j0 = 0; j0 < N; j0 += 32) {
      const int j = j0 + lane;
      const float v = j < N ? row[j] : 0.0f;
      const unsigned m = __ballot_sync(0xffffffffu, v != 0.0f);
      const int k = count + __popc(m & ((1u << lane) - 1u));
      if (v != 0.0f && k < dmax) {
        col[size_t(k) * Np + i] = j;
        val[size_t(k) * Np + i] = v;
      }
      count += __popc(m);
    }
  }
  if (lane == 0) {
    deg[i] = count < dmax ? count : dmax;
    atomicMax(maxdeg, count);
  }
}

}  // namespace

cudaError_t launch_transpose_state(const float* x, int Np, int Cp, float* out, cudaStream_t s) {
  k_transpose_state<<<dim3(Cp / 32, Np / 32), dim3(32, 8), 0, s>>>(x, Np, Cp, out);
  return cudaGetLastError();
}

cudaError_t launch_prepare_ell(const float* J32, int N, int Np, int dmax, int* col, float* val, int* deg, int* maxdeg,
                               cudaStream_t s) {
  const int blocks = (Np * 32 + 255) / 256;
  k_prepare_ell<<<blocks, 256, 0, s>>>(J32, N, Np, dmax, col, val, deg, maxdeg);
  return cudaGetLastError();
}

}  // namespace gda
