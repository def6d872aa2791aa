// Internal types shared by the host runtime and the kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

namespace gda {

// What one launch of a step kernel computes in its epilogue.
enum Mode : int {
  M_EULER = 0,   // forward Euler step (plus noise)
  M_RK1 = 1,     // RK4 stages 1..4 (stage 4 completes the step, plus noise)
  M_RK2 = 2,
  M_RK3 = 3,
  M_RK4 = 4,
  M_ENERGY = 5,  // per-restart Eq. (1) partial energies of the projected spins
  M_RAW = 6,     // writes Y = J0 X itself (the coupling product alone)
};

// |psi|^2 with a fixed rounding sequence, so every kernel that forms a
// density gets the same bits.
__host__ __device__ __forceinline__ float density(float re, float im) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im));
#else
  return re * re + im * im;
#endif
}

// Device error bits (OR-ed into a flag the host reads at sync points).
enum DevErr : int { E_DIVERGED = 1, E_TIMEOUT = 2 };

// Layout: spins are padded to Np (a multiple of 128) and columns to Cp (a
// multiple of 256).  A "column" c is one real amplitude series: c = r for
// Ising, c = 2r (real part) and 2r+1 (imaginary part) for XY.  Column-major
// state: x[c * Np + i].  Per-restart arrays: y[r * Np + i].  Padding is zero
// and never written.
struct StepArgs {
  int N, Np, C, R, Cp, Rp;
  int mode;
  int cplx;
  int mt_count;          // M tiles of the launching kernel (rho / energy partials)
  float dt, eps, rho_th, eps_hat;
  float noise_D;
  int noise_decay;
  unsigned long long seed;
  unsigned int step;     // global step index n of this transition n -> n+1
  const float* psi_n;    // psi^n, FP32 [Cp][Np]
  float* psi_out;        // Euler: psi^{n+1}; RK stage 4: psi^n updated in place
  const float* xs;       // RK stage input X_s (stage 1: psi_n)
  float* xs_next;        // RK stages 1-3: X_{s+1}
  float* acc;            // RK accumulator of psi increments [Cp][Np]
  float* gam;            // gamma^n [Rp][Np] (updated in place at the end of a step)
  float* gstg;           // RK stage gains [Rp][Np]
  float* gacc;           // RK accumulator of gamma increments [Rp][Np]
  __nv_bfloat16* op_out; // BF16 copy of the next GEMM operand, or nullptr
  int op_pitch;          // row pitch (elements) of op_out; Np except in packed batches
  unsigned char* op8_out;  // E4M3 copy of the next GEMM operand (FP8 path), or nullptr
  float op8_inv;         // 1 / scale of the FP8 amplitude operand
  float* opT_out;        // sparse path: next operand, spin-major [Np][Cp] (FP32), or nullptr
  const float* opT_in;   // sparse path: this launch's operand in that layout, or nullptr
  int q;                 // resonant drive h_q conj(psi)^(q-1) of Eq. (2) (complex only; 0: none)
  float hq;
  const float* row_scale;  // FP8 path: Y_i = row_scale[i] * (J8 X8)_i, else nullptr
  const float* h1;       // drive h_1i = -g_i sqrt(rho_th), [Np]
  const float* beta_in;  // beta^n [Rp]
  float* beta_out;       // beta^{n+1} [Rp]
  const float* rho_in;   // [mt_count][Rp] partial sums of |psi^n|^2 over spins
  float* rho_out;        // [mt_count][Rp] partial sums of |psi^{n+1}|^2
  const float* g;        // field g_i [Np] (energy mode)
  float* e_part;         // [mt_count][Rp] partial energies (energy mode)
  int* err;
  unsigned long long* stamps;  // per-CTA timestamps [ctas][8], or nullptr
  long long wait_cycles;       // limit of every device-side wait (SM clock cycles)
};

// Nanosecond device clock for the optional per-CTA timestamps.
__device__ __forceinline__ void stamp(const StepArgs& a, int k) {
  if (a.stamps) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    a.stamps[(size_t(blockIdx.y) * gridDim.x + blockIdx.x) * 8 + k] = t;
  }
}

// Default limit of a device-side wait (SM clock cycles, about 2 s) and the
// cycles per second used to convert a limit given in seconds.
long long ptx_default_wait_cycles();
double ptx_cycles_per_second();

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_step_simt(const StepArgs& a, const float* J32, const float* operand, cudaStream_t s);
int simt_mtiles(int N);
// Sparse J0 (ELL [dmax][Np], ascending columns): the SIMT step with the SGEMM
// replaced by a gather over the nonzeros; same tiles and epilogue.
cudaError_t launch_step_sparse(const StepArgs& a, const int* col, const float* val, const int* deg,
                               const float* operand, int maxdeg, cudaStream_t s);
cudaError_t launch_prepare_ell(const float* J32, int N, int Np, int dmax, int* col, float* val, int* deg, int* maxdeg,
                               cudaStream_t s);
// out[i][c] = x[c][i] for c < Cp, i < Np (column-major state -> spin-major operand).
cudaError_t launch_transpose_state(const float* x, int Np, int Cp, float* out, cudaStream_t s);

// One launch of the persistent multi-step tensor-core kernel (step_tcs.cuh):
// forward-Euler steps whose buffers alternate with the step's parity.
struct SegArgs {
  int steps;                // steps of this launch
  int buf0;                 // operand buffer holding the first step's operand
  int Cp;                   // rows of one operand buffer
  unsigned* flags;          // [column blocks][128-row blocks], zero at launch
  float* psi[2];            // psi[0]: the first step's amplitudes; alternate per step
  float* beta[2];           // likewise the coupling scales
  float* rho[2];            // likewise the density partial sums (noise decay)
  __nv_bfloat16* ops;       // BF16 operand buffers [2][Cp][Np] (or nullptr)
  unsigned char* ops8;      // E4M3 operand buffers [2][Cp][Np] (FP8 path, or nullptr)
};

struct TcPlan;  // opaque plan holding the tensor maps of one context
cudaError_t tc_plan_create(TcPlan** plan, const __nv_bfloat16* J16, int Np,
                           const __nv_bfloat16* ops, int n_op_bufs, int Cp);
void tc_plan_destroy(TcPlan* plan);
// pair: two-SM tiles (cta_group::2, clusters of 2 CTAs); needs an even number
// of 128-row blocks (cudaErrorInvalidValue otherwise).
cudaError_t launch_step_tc(const TcPlan* plan, const StepArgs& a, int op_buf, cudaStream_t s, bool pair = false);
// FP8 operands (E4M3 J with per-row scales, E4M3 amplitudes at a fixed scale):
// plan over J8 [Np][Np] and ops8 [n_op_bufs * Cp][Np] (bytes).
cudaError_t tc_plan8_create(TcPlan** plan, const unsigned char* J8, int Np, const unsigned char* ops8, int n_op_bufs,
                            int Cp);
cudaError_t launch_step_tc8(const TcPlan* plan, const StepArgs& a, int op_buf, cudaStream_t s, bool pair = false);
// g.steps forward-Euler steps in one persistent launch (BF16 / FP8 plans).
cudaError_t launch_step_tcs(const TcPlan* plan, const StepArgs& a, const SegArgs& g, cudaStream_t s, bool pair);
cudaError_t launch_step_tcs8(const TcPlan* plan, const StepArgs& a, const SegArgs& g, cudaStream_t s, bool pair);
// q-state Potts projection (Sec. 1), in double: the q-th root of unity w_k = exp(2 pi i k / q)
// maximising Re(conj(w_k) psi); ties and psi = 0 go to the lowest k.  In the
// projection kernels the `cplx` argument is 0 (real spins), 1 (XY: psi / |psi|)
// or q >= 2 (Potts onto the q-th roots).
__device__ __forceinline__ void potts_project(double re, double im, int q, double& sr, double& si) {
  double bs = -DBL_MAX;
  sr = 1.0;
  si = 0.0;
  for (int k = 0; k < q; ++k) {
    double sn, cs;
    sincospi(2.0 * k / q, &sn, &cs);
    const double sc = re * cs + im * sn;
    if (sc > bs) {
      bs = sc;
      sr = cs;
      si = sn;
    }
  }
}

constexpr float kFp8PsiScale = 1.0f / 64.0f;
// J8_ij = e4m3(J32_ij / s_i), s_i = max_j |J32_ij| / 448 (1 for a zero row).
cudaError_t launch_prepare_J8(const float* J32, int Np, unsigned char* J8, float* scale, cudaStream_t s);
// GD-mod (Eq. 6 with Delta_ij = gamma_i^inj + gamma_j^inj): K[r][i][j] =
// beta0 J[i][j] for R restarts; one forward-Euler step reading gin, writing
// gout and updating K in place.
size_t gdmod_smem_bytes(int Np, bool cplx);
cudaError_t launch_gdmod_init(float* K, const float* J, float beta0, int N, int Np, int R, cudaStream_t s);
cudaError_t launch_gdmod_step(const StepArgs& a, const float* J, float* K, const float* gin, float* gout,
                              float gamma_c, float ceh, cudaStream_t s);
// y = e4m3(x / kFp8PsiScale), n elements.
cudaError_t launch_to_e4m3(const float* x, unsigned char* y, size_t n, cudaStream_t s);
int tc_mtiles(int N);
int tc_pick_bn(int N, int C);
int tc_pick_bn_pair(int N, int C);
bool tc_pair_pays(int N, int C);
bool tc_supported(int device);

}  // namespace gda
