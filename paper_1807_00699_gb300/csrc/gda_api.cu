// C ABI of the GD solver (include/gda.h): context, device memory, the step
// loop and the energy / argmin calls.  The arithmetic runs in the kernels of
// step_simt.cu, step_tc.cu and energy.cu; this file only orders launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gda.h"
#include "gda_internal.h"
#include "kernels.h"
#include "res.h"

using namespace gda;

namespace {

constexpr int kTraceCap = 1 << 16;
constexpr size_t kHistBytes = size_t(256) << 20;  // bound on the kept trace configurations
constexpr int kMaxResidentTiles = 1024;  // bound on the CTAs of a resident launch

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct gda_ctx {
  int dev = 0;
  int N = 0, Np = 0, model = 0, cplx = 0;
  cudaStream_t stream = nullptr;
  bool tc_ok = false;
  // instance
  double* J64 = nullptr;  // [Np][Np], diagonal kept
  float* J32 = nullptr;   // [Np][Np], diagonal removed
  __nv_bfloat16* J16 = nullptr;
  unsigned char* J8 = nullptr;  // [Np][Np] E4M3, row-scaled (FP8 path, on first use)
  float* jscale = nullptr;      // [Np] row scales of J8
  bool j8_ready = false;
  int* Jint = nullptr;
  double* g64 = nullptr;  // [Np]
  float* g32 = nullptr;   // [Np]
  float* h1 = nullptr;    // [Np]
  bool int_exact = false;
  double diag = 0.0;      // -sum_i J_ii
  // instance checks
  int* d_flags = nullptr;
  unsigned long long* d_maxabs = nullptr;
  double* d_diag = nullptr;
  // state
  int R = 0, C = 0, Cp = 0, Rp = 0, Rcap_cols = 0, MT = 0;
  float* psi[2] = {nullptr, nullptr};
  float* stg[2] = {nullptr, nullptr};
  float* acc = nullptr;
  float* S32 = nullptr;
  float* gam = nullptr;
  float* gstg = nullptr;
  float* gacc = nullptr;
  float* beta[2] = {nullptr, nullptr};
  float* rho[2] = {nullptr, nullptr};
  float* epart = nullptr;
  __nv_bfloat16* ops = nullptr;  // [3][Cp][Np]: operand ping-pong + projected spins
  unsigned char* ops8 = nullptr;  // [2][Cp][Np]: E4M3 operand ping-pong (FP8 path)
  TcPlan* plan8 = nullptr;
  int* ell_col = nullptr;     // sparse J0: [GDA_SPARSE_MAX_DEG][Np] column indices
  float* ell_val = nullptr;   // [GDA_SPARSE_MAX_DEG][Np] values
  int* ell_deg = nullptr;     // [Np] nonzeros per row
  int* d_maxdeg = nullptr;
  int ell_maxdeg = -1;        // largest row count of the current J (-1: not built)
  bool run_sparse = false;    // steps of the current call use the sparse product
  float* opT[3] = {nullptr, nullptr, nullptr};  // sparse: spin-major operand copies [Np][Cp]
  size_t opT_cap = 0;
  bool run_pair = false;      // tensor-core launches of the current call use two-SM tiles
  int potts_q = 0;            // q >= 2: spins project onto the q-th roots (last run's resonant drive)
  float* K = nullptr;  // GD-mod per-restart couplings [K_R][N][Np]
  size_t K_cap = 0;
  int K_R = 0;         // restarts K was initialised for (0: none)
  double* S64 = nullptr;
  int* Sint = nullptr;
  double* part64 = nullptr;
  long long* partint = nullptr;
  double* E64 = nullptr;
  double* bestE = nullptr;
  int* bestR = nullptr;
  double* E32 = nullptr;    // ranking: compensated FP32 energies [rank_cap]
  int* cidx = nullptr;      // ranking: candidate restarts [rank_cap]
  int* d_count = nullptr;
  double* d_abs = nullptr;
  int rank_cap = 0;
  double abs_sum = -1.0;    // sum |J0| + sum |g| of the current instance (-1: not computed)
  signed char* cfg8 = nullptr;
  double* cfgth = nullptr;
  long long* t_step = nullptr;
  double* t_E = nullptr;
  int* t_r = nullptr;
  int* t_count = nullptr;
  double* lastE = nullptr;     // lowest tracking energy of the latest evaluation, its restart
  int* lastR = nullptr;
  double* snapE = nullptr;     // running best of the trace: tracking energy, restart, step,
  int* snapR = nullptr;        // and the restart's amplitudes [2][Np] at that step
  long long* snapStep = nullptr;
  float* snap = nullptr;
  float* hist = nullptr;       // tracked-best amplitudes of every trace entry [hist_cap][W][Np]
  size_t hist_bytes = 0;
  int hist_run = 0;            // entries the current run keeps (<= kept capacity)
  int* d_zero = nullptr;
  int* err = nullptr;
  unsigned* flags = nullptr;  // per-tile step flags of the resident kernel
  unsigned* seg_flags = nullptr;  // per-tile step flags of the persistent streaming kernel
  size_t seg_flags_cap = 0;
  TcPlan* plan = nullptr;
  int cur = 0, bcur = 0, rcur = 0, opcur = 0;
  long long step = 0;
  bool have_state = false;
  long long launches = 0;
  double* fw[2] = {nullptr, nullptr};    // feature scratch [Np]
  float* base = nullptr;                 // per-spin base amplitude (re, im) for init_mode 3
  unsigned long long* stamps = nullptr;  // per-CTA timestamps of the last step launch
  int stamp_cap = 0;
  std::string msg;
};

namespace {

// Spin projection of the energy kernels: 0 real, 1 XY (psi / |psi|), q >= 2
// the q-th roots of unity (the last run's resonant drive).
int pmode(const gda_ctx* c) { return c->cplx ? (c->potts_q >= 2 ? c->potts_q : 1) : 0; }

gda_status fail(gda_ctx* c, gda_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->msg = buf;
  return s;
}

gda_status cuda_fail(gda_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? GDA_ERR_OOM : GDA_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(expr)                                            \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
  } while (0)

#define LK(expr)                                            \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    ++c->launches;                                          \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_state(gda_ctx* c) {
  for (int k = 0; k < 2; ++k) {
    dfree(c->psi[k]);
    dfree(c->stg[k]);
    dfree(c->beta[k]);
    dfree(c->rho[k]);
  }
  dfree(c->acc); dfree(c->S32); dfree(c->gam); dfree(c->gstg); dfree(c->gacc); dfree(c->epart);
  dfree(c->ops); dfree(c->S64); dfree(c->Sint); dfree(c->part64); dfree(c->partint); dfree(c->E64);
  if (c->plan) tc_plan_destroy(c->plan);
  c->plan = nullptr;
  dfree(c->ops8);
  if (c->plan8) tc_plan_destroy(c->plan8);
  c->plan8 = nullptr;
  c->R = c->C = c->Cp = c->Rp = c->Rcap_cols = 0;
  c->have_state = false;
}

// Allocates (or keeps) the state for R restarts; padding stays zero.
gda_status ensure_state(gda_ctx* c, int R) {
  const int C = c->cplx ? 2 * R : R;
  if (c->Rcap_cols >= C && c->psi[0]) {
    c->R = R;
    c->C = C;
    return GDA_OK;
  }
  free_state(c);
  const size_t Cp = round_up(C, 256), Np = c->Np;
  const size_t Rp = round_up(R, 256);
  const size_t MT = (c->N + 63) / 64;
  const size_t cn = Cp * Np, rn = Rp * Np;
  for (int k = 0; k < 2; ++k) {
    CK(dalloc(&c->psi[k], cn));
    CK(dalloc(&c->stg[k], cn));
    CK(dalloc(&c->beta[k], Rp));
    CK(dalloc(&c->rho[k], MT * Rp));
  }
  CK(dalloc(&c->acc, cn));
  CK(dalloc(&c->S32, cn));
  CK(dalloc(&c->gam, rn));
  CK(dalloc(&c->gstg, rn));
  CK(dalloc(&c->gacc, rn));
  CK(dalloc(&c->epart, MT * Rp));
  CK(dalloc(&c->S64, cn));
  CK(dalloc(&c->part64, MT * Rp));
  CK(dalloc(&c->E64, Rp));
  if (c->int_exact || c->model == GDA_ISING) {
    CK(dalloc(&c->Sint, cn));
    CK(dalloc(&c->partint, MT * Rp));
  }
  float* zf[] = {c->psi[0], c->psi[1], c->stg[0], c->stg[1], c->acc, c->S32};
  for (float* p : zf) CK(cudaMemsetAsync(p, 0, cn * sizeof(float), c->stream));
  CK(cudaMemsetAsync(c->S64, 0, cn * sizeof(double), c->stream));
  if (c->Sint) CK(cudaMemsetAsync(c->Sint, 0, cn * sizeof(int), c->stream));
  CK(cudaMemsetAsync(c->gam, 0, rn * sizeof(float), c->stream));
  CK(cudaMemsetAsync(c->gstg, 0, rn * sizeof(float), c->stream));
  CK(cudaMemsetAsync(c->gacc, 0, rn * sizeof(float), c->stream));
  if (c->tc_ok) {
    CK(dalloc(&c->ops, 3 * cn));
    CK(cudaMemsetAsync(c->ops, 0, 3 * cn * sizeof(__nv_bfloat16), c->stream));
    CK(tc_plan_create(&c->plan, c->J16, int(Np), c->ops, 3, int(Cp)));
  }
  c->R = R;
  c->C = C;
  c->Cp = int(Cp);
  c->Rp = int(Rp);
  c->MT = int(MT);
  c->Rcap_cols = int(Cp);
  return GDA_OK;
}

// Uploads J (N x N, row-major) and g into the padded FP64 copies, checks the
// instance on the device and derives the coupling operands.
gda_status load_instance(gda_ctx* c, const double* J, const double* g, cudaMemcpyKind kind) {
  const size_t Np = c->Np, N = c->N;
  CK(cudaMemsetAsync(c->J64, 0, Np * Np * sizeof(double), c->stream));
  CK(cudaMemcpy2DAsync(c->J64, Np * sizeof(double), J, N * sizeof(double), N * sizeof(double), N, kind, c->stream));
  CK(cudaMemsetAsync(c->g64, 0, Np * sizeof(double), c->stream));
  if (g) CK(cudaMemcpyAsync(c->g64, g, N * sizeof(double), kind, c->stream));
  c->K_R = 0;  // a GD-mod coupling state belongs to the previous J
  LK(launch_snapshot_reset(c->snapE, c->snapR, c->snapStep, c->stream));
  c->ell_maxdeg = -1;
  c->abs_sum = -1.0;
  CK(cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  CK(cudaMemsetAsync(c->d_maxabs, 0, sizeof(unsigned long long), c->stream));
  LK(launch_check_instance(c->J64, c->g64, c->N, c->Np, c->d_flags, c->d_maxabs, c->d_diag, c->stream));
  int flags = 0;
  unsigned long long mbits = 0;
  CK(cudaMemcpyAsync(&flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&mbits, c->d_maxabs, sizeof(mbits), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&c->diag, c->d_diag, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flags & 1) return fail(c, GDA_ERR_INVALID, "J has a non-finite entry");
  if (flags & 2) return fail(c, GDA_ERR_INVALID, "J is not symmetric");
  if (flags & 8) return fail(c, GDA_ERR_INVALID, "g has a non-finite entry");
  double maxabs;
  std::memcpy(&maxabs, &mbits, sizeof(maxabs));
  const bool was_int = c->int_exact;
  c->int_exact = c->model == GDA_ISING && !(flags & 4) && !(flags & 16) && maxabs * double(N) < 2147483647.0;
  if (c->int_exact && !c->Jint) CK(dalloc(&c->Jint, Np * Np));
  if (c->int_exact && !was_int && c->psi[0] && !c->Sint) {
    CK(dalloc(&c->Sint, size_t(c->Cp) * Np));
    CK(cudaMemsetAsync(c->Sint, 0, size_t(c->Cp) * Np * sizeof(int), c->stream));
    CK(dalloc(&c->partint, size_t(c->MT) * c->Rp));
  }
  LK(launch_prepare_J(c->J64, c->Np, c->J32, c->J16, c->int_exact ? c->Jint : nullptr, c->stream));
  c->j8_ready = false;
  return GDA_OK;
}

// Sparse J0 on first use: the ELL table of the nonzeros (at most
// GDA_SPARSE_MAX_DEG per row).  Synchronises once to read the largest count.
gda_status ensure_ell(gda_ctx* c) {
  const size_t Np = c->Np;
  if (!c->ell_col) {
    CK(dalloc(&c->ell_col, size_t(GDA_SPARSE_MAX_DEG) * Np));
    CK(dalloc(&c->ell_val, size_t(GDA_SPARSE_MAX_DEG) * Np));
    CK(dalloc(&c->ell_deg, Np));
    CK(dalloc(&c->d_maxdeg, 1));
  }
  if (c->ell_maxdeg < 0) {
    CK(cudaMemsetAsync(c->ell_col, 0, size_t(GDA_SPARSE_MAX_DEG) * Np * sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->ell_val, 0, size_t(GDA_SPARSE_MAX_DEG) * Np * sizeof(float), c->stream));
    CK(cudaMemsetAsync(c->d_maxdeg, 0, sizeof(int), c->stream));
    LK(launch_prepare_ell(c->J32, c->N, int(Np), GDA_SPARSE_MAX_DEG, c->ell_col, c->ell_val, c->ell_deg,
                          c->d_maxdeg, c->stream));
    int m = 0;
    CK(cudaMemcpyAsync(&m, c->d_maxdeg, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->ell_maxdeg = m;
  }
  if (c->ell_maxdeg > GDA_SPARSE_MAX_DEG)
    return fail(c, GDA_ERR_UNSUPPORTED, "J has %d nonzeros in a row; the sparse product takes at most %d",
                c->ell_maxdeg, GDA_SPARSE_MAX_DEG);
  return GDA_OK;
}

// FP8 operands on first use: row-scaled E4M3 couplings, the E4M3 operand
// buffers of the current state and their tensor maps.
gda_status ensure_fp8(gda_ctx* c) {
  const size_t Np = c->Np;
  if (!c->J8) {
    CK(dalloc(&c->J8, Np * Np));
    CK(dalloc(&c->jscale, Np));
  }
  if (!c->j8_ready) {
    LK(launch_prepare_J8(c->J32, int(Np), c->J8, c->jscale, c->stream));
    c->j8_ready = true;
  }
  if (!c->ops8) {
    const size_t cn = size_t(c->Cp) * Np;
    CK(dalloc(&c->ops8, 2 * cn));
    CK(cudaMemsetAsync(c->ops8, 0, 2 * cn, c->stream));
    CK(tc_plan8_create(&c->plan8, c->J8, int(Np), c->ops8, 2, c->Cp));
  }
  return GDA_OK;
}

bool finite(double x) { return std::isfinite(x); }

gda_status check_params(gda_ctx* c, const gda_params* p) {
  if (!p) return fail(c, GDA_ERR_INVALID, "params is NULL");
  if (p->integ != GDA_EULER && p->integ != GDA_RK4) return fail(c, GDA_ERR_INVALID, "unknown integrator %d", p->integ);
  if (p->prec != GDA_FP32 && p->prec != GDA_BF16 && p->prec != GDA_FP8 && p->prec != GDA_SPARSE)
    return fail(c, GDA_ERR_INVALID, "unknown precision %d", p->prec);
  const double v[] = {p->dt, p->eps, p->rho_th, p->gamma0, p->beta0, p->eps_hat, p->noise_D, p->init_amp};
  for (double x : v)
    if (!finite(x)) return fail(c, GDA_ERR_INVALID, "non-finite parameter");
  if (!(p->dt > 0)) return fail(c, GDA_ERR_INVALID, "dt must be > 0");
  if (!(p->rho_th > 0)) return fail(c, GDA_ERR_INVALID, "rho_th must be > 0");
  if (p->noise_D < 0) return fail(c, GDA_ERR_INVALID, "noise_D must be >= 0");
  if (p->init_mode < 0 || p->init_mode > 3) return fail(c, GDA_ERR_INVALID, "init_mode must be 0, 1, 2 or 3");
  if (p->init_mode == 3 && !c->base) return fail(c, GDA_ERR_STATE, "init_mode 3 needs gda_set_init_base first");
  if (p->energy_every < 0) return fail(c, GDA_ERR_INVALID, "energy_every must be >= 0");
  if (p->schedule < GDA_SCHEDULE_AUTO || p->schedule > GDA_SCHEDULE_RESIDENT_PAIR)
    return fail(c, GDA_ERR_INVALID, "unknown schedule %d", p->schedule);
  if ((p->prec == GDA_BF16 || p->prec == GDA_FP8) && !c->tc_ok)
    return fail(c, GDA_ERR_UNSUPPORTED, "tensor-core path needs an sm_103 device");
  const bool res_sched = p->schedule == GDA_SCHEDULE_RESIDENT || p->schedule == GDA_SCHEDULE_RESIDENT_PAIR;
  if (p->prec == GDA_SPARSE && res_sched)
    return fail(c, GDA_ERR_UNSUPPORTED, "the sparse product runs per step");
  if ((p->schedule == GDA_SCHEDULE_PAIR || p->schedule == GDA_SCHEDULE_STREAM_PAIR) &&
      (!(p->prec == GDA_BF16 || p->prec == GDA_FP8) || (c->Np / 128) % 2 != 0 || p->coupling != GDA_COUPLING_GD))
    return fail(c, GDA_ERR_UNSUPPORTED, "two-SM tiles need BF16 or FP8 and an even number of 128-row blocks");
  if ((p->schedule == GDA_SCHEDULE_STREAM || p->schedule == GDA_SCHEDULE_STREAM_PAIR) &&
      (!(p->prec == GDA_BF16 || p->prec == GDA_FP8) || p->integ != GDA_EULER || p->coupling != GDA_COUPLING_GD))
    return fail(c, GDA_ERR_UNSUPPORTED, "the streaming schedule runs forward-Euler BF16 / FP8 steps");
  if (p->q != 0 && (p->q < 2 || p->q > 16)) return fail(c, GDA_ERR_INVALID, "q must be 0 or 2..16");
  if (!finite(p->wait_s) || p->wait_s < 0 || p->wait_s > 1e3)
    return fail(c, GDA_ERR_INVALID, "wait_s must be in [0, 1000] seconds");
  if (p->withhold_flag < 0) return fail(c, GDA_ERR_INVALID, "withhold_flag must be >= 0");
  if (!finite(p->hq)) return fail(c, GDA_ERR_INVALID, "non-finite hq");
  if (p->q != 0 && (!c->cplx || res_sched || p->coupling == GDA_COUPLING_GDMOD))
    return fail(c, GDA_ERR_UNSUPPORTED, "the resonant drive needs complex amplitudes (GDA_XY) and per-step GD");
  if (p->coupling != GDA_COUPLING_GD && p->coupling != GDA_COUPLING_GDMOD)
    return fail(c, GDA_ERR_INVALID, "unknown coupling mode %d", p->coupling);
  if (p->coupling == GDA_COUPLING_GDMOD) {
    if (!finite(p->gamma_c)) return fail(c, GDA_ERR_INVALID, "non-finite gamma_c");
    if (p->prec != GDA_FP32 || p->integ != GDA_EULER || res_sched)
      return fail(c, GDA_ERR_UNSUPPORTED, "GD-mod runs FP32 forward Euler, per step");
    if (p->noise_D != 0.0 && p->noise_decay) return fail(c, GDA_ERR_UNSUPPORTED, "GD-mod has no noise decay");
    if (gdmod_smem_bytes(c->Np, c->cplx) > 227 * 1024) return fail(c, GDA_ERR_UNSUPPORTED, "N too large for GD-mod");
  }
  return GDA_OK;
}

StepArgs base_args(gda_ctx* c, const gda_params* p, bool tc) {
  StepArgs a{};
  a.N = c->N; a.Np = c->Np; a.C = c->C; a.R = c->R; a.Cp = c->Cp; a.Rp = c->Rp;
  a.op_pitch = c->Np;
  a.cplx = c->cplx;
  a.mt_count = tc ? tc_mtiles(c->N) : simt_mtiles(c->N);
  a.dt = float(p->dt); a.eps = float(p->eps); a.rho_th = float(p->rho_th); a.eps_hat = float(p->eps_hat);
  a.noise_D = float(p->noise_D);
  a.q = c->cplx ? p->q : 0;
  a.hq = float(p->hq);
  a.noise_decay = p->noise_decay ? 1 : 0;
  a.seed = p->seed;
  a.acc = c->acc; a.gam = c->gam; a.gstg = c->gstg; a.gacc = c->gacc;
  a.h1 = c->h1;
  a.g = c->g32;
  a.e_part = c->epart;
  a.err = c->err;
  const long long ctas = (long long)((c->C + 127) / 128) * ((c->N + 127) / 128);
  a.stamps = (c->stamps && tc && ctas <= c->stamp_cap) ? c->stamps : nullptr;
  a.wait_cycles = p->wait_s > 0 ? (long long)(p->wait_s * ptx_cycles_per_second()) : ptx_default_wait_cycles();
  return a;
}

gda_status launch_step(gda_ctx* c, const StepArgs& a, bool tc, const float* operand32, int op_buf) {
  if (c->run_sparse && !tc) {
    LK(launch_step_sparse(a, c->ell_col, c->ell_val, c->ell_deg, operand32, c->ell_maxdeg, c->stream));
  } else if (a.row_scale) {
    LK(launch_step_tc8(c->plan8, a, op_buf, c->stream, c->run_pair));
  } else if (tc) {
    LK(launch_step_tc(c->plan, a, op_buf, c->stream, c->run_pair));
  } else {
    LK(launch_step_simt(a, c->J32, operand32, c->stream));
  }
  return GDA_OK;
}

// One tracking evaluation of the projected spins of psi[cur].
gda_status track(gda_ctx* c, const gda_params* p, bool tc, long long step) {
  StepArgs a = base_args(c, p, tc);
  a.mode = M_ENERGY;
  a.psi_n = c->psi[c->cur];
  a.beta_in = c->beta[c->bcur];
  if (tc) {
    LK(launch_project_bf16(c->psi[c->cur], c->ops + size_t(2) * c->Cp * c->Np, c->N, c->Np, c->R, pmode(c),
                           c->stream));
  } else {
    LK(launch_project_f32(c->psi[c->cur], c->S32, c->N, c->Np, c->R, pmode(c), c->stream));
  }
  gda_status s = launch_step(c, a, tc, c->S32, 2);
  if (s != GDA_OK) return s;
  LK(launch_track_reduce(c->epart, a.mt_count, c->R, c->Rp, c->diag, step, c->t_step, c->t_E, c->t_r, kTraceCap,
                         c->t_count, c->lastE, c->lastR, c->stream));
  LK(launch_snapshot(c->psi[c->cur], c->Np, c->cplx ? 2 : 1, c->lastE, c->lastR, step, c->snapE, c->snapR,
                     c->snapStep, c->snap, c->hist, c->hist_run, c->t_count, c->stream));
  return GDA_OK;
}

// GD-mod (Sec. 2): one K-streaming launch per step, FP32, forward Euler.
gda_status run_gdmod(gda_ctx* c, const gda_params* p, int R, int64_t steps) {
  const size_t need = size_t(R) * c->N * c->Np;
  const long long nrb = (c->N + 31) / 32;
  if (nrb * R >= (1LL << 31)) return fail(c, GDA_ERR_UNSUPPORTED, "too many GD-mod row blocks");
  if (p->init_mode == 2) {
    if (!c->K || c->K_R != R) return fail(c, GDA_ERR_STATE, "GD-mod continuation needs a GD-mod state with the same R");
  } else {
    if (c->K_cap < need) {
      dfree(c->K);
      c->K_cap = 0;
      CK(dalloc(&c->K, need));
      c->K_cap = need;
    }
    LK(launch_gdmod_init(c->K, c->J32, float(p->beta0), c->N, c->Np, R, c->stream));
    c->K_R = R;
  }
  const StepArgs base = base_args(c, p, false);
  const float ceh = float(p->dt * p->eps_hat);
  for (int64_t k = 0; k < steps; ++k) {
    const long long n = c->step + k;
    StepArgs a = base;
    a.step = static_cast<unsigned int>(n);
    a.psi_n = c->psi[c->cur];
    a.psi_out = c->psi[c->cur ^ 1];
    a.beta_in = c->beta[c->bcur];
    LK(launch_gdmod_step(a, c->J32, c->K, c->gam, c->gstg, float(p->gamma_c), ceh, c->stream));
    std::swap(c->gam, c->gstg);
    c->cur ^= 1;
    if (p->energy_every > 0 && (k + 1) % p->energy_every == 0) {
      gda_status s = track(c, p, false, n + 1);
      if (s != GDA_OK) return s;
    }
  }
  c->step += steps;
  return GDA_OK;
}

gda_status compute_energies(gda_ctx* c) {
  if (!c->have_state) return fail(c, GDA_ERR_STATE, "no state: call gda_run or gda_set_state first");
  if (c->int_exact) {
    LK(launch_energy_int(c->psi[c->cur], c->Jint, c->Sint, c->partint, c->E64, c->N, c->Np, c->R, c->Rp, c->C,
                         c->stream));
  } else {
    LK(launch_energy64(c->psi[c->cur], c->J64, c->g64, c->S64, c->part64, c->E64, c->N, c->Np, c->R, c->Rp, c->C,
                       pmode(c), c->stream));
  }
  return GDA_OK;
}

gda_status check_err(gda_ctx* c) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (e) {
    CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (e & E_TIMEOUT) return fail(c, GDA_ERR_TIMEOUT, "a device-side wait timed out");
    return fail(c, GDA_ERR_DIVERGED, "non-finite or overflowing amplitude");
  }
  return GDA_OK;
}

}  // namespace

extern "C" {

void gda_default_params(gda_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->integ = GDA_EULER;
  p->prec = GDA_FP32;
  p->dt = 0.01;
  p->eps = 0.1;
  p->rho_th = 1.0;
  p->gamma0 = 0.0;
  p->beta0 = 1.0;
  p->eps_hat = 0.0;
  p->noise_D = 0.0;
  p->noise_decay = 0;
  p->energy_every = 0;
  p->seed = 0;
  p->init_mode = 1;
  p->init_amp = 1e-3;
  p->coupling = GDA_COUPLING_GD;
  p->gamma_c = 1.0;
  p->q = 0;
  p->hq = 0.0;
}

const char* gda_status_string(gda_status s) {
  switch (s) {
    case GDA_OK: return "ok";
    case GDA_ERR_INVALID: return "invalid argument";
    case GDA_ERR_CUDA: return "CUDA error";
    case GDA_ERR_OOM: return "out of device memory";
    case GDA_ERR_DIVERGED: return "amplitudes diverged";
    case GDA_ERR_TIMEOUT: return "device wait timed out";
    case GDA_ERR_UNSUPPORTED: return "unsupported on this device";
    case GDA_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* gda_last_error(const gda_ctx* c) { return c ? c->msg.c_str() : "NULL context"; }

int64_t gda_kernel_launches(const gda_ctx* c) { return c ? c->launches : 0; }

void gda_destroy(gda_ctx* c) {
  if (!c) return;
  free_state(c);
  dfree(c->J64); dfree(c->J32); dfree(c->J16); dfree(c->J8); dfree(c->jscale); dfree(c->Jint); dfree(c->g64); dfree(c->g32); dfree(c->h1);
  dfree(c->d_flags); dfree(c->d_maxabs); dfree(c->d_diag);
  dfree(c->bestE); dfree(c->bestR); dfree(c->cfg8); dfree(c->cfgth);
  dfree(c->E32); dfree(c->cidx); dfree(c->d_count); dfree(c->d_abs);
  dfree(c->t_step); dfree(c->t_E); dfree(c->t_r); dfree(c->t_count); dfree(c->err); dfree(c->flags);
  dfree(c->seg_flags);
  dfree(c->lastE); dfree(c->lastR); dfree(c->snapE); dfree(c->snapR); dfree(c->snapStep); dfree(c->snap);
  dfree(c->hist);
  dfree(c->d_zero);
  dfree(c->stamps);
  dfree(c->K);
  dfree(c->ell_col); dfree(c->ell_val); dfree(c->ell_deg); dfree(c->d_maxdeg);
  for (float*& t : c->opT) dfree(t);
  dfree(c->fw[0]);
  dfree(c->fw[1]);
  dfree(c->base);
  delete c;
}

static gda_status create_impl(const double* J, const double* g, int32_t N, int32_t model, gda_ctx** out,
                              cudaMemcpyKind kind) {
  if (!out) return GDA_ERR_INVALID;
  *out = nullptr;
  if (!J || N < 1 || N > 65536 || (model != GDA_ISING && model != GDA_XY)) return GDA_ERR_INVALID;
  if (kind == cudaMemcpyHostToDevice) {
    // host-side screening of the cheap conditions before any allocation
    for (int64_t k = 0; k < int64_t(N) * N; ++k)
      if (!std::isfinite(J[k])) return GDA_ERR_INVALID;
    for (int32_t i = 0; i < N; ++i)
      for (int32_t j = i + 1; j < N; ++j)
        if (J[int64_t(i) * N + j] != J[int64_t(j) * N + i]) return GDA_ERR_INVALID;
    if (g)
      for (int32_t i = 0; i < N; ++i)
        if (!std::isfinite(g[i])) return GDA_ERR_INVALID;
  }
  gda_ctx* c = new gda_ctx();
  c->N = N;
  c->Np = int(round_up(N, 128));
  c->model = model;
  c->cplx = model == GDA_XY;
  if (cudaGetDevice(&c->dev) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return GDA_ERR_CUDA;
  }
  c->tc_ok = tc_supported(c->dev);
  const size_t Np = c->Np;
  gda_status st = GDA_OK;
  auto step = [&](cudaError_t e) {
    if (st == GDA_OK && e != cudaSuccess) st = cuda_fail(c, e, "gda_create allocation");
  };
  step(dalloc(&c->J64, Np * Np));
  step(dalloc(&c->J32, Np * Np));
  if (c->tc_ok) step(dalloc(&c->J16, Np * Np));
  step(dalloc(&c->g64, Np));
  step(dalloc(&c->g32, Np));
  step(dalloc(&c->h1, Np));
  step(dalloc(&c->d_flags, 1));
  step(dalloc(&c->d_maxabs, 1));
  step(dalloc(&c->d_diag, 1));
  step(dalloc(&c->bestE, 1));
  step(dalloc(&c->bestR, 1));
  step(dalloc(&c->cfg8, Np));
  step(dalloc(&c->cfgth, Np));
  step(dalloc(&c->t_step, kTraceCap));
  step(dalloc(&c->t_E, kTraceCap));
  step(dalloc(&c->t_r, kTraceCap));
  step(dalloc(&c->t_count, 1));
  step(dalloc(&c->lastE, 1));
  step(dalloc(&c->lastR, 1));
  step(dalloc(&c->snapE, 1));
  step(dalloc(&c->snapR, 1));
  step(dalloc(&c->snapStep, 1));
  step(dalloc(&c->snap, 2 * Np));
  step(dalloc(&c->d_zero, 1));
  step(dalloc(&c->err, 1));
  step(dalloc(&c->flags, kMaxResidentTiles));
  if (st == GDA_OK) step(cudaMemset(c->err, 0, sizeof(int)));
  if (st == GDA_OK) step(cudaMemset(c->t_count, 0, sizeof(int)));
  if (st == GDA_OK) step(cudaMemset(c->d_zero, 0, sizeof(int)));
  if (st == GDA_OK) step(cudaMemset(c->snap, 0, 2 * Np * sizeof(float)));
  if (st == GDA_OK) step(cudaMemset(c->h1, 0, Np * sizeof(float)));
  if (st == GDA_OK) step(cudaMemset(c->g32, 0, Np * sizeof(float)));
  if (st == GDA_OK) st = load_instance(c, J, g, kind);
  if (st != GDA_OK) {
    gda_destroy(c);
    return st;
  }
  *out = c;
  return GDA_OK;
}

gda_status gda_create(const double* J, const double* g, int32_t N, int32_t model, gda_ctx** out) {
  return create_impl(J, g, N, model, out, cudaMemcpyHostToDevice);
}

static gda_status load_common(gda_ctx* c, const double* J, const double* g, cudaMemcpyKind kind) {
  if (!c) return GDA_ERR_INVALID;
  if (!J) return fail(c, GDA_ERR_INVALID, "J is NULL");
  gda_status s = load_instance(c, J, g, kind);
  if (s == GDA_OK) c->have_state = false;
  return s;
}

gda_status gda_load(gda_ctx* c, const double* J, const double* g) {
  return load_common(c, J, g, cudaMemcpyHostToDevice);
}

gda_status gda_load_dev(gda_ctx* c, const double* J_dev, const double* g_dev) {
  return load_common(c, J_dev, g_dev, cudaMemcpyDeviceToDevice);
}

gda_status gda_set_stream(gda_ctx* c, void* stream) {
  if (!c) return GDA_ERR_INVALID;
  c->stream = static_cast<cudaStream_t>(stream);
  return GDA_OK;
}

gda_status gda_run(gda_ctx* c, const gda_params* p, int32_t R, int64_t steps) {
  if (!c) return GDA_ERR_INVALID;
  gda_status s = check_params(c, p);
  if (s != GDA_OK) return s;
  if (R < 1) return fail(c, GDA_ERR_INVALID, "R must be >= 1");
  if (steps < 0) return fail(c, GDA_ERR_INVALID, "steps must be >= 0");
  if (size_t(c->cplx ? 2 : 1) * size_t(R) > size_t(1) << 24) return fail(c, GDA_ERR_INVALID, "R too large");
  const bool tc = p->prec == GDA_BF16 || p->prec == GDA_FP8;
  const bool f8 = p->prec == GDA_FP8;
  c->run_sparse = false;
  c->run_pair = p->schedule == GDA_SCHEDULE_PAIR || p->schedule == GDA_SCHEDULE_STREAM_PAIR;
  c->potts_q = (c->cplx && p->q >= 2) ? p->q : 0;
  if (p->prec == GDA_SPARSE && p->coupling != GDA_COUPLING_GDMOD) {
    s = ensure_ell(c);
    if (s != GDA_OK) return s;
    c->run_sparse = true;
  }
  if (p->init_mode == 2) {
    if (!c->have_state || c->R != R) return fail(c, GDA_ERR_STATE, "init_mode 2 needs a state with the same R");
  } else {
    s = ensure_state(c, R);
    if (s != GDA_OK) return s;
    LK(launch_init_state(c->psi[0], c->gam, c->beta[0], c->N, c->Np, R, c->cplx, p->init_mode, float(p->init_amp),
                         float(p->gamma0), float(p->beta0), p->seed, c->base, c->stream));
    c->cur = 0;
    c->bcur = 0;
    c->step = 0;
    c->have_state = true;
    LK(launch_snapshot_reset(c->snapE, c->snapR, c->snapStep, c->stream));
  }
  CK(cudaMemsetAsync(c->t_count, 0, sizeof(int), c->stream));
  // keep the tracked-best configuration of every trace entry of this run
  c->hist_run = 0;
  if (p->energy_every > 0 && steps >= p->energy_every) {
    const size_t row = size_t(c->cplx ? 2 : 1) * c->Np * sizeof(float);
    const size_t want = std::min<size_t>(size_t(steps / p->energy_every), size_t(kTraceCap));
    const size_t n = std::min(want, kHistBytes / row);
    if (c->hist_bytes < n * row) {
      dfree(c->hist);
      c->hist_bytes = 0;
      CK(dalloc(reinterpret_cast<unsigned char**>(&c->hist), n * row));
      c->hist_bytes = n * row;
    }
    c->hist_run = int(n);
  }
  LK(launch_fill_h1(c->g64, c->h1, c->N, float(std::sqrt(p->rho_th)), c->stream));
  // field in FP32 for the tracking energy
  LK(launch_fill_h1(c->g64, c->g32, c->N, -1.0f, c->stream));
  if (p->coupling == GDA_COUPLING_GDMOD) return run_gdmod(c, p, R, steps);
  const size_t cn = size_t(c->Cp) * c->Np;
  c->opcur = 0;
  if (f8) {
    s = ensure_fp8(c);
    if (s != GDA_OK) return s;
    LK(launch_to_e4m3(c->psi[c->cur], c->ops8, cn, c->stream));
  } else if (tc) {
    LK(launch_to_bf16(c->psi[c->cur], c->ops, cn, c->stream));
  }
  const bool decay = p->noise_D != 0.0 && p->noise_decay;
  c->rcur = 0;
  if (decay) LK(launch_rho_partials(tc, c->psi[c->cur], c->N, c->Np, c->R, c->Rp, c->cplx, c->rho[0], c->stream));

  // sparse product: the gathers read a spin-major copy of the operand (the 4
  // columns of a thread's quad in one 16-byte load), kept in step by the epilogue
  int tcur = 0;
  if (c->run_sparse) {
    const size_t tn = size_t(c->Np) * c->Cp;
    if (c->opT_cap < tn) {
      for (float*& t : c->opT) dfree(t);
      c->opT_cap = 0;
      for (float*& t : c->opT) CK(dalloc(&t, tn));
      c->opT_cap = tn;
    }
    LK(launch_transpose_state(c->psi[c->cur], c->Np, c->Cp, c->opT[0], c->stream));
  }
  StepArgs base = base_args(c, p, tc);
  if (f8) {
    base.row_scale = c->jscale;
    base.op8_inv = 1.0f / kFp8PsiScale;
  }
  const size_t opsz = cn;
  // Resident persistent kernel: BF16 Euler runs whose tiles all fit on the
  // device at once run as one launch per tracking segment.
  const bool res_sched = p->schedule == GDA_SCHEDULE_AUTO || p->schedule == GDA_SCHEDULE_RESIDENT ||
                         p->schedule == GDA_SCHEDULE_RESIDENT_PAIR;
  const bool resident = p->prec == GDA_BF16 && p->integ == GDA_EULER && p->q == 0 && res_sched &&
                        res_fits(c->N, c->C, c->dev) &&
                        (long long)((c->C + 127) / 128) * ((c->N + 127) / 128) <= kMaxResidentTiles;
  if ((p->schedule == GDA_SCHEDULE_RESIDENT || p->schedule == GDA_SCHEDULE_RESIDENT_PAIR) && !resident)
    return fail(c, GDA_ERR_UNSUPPORTED, "resident schedule needs BF16, Euler and a grid that fits the device");
  // two-SM tiles in the resident kernel: on request
  const bool res_pair = resident && p->schedule == GDA_SCHEDULE_RESIDENT_PAIR;
  if (res_pair && !res_pair_fits(c->N, c->C))
    return fail(c, GDA_ERR_UNSUPPORTED, "two-SM resident tiles need an even number of 128-row blocks and room for every cluster");
  if (tc && !resident && (p->schedule == GDA_SCHEDULE_AUTO || p->schedule == GDA_SCHEDULE_STREAM) &&
      tc_pair_pays(c->N, c->C))
    c->run_pair = true;
  // persistent streaming launches: one per tracking segment, steps ordered by
  // tile flags.  AUTO takes them for Euler runs whose coupling operand fits
  // well inside L2 (the column-major tile order re-reads J from L2 for every
  // column block; measured 13 % faster per step at N = R = 4096, 4 % slower at
  // N = R = 8192, whose BF16 J is larger than L2)
  const size_t j_bytes = size_t(c->Np) * c->Np * (f8 ? 1 : 2);
  const bool stream_auto = tc && !resident && p->schedule == GDA_SCHEDULE_AUTO && p->integ == GDA_EULER &&
                           j_bytes <= (size_t(48) << 20);
  if (tc && (stream_auto || p->schedule == GDA_SCHEDULE_STREAM || p->schedule == GDA_SCHEDULE_STREAM_PAIR)) {
    const size_t nflags = size_t((c->C + 127) / 128) * size_t((c->N + 127) / 128);
    if (c->seg_flags_cap < nflags) {
      dfree(c->seg_flags);
      c->seg_flags_cap = 0;
      CK(dalloc(&c->seg_flags, nflags));
      c->seg_flags_cap = nflags;
    }
    const int64_t seg = p->energy_every > 0 ? p->energy_every : steps;
    for (int64_t k = 0; k < steps; k += seg) {
      const int64_t len = std::min<int64_t>(seg, steps - k);
      const int flip = int(len & 1);
      StepArgs a = base;
      a.mode = M_EULER;
      a.step = static_cast<unsigned int>(c->step + k);
      a.psi_n = c->psi[c->cur];
      a.xs = c->psi[c->cur];
      a.psi_out = c->psi[c->cur ^ 1];
      a.beta_in = c->beta[c->bcur];
      a.beta_out = c->beta[c->bcur ^ 1];
      a.rho_in = c->rho[c->rcur];
      a.rho_out = decay ? c->rho[c->rcur ^ 1] : nullptr;
      SegArgs g{};
      g.steps = int(len);
      g.buf0 = c->opcur;
      g.Cp = c->Cp;
      g.flags = c->seg_flags;
      g.psi[0] = c->psi[c->cur];
      g.psi[1] = c->psi[c->cur ^ 1];
      g.beta[0] = c->beta[c->bcur];
      g.beta[1] = c->beta[c->bcur ^ 1];
      g.rho[0] = c->rho[c->rcur];
      g.rho[1] = c->rho[c->rcur ^ 1];
      g.ops = f8 ? nullptr : c->ops;
      g.ops8 = f8 ? c->ops8 : nullptr;
      CK(cudaMemsetAsync(c->seg_flags, 0, nflags * sizeof(unsigned), c->stream));
      LK(f8 ? launch_step_tcs8(c->plan8, a, g, c->stream, c->run_pair)
            : launch_step_tcs(c->plan, a, g, c->stream, c->run_pair));
      c->cur ^= flip;
      c->bcur ^= flip;
      c->opcur ^= flip;
      if (decay) c->rcur ^= flip;
      if (p->energy_every > 0 && len == seg) {
        s = track(c, p, tc, c->step + k + len);
        if (s != GDA_OK) return s;
      }
    }
    c->step += steps;
    return GDA_OK;
  }
  if (resident) {
    const int64_t seg = p->energy_every > 0 ? p->energy_every : steps;
    for (int64_t k = 0; k < steps; k += seg) {
      const int64_t len = std::min<int64_t>(seg, steps - k);
      const int flip = int(len & 1);
      StepArgs a = base;
      a.mode = M_EULER;
      a.step = static_cast<unsigned int>(c->step + k);
      a.psi_n = c->psi[c->cur];
      a.beta_in = c->beta[c->bcur];
      ResArgs ra{};
      ra.steps = int(len);
      ra.buf0 = c->opcur;
      ra.Cp = c->Cp;
      ra.flags = c->flags;
      ra.psi_final = c->psi[c->cur ^ flip];
      ra.beta_final = c->beta[c->bcur ^ flip];
      ra.rho[0] = c->rho[c->rcur];
      ra.rho[1] = c->rho[c->rcur ^ 1];
      ra.ops = c->ops;
      ra.withhold_tile = p->withhold_flag > 0 ? int((c->C + 127) / 128) * int((c->N + 127) / 128) - 1 : -1;
      ra.withhold_step = p->withhold_flag > 0 ? p->withhold_flag : -1;
      CK(cudaMemsetAsync(c->flags, 0, kMaxResidentTiles * sizeof(unsigned), c->stream));
      LK(launch_step_res(c->plan, ra, a, c->stream, res_pair));
      c->cur ^= flip;
      c->bcur ^= flip;
      c->opcur ^= flip;
      if (decay) c->rcur ^= flip;
      if (p->energy_every > 0 && len == seg) {
        s = track(c, p, tc, c->step + k + len);
        if (s != GDA_OK) return s;
      }
    }
    c->step += steps;
    return GDA_OK;
  }

  for (int64_t k = 0; k < steps; ++k) {
    const long long n = c->step + k;
    StepArgs a = base;
    a.step = static_cast<unsigned int>(n);
    a.beta_in = c->beta[c->bcur];
    a.beta_out = c->beta[c->bcur ^ 1];
    a.rho_in = c->rho[c->rcur];
    a.rho_out = decay ? c->rho[c->rcur ^ 1] : nullptr;
    if (p->integ == GDA_EULER) {
      a.mode = M_EULER;
      a.psi_n = c->psi[c->cur];
      a.xs = c->psi[c->cur];
      a.psi_out = c->psi[c->cur ^ 1];
      a.op_out = (tc && !f8) ? c->ops + (c->opcur ^ 1) * opsz : nullptr;
      a.op8_out = f8 ? c->ops8 + (c->opcur ^ 1) * opsz : nullptr;
      if (c->run_sparse) {
        a.opT_in = c->opT[tcur];
        a.opT_out = c->opT[(tcur + 1) % 3];
      }
      s = launch_step(c, a, tc, c->psi[c->cur], c->opcur);
      if (s != GDA_OK) return s;
      c->cur ^= 1;
      c->opcur ^= 1;
      tcur = (tcur + 1) % 3;
    } else {
      const float* xin[4] = {c->psi[c->cur], c->stg[0], c->stg[1], c->stg[0]};
      float* xout[3] = {c->stg[0], c->stg[1], c->stg[0]};
      for (int st = 0; st < 4; ++st) {
        a.mode = M_RK1 + st;
        a.psi_n = c->psi[c->cur];
        a.xs = xin[st];
        a.xs_next = st < 3 ? xout[st] : nullptr;
        a.psi_out = c->psi[c->cur];
        const int in_buf = c->opcur ^ (st & 1);
        a.op_out = (tc && !f8) ? c->ops + (in_buf ^ 1) * opsz : nullptr;
        a.op8_out = f8 ? c->ops8 + (in_buf ^ 1) * opsz : nullptr;
        if (c->run_sparse) {  // psi in T[tcur]; stages through T[A], T[B], T[A]; psi^{n+1} back to T[tcur]
          const int A = (tcur + 1) % 3, B = (tcur + 2) % 3;
          const int tin[4] = {tcur, A, B, A}, tout[4] = {A, B, A, tcur};
          a.opT_in = c->opT[tin[st]];
          a.opT_out = c->opT[tout[st]];
        }
        s = launch_step(c, a, tc, xin[st], in_buf);
        if (s != GDA_OK) return s;
      }
    }
    c->bcur ^= 1;
    if (decay) c->rcur ^= 1;
    if (p->energy_every > 0 && (k + 1) % p->energy_every == 0) {
      s = track(c, p, tc, n + 1);
      if (s != GDA_OK) return s;
    }
  }
  c->step += steps;
  return GDA_OK;
}

gda_status gda_sync(gda_ctx* c) {
  if (!c) return GDA_ERR_INVALID;
  CK(cudaStreamSynchronize(c->stream));
  return check_err(c);
}

gda_status gda_energy_dev(gda_ctx* c, double* E_dev) {
  if (!c) return GDA_ERR_INVALID;
  if (!E_dev) return fail(c, GDA_ERR_INVALID, "E_dev is NULL");
  gda_status s = compute_energies(c);
  if (s != GDA_OK) return s;
  CK(cudaMemcpyAsync(E_dev, c->E64, size_t(c->R) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return GDA_OK;
}

gda_status gda_energy(gda_ctx* c, double* E) {
  if (!c) return GDA_ERR_INVALID;
  if (!E) return fail(c, GDA_ERR_INVALID, "E is NULL");
  gda_status s = compute_energies(c);
  if (s != GDA_OK) return s;
  CK(cudaMemcpyAsync(E, c->E64, size_t(c->R) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check_err(c);
}

// FP64 argmin through candidate ranking (non-integer energies, R >= 32):
// compensated FP32 energies of all restarts carry an error below
// delta = 48 u (sum |J0| + sum |g|) (u = 2^-24: J rounded to FP32, spins
// rounded once, 16-term FMA blocks plus an exact two-sum, double partials);
// every restart within 2 (delta + delta64) of the lowest FP32 value is
// evaluated in FP64 (delta64 covers the FP64 sums themselves), which contains
// the FP64 argmin over all restarts.  Sets *done = false when ranking does
// not narrow the set (the caller then evaluates every restart).
gda_status best_ranked(gda_ctx* c, bool* done) {
  *done = false;
  if (c->int_exact || c->R < 32) return GDA_OK;
  if (c->rank_cap < c->Rp) {
    dfree(c->E32);
    dfree(c->cidx);
    c->rank_cap = 0;
    CK(dalloc(&c->E32, size_t(c->Rp)));
    CK(dalloc(&c->cidx, size_t(c->Rp)));
    c->rank_cap = c->Rp;
  }
  if (!c->d_count) CK(dalloc(&c->d_count, 1));
  if (!c->d_abs) CK(dalloc(&c->d_abs, 1));
  if (c->abs_sum < 0.0) {
    LK(launch_abs_sum(c->J64, c->g64, c->N, c->Np, c->d_abs, c->stream));
    CK(cudaMemcpyAsync(&c->abs_sum, c->d_abs, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  const double u = std::ldexp(1.0, -24);
  const double delta = 48.0 * u * c->abs_sum;
  const double delta64 = 1e-9 * (c->abs_sum + std::fabs(c->diag)) + 1e-300;
  const double margin = 2.0 * (delta + delta64);
  LK(launch_rank(c->psi[c->cur], c->J32, c->g64, c->S32, c->part64, c->E32, c->cidx, c->d_count, c->N, c->Np, c->R,
                 c->Rp, c->C, pmode(c), c->diag, margin, c->stream));
  int count = 0;
  CK(cudaMemcpyAsync(&count, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (count < 1 || count > c->R / 2) return GDA_OK;
  LK(launch_gather_cols(c->psi[c->cur], c->Np, c->cidx, count, c->cplx, c->stg[0], c->stream));
  LK(launch_energy64(c->stg[0], c->J64, c->g64, c->S64, c->part64, c->E64, c->N, c->Np, count, c->Rp,
                     count * (c->cplx ? 2 : 1), pmode(c), c->stream));
  LK(launch_argmin(c->E64, count, c->bestE, c->bestR, c->stream));
  LK(launch_map_best(c->cidx, c->bestR, c->stream));
  *done = true;
  return GDA_OK;
}

gda_status gda_best(gda_ctx* c, double* E, int32_t* r, void* cfg) {
  if (!c) return GDA_ERR_INVALID;
  if (!c->have_state) return fail(c, GDA_ERR_STATE, "no state: call gda_run or gda_set_state first");
  bool ranked = false;
  gda_status s = best_ranked(c, &ranked);
  if (s != GDA_OK) return s;
  if (!ranked) {
    s = compute_energies(c);
    if (s != GDA_OK) return s;
    LK(launch_argmin(c->E64, c->R, c->bestE, c->bestR, c->stream));
  }
  double e = 0.0;
  int rr = 0;
  CK(cudaMemcpyAsync(&e, c->bestE, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&rr, c->bestR, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  if (cfg) {
    LK(launch_best_cfg(c->psi[c->cur], c->bestR, c->N, c->Np, pmode(c), c->cfg8, c->cfgth, c->stream));
    if (c->cplx)
      CK(cudaMemcpyAsync(cfg, c->cfgth, size_t(c->N) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    else
      CK(cudaMemcpyAsync(cfg, c->cfg8, size_t(c->N), cudaMemcpyDeviceToHost, c->stream));
  }
  s = check_err(c);
  if (s != GDA_OK) return s;
  if (E) *E = e;
  if (r) *r = rr;
  return GDA_OK;
}

gda_status gda_best_seen(gda_ctx* c, double* E, int32_t* r, int64_t* step, void* cfg) {
  if (!c) return GDA_ERR_INVALID;
  int rr = -1;
  long long st = -1;
  CK(cudaMemcpyAsync(&rr, c->snapR, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&st, c->snapStep, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (rr < 0 || !c->have_state) return fail(c, GDA_ERR_STATE, "no tracked state: run with energy_every > 0 first");
  const int W = c->cplx ? 2 : 1;
  if (c->int_exact) {
    LK(launch_energy_int(c->snap, c->Jint, c->Sint, c->partint, c->E64, c->N, c->Np, 1, c->Rp, W, c->stream));
  } else {
    LK(launch_energy64(c->snap, c->J64, c->g64, c->S64, c->part64, c->E64, c->N, c->Np, 1, c->Rp, W, pmode(c),
                       c->stream));
  }
  double e = 0.0;
  CK(cudaMemcpyAsync(&e, c->E64, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (cfg) {
    LK(launch_best_cfg(c->snap, c->d_zero, c->N, c->Np, pmode(c), c->cfg8, c->cfgth, c->stream));
    if (c->cplx)
      CK(cudaMemcpyAsync(cfg, c->cfgth, size_t(c->N) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    else
      CK(cudaMemcpyAsync(cfg, c->cfg8, size_t(c->N), cudaMemcpyDeviceToHost, c->stream));
  }
  gda_status s = check_err(c);
  if (s != GDA_OK) return s;
  if (E) *E = e;
  if (r) *r = rr;
  if (step) *step = st;
  return GDA_OK;
}

gda_status gda_trace_energy(gda_ctx* c, int32_t first, int32_t count, double* E) {
  if (!c) return GDA_ERR_INVALID;
  if (!E || first < 0 || count < 0) return fail(c, GDA_ERR_INVALID, "E NULL, first < 0 or count < 0");
  int n = 0;
  CK(cudaMemcpyAsync(&n, c->t_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int kept = std::min(n, c->hist_run);
  if (!c->have_state || int64_t(first) + count > kept)
    return fail(c, GDA_ERR_INVALID, "trace entries [%d, %d) requested, %d kept", first, first + count, kept);
  const int W = c->cplx ? 2 : 1;
  // evaluate in chunks of at most R configurations (the energy scratch holds R columns)
  for (int k0 = 0; k0 < count; k0 += c->R) {
    const int m = std::min(c->R, count - k0);
    const float* src = c->hist + size_t(first + k0) * W * c->Np;
    if (c->int_exact) {
      LK(launch_energy_int(src, c->Jint, c->Sint, c->partint, c->E64, c->N, c->Np, m, c->Rp, m * W, c->stream));
    } else {
      LK(launch_energy64(src, c->J64, c->g64, c->S64, c->part64, c->E64, c->N, c->Np, m, c->Rp, m * W, pmode(c),
                         c->stream));
    }
    CK(cudaMemcpyAsync(E + k0, c->E64, size_t(m) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  return check_err(c);
}

gda_status gda_get_state(gda_ctx* c, float* psi, float* gamma, float* beta, int64_t* step) {
  if (!c) return GDA_ERR_INVALID;
  if (!c->have_state) return fail(c, GDA_ERR_STATE, "no state");
  const size_t rn = size_t(c->R) * c->N, W = c->cplx ? 2 : 1;
  // stage in the RK buffers (scratch between runs), then one copy each
  float* hp = c->stg[1];
  float* hg = c->gstg;
  float* hb = c->beta[c->bcur ^ 1];
  LK(launch_pack_state(c->psi[c->cur], c->gam, c->beta[c->bcur], c->N, c->Np, c->R, c->cplx, hp, hg, hb, c->stream));
  if (psi) CK(cudaMemcpyAsync(psi, hp, rn * W * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (gamma) CK(cudaMemcpyAsync(gamma, hg, rn * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (beta) CK(cudaMemcpyAsync(beta, hb, size_t(c->R) * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  gda_status s = check_err(c);
  if (s != GDA_OK) return s;
  if (step) *step = c->step;
  return GDA_OK;
}

gda_status gda_set_state(gda_ctx* c, const float* psi, const float* gamma, const float* beta, int32_t R,
                         int64_t step) {
  if (!c) return GDA_ERR_INVALID;
  if (!psi || R < 1 || step < 0) return fail(c, GDA_ERR_INVALID, "psi NULL, R < 1 or step < 0");
  gda_status s = ensure_state(c, R);
  if (s != GDA_OK) return s;
  const size_t rn = size_t(R) * c->N, W = c->cplx ? 2 : 1;
  float* hp = c->stg[1];
  float* hg = c->gstg;
  float* hb = c->beta[1];
  CK(cudaMemcpyAsync(hp, psi, rn * W * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  if (gamma) CK(cudaMemcpyAsync(hg, gamma, rn * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  if (beta) CK(cudaMemcpyAsync(hb, beta, size_t(R) * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  LK(launch_unpack_state(c->psi[0], c->gam, c->beta[0], c->N, c->Np, R, c->cplx, hp, gamma ? hg : nullptr,
                         beta ? hb : nullptr, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->cur = 0;
  c->bcur = 0;
  c->step = step;
  LK(launch_snapshot_reset(c->snapE, c->snapR, c->snapStep, c->stream));
  c->have_state = true;
  return GDA_OK;
}

gda_status gda_trace(gda_ctx* c, int64_t* step, double* E, int32_t* r, int32_t cap, int32_t* count) {
  if (!c) return GDA_ERR_INVALID;
  int n = 0;
  CK(cudaMemcpyAsync(&n, c->t_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int m = std::min(std::min(n, cap), kTraceCap);
  if (m > 0) {
    if (step) CK(cudaMemcpyAsync(step, c->t_step, m * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    if (E) CK(cudaMemcpyAsync(E, c->t_E, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (r) CK(cudaMemcpyAsync(r, c->t_r, m * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  }
  gda_status s = check_err(c);
  if (s != GDA_OK) return s;
  if (count) *count = n;
  return GDA_OK;
}

gda_status gda_profile(gda_ctx* c, int32_t enable) {
  if (!c) return GDA_ERR_INVALID;
  if (!enable) {
    CK(cudaStreamSynchronize(c->stream));
    dfree(c->stamps);
    c->stamp_cap = 0;
    return GDA_OK;
  }
  if (!c->stamps) {
    const int ctas = (c->Np / 64) * 4096;  // bound on the CTAs of any step launch
    CK(dalloc(&c->stamps, size_t(ctas) * 8));
    CK(cudaMemsetAsync(c->stamps, 0, size_t(ctas) * 8 * sizeof(unsigned long long), c->stream));
    c->stamp_cap = ctas;
  }
  return GDA_OK;
}

gda_status gda_profile_read(gda_ctx* c, uint64_t* out, int32_t cap_ctas, int32_t* nctas) {
  if (!c) return GDA_ERR_INVALID;
  if (!c->stamps) return fail(c, GDA_ERR_STATE, "profiling is not enabled");
  const int n = std::min(cap_ctas, c->stamp_cap);
  CK(cudaMemcpyAsync(out, c->stamps, size_t(n) * 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (nctas) *nctas = n;
  return GDA_OK;
}

gda_status gda_set_init_base(gda_ctx* c, const float* base, int32_t on_device) {
  if (!c) return GDA_ERR_INVALID;
  if (!base) return fail(c, GDA_ERR_INVALID, "base is NULL");
  if (!c->base) {
    CK(dalloc(&c->base, size_t(2) * c->N));
  }
  const size_t W = c->cplx ? 2 : 1;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (W == 2) {
    CK(cudaMemcpyAsync(c->base, base, size_t(2) * c->N * sizeof(float), kind, c->stream));
  } else {
    // real amplitudes: imaginary parts are zero
    CK(cudaMemsetAsync(c->base, 0, size_t(2) * c->N * sizeof(float), c->stream));
    CK(cudaMemcpy2DAsync(c->base, 2 * sizeof(float), base, sizeof(float), sizeof(float), c->N, kind, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return GDA_OK;
}

gda_status gda_features(gda_ctx* c, float* F) {
  if (!c) return GDA_ERR_INVALID;
  if (!F) return fail(c, GDA_ERR_INVALID, "F is NULL");
  for (int k = 0; k < 2; ++k)
    if (!c->fw[k]) CK(dalloc(&c->fw[k], size_t(c->Np)));
  LK(launch_features(c->J64, c->g64, c->N, c->Np, c->cplx, c->fw[0], c->fw[1], F, c->stream));
  return GDA_OK;
}

gda_status gda_coupling(gda_ctx* c, int32_t prec, int32_t R, const float* X, float* Y) {
  if (!c) return GDA_ERR_INVALID;
  if (!X || !Y || R < 1) return fail(c, GDA_ERR_INVALID, "X or Y NULL, or R < 1");
  if (prec != GDA_FP32 && prec != GDA_BF16 && prec != GDA_FP8 && prec != GDA_SPARSE)
    return fail(c, GDA_ERR_INVALID, "unknown precision");
  const bool tc = prec == GDA_BF16 || prec == GDA_FP8;
  if (tc && !c->tc_ok) return fail(c, GDA_ERR_UNSUPPORTED, "tensor-core path needs an sm_103 device");
  c->run_sparse = false;
  c->run_pair = false;
  if (prec == GDA_SPARSE) {
    gda_status se = ensure_ell(c);
    if (se != GDA_OK) return se;
    c->run_sparse = true;
  }
  gda_status s = gda_set_state(c, X, nullptr, nullptr, R, 0);
  if (s != GDA_OK) return s;
  gda_params p;
  gda_default_params(&p);
  StepArgs a = base_args(c, &p, tc);
  if (prec == GDA_FP8) {
    s = ensure_fp8(c);
    if (s != GDA_OK) return s;
    a.row_scale = c->jscale;
    LK(launch_to_e4m3(c->psi[0], c->ops8, size_t(c->Cp) * c->Np, c->stream));
  } else if (tc) {
    LK(launch_to_bf16(c->psi[0], c->ops, size_t(c->Cp) * c->Np, c->stream));
  }
  a.mode = M_RAW;
  a.psi_n = c->psi[0];
  a.xs = c->psi[0];
  a.psi_out = c->stg[0];
  a.beta_in = c->beta[0];
  s = launch_step(c, a, tc, c->psi[0], 0);
  if (s != GDA_OK) return s;
  const size_t rn = size_t(R) * c->N, W = c->cplx ? 2 : 1;
  LK(launch_pack_state(c->stg[0], c->gam, c->beta[0], c->N, c->Np, R, c->cplx, c->stg[1], nullptr, nullptr,
                       c->stream));
  CK(cudaMemcpyAsync(Y, c->stg[1], rn * W * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  return check_err(c);
}

}  // extern "C"
