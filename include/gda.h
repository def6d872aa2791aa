/*
 * gda.h — C ABI of the GB300 gain-dissipative (GD) solver.
 *
 * The library time-steps R independent restarts of the GD rate equations of
 * Kalinin & Berloff, "Global optimization of spin Hamiltonians with
 * gain-dissipative systems" (2018):
 *
 *   dpsi_i/dt   = psi_i (gamma_i - |psi_i|^2) + beta * sum_{j != i} J_ij psi_j + h_1i   (Eq. 2)
 *   dgamma_i/dt = eps (rho_th - |psi_i|^2)                                           (Eq. 5)
 *   dbeta/dt    = eps_hat (1 - beta)        (Eq. 6 with Delta_ij = 1, K(t) = beta(t) J)
 *
 * with h_1i = -g_i sqrt(rho_th) and optional Euler-Maruyama noise D xi_i, and
 * evaluates the spin Hamiltonian of Eq. (1),
 *
 *   H = - sum_i sum_j J_ij cos(theta_i - theta_j) + sum_i g_i cos(theta_i),
 *
 * on the projected spins of every restart.  Ising runs use real amplitudes
 * (theta in {0, pi}); XY runs use complex amplitudes.  Options of gda_params
 * extend this to the paper's other forms: the GD-mod coupling feedback (Eq. 6
 * with Delta_ij = gamma_i^inj + gamma_j^inj and a coupling matrix per
 * restart), a resonant q:1 drive h_q conj(psi)^(q-1) of Eq. (2) with spins
 * projected onto the q-th roots of unity (the q-state Potts model; q = 2 is
 * the complex-amplitude Ising form with the h_2 penalty), and the coupling
 * product in FP32, BF16 or FP8 on tensor cores, or over the nonzeros of a
 * sparse J.
 *
 * Typical use: gda_create (J, g, model) -> gda_run (params, R, steps) ->
 * gda_best (lowest FP64 energy, its restart and configuration) or
 * gda_energy (every restart's energy) -> gda_destroy.  gda_get_state /
 * gda_set_state checkpoint and resume; gda_batch_* runs many instances of
 * different sizes in one launch per step.
 *
 * Conventions for every entry point:
 *   - Host pointers are plain C arrays owned by the caller; the library copies
 *     what it needs and never keeps a host pointer after the call returns.
 *   - `_dev` entry points take device pointers (e.g. torch data pointers) on
 *     the context's device; the caller keeps ownership.
 *   - The context owns all device memory it allocates; gda_destroy frees it.
 *   - Work is queued on the context's stream (gda_set_stream; default: the
 *     legacy default stream).  gda_run returns after queuing; device-side
 *     errors (divergence, a barrier timeout) are reported by the next
 *     synchronising call (gda_sync, gda_energy, gda_best, gda_get_state,
 *     gda_trace).
 *   - Every call returns a gda_status; on failure the context keeps a
 *     message readable with gda_last_error.  No C++ exception crosses the ABI.
 *   - Calls on one context are not thread safe; use one context per thread.
 */
#ifndef GDA_H
#define GDA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gda_ctx gda_ctx;

typedef enum {
  GDA_ISING = 0, /* real amplitudes, spins s_i = sign(psi_i)            */
  GDA_XY = 1     /* complex amplitudes, spins s_i = psi_i / |psi_i|     */
} gda_model;

typedef enum {
  GDA_OK = 0,
  GDA_ERR_INVALID = 1,     /* bad argument (sizes, NaN/asymmetric J, NULL)  */
  GDA_ERR_CUDA = 2,        /* a CUDA runtime/driver call failed              */
  GDA_ERR_OOM = 3,         /* device allocation failed                       */
  GDA_ERR_DIVERGED = 4,    /* a non-finite or overflowing amplitude appeared */
  GDA_ERR_TIMEOUT = 5,     /* a device-side wait ran out of its time limit   */
  GDA_ERR_UNSUPPORTED = 6, /* option not available on this device / build    */
  GDA_ERR_STATE = 7        /* call out of order (e.g. gda_energy before run) */
} gda_status;

typedef enum { GDA_EULER = 0, GDA_RK4 = 1 } gda_integrator;

typedef enum {
  GDA_FP32 = 0, /* J.Psi on CUDA cores in FP32 (the plain reference path)     */
  GDA_BF16 = 1, /* J.Psi on tcgen05 tensor cores, BF16 operands, FP32 accum   */
  GDA_FP8 = 2,  /* J.Psi on tcgen05 tensor cores, E4M3 operands, FP32 accum:
                 * J0_ij stored as e4m3(J0_ij / s_i), s_i = max_j |J0_ij| / 448
                 * (row scale), amplitudes as e4m3(psi * 64) (|psi| up to 7
                 * before saturation), Y_i = acc_i * s_i / 64.  Per-step
                 * schedule only; the energy tracking of energy_every uses
                 * the BF16 product of the projected spins. */
  GDA_SPARSE = 3 /* J.Psi over the nonzeros of J only (the paper's sparse
                 * 3-regular instances, Sec. 2): on first use J0 is compacted
                 * on the device into an ELL table of at most
                 * GDA_SPARSE_MAX_DEG nonzeros per row (column index and FP32
                 * value, ascending column order); every step gathers those
                 * entries on CUDA cores in FP32.  Amplitudes, gains, noise
                 * (with decay), RK4 and the energy tracking as in GDA_FP32.
                 * A row with more nonzeros gives GDA_ERR_UNSUPPORTED. */
} gda_precision;

#define GDA_SPARSE_MAX_DEG 64

/* Run parameters (Eqs. 2, 5, 6; Sec. 2 integrator).  Fill with
 * gda_default_params, then override.  All rates are per unit of time t. */
typedef struct {
  int32_t integ;        /* gda_integrator                                      */
  int32_t prec;         /* gda_precision of the coupling product               */
  double dt;            /* time step                                           */
  double eps;           /* gain adjustment speed epsilon, Eq. (5)              */
  double rho_th;        /* threshold density rho_th, Eq. (5)                   */
  double gamma0;        /* initial effective gain gamma^inj - gamma_c          */
  double beta0;         /* initial coupling scale, K(0) = beta0 J              */
  double eps_hat;       /* coupling adjustment speed, Eq. (6)                  */
  double noise_D;       /* noise strength D, Eq. (2); 0 disables noise         */
  int32_t noise_decay;  /* 1: D_r = D max(0, 1 - mean_i rho_i / rho_th)        */
  int32_t energy_every; /* k > 0: record the best projected energy every k steps */
  uint64_t seed;        /* Philox4x32-10 key for noise and initial amplitudes  */
  int32_t init_mode;    /* 0: psi = 0; 1: seeded U(-a, a) per real component;
                           2: continue from the current state (resume);
                           3: as 1 plus the per-spin base of gda_set_init_base */
  int32_t schedule;     /* gda_schedule: how BF16 steps are launched           */
  double init_amp;      /* a for init_mode 1                                   */
  int32_t coupling;     /* gda_coupling_mode: GD (K = beta J) or GD-mod        */
  int32_t withhold_flag; /* testing only, 0 otherwise: k >= 1 makes the last
                           tile of the resident kernel (GDA_SCHEDULE_RESIDENT)
                           withhold the step flag it would publish after step
                           k of each launch, so every wait on it in its
                           column runs out after wait_s and the run reports
                           GDA_ERR_TIMEOUT; the context stays usable          */
  double gamma_c;       /* GD-mod: loss rate, gamma^inj = gamma + gamma_c      */
  int32_t q;            /* resonant q:1 drive of Eq. (2), h_q conj(psi)^(q-1),
                           for GDA_XY contexts: 0 none, 2 <= q <= 16.  With
                           q >= 2 the energies, the trace and gda_best project
                           onto the q-th roots of unity (the q-state Potts
                           model of Sec. 1; q = 2 is the paper's complex
                           Ising formulation with the h_2 penalty).  Per-step
                           GD only (not RESIDENT, not GD-mod).  The projection
                           stays with the context until the next gda_run. */
  int32_t reserved2;    /* 0                                                   */
  double hq;            /* h_q of that drive                                   */
  double wait_s;        /* limit of every device-side wait of the tensor-core
                           step kernels, in seconds (0: about 2 s); a wait
                           that runs out aborts the launch, which drains its
                           copies and MMAs, frees its tensor memory and
                           reports GDA_ERR_TIMEOUT                             */
} gda_params;

/* Coupling feedback of Eq. (6).
 * GDA_COUPLING_GD: Delta_ij = 1 and K(0) = beta0 J, so K(t) = beta(t) J with
 *   d beta/dt = eps_hat (1 - beta) per restart: one GEMM per step.
 * GDA_COUPLING_GDMOD (Sec. 2, the GD-mod algorithm): Delta_ij = gamma_i^inj +
 *   gamma_j^inj with gamma^inj = gamma + gamma_c, and a full coupling matrix
 *   K_r per restart, K_r(0) = beta0 J, dK_ij/dt = eps_hat (J_ij - Delta_ij
 *   K_ij); the coupling sum is sum_{j != i} Delta_ij K_ij psi_j.  K takes
 *   R * N * Np * 4 bytes of device memory (Np = N rounded up to 128) and is
 *   streamed from HBM every step.  Requires GDA_FP32, GDA_EULER, no noise
 *   decay, Np * 12 bytes <= 227 KB; else GDA_ERR_UNSUPPORTED.  K lives in the
 *   context: init_mode 2 continues it, gda_set_state does not touch it, and
 *   gda_get_state does not return it. */
typedef enum { GDA_COUPLING_GD = 0, GDA_COUPLING_GDMOD = 1 } gda_coupling_mode;

/* Launch schedule of the tensor-core path.  AUTO picks the resident kernel
 * for Euler runs whose 128 x 128 tiles all fit on the device at once (every
 * CTA keeps its tile's FP32 state in tensor memory for a whole segment of
 * steps, with per-tile flags between steps); else, for Euler runs whose
 * coupling operand (N'^2 BF16 or E4M3 values) fits in 48 MiB, the persistent
 * streaming launch (GDA_SCHEDULE_STREAM); else one launch per step (RK4
 * stage), with two-SM tiles where they pay.  All give the same numbers. */
typedef enum {
  GDA_SCHEDULE_AUTO = 0,
  GDA_SCHEDULE_PER_STEP = 1,
  GDA_SCHEDULE_RESIDENT = 2, /* GDA_ERR_UNSUPPORTED if not applicable */
  GDA_SCHEDULE_PAIR = 3,     /* per-step launches with two-SM tiles: clusters of
                              * two CTAs share 256 x BN tensor-core tiles
                              * (tcgen05 cta_group::2), each SM staging its 128
                              * rows of J and half of the operand columns;
                              * BF16 / FP8 only, N rounded up to 128 must be a
                              * multiple of 256, else GDA_ERR_UNSUPPORTED.
                              * AUTO uses them for per-step runs whose pair
                              * tiles fill three or more waves of clusters */
  GDA_SCHEDULE_STREAM = 4    /* forward-Euler BF16 / FP8 steps of instances too
                              * large for the resident kernel in one persistent
                              * launch per tracking segment: the state streams
                              * from HBM every step as with per-step launches,
                              * but steps are ordered by per-tile flags, so the
                              * next step's first tiles overlap the last
                              * epilogues of the step before (two-SM tiles where
                              * AUTO would take them); GDA_ERR_UNSUPPORTED for
                              * RK4 or FP32 */,
  GDA_SCHEDULE_STREAM_PAIR = 5, /* GDA_SCHEDULE_STREAM with two-SM tiles always
                              * (conditions of GDA_SCHEDULE_PAIR) */
  GDA_SCHEDULE_RESIDENT_PAIR = 6 /* the resident kernel with two-SM tiles: the
                              * CTAs of row blocks 2p, 2p + 1 form a cluster and
                              * share M = 256 tensor-core instructions, each
                              * keeping its own rows' state in tensor memory;
                              * conditions of GDA_SCHEDULE_RESIDENT plus an even
                              * number of 128-row blocks and every cluster
                              * resident at once, else GDA_ERR_UNSUPPORTED */
} gda_schedule;

/* Fills p with dt = 0.01, eps = 0.1, rho_th = 1, gamma0 = 0, beta0 = 1,
 * eps_hat = 0, noise off, Euler, FP32, init_mode 1 with a = 1e-3, seed 0,
 * GDA_COUPLING_GD, gamma_c = 1, no resonant drive (q = 0, hq = 0), the
 * default wait limit (wait_s = 0) and no withheld flag. */
void gda_default_params(gda_params* p);

/* Creates a context for an N-spin instance on the current CUDA device.
 * J: N*N row-major doubles (host), symmetric and finite, copied.  The
 *    diagonal is left out of the dynamics (Eq. 2 sums j != i) but counted in
 *    the energy (Eq. 1 sums all ordered pairs).
 * g: N doubles (host) or NULL for g = 0.
 * Errors: GDA_ERR_INVALID for N < 1, N > 65536, NULL J or out, non-finite or
 * asymmetric J, non-finite g, or model not in gda_model; GDA_ERR_OOM/CUDA.
 * On failure *out is NULL. */
gda_status gda_create(const double* J, const double* g, int32_t N, int32_t model, gda_ctx** out);

/* Replaces J and g of an existing context with a new instance of the same N
 * (host pointers, copied).  Same checks as gda_create.  Ordered on the stream. */
gda_status gda_load(gda_ctx* ctx, const double* J, const double* g);

/* Same as gda_load with device pointers (N*N and N doubles on the device). */
gda_status gda_load_dev(gda_ctx* ctx, const double* J_dev, const double* g_dev);

/* Sets the CUDA stream (a cudaStream_t passed as void*) used by every later
 * call.  NULL selects the legacy default stream. */
gda_status gda_set_stream(gda_ctx* ctx, void* stream);

/* Runs `steps` steps for R restarts with parameters p (Eqs. 2, 5, 6).
 * init_mode 0/1 starts a new run at step 0; init_mode 2 continues from the
 * current state (R must equal the current restart count).  If
 * p->energy_every = k > 0, the best projected energy over the restarts
 * (FP32 tracking value) is recorded after every k-th step (gda_trace).
 * Asynchronous on the context's stream.
 * Errors: GDA_ERR_INVALID (R < 1, steps < 0, dt <= 0, non-finite params),
 * GDA_ERR_UNSUPPORTED (BF16 on a device other than sm_103), GDA_ERR_OOM. */
gda_status gda_run(gda_ctx* ctx, const gda_params* p, int32_t R, int64_t steps);

/* Waits for the stream and reports device-side errors of earlier runs
 * (GDA_ERR_DIVERGED, GDA_ERR_TIMEOUT).  The error flags are cleared. */
gda_status gda_sync(gda_ctx* ctx);

/* Eq. (1) energy of the projected spins of every restart, in FP64 (exact,
 * through an int64 reduction, for Ising runs with integer J and g = 0).
 * E: R doubles on the host.  Synchronises. */
gda_status gda_energy(gda_ctx* ctx, double* E);

/* Same as gda_energy into R doubles on the device; stream ordered, does not
 * synchronise. */
gda_status gda_energy_dev(gda_ctx* ctx, double* E_dev);

/* Lowest Eq. (1) energy over the restarts (ties: lowest restart index), the
 * same answer and FP64 value as the argmin of gda_energy.  For non-integer
 * energies and R >= 32 it first bounds every restart's energy with
 * compensated FP32 sums (error below 48 * 2^-24 * (sum |J0| + sum |g|)) and
 * evaluates in FP64 only the restarts within twice that bound of the lowest.
 * E, r: host scalars (either may be NULL).  cfg (may be NULL): N int8 spins
 * (+1/-1) for Ising, or N doubles theta_i in (-pi, pi] for XY (on the q-th
 * roots of unity after a run with a resonant drive), host.  Synchronises. */
gda_status gda_best(gda_ctx* ctx, double* E, int32_t* r, void* cfg);

/* Copies the state out (host).  psi: R*N floats (Ising) or R*N interleaved
 * (re, im) float pairs (XY), restart-major; gamma: R*N floats; beta: R
 * floats; step: global step count.  Any pointer may be NULL.  Synchronises. */
gda_status gda_get_state(gda_ctx* ctx, float* psi, float* gamma, float* beta, int64_t* step);

/* Sets the state (host arrays in the layout of gda_get_state) for R restarts
 * at global step `step`; a following gda_run with init_mode 2 resumes from it,
 * bit-identical to an uninterrupted run.  gamma/beta NULL: gamma0 = 0,
 * beta = 1. */
gda_status gda_set_state(gda_ctx* ctx, const float* psi, const float* gamma, const float* beta,
                         int32_t R, int64_t step);

/* The running best of the energy trace (S8): whenever a tracking evaluation
 * (energy_every > 0) finds a lower energy than any before it, the library
 * keeps that restart's amplitudes; this call evaluates the kept configuration
 * in FP64 (exact for integer-J Ising) and returns that energy, the restart,
 * the step of the evaluation and optionally the configuration (cfg as in
 * gda_best).  The running best spans runs continued with init_mode 2 and is
 * cleared by a fresh run, gda_set_state and gda_load.  GDA_ERR_STATE if no
 * evaluation has run.  Synchronises.  (Sec. 2-3: the best state any restart
 * visits, verified at the end.) */
gda_status gda_best_seen(gda_ctx* ctx, double* E, int32_t* r, int64_t* step, void* cfg);

/* FP64 Eq. (1) energies (exact for integer-J Ising) of the configurations the
 * trace of the last run names: trace entry k's configuration is the restart
 * with the lowest tracking energy at that evaluation, as it was at that step
 * (kept on the device when the evaluation ran).  E: `count` doubles (host)
 * for entries first .. first+count-1, in trace order.  The run keeps up to
 * min(steps / energy_every, 65536, 256 MiB / (4 N' W)) entries (N' = N
 * rounded up to 128, W = 2 for XY, 1 for Ising); GDA_ERR_INVALID for entries
 * beyond what was recorded and kept.  Synchronises.  (Sec. 2-3: the energy
 * of the state a run holds at each evaluation, verified in FP64.) */
gda_status gda_trace_energy(gda_ctx* ctx, int32_t first, int32_t count, double* E);

/* Copies out the energy trace of the last run (host arrays of capacity cap):
 * step index, best tracking energy and its restart.  *count receives the
 * number of entries recorded (may exceed cap).  Synchronises. */
gda_status gda_trace(gda_ctx* ctx, int64_t* step, double* E, int32_t* r, int32_t cap, int32_t* count);

/* The coupling product alone (the GEMM of Eq. 2's sum over j != i):
 * Y = J0 X for R restarts, with J0 = J minus its diagonal, through the
 * FP32 (prec = GDA_FP32), tensor-core BF16 (GDA_BF16) or tensor-core FP8
 * (GDA_FP8) path.  X, Y: host
 * arrays in the psi layout of gda_get_state.  Replaces the context's state
 * (a following gda_run must start with init_mode 0 or 1).  Synchronises. */
gda_status gda_coupling(gda_ctx* ctx, int32_t prec, int32_t R, const float* X, float* Y);

/* Tracing: enable (1) or disable (0) per-CTA device timestamps of the
 * tensor-core step kernel.  When enabled, every step launch overwrites, for
 * each CTA, eight %globaltimer readings (ns): entry, set-up done, first
 * operand tile arrived, last MMA issued, accumulator ready, epilogue done,
 * partial sums written, exit.  Costs one buffer of at most (N/64+1)*4096*64
 * bytes; timing of a profiled run is not representative of an unprofiled one. */
gda_status gda_profile(gda_ctx* ctx, int32_t enable);

/* Copies the timestamps of the last profiled step launch to out
 * (cap_ctas * 8 uint64, CTA-major in launch order y*gridDim.x + x);
 * *nctas receives the number of CTA records copied.  Synchronises. */
gda_status gda_profile_read(gda_ctx* ctx, uint64_t* out, int32_t cap_ctas, int32_t* nctas);

/* Allocation-free energy evaluation.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory while
 * they run, such as a host that has reserved all GPU memory for its own
 * pool, or a serving process whose allocator is frozen after start-up; the
 * context-based calls above allocate on gda_create / gda_run, this one never
 * calls cudaMalloc, cudaFree or any allocating routine.
 *
 * Computes the same FP64 energies of the projected spins of R restarts as
 * gda_energy does (J's diagonal counted), from caller-owned device buffers:
 *   J_dev   N*N doubles, row-major, symmetric;
 *   g_dev   N doubles, or NULL for g = 0;
 *   psi_dev amplitudes in the gda_get_state layout: R*N floats (Ising) or
 *           R*N interleaved (re, im) float pairs (XY), restart-major;
 *   E_dev   R doubles, written;
 *   stream  a cudaStream_t (NULL: legacy default stream).
 * Its scratch is one file-scope device array of
 * GDA_NOALLOC_MAX_N/64 * GDA_NOALLOC_MAX_R doubles (2 MiB) that every GPU
 * loading this library keeps until the process exits.  Sizes beyond
 * N <= GDA_NOALLOC_MAX_N and R <= GDA_NOALLOC_MAX_R return GDA_ERR_INVALID,
 * as do NULL buffers, N < 1, R < 1 or an unknown model.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Under
 * CUDA's default lazy module loading that first call is also when the module
 * holding the array, and so the array itself, is placed in device memory: a
 * caller that will reserve the rest of the GPU for its own pool, or freeze
 * its allocator, makes its first call before doing so (or sets
 * CUDA_MODULE_LOADING=EAGER, which places it when the library loads).  All calls
 * share the array: calls whose work overlaps on the GPU (different streams,
 * or different threads on one device) race and must be serialised by the
 * caller.  Asynchronous on `stream`; returns GDA_ERR_CUDA if a launch fails. */
#define GDA_NOALLOC_MAX_N 4096
#define GDA_NOALLOC_MAX_R 4096
gda_status gda_energy_noalloc(const double* J_dev, const double* g_dev, int32_t N, int32_t model,
                              const float* psi_dev, int32_t R, double* E_dev, void* stream);

/* ---- Learned proposal (not in the paper) --------------------------------
 * A network that maps an instance's couplings to initial amplitudes and run
 * settings, trained on configurations the GD algorithm itself finds.  Inputs
 * are per-spin features (gda_features); the network is a 3-layer MLP
 * GDA_MLP_IN -> GDA_MLP_HIDDEN -> GDA_MLP_HIDDEN -> GDA_MLP_OUT with ReLU
 * hidden layers; parameters are one float vector of GDA_MLP_PARAMS entries:
 * W1 [128][8], b1 [128], W2 [128][128], b2 [128], W3 [5][128], b3 [5].
 * Outputs per spin: 0, 1 the initial amplitude (real, imaginary part); the
 * mean over an instance's spins of outputs 2, 3, 4 the instance's settings
 * (their mapping to epsilon, rho_th and the ramp is the caller's).  All
 * pointers below are device pointers; calls are asynchronous on `stream`. */
#define GDA_MLP_IN 8
#define GDA_MLP_HIDDEN 128
#define GDA_MLP_OUT 5
#define GDA_MLP_PARAMS 18309

/* Base amplitude for init_mode 3 (used by the learned proposal): N floats
 * (Ising) or N interleaved (re, im) float pairs (XY), on the host
 * (on_device = 0) or the device (1); copied.  A run with init_mode 3 starts
 * restart r at psi_i = base_i + the init_mode 1 perturbation of (i, r).
 * Synchronises. */
gda_status gda_set_init_base(gda_ctx* ctx, const float* base, int32_t on_device);

/* Per-spin features of the context's instance into F_dev [N][8]:
 * f0 = sum_j J0_ij / |J0_i|, f1 = sum_j |J0_ij| / (sqrt(N) |J0_i|),
 * f2 = |J0_i|, f3 = max_j |J0_ij| / |J0_i|, f4 = g_i,
 * f5 = (J0 v1)_i / rms(J0 v1) with v1 = J0 1 / rms(J0 1),
 * f6 = (J0 f5)_i / rms(J0 f5), f7 = 1 (XY) or 0 (Ising);
 * J0 = J without its diagonal, |.| Euclidean, rms over spins, 0/0 = 0.
 * Stream ordered on the context's stream. */
gda_status gda_features(gda_ctx* ctx, float* F_dev);

/* O [M][5] = MLP(X [M][8]); H (may be NULL) caches the hidden activations
 * [M][256] for gda_mlp_backward. */
gda_status gda_mlp_forward(const float* params, const float* X, int32_t M, float* O, float* H, void* stream);

/* G [GDA_MLP_PARAMS] += d(sum_m dO[m] . O[m]) / d params, from the cache of a
 * forward pass on the same X (G is accumulated with atomics: zero it first). */
gda_status gda_mlp_backward(const float* params, const float* X, const float* H, const float* dO, int32_t M,
                            float* G, void* stream);

/* Training loss of n_inst instances (rows [offsets[b], offsets[b+1]) of O):
 * loss_b = mean_i |a_i - u s_i|^2 + wset * sum_k (mean_i O[i][2+k] - Tset[b][k])^2,
 * a_i = O[i][0] (+ i O[i][1] if cplx[b]), target spins S [M][2] (re, im),
 * u the global sign (Ising) or phase (XY) that aligns s with a.  Writes dO
 * [M][5] = d loss_b / d O and loss [n_inst].  offsets, cplx: device int32. */
gda_status gda_proposal_loss(const float* O, const float* S, const float* Tset, const int32_t* offsets,
                             const int32_t* cplx, int32_t n_inst, float wset, float* dO, float* loss,
                             void* stream);

/* The proposal's head, on the device, for one instance of N spins: from the
 * network outputs O [N][5] (gda_mlp_forward), the init_mode 3 base amplitudes
 * for gda_set_init_base / gda_batch_set_init_base with on_device = 1 --
 * base [N] = amp * O[:, 0] (Ising, cplx = 0) or base [N][2] = amp * (O[:, 0],
 * O[:, 1]) (XY), each the float rounding of the double product -- and the
 * instance's settings [3] (double) = (eps, rho_th, beta0) =
 * (0.02 + 0.48 s(m0), 0.5 + 1.5 s(m1), 0.1 + 0.9 s(m2)), s the logistic
 * function, m_k the mean over the spins of O[:, 2 + k] (summed in double).
 * Device pointers, owned by the caller; asynchronous on `stream`.
 * GDA_ERR_INVALID for a null pointer or N < 1. */
gda_status gda_proposal_head(const float* O, int32_t N, int32_t cplx, double amp, float* base, double* settings,
                             void* stream);

/* One Adam step (bias corrected, step t >= 1) on P parameters. */
gda_status gda_adam_step(float* params, const float* grad, float* m1, float* m2, int32_t P, float lr,
                         float beta1, float beta2, float eps, int32_t t, void* stream);

/* ---- Batched serving (not in the paper) -----------------------------------
 * Many independent instances (own N, model and R each) stepped together: one
 * persistent cooperative tensor-core launch runs a chunk of 100 steps of
 * every instance (both model types) over all their 128 x BN output tiles,
 * with steps ordered by per-tile dataflow flags (or, by choice, one launch per
 * step: gda_batch_set_schedule); chunks replay from a captured CUDA graph
 * where the CUDA runtime captures the launch (gda_batch_launch_mode).
 * Every instance follows exactly the single-instance forward-Euler BF16
 * dynamics (Eqs. 2, 5, 6) with its own Philox seed and, optionally, its own
 * settings and start (gda_batch_set_params, gda_batch_set_init_base).  The
 * batch owns its device memory.  Layout conventions are those of the
 * single-instance calls. */
typedef struct gda_batch gda_batch;

/* n instances: N[k] spins, model[k], R[k] restarts, J[k] (N[k]^2 doubles,
 * host, symmetric, finite), g[k] (N[k] doubles or NULL; g may be NULL).
 * Instance k uses Philox key seed + k * 0x9E3779B97F4A7C15 (mod 2^64).
 * Errors: GDA_ERR_INVALID, GDA_ERR_UNSUPPORTED (not an sm_103 device), OOM. */
gda_status gda_batch_create(int32_t n, const int32_t* N, const int32_t* model, const int32_t* R,
                            const double* const* J, const double* const* g, uint64_t seed, gda_batch** out);
gda_status gda_batch_set_stream(gda_batch* b, void* stream);

/* Tile width of the coupling product: 128 or 256 columns (the caller times
 * both and keeps the faster). */
gda_status gda_batch_set_tile(gda_batch* b, int32_t bn);

/* Launch schedule of the batch: GDA_SCHEDULE_RESIDENT (the default) runs each
 * chunk of 100 steps as one persistent launch with steps ordered by per-tile
 * flags; GDA_SCHEDULE_PER_STEP launches every step separately (the kernel
 * boundary orders the steps).  Same numbers either way; which is faster
 * depends on the mix (the caller times both).  GDA_ERR_INVALID otherwise. */
gda_status gda_batch_set_schedule(gda_batch* b, int32_t schedule);

/* Runs `steps` forward-Euler BF16 steps of every instance (p->integ must be
 * GDA_EULER, p->prec GDA_BF16; noise without decay; init_mode 0, 1, 2 or 3;
 * p->seed is ignored: instances use their own keys).  dt, eps, rho_th, beta0
 * and eps_hat of p apply to the instances without their own settings;
 * noise_D, init_amp, gamma0 and wait_s to all.  Asynchronous. */
gda_status gda_batch_run(gda_batch* b, const gda_params* p, int64_t steps);

/* Instance k's own settings: dt, eps, rho_th, beta0 and eps_hat of p replace
 * the run's for instance k in later runs (the learned proposal gives each
 * instance its own; instances of different coupling scales need their own
 * dt); p = NULL returns instance k to the run's settings.  GDA_ERR_INVALID
 * for k out of range, non-finite values, dt <= 0 or rho_th <= 0. */
gda_status gda_batch_set_params(gda_batch* b, int32_t k, const gda_params* p);

/* Base amplitudes of instance k for init_mode 3, as gda_set_init_base: N[k]
 * floats (Ising) or N[k] interleaved (re, im) pairs (XY), host (on_device =
 * 0) or device (1), copied; a run with init_mode 3 starts restart r of
 * instance k at base_i + the init_mode 1 perturbation of (i, r) (instances
 * without a base: the perturbation alone).  base = NULL clears it.
 * Synchronises. */
gda_status gda_batch_set_init_base(gda_batch* b, int32_t k, const float* base, int32_t on_device);

/* 1 if the batch's chunks replay a captured CUDA graph, 0 if they are
 * launched directly (the CUDA runtime declined to capture the cooperative launch),
 * -1 for b = NULL. */
int32_t gda_batch_launch_mode(const gda_batch* b);

/* FP64 Eq. (1) energy of the best restart of every instance (ties: lowest
 * restart) into E[n], r[n] (host, either may be NULL).  Synchronises and
 * reports device errors of earlier runs. */
gda_status gda_batch_best(gda_batch* b, double* E, int32_t* r);

/* State of instance k in the gda_get_state layout (host).  Synchronises. */
gda_status gda_batch_get_state(gda_batch* b, int32_t k, float* psi, float* gamma, float* beta);
const char* gda_batch_last_error(const gda_batch* b);
void gda_batch_destroy(gda_batch* b);

/* Number of kernels the library launched on this context since creation. */
int64_t gda_kernel_launches(const gda_ctx* ctx);

/* Last error message of this context ("" if none). */
const char* gda_last_error(const gda_ctx* ctx);

/* Static description of a status code. */
const char* gda_status_string(gda_status s);

/* Frees the context and all its device memory (NULL is a no-op). */
void gda_destroy(gda_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GDA_H */
