// Launchers of the small kernels in energy.cu (projection, energies, argmin,
// state initialisation).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "philox.cuh"

namespace gda {

cudaError_t launch_init_state(float* psi, float* gam, float* beta, int N, int Np, int R, int cplx, int mode,
                              float amp, float gamma0, float beta0, unsigned long long seed, const float* base,
                              cudaStream_t s);
cudaError_t launch_fill_h1(const double* g, float* h1, int N, float sq, cudaStream_t s);
cudaError_t launch_to_bf16(const float* x, __nv_bfloat16* y, size_t n, cudaStream_t s);
cudaError_t launch_rho_partials(bool tc, const float* psi, int N, int Np, int R, int Rp, int cplx, float* out,
                                cudaStream_t s);
cudaError_t launch_project_f32(const float* psi, float* S, int N, int Np, int R, int cplx, cudaStream_t s);
cudaError_t launch_project_bf16(const float* psi, __nv_bfloat16* S, int N, int Np, int R, int cplx, cudaStream_t s);
cudaError_t launch_track_reduce(const float* e_part, int mt, int R, int Rp, double diag, long long step,
                                long long* t_step, double* t_E, int* t_r, int cap, int* count, double* lastE,
                                int* lastR, cudaStream_t s);
// Running best of the trace (energy.cu): copy restart *lastR's amplitudes to
// snap when *lastE improves on *snapE; reset before a fresh run.  With hist,
// also keep them as trace entry *count - 1 (if below hist_cap).
cudaError_t launch_snapshot(const float* psi, int Np, int W, const double* lastE, const int* lastR, long long step,
                            double* snapE, int* snapR, long long* snapStep, float* snap, float* hist, int hist_cap,
                            const int* count, cudaStream_t s);
cudaError_t launch_snapshot_reset(double* snapE, int* snapR, long long* snapStep, cudaStream_t s);
cudaError_t launch_energy64(const float* psi, const double* J64, const double* g, double* S64, double* part,
                            double* E, int N, int Np, int R, int Rp, int C, int cplx, cudaStream_t s);
cudaError_t launch_energy_int(const float* psi, const int* Jint, int* Sint, long long* part, double* E, int N,
                              int Np, int R, int Rp, int C, cudaStream_t s);
cudaError_t launch_argmin(const double* E, int R, double* bestE, int* bestR, cudaStream_t s);
cudaError_t launch_best_cfg(const float* psi, const int* bestR, int N, int Np, int cplx, signed char* s8, double* th,
                            cudaStream_t s);

}  // namespace gda

namespace gda {
cudaError_t launch_pack_state(const float* psi, const float* gam, const float* beta, int N, int Np, int R, int cplx,
                              float* hpsi, float* hgam, float* hbeta, cudaStream_t s);
cudaError_t launch_unpack_state(float* psi, float* gam, float* beta, int N, int Np, int R, int cplx, const float* hpsi,
                                const float* hgam, const float* hbeta, cudaStream_t s);
cudaError_t launch_check_instance(const double* J64, const double* g, int N, int Np, int* flags,
                                  unsigned long long* maxabs, double* diag, cudaStream_t s);
cudaError_t launch_prepare_J(const double* J64, int Np, float* J32, __nv_bfloat16* J16, int* Jint, cudaStream_t s);
// Candidate ranking for the FP64 argmin (energy.cu): *out = sum_ij |J0_ij| + sum |g|;
// compensated FP32 energies of all restarts into E32 and the restarts within
// margin of their minimum (ascending) into idx[0 .. *count); candidate columns
// gathered into a compact buffer; bestR mapped back through idx.
cudaError_t launch_abs_sum(const double* J64, const double* g, int N, int Np, double* out, cudaStream_t s);
cudaError_t launch_rank(const float* psi, const float* J32, const double* g, float* S32, double* part, double* E32,
                        int* idx, int* count, int N, int Np, int R, int Rp, int C, int cplx, double diag,
                        double margin, cudaStream_t s);
cudaError_t launch_gather_cols(const float* psi, int Np, const int* idx, int count, int cplx, float* out,
                               cudaStream_t s);
cudaError_t launch_map_best(const int* idx, int* bestR, cudaStream_t s);
cudaError_t launch_features(const double* J, const double* g, int N, int Np, int cplx, double* w0, double* w1,
                            float* F, cudaStream_t s);
}  // namespace gda
