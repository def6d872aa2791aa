// Launch interface of the resident persistent kernel (step_res.cu).
#pragma once
#include <cuda.h>

#include "gda_internal.h"

namespace gda {

struct ResArgs {
  int steps;                // steps run by this launch
  int buf0;                 // operand buffer holding bf16(psi) of the first step
  int Cp;                   // rows of one operand buffer
  unsigned* flags;          // per-tile step flags [column block][row block], zero at launch
  float* psi_final;         // FP32 amplitudes written after the last step [Cp][Np]
  float* beta_final;        // coupling scale after the last step [Rp]
  float* rho[2];            // density partial sums: rho[0] of the first step's state
  __nv_bfloat16* ops;       // operand buffers [2][Cp][Np]
  int withhold_tile;        // testing: tile (column block * row blocks + row block) that
  int withhold_step;        // does not release its flag value withhold_step (-1: none)
};

// True if every CTA of the launch for N spins and C columns fits on the device at once.
bool res_fits(int N, int C, int device);
// The same for the two-SM form (clusters of two row blocks; the current
// device): an even number of row blocks and every cluster resident at once.
bool res_pair_fits(int N, int C);
cudaError_t launch_step_res(const TcPlan* plan, const ResArgs& ra, const StepArgs& a, cudaStream_t s, bool pair);
const CUtensorMap* tc_plan_A(const TcPlan* plan);
const CUtensorMap* tc_plan_B(const TcPlan* plan);    // 128-row operand boxes
const CUtensorMap* tc_plan_B64(const TcPlan* plan);  // 64-row operand boxes (halves of a pair's tile)

}  // namespace gda
