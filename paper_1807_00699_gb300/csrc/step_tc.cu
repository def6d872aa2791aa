// BF16 instantiation of the tensor-core step kernel (step_tc.cuh) and the
// tile-width choice shared by both precisions.
#include "step_tc.cuh"

namespace gda {

int tc_mtiles(int N) { return (N + BM - 1) / BM; }

// Tile width for N spins and C columns: the busiest CTA runs ceil(tiles / SMs)
// tiles, and a 128 x BN tile costs about (128 + BN) shared-memory cycles per
// K-slice of 16 (MMA reads plus TMA writes of A and B at ~128 B/clk), so pick
// the width minimising rounds x (128 + BN).
int tc_pick_bn(int N, int C) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
  }
  const int widths[3] = {128, 224, 256};
  int best = 128;
  long long best_cost = -1;
  for (int bn : widths) {
    const long long tiles = (long long)((C + bn - 1) / bn) * ((N + BM - 1) / BM);
    const long long cost = ((tiles + sms - 1) / sms) * (128 + bn);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = bn;
    }
  }
  return best;
}

bool tc_supported(int device) {
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) return false;
  return major == 10 && minor == 3 && get_encode() != nullptr;
}

cudaError_t tc_plan_create(TcPlan** plan, const __nv_bfloat16* J16, int Np, const __nv_bfloat16* ops, int n_op_bufs,
                           int Cp) {
  TcPlan* p = new TcPlan();
  p->Cp = Cp;
  if (!make_map(&p->A, J16, Np, Np, BM) || !make_map(&p->B128, ops, Np, n_op_bufs * Cp, 128) ||
      !make_map(&p->B224, ops, Np, n_op_bufs * Cp, 224) || !make_map(&p->B256, ops, Np, n_op_bufs * Cp, 256)) {
    delete p;
    return cudaErrorInvalidValue;
  }
  *plan = p;
  return cudaSuccess;
}

void tc_plan_destroy(TcPlan* plan) { delete plan; }

const CUtensorMap* tc_plan_A(const TcPlan* plan) { return &plan->A; }
const CUtensorMap* tc_plan_B(const TcPlan* plan) { return &plan->B128; }

cudaError_t launch_step_tc(const TcPlan* plan, const StepArgs& a, int op_buf, cudaStream_t s) {
  const int b_row0 = op_buf * plan->Cp;
  const int bn = tc_pick_bn(a.N, a.C);
  if (bn == 256) return dispatch_mode<256, 4, false>(plan->A, plan->B256, b_row0, a, s);
  if (bn == 224) return dispatch_mode<224, 4, false>(plan->A, plan->B224, b_row0, a, s);
  return dispatch_mode<128, 6, false>(plan->A, plan->B128, b_row0, a, s);
}

}  // namespace gda
