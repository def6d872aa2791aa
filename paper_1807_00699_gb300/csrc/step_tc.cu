// BF16 instantiation of the tensor-core step kernel (step_tc.cuh) and the
// tile-width choice shared by both precisions.
#include "step_tc.cuh"

namespace gda {

int tc_mtiles(int N) { return (N + BM - 1) / BM; }

long long ptx_default_wait_cycles() { return kWaitCycles; }
double ptx_cycles_per_second() { return kCyclesPerSecond; }

// Two-SM pairs: a 256 x BN pair tile costs each SM about max(BN, 128 + BN / 2)
// cycles per 16-deep K slice (MMA time against its shared-memory feed: own A
// rows plus half of B), over ceil(pair tiles / clusters) rounds.
int tc_pick_bn_pair(int N, int C) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 2) sms = 148;
  }
  const int clusters = sms / 2;
  const int widths[3] = {128, 224, 256};
  int best = 128;
  long long best_cost = -1;
  for (int bn : widths) {
    const long long ptiles = (long long)((C + bn - 1) / bn) * (((N + BM - 1) / BM) / 2);
    const long long per = bn > 128 + bn / 2 ? bn : 128 + bn / 2;
    const long long cost = ((ptiles + clusters - 1) / clusters) * per;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = bn;
    }
  }
  return best;
}

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

// AUTO's choice: two-SM tiles when the row blocks pair up and the pair tiles
// fill at least three waves of clusters (measured on GB300: 5-10 % faster at
// N = R = 4096 and above, 5-15 % slower on one or two waves).
bool tc_pair_pays(int N, int C) {
  const int mt = (N + BM - 1) / BM;
  if (mt % 2) return false;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 2) return false;
  const int bn = tc_pick_bn_pair(N, C);
  const long long ptiles = (long long)((C + bn - 1) / bn) * (mt / 2);
  return ptiles >= 3LL * (sms / 2);
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
  if (!plan_maps<false>(p, J16, Np, ops, n_op_bufs, Cp)) {
    delete p;
    return cudaErrorInvalidValue;
  }
  *plan = p;
  return cudaSuccess;
}

void tc_plan_destroy(TcPlan* plan) { delete plan; }

const CUtensorMap* tc_plan_A(const TcPlan* plan) { return &plan->A; }
const CUtensorMap* tc_plan_B(const TcPlan* plan) { return &plan->B128; }
const CUtensorMap* tc_plan_B64(const TcPlan* plan) { return &plan->B64; }

cudaError_t launch_step_tc(const TcPlan* plan, const StepArgs& a, int op_buf, cudaStream_t s, bool pair) {
  return launch_plan<false>(plan, a, op_buf, pair, s);
}

cudaError_t launch_step_tcs(const TcPlan* plan, const StepArgs& a, const SegArgs& g, cudaStream_t s, bool pair) {
  return launch_seg_plan<false>(plan, a, g, pair, s);
}

}  // namespace gda
