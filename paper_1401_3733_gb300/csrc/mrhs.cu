// mrhs.cu -- launch of the multi-RHS hopping block with an autotuned RHS
// block: the first launch for a (precision, d, n_rhs, V_h) shape times every
// compiled block size RB that divides n_rhs, the f32x2-paired kernels (2 or 4
// RHS per thread as lane pairs) and the tensor-core kernel where it applies
// (BF16, d = 4, 6, 8), on the caller's stream and keeps the fastest for the
// rest of the process.
#include <map>
#include <mutex>
#include <tuple>

#include <stdlib.h>

#include "mrhs.cuh"

namespace bsm {

bool launch_mrhs_f32(int d, bool real, int rb, const MrhsArgs& A, cudaStream_t s);
bool launch_mrhs_bf16(int d, bool real, int rb, const MrhsArgs& A, cudaStream_t s);
bool launch_mrhs_tc(int prec, int d, bool real, const MrhsArgs& A, cudaStream_t s);

// RHS-block code of the tensor-core kernel (one warp per site, all RHS)
constexpr int kTensorCoreBlock = 16;

namespace {

using TuneKey = std::tuple<int, int, bool, int, int>;  // prec, d, real, nrhs, V_h
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

bool launch_rb(int prec, int d, bool real, int rb, const MrhsArgs& A, cudaStream_t s) {
  if (rb == kTensorCoreBlock) return launch_mrhs_tc(prec, d, real, A, s);
  if (prec == BSM_F32) return launch_mrhs_f32(d, real, rb, A, s);
  if (prec == BSM_BF16) return launch_mrhs_bf16(d, real, rb, A, s);
  return false;
}

int max_rb(int d) { return d <= 3 ? 4 : 2; }

// time one candidate: one warm-up launch, then the mean of three
float time_rb(int prec, int d, bool real, int rb, const MrhsArgs& A, cudaStream_t s, cudaEvent_t e0,
              cudaEvent_t e1) {
  if (!launch_rb(prec, d, real, rb, A, s)) return -1.f;
  cudaEventRecord(e0, s);
  for (int k = 0; k < 3; ++k) launch_rb(prec, d, real, rb, A, s);
  cudaEventRecord(e1, s);
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
  float ms = -1.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

}  // namespace

// pins the block of a shape (0 forgets it, so the next launch tunes again);
// false if that block is not available for the shape
bool mrhs_set_block(int prec, int d, bool real, int nrhs, int Vh, int block) {
  const TuneKey key(prec, d, real, nrhs, Vh);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (block == 0) {
    g_tuned.erase(key);
    return true;
  }
  if (block == kTensorCoreBlock) {
    if (prec != BSM_BF16 || real || !(d == 4 || d == 6 || d == 8) || nrhs % 4 != 0 || nrhs > 16) return false;
  } else if (block == kPairedBlock + 2 || block == kPairedBlock + 4) {
    if (block - kPairedBlock > max_rb(d) || nrhs % (block - kPairedBlock) != 0) return false;
  } else if (block < 1 || block > max_rb(d) || nrhs % block != 0) {
    return false;
  }
  g_tuned[key] = block;
  return true;
}

int mrhs_tuned_block(int prec, int d, bool real, int nrhs, int Vh) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const auto it = g_tuned.find(TuneKey(prec, d, real, nrhs, Vh));
  return it == g_tuned.end() ? 0 : it->second;
}

// returns 0 or a bsm_status
int launch_mrhs(int prec, int d, bool real, const MrhsArgs& A, cudaStream_t s) {
  const TuneKey key(prec, d, real, A.nrhs, A.g.Vh);
  int rb = 0;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto it = g_tuned.find(key);
    if (it != g_tuned.end()) rb = it->second;
  }
  if (rb == 0) {
    const char* env = getenv("BSM_MRHS_TUNE");
    const bool tune = !(env != nullptr && env[0] == '0');
    int best = 1;
    if (tune) {
      cudaEvent_t e0, e1;
      if (cudaEventCreate(&e0) != cudaSuccess) return BSM_ECUDA;
      if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return BSM_ECUDA;
      }
      float best_ms = -1.f;
      for (int c = 1; c <= kPairedBlock + 4; ++c) {
        const bool paired = c == kPairedBlock + 2 || c == kPairedBlock + 4;
        const int rhs = paired ? c - kPairedBlock : c;
        if (!paired && c > max_rb(d) && c != kTensorCoreBlock) continue;
        if (paired && rhs > max_rb(d)) continue;
        if (c != kTensorCoreBlock && A.nrhs % rhs != 0) continue;
        const float ms = time_rb(prec, d, real, c, A, s, e0, e1);
        if (ms > 0.f && (best_ms < 0.f || ms < best_ms)) {
          best_ms = ms;
          best = c;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    } else {
      for (int c = max_rb(d) > 2 ? 2 : max_rb(d); c >= 1; --c)
        if (A.nrhs % c == 0) {
          best = c;
          break;
        }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = best;
    rb = best;
  }
  return launch_rb(prec, d, real, rb, A, s) ? 0 : BSM_EUNSUPPORTED;
}

}  // namespace bsm
