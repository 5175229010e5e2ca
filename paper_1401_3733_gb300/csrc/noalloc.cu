// noalloc.cu -- bsm_dirac_eo_noalloc: the even-odd Schur operator with its
// scratch in a fixed, library-owned device array instead of a caller
// workspace.  For callers that cannot allocate device memory (see bsm.h).
//
// The scratch is a file-scope __device__ array.  Its name in host code is
// only a host-side stand-in, not a device address, so the address is asked
// from the runtime once per device (cudaGetSymbolAddress with that device
// current) and cached; every call on that device then shares the array.
#include <mutex>

#include "operators.cuh"

namespace bsm {
namespace {

constexpr size_t kNoAllocScratchBytes = BSM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_eo_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// device address of g_eo_scratch on the current device (set up on first use)
int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return BSM_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_eo_scratch);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return BSM_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BSM_OK;
}

int check_lattice_local(const bsm_lattice* L) {
  if (L == nullptr) return BSM_EINVAL;
  int64_t V = 1;
  for (int m = 0; m < 4; ++m) {
    if (L->dims[m] < 2 || (L->dims[m] & 1)) return BSM_EINVAL;
    V *= L->dims[m];
    if (!isfinite(L->bc_phase[m])) return BSM_EINVAL;
  }
  if (V > ((int64_t)1 << 30)) return BSM_EUNSUPPORTED;
  if (!isfinite(L->m0) || 4.0 + L->m0 == 0.0) return BSM_EINVAL;
  const RepInfo ri = rep_info(L->N, L->rep);
  if (ri.d < 0) return BSM_EUNSUPPORTED;
  if (ri.real)
    for (int m = 0; m < 4; ++m) {
      const double k = L->bc_phase[m] / M_PI;
      if (fabs(k - nearbyint(k)) > 1e-12) return BSM_EUNSUPPORTED;
    }
  return BSM_OK;
}

bool aligned16(const void* p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace
}  // namespace bsm

using namespace bsm;

extern "C" int bsm_dirac_eo_noalloc(const bsm_lattice* lat, const void* U_rep, const void* in_e, void* out_e,
                                    int32_t op, int32_t prec, void* stream) {
  int rc = check_lattice_local(lat);
  if (rc != BSM_OK) return rc;
  if (prec != BSM_F64 && prec != BSM_F32) return BSM_EUNSUPPORTED;
  if (!aligned16(U_rep) || !aligned16(in_e) || !aligned16(out_e)) return BSM_EINVAL;
  if (op != BSM_OP_DHAT && op != BSM_OP_DHAT_DAG && op != BSM_OP_DHAT_DAG_DHAT) return BSM_EINVAL;
  const OpCtx c = make_ctx(*lat, U_rep, prec, (cudaStream_t)stream);
  if (2 * c.half_bytes > kNoAllocScratchBytes) return BSM_EWORKSPACE;  // lattice too large for the array
  {
    const uintptr_t a = reinterpret_cast<uintptr_t>(in_e), b = reinterpret_cast<uintptr_t>(out_e);
    if (a < b + c.half_bytes && b < a + c.half_bytes) return BSM_EINVAL;
  }
  void* scratch = nullptr;
  if ((rc = scratch_address(&scratch)) != BSM_OK) return rc;
  // both scratch halves are written in full before they are read, so the
  // previous call's contents need no clearing
  char* t = reinterpret_cast<char*>(scratch);
  char* u = t + c.half_bytes;
  if (op == BSM_OP_DHAT_DAG_DHAT) {
    rc = op_dhat(c, in_e, u, t, 0, nullptr, nullptr);
    if (rc >= 0) rc = op_dhat(c, u, out_e, t, 1, nullptr, nullptr);
  } else {
    rc = op_dhat(c, in_e, out_e, t, op == BSM_OP_DHAT_DAG, nullptr, nullptr);
  }
  if (rc < 0) return rc;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return BSM_OK;
}
