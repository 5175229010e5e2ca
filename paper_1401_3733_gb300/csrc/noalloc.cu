// noalloc.cu -- bsm_dirac_eo_noalloc: the even-odd Schur operator with its
// scratch in a fixed, library-owned device array instead of a caller
// workspace.  For callers that cannot allocate device memory (see bsm.h).
//
// The scratch is a file-scope __device__ array.  Its name in host code is
// only a host-side stand-in, not a device address, so the address is asked
// from the runtime once per device (cudaGetSymbolAddress with that device
// current) and cached; every call on that device then shares the array.
// The runtime reserves the array when it loads this module on a device:
// under lazy module loading (the default) inside that first lookup, under
// eager loading when the context is created.  Calls after the first on a
// device therefore reserve no device memory.
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

}  // namespace
}  // namespace bsm

using namespace bsm;

extern "C" int bsm_dirac_eo_noalloc(const bsm_lattice* lat, const void* U_rep, const void* in_e, void* out_e,
                                    int32_t op, int32_t prec, void* stream) {
  // the same argument checks as bsm_dirac_eo
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if (!prec_lat_ok(lat, prec)) return BSM_EUNSUPPORTED;
  if (!aligned(U_rep) || !aligned(in_e) || !aligned(out_e)) return BSM_EINVAL;
  if (op != BSM_OP_DHAT && op != BSM_OP_DHAT_DAG && op != BSM_OP_DHAT_DAG_DHAT) return BSM_EINVAL;
  const OpCtx c = make_ctx(*lat, U_rep, prec, (cudaStream_t)stream);
  if (2 * c.half_bytes > kNoAllocScratchBytes) return BSM_EWORKSPACE;  // lattice too large for the array
  if (overlap(in_e, c.half_bytes, out_e, c.half_bytes)) return BSM_EINVAL;
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
