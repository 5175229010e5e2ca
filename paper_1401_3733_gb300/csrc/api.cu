// api.cu -- the extern "C" entry points declared in include/bsm.h: argument
// validation (before any launch), size queries, dispatch to the kernels, and
// CUDA error mapping.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "blas.cuh"
#include "mrhs.cuh"
#include "operators.cuh"

namespace bsm {

int links_to_rep_launch(const bsm_lattice& L, const double* U, void* out, int prec, cudaStream_t s);
void pack_spinor_launch(const bsm_lattice& L, const double* canon, void* dev, int d, int prec, bool unpack,
                        int nrhs, bool site_major, cudaStream_t s);
int launch_mrhs(int prec, int d, bool real, const MrhsArgs& A, cudaStream_t s);
int mrhs_tuned_block(int prec, int d, bool real, int nrhs, int Vh);
size_t batch_workspace_bytes(const bsm_batch_item* items, int count, int op);
int batch_launch(const bsm_batch_item* items, int count, const bsm_batch_opts& o, void* ws, cudaStream_t s,
                 bool sync);
int batch_status(void* ws, cudaStream_t s);
void batch_last_config(int* rb, int* grab);
bool mrhs_set_block(int prec, int d, bool real, int nrhs, int Vh, int block);
size_t cg_workspace_bytes(const bsm_lattice& L, int prec_inner, int eo, int prec_outer);
size_t cg_batch_workspace_bytes(const bsm_cg_batch_item* items, int count);
int cg_solve_batch(const bsm_cg_batch_item* items, int count, const bsm_cg_opts& o, bsm_cg_stats* stats, void* ws,
                   cudaStream_t s);
int cg_solve(const bsm_lattice& L, const void* U64, const void* U32, const void* b, void* x,
             const bsm_cg_opts& o, bsm_cg_stats* stats, void* ws, cudaStream_t s);
size_t ptc_workspace_bytes(const bsm_lattice& L, int C, int nb, bool train);
int ptc_pack(const bsm_lattice& L, const double* psi, void* F, bool unpack, bool even_only, cudaStream_t s);
int ptc_apply(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* in,
              void* out, int nb, int prec, void* ws, cudaStream_t s, bool even_only = false, bool reset_err = true);
int ptc_loss_grad(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* r,
                  const void* e, int nb, void* GW1, void* GW2, double* loss, void* ws, cudaStream_t s);
int ptc_adam(void* W, const void* G, void* m, void* v, long long nfloat, double lr, int step, cudaStream_t s);
size_t fgcr_workspace_bytes(const bsm_lattice& L, const bsm_fgcr_opts& o);
int fgcr_solve(const bsm_lattice& L, const void* U64, const void* U32, const void* W1, const void* W2,
               const void* b, void* x, const bsm_fgcr_opts& o, bsm_fgcr_stats* stats, void* ws, cudaStream_t s);

// FGCR's workspace, or the larger of FGCR's and its fallback CG's
size_t fgcr_total_workspace_bytes(const bsm_lattice& L, const bsm_fgcr_opts& o) {
  size_t n = fgcr_workspace_bytes(L, o);
  if (o.fallback != 0) {
    const size_t c = cg_workspace_bytes(L, BSM_F32, o.eo, o.prec_outer);
    const size_t p = cg_workspace_bytes(L, o.prec_outer, o.eo, o.prec_outer);
    n = std::max(n, std::max(c, p));
  }
  return n;
}

RepInfo rep_info(int N, int rep) {
  RepInfo r{-1, false};
  switch (rep) {
    case BSM_FUND:
      if (N == 2 || N == 3 || N == 4 || N == 6 || N == 8) r.d = N;
      break;
    case BSM_ADJ:
      if (N == 2 || N == 3) {
        r.d = N * N - 1;
        r.real = true;
      }
      break;
    case BSM_SYM:
      if (N == 2 || N == 3) r.d = N * (N + 1) / 2;
      break;
    case BSM_ASYM:
      if (N == 3 || N == 4) r.d = N * (N - 1) / 2;
      break;
    default:
      break;
  }
  return r;
}

namespace {
thread_local char g_cuda_err[256] = "";
}

void set_cuda_error(cudaError_t e) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

// checks every field of the lattice; BSM_OK, BSM_EINVAL or BSM_EUNSUPPORTED
int check_lattice(const bsm_lattice* L) {
  if (L == nullptr) return BSM_EINVAL;
  int64_t V = 1;
  for (int m = 0; m < 4; ++m) {
    if (L->dims[m] < 2 || (L->dims[m] & 1)) return BSM_EINVAL;
    V *= L->dims[m];
    if (!isfinite(L->bc_phase[m])) return BSM_EINVAL;
  }
  if (V > ((int64_t)1 << 30)) return BSM_EUNSUPPORTED;  // 32-bit site indexing with headroom
  if (!isfinite(L->m0) || 4.0 + L->m0 == 0.0) return BSM_EINVAL;
  const RepInfo ri = rep_info(L->N, L->rep);
  if (ri.d < 0) return BSM_EUNSUPPORTED;
  if (ri.real) {
    // a real representation stays real only for phases that are multiples of pi
    for (int m = 0; m < 4; ++m) {
      const double k = L->bc_phase[m] / M_PI;
      if (fabs(k - nearbyint(k)) > 1e-12) return BSM_EUNSUPPORTED;
    }
  }
  return BSM_OK;
}

bool aligned(const void* p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
bool prec_ok(int prec) {
  return prec == BSM_F64 || prec == BSM_F32 || prec == BSM_DF64 || prec == BSM_BF16 || prec == BSM_F32R12;
}
// two-row links exist for SU(3) fundamental only
bool prec_lat_ok(const bsm_lattice* L, int prec) {
  return prec_ok(prec) && (prec != BSM_F32R12 || (L->N == 3 && L->rep == BSM_FUND));
}

// true when the byte ranges [a, a + na) and [b, b + nb) intersect
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

namespace {

int finish(int rc) {
  if (rc != BSM_OK) return rc;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return BSM_OK;
}

// multi-RHS: supported precisions and the 32-bit (site, rhs) index bound
int check_mrhs(const bsm_lattice* L, int nrhs, int prec) {
  if (nrhs < 1) return BSM_EINVAL;
  if (prec != BSM_F32 && prec != BSM_BF16) return BSM_EUNSUPPORTED;
  const int64_t V = (int64_t)L->dims[0] * L->dims[1] * L->dims[2] * L->dims[3];
  if (V * nrhs > ((int64_t)1 << 30)) return BSM_EUNSUPPORTED;
  return BSM_OK;
}

// batch: SU(2)/SU(3) fundamental items, FP32, sane options
int check_batch(const bsm_batch_item* items, int count, const bsm_batch_opts* o) {
  if (items == nullptr || o == nullptr || count < 1 || count > 32) return BSM_EINVAL;
  if (o->op != BSM_BATCH_D && o->op != BSM_BATCH_DHAT) return BSM_EINVAL;
  if (o->prec != BSM_F32) return BSM_EUNSUPPORTED;
  if (!(o->timeout_s >= 0.0) || o->timeout_s > 60.0) return BSM_EINVAL;
  for (int k = 0; k < count; ++k) {
    const bsm_batch_item& it = items[k];
    int rc = check_lattice(&it.lat);
    if (rc != BSM_OK) return rc;
    if (it.lat.rep != BSM_FUND || (it.lat.N != 2 && it.lat.N != 3)) return BSM_EUNSUPPORTED;
    if ((rc = check_mrhs(&it.lat, it.nrhs, o->prec)) != BSM_OK) return rc;
    if (!aligned(it.U_rep) || !aligned(it.in) || !aligned(it.out)) return BSM_EINVAL;
    const Geom g = make_geom(it.lat);
    const size_t n = half_spinor_bytes(g.Vh, it.lat.N, BSM_F32) * it.nrhs * (o->op == BSM_BATCH_D ? 2 : 1);
    if (overlap(it.in, n, it.out, n)) return BSM_EINVAL;
  }
  return BSM_OK;
}

// learned preconditioner: complex d = 2, 3; channels 1..64; 32-bit GEMM rows
int check_ptc(const bsm_lattice* L, int C, int nb) {
  const int rc = check_lattice(L);
  if (rc != BSM_OK) return rc;
  if (C < 1 || C > 64 || nb < 1) return BSM_EINVAL;
  const RepInfo ri = rep_info(L->N, L->rep);
  if (ri.real || (ri.d != 2 && ri.d != 3)) return BSM_EUNSUPPORTED;
  const int64_t V = (int64_t)L->dims[0] * L->dims[1] * L->dims[2] * L->dims[3];
  if (V * ri.d * nb > ((int64_t)1 << 28)) return BSM_EUNSUPPORTED;
  return BSM_OK;
}

}  // namespace
}  // namespace bsm

using namespace bsm;

extern "C" {

int bsm_rep_dim(int32_t N, int32_t rep) {
  const RepInfo r = rep_info(N, rep);
  return r.d < 0 ? BSM_EUNSUPPORTED : r.d;
}

size_t bsm_field_bytes(const bsm_lattice* lat, int32_t kind, int32_t prec) {
  if (check_lattice(lat) != BSM_OK) return 0;
  const Geom g = make_geom(*lat);
  const RepInfo ri = rep_info(lat->N, lat->rep);
  const size_t V = 2 * (size_t)g.Vh;
  switch (kind) {
    case BSM_FIELD_FUND_CANON: return V * 4 * lat->N * lat->N * 16;
    case BSM_FIELD_SPINOR_CANON: return V * 4 * ri.d * 16;
    default: break;
  }
  if (!prec_lat_ok(lat, prec)) return 0;
  switch (kind) {
    case BSM_FIELD_LINKS: return 2 * link_block_bytes(g.Vh, ri.d, ri.real, prec);
    case BSM_FIELD_SPINOR: return 2 * half_spinor_bytes(g.Vh, ri.d, prec);
    case BSM_FIELD_HALF_SPINOR: return half_spinor_bytes(g.Vh, ri.d, prec);
    default: return 0;
  }
}

size_t bsm_workspace_bytes(const bsm_lattice* lat, int32_t call, int32_t prec) {
  if (check_lattice(lat) != BSM_OK || !prec_lat_ok(lat, prec)) return 0;
  const Geom g = make_geom(*lat);
  const RepInfo ri = rep_info(lat->N, lat->rep);
  if (call == BSM_CALL_DIRAC_EO) return 2 * half_spinor_bytes(g.Vh, ri.d, prec);
  if (call == BSM_CALL_CG) {
    // the largest layout over even-odd/full and, for a mixed inner
    // precision, over both outer precisions
    size_t m = 0;
    const bool mixed = prec == BSM_F32 || prec == BSM_F32R12;
    const int outers[2] = {mixed ? BSM_F64 : prec, mixed ? BSM_DF64 : prec};
    for (int k = 0; k < 2; ++k)
      for (int eo = 0; eo < 2; ++eo) {
        const size_t v = cg_workspace_bytes(*lat, prec, eo, outers[k]);
        m = v > m ? v : m;
      }
    return m;
  }
  return 0;
}

int bsm_pack_spinor(const bsm_lattice* lat, const double* canon, void* dev, int32_t prec, void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if (!prec_lat_ok(lat, prec)) return BSM_EUNSUPPORTED;
  if (!aligned(canon) || !aligned(dev)) return BSM_EINVAL;
  pack_spinor_launch(*lat, canon, dev, rep_info(lat->N, lat->rep).d, prec, false, 1, false, (cudaStream_t)stream);
  return finish(BSM_OK);
}

int bsm_unpack_spinor(const bsm_lattice* lat, const void* dev, double* canon, int32_t prec, void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if (!prec_lat_ok(lat, prec)) return BSM_EUNSUPPORTED;
  if (!aligned(canon) || !aligned(dev)) return BSM_EINVAL;
  pack_spinor_launch(*lat, canon, const_cast<void*>(dev), rep_info(lat->N, lat->rep).d, prec, true, 1, false,
                     (cudaStream_t)stream);
  return finish(BSM_OK);
}

int bsm_links_to_rep(const bsm_lattice* lat, const double* U_fund, void* U_rep, int32_t prec, void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if (!prec_lat_ok(lat, prec)) return BSM_EUNSUPPORTED;
  if (!aligned(U_fund) || !aligned(U_rep)) return BSM_EINVAL;
  return finish(links_to_rep_launch(*lat, U_fund, U_rep, prec, (cudaStream_t)stream));
}

int bsm_dslash(const bsm_lattice* lat, const void* U_rep, const void* in, void* out, int32_t out_parity,
               int32_t dagger, int32_t prec, void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if (!prec_lat_ok(lat, prec)) return BSM_EUNSUPPORTED;
  if (!aligned(U_rep) || !aligned(in) || !aligned(out)) return BSM_EINVAL;
  if (out_parity != BSM_EVEN && out_parity != BSM_ODD && out_parity != BSM_FULL) return BSM_EINVAL;
  const OpCtx c = make_ctx(*lat, U_rep, prec, (cudaStream_t)stream);
  const size_t n = out_parity == BSM_FULL ? 2 * c.half_bytes : c.half_bytes;
  if (overlap(in, n, out, n)) return BSM_EINVAL;  // the stencil reads neighbours of what it writes
  if (out_parity == BSM_FULL) rc = op_dirac(c, in, out, dagger != 0, nullptr, nullptr);
  else rc = op_hop(c, out_parity, in, out, dagger != 0, nullptr, 0.0, 1.0, nullptr, nullptr);
  return finish(rc < 0 ? rc : BSM_OK);
}

int bsm_pack_spinor_mrhs(const bsm_lattice* lat, const double* canon, void* dev, int32_t nrhs, int32_t prec,
                         void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if ((rc = check_mrhs(lat, nrhs, prec)) != BSM_OK) return rc;
  if (!aligned(canon) || !aligned(dev)) return BSM_EINVAL;
  pack_spinor_launch(*lat, canon, dev, rep_info(lat->N, lat->rep).d, prec, false, nrhs, true, (cudaStream_t)stream);
  return finish(BSM_OK);
}

int bsm_unpack_spinor_mrhs(const bsm_lattice* lat, const void* dev, double* canon, int32_t nrhs, int32_t prec,
                           void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if ((rc = check_mrhs(lat, nrhs, prec)) != BSM_OK) return rc;
  if (!aligned(canon) || !aligned(dev)) return BSM_EINVAL;
  pack_spinor_launch(*lat, canon, const_cast<void*>(dev), rep_info(lat->N, lat->rep).d, prec, true, nrhs, true,
                     (cudaStream_t)stream);
  return finish(BSM_OK);
}

int bsm_dslash_mrhs(const bsm_lattice* lat, const void* U_rep, const void* in, void* out, int32_t nrhs,
                    int32_t out_parity, int32_t dagger, int32_t prec, void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if ((rc = check_mrhs(lat, nrhs, prec)) != BSM_OK) return rc;
  if (!aligned(U_rep) || !aligned(in) || !aligned(out)) return BSM_EINVAL;
  if (out_parity != BSM_EVEN && out_parity != BSM_ODD && out_parity != BSM_FULL) return BSM_EINVAL;
  const OpCtx c = make_ctx(*lat, U_rep, prec, (cudaStream_t)stream);
  const size_t half = c.half_bytes * nrhs;
  const size_t n = out_parity == BSM_FULL ? 2 * half : half;
  if (overlap(in, n, out, n)) return BSM_EINVAL;
  MrhsArgs A;
  A.g = c.g;
  A.dagger = dagger != 0;
  A.nrhs = nrhs;
  const char* ic = reinterpret_cast<const char*>(in);
  char* oc = reinterpret_cast<char*>(out);
  const int first = out_parity == BSM_ODD ? 1 : 0, last = out_parity == BSM_EVEN ? 0 : 1;
  for (int p = first; p <= last; ++p) {
    A.links = c.links + (size_t)p * c.link_block;
    A.p = p;
    if (out_parity == BSM_FULL) {  // out_p = A in_p - 1/2 H in_{1-p}
      A.in = ic + (size_t)(1 - p) * half;
      A.out = oc + (size_t)p * half;
      A.x = ic + (size_t)p * half;
      A.a = c.A;
      A.b = -0.5;
    } else {  // the raw hopping block on half spinors
      A.in = in;
      A.out = out;
      A.x = nullptr;
      A.a = 0.0;
      A.b = 1.0;
    }
    if ((rc = launch_mrhs(prec, c.d, c.real, A, (cudaStream_t)stream)) != 0) return rc;
  }
  return finish(BSM_OK);
}

int bsm_dslash_mrhs_block(const bsm_lattice* lat, int32_t nrhs, int32_t prec) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if ((rc = check_mrhs(lat, nrhs, prec)) != BSM_OK) return rc;
  const RepInfo ri = rep_info(lat->N, lat->rep);
  return mrhs_tuned_block(prec, ri.d, ri.real, nrhs, make_geom(*lat).Vh);
}

int bsm_dslash_mrhs_set_block(const bsm_lattice* lat, int32_t nrhs, int32_t prec, int32_t block) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if ((rc = check_mrhs(lat, nrhs, prec)) != BSM_OK) return rc;
  const RepInfo ri = rep_info(lat->N, lat->rep);
  return mrhs_set_block(prec, ri.d, ri.real, nrhs, make_geom(*lat).Vh, block) ? BSM_OK : BSM_EUNSUPPORTED;
}

size_t bsm_batch_workspace_bytes(const bsm_batch_item* items, int32_t count, const bsm_batch_opts* opts) {
  if (check_batch(items, count, opts) != BSM_OK) return 0;
  return batch_workspace_bytes(items, count, opts->op);
}

namespace {
int dslash_batch(const bsm_batch_item* items, int32_t count, const bsm_batch_opts* opts, void* workspace,
                 size_t workspace_bytes, void* stream, bool sync) {
  const int rc = check_batch(items, count, opts);
  if (rc != BSM_OK) return rc;
  if (!aligned(workspace)) return BSM_EINVAL;
  if (workspace_bytes < batch_workspace_bytes(items, count, opts->op)) return BSM_EWORKSPACE;
  const cudaError_t pre = cudaGetLastError();
  if (pre != cudaSuccess) {
    set_cuda_error(pre);
    return BSM_ECUDA;
  }
  return batch_launch(items, count, *opts, workspace, (cudaStream_t)stream, sync);
}
}  // namespace

int bsm_dslash_batch(const bsm_batch_item* items, int32_t count, const bsm_batch_opts* opts, void* workspace,
                     size_t workspace_bytes, void* stream) {
  return dslash_batch(items, count, opts, workspace, workspace_bytes, stream, true);
}

int bsm_dslash_batch_async(const bsm_batch_item* items, int32_t count, const bsm_batch_opts* opts,
                           void* workspace, size_t workspace_bytes, void* stream) {
  return dslash_batch(items, count, opts, workspace, workspace_bytes, stream, false);
}

int bsm_batch_last_config(int32_t* rhs_per_thread, int32_t* chunks_per_grab) {
  if (rhs_per_thread == nullptr || chunks_per_grab == nullptr) return BSM_EINVAL;
  int rb = 1, grab = 4;
  batch_last_config(&rb, &grab);
  *rhs_per_thread = rb;
  *chunks_per_grab = grab;
  return BSM_OK;
}

int bsm_dslash_batch_status(void* workspace, void* stream) {
  if (!aligned(workspace)) return BSM_EINVAL;
  return batch_status(workspace, (cudaStream_t)stream);
}

namespace {
int check_cg_batch(const bsm_cg_batch_item* items, int count) {
  if (items == nullptr || count < 1 || count > 32) return BSM_EINVAL;
  for (int k = 0; k < count; ++k) {
    const bsm_cg_batch_item& it = items[k];
    int rc = check_lattice(&it.lat);
    if (rc != BSM_OK) return rc;
    if (it.lat.rep != BSM_FUND || (it.lat.N != 2 && it.lat.N != 3)) return BSM_EUNSUPPORTED;
    if (it.nrhs != 1 && it.nrhs != 2 && it.nrhs != 4 && it.nrhs != 8 && it.nrhs != 16) return BSM_EINVAL;
    if ((rc = check_mrhs(&it.lat, it.nrhs, BSM_F32)) != BSM_OK) return rc;
    if (!aligned(it.U_rep64) || !aligned(it.U_rep32) || !aligned(it.b) || !aligned(it.x)) return BSM_EINVAL;
    const size_t n = bsm_field_bytes(&it.lat, BSM_FIELD_SPINOR, BSM_F64) * it.nrhs;
    if (overlap(it.b, n, it.x, n)) return BSM_EINVAL;
  }
  return BSM_OK;
}
}  // namespace

size_t bsm_cg_batch_workspace_bytes(const bsm_cg_batch_item* items, int32_t count) {
  if (check_cg_batch(items, count) != BSM_OK) return 0;
  return cg_batch_workspace_bytes(items, count);
}

int bsm_cg_solve_batch(const bsm_cg_batch_item* items, int32_t count, const bsm_cg_opts* opts, bsm_cg_stats* stats,
                       void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_cg_batch(items, count);
  if (rc != BSM_OK) return rc;
  if (opts == nullptr || !(opts->tol > 0.0) || opts->max_iter < 1 || opts->delta < 0.0 || opts->delta >= 1.0 ||
      opts->check_every < 0)
    return BSM_EINVAL;
  if (opts->prec_inner != BSM_F32 || opts->eo == 0 || opts->use_x0 != 0) return BSM_EUNSUPPORTED;
  if (opts->prec_outer != BSM_F64 && opts->prec_outer != BSM_DF64) return BSM_EUNSUPPORTED;
  if (!aligned(workspace)) return BSM_EINVAL;
  if (workspace_bytes < cg_batch_workspace_bytes(items, count)) return BSM_EWORKSPACE;
  const cudaError_t pre = cudaGetLastError();
  if (pre != cudaSuccess) {
    set_cuda_error(pre);
    return BSM_ECUDA;
  }
  rc = cg_solve_batch(items, count, *opts, stats, workspace, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return rc;
}

int bsm_dirac_eo(const bsm_lattice* lat, const void* U_rep, const void* in_e, void* out_e, int32_t op,
                 int32_t prec, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if (!prec_lat_ok(lat, prec)) return BSM_EUNSUPPORTED;
  if (!aligned(U_rep) || !aligned(in_e) || !aligned(out_e) || !aligned(workspace)) return BSM_EINVAL;
  if (op != BSM_OP_DHAT && op != BSM_OP_DHAT_DAG && op != BSM_OP_DHAT_DAG_DHAT) return BSM_EINVAL;
  const OpCtx c = make_ctx(*lat, U_rep, prec, (cudaStream_t)stream);
  if (workspace_bytes < 2 * c.half_bytes) return BSM_EWORKSPACE;
  if (overlap(in_e, c.half_bytes, out_e, c.half_bytes)) return BSM_EINVAL;
  char* t = reinterpret_cast<char*>(workspace);
  char* u = t + c.half_bytes;
  if (op == BSM_OP_DHAT_DAG_DHAT) {
    rc = op_dhat(c, in_e, u, t, 0, nullptr, nullptr);
    if (rc >= 0) rc = op_dhat(c, u, out_e, t, 1, nullptr, nullptr);
  } else {
    rc = op_dhat(c, in_e, out_e, t, op == BSM_OP_DHAT_DAG, nullptr, nullptr);
  }
  return finish(rc < 0 ? rc : BSM_OK);
}

int bsm_cg_solve(const bsm_lattice* lat, const void* U_rep64, const void* U_rep32, const void* b, void* x,
                 const bsm_cg_opts* opts, bsm_cg_stats* stats, void* workspace, size_t workspace_bytes,
                 void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if (opts == nullptr || !(opts->tol > 0.0) || opts->max_iter < 1 || opts->delta < 0.0 || opts->delta >= 1.0)
    return BSM_EINVAL;
  if (opts->prec_outer != BSM_F64 && opts->prec_outer != BSM_DF64) return BSM_EUNSUPPORTED;
  const bool mixed = opts->prec_inner == BSM_F32 || opts->prec_inner == BSM_F32R12;
  if (!mixed && opts->prec_inner != opts->prec_outer) return BSM_EUNSUPPORTED;
  if (!prec_lat_ok(lat, opts->prec_inner)) return BSM_EUNSUPPORTED;
  if (!aligned(U_rep64) || !aligned(b) || !aligned(x) || !aligned(workspace)) return BSM_EINVAL;
  if (mixed && !aligned(U_rep32)) return BSM_EINVAL;
  if (workspace_bytes < cg_workspace_bytes(*lat, opts->prec_inner, opts->eo != 0, opts->prec_outer))
    return BSM_EWORKSPACE;
  const size_t full = bsm_field_bytes(lat, BSM_FIELD_SPINOR, BSM_F64);
  if (overlap(b, full, x, full)) return BSM_EINVAL;
  const cudaError_t pre = cudaGetLastError();
  if (pre != cudaSuccess) {
    set_cuda_error(pre);
    return BSM_ECUDA;
  }
  rc = cg_solve(*lat, U_rep64, U_rep32, b, x, *opts, stats, workspace, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return rc;
}

int bsm_ptc_pack(const bsm_lattice* lat, const void* psi, void* field, void* stream) {
  int rc = check_ptc(lat, 1, 1);
  if (rc != BSM_OK) return rc;
  if (!aligned(psi) || !aligned(field)) return BSM_EINVAL;
  return finish(ptc_pack(*lat, reinterpret_cast<const double*>(psi), field, false, false, (cudaStream_t)stream));
}

int bsm_ptc_unpack(const bsm_lattice* lat, const void* field, void* psi, void* stream) {
  int rc = check_ptc(lat, 1, 1);
  if (rc != BSM_OK) return rc;
  if (!aligned(psi) || !aligned(field)) return BSM_EINVAL;
  return finish(ptc_pack(*lat, reinterpret_cast<const double*>(psi), const_cast<void*>(field), true, false,
                         (cudaStream_t)stream));
}

size_t bsm_ptc_workspace_bytes(const bsm_lattice* lat, int32_t channels, int32_t nbatch, int32_t train) {
  if (check_ptc(lat, channels, nbatch) != BSM_OK) return 0;
  return ptc_workspace_bytes(*lat, channels, nbatch, train != 0);
}

int bsm_ptc_apply(const bsm_lattice* lat, const void* U_rep32, const void* W1, const void* W2, int32_t channels,
                  const void* in, void* out, int32_t nbatch, int32_t prec, void* workspace, size_t workspace_bytes,
                  void* stream) {
  int rc = check_ptc(lat, channels, nbatch);
  if (rc != BSM_OK) return rc;
  if (prec != BSM_F32 && prec != BSM_BF16) return BSM_EUNSUPPORTED;
  if (!aligned(U_rep32) || !aligned(W1) || !aligned(W2) || !aligned(in) || !aligned(out) || !aligned(workspace))
    return BSM_EINVAL;
  if (workspace_bytes < ptc_workspace_bytes(*lat, channels, nbatch, false)) return BSM_EWORKSPACE;
  const int64_t V = (int64_t)lat->dims[0] * lat->dims[1] * lat->dims[2] * lat->dims[3];
  const size_t fb = (size_t)V * nbatch * rep_info(lat->N, lat->rep).d * 4 * 8;
  if (overlap(in, fb, out, fb)) return BSM_EINVAL;
  return finish(ptc_apply(*lat, U_rep32, W1, W2, channels, in, out, nbatch, prec, workspace, (cudaStream_t)stream));
}

int bsm_ptc_status(void* workspace, void* stream) {
  if (!aligned(workspace)) return BSM_EINVAL;
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, workspace, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return err ? BSM_ETIMEOUT : BSM_OK;
}

int bsm_ptc_loss_grad(const bsm_lattice* lat, const void* U_rep32, const void* W1, const void* W2, int32_t channels,
                      const void* r, const void* e, int32_t nbatch, void* G_W1, void* G_W2, double* loss,
                      void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_ptc(lat, channels, nbatch);
  if (rc != BSM_OK) return rc;
  if (!aligned(U_rep32) || !aligned(W1) || !aligned(W2) || !aligned(r) || !aligned(e) || !aligned(G_W1) ||
      !aligned(G_W2) || !aligned(workspace) || loss == nullptr)
    return BSM_EINVAL;
  if (workspace_bytes < ptc_workspace_bytes(*lat, channels, nbatch, true)) return BSM_EWORKSPACE;
  return finish(ptc_loss_grad(*lat, U_rep32, W1, W2, channels, r, e, nbatch, G_W1, G_W2, loss, workspace,
                              (cudaStream_t)stream));
}

int bsm_ptc_adam_step(void* W, const void* G, void* m, void* v, int64_t n, double lr, int32_t step, void* stream) {
  if (!aligned(W) || !aligned(G) || !aligned(m) || !aligned(v) || n < 1 || step < 1 || !(lr > 0.0))
    return BSM_EINVAL;
  return finish(ptc_adam(W, G, m, v, n, lr, step, (cudaStream_t)stream));
}

size_t bsm_fgcr_workspace_bytes(const bsm_lattice* lat, const bsm_fgcr_opts* opts) {
  if (opts == nullptr || check_lattice(lat) != BSM_OK || opts->restart < 1 || opts->restart > 64) return 0;
  if (opts->precond == BSM_FGCR_PTC && check_ptc(lat, opts->channels, 1) != BSM_OK) return 0;
  return fgcr_total_workspace_bytes(*lat, *opts);
}

int bsm_fgcr_solve(const bsm_lattice* lat, const void* U_rep64, const void* U_rep32, const void* W1, const void* W2,
                   const void* b, void* x, const bsm_fgcr_opts* opts, bsm_fgcr_stats* stats, void* workspace,
                   size_t workspace_bytes, void* stream) {
  int rc = check_lattice(lat);
  if (rc != BSM_OK) return rc;
  if (opts == nullptr || !(opts->tol > 0.0) || opts->max_iter < 1 || opts->restart < 1 || opts->restart > 64)
    return BSM_EINVAL;
  if (opts->precond != BSM_FGCR_NONE && opts->precond != BSM_FGCR_PTC) return BSM_EINVAL;
  if (opts->prec_inner != BSM_F64 && opts->prec_inner != BSM_F32) return BSM_EUNSUPPORTED;
  if (opts->prec_outer != BSM_F64 && opts->prec_outer != BSM_DF64) return BSM_EUNSUPPORTED;
  if (opts->prec_outer == BSM_DF64 && opts->prec_inner != BSM_F32) return BSM_EUNSUPPORTED;  // no FP64 links then
  if (!(opts->inner_tol >= 0.0) || opts->inner_tol >= 1.0 || opts->check_every < 0) return BSM_EINVAL;
  if (opts->prec_inner == BSM_F32 && !aligned(U_rep32)) return BSM_EINVAL;
  if (opts->precond == BSM_FGCR_PTC) {
    if ((rc = check_ptc(lat, opts->channels, 1)) != BSM_OK) return rc;
    if (opts->ptc_prec != BSM_F32 && opts->ptc_prec != BSM_BF16) return BSM_EUNSUPPORTED;
    if (!aligned(U_rep32) || !aligned(W1) || !aligned(W2)) return BSM_EINVAL;
  }
  if (!aligned(U_rep64) || !aligned(b) || !aligned(x) || !aligned(workspace)) return BSM_EINVAL;
  if (opts->fallback != 0 && opts->fallback_max_iter < 0) return BSM_EINVAL;
  if (workspace_bytes < fgcr_total_workspace_bytes(*lat, *opts)) return BSM_EWORKSPACE;
  const size_t full = bsm_field_bytes(lat, BSM_FIELD_SPINOR, BSM_F64);
  if (overlap(b, full, x, full)) return BSM_EINVAL;
  const cudaError_t pre = cudaGetLastError();
  if (pre != cudaSuccess) {
    set_cuda_error(pre);
    return BSM_ECUDA;
  }
  const auto t0 = std::chrono::steady_clock::now();
  bsm_fgcr_stats st{};
  rc = fgcr_solve(*lat, U_rep64, U_rep32, W1, W2, b, x, *opts, &st, workspace, (cudaStream_t)stream);
  st.fgcr_status = rc;
  st.fallback_iters = 0;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  if (opts->fallback != 0 && (rc == BSM_ENOCONV || rc == BSM_ENAN || rc == BSM_ETIMEOUT)) {
    // the plain solver of the paper's method on the same system: mixed
    // precision CG on the normal equations (reliable updates at prec_outer)
    bsm_cg_opts co{};
    co.tol = opts->tol;
    co.max_iter = opts->fallback_max_iter > 0 ? opts->fallback_max_iter : 20000;
    const bool mixed = U_rep32 != nullptr;
    co.prec_inner = mixed ? BSM_F32 : opts->prec_outer;
    co.prec_outer = opts->prec_outer;
    co.delta = 0.1;
    co.use_x0 = rc == BSM_ENOCONV;  // a NaN iterate is no starting point
    co.eo = opts->eo;
    co.check_every = 16;
    co.use_graph = 0;
    bsm_cg_stats cs{};
    rc = cg_solve(*lat, U_rep64, mixed ? U_rep32 : nullptr, b, x, co, &cs, workspace, (cudaStream_t)stream);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      set_cuda_error(e);
      return BSM_ECUDA;
    }
    st.fallback_iters = cs.iters;
    st.true_res = cs.true_res_full;
  }
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return rc;
}

const char* bsm_strerror(int status) {
  switch (status) {
    case BSM_OK: return "ok";
    case BSM_EINVAL: return "invalid argument";
    case BSM_EUNSUPPORTED: return "unsupported configuration";
    case BSM_ECUDA: return "CUDA error";
    case BSM_EWORKSPACE: return "workspace too small";
    case BSM_ENOCONV: return "solver did not converge within max_iter";
    case BSM_EBREAKDOWN: return "CG breakdown (<p, M p> <= 0)";
    case BSM_ENAN: return "NaN or Inf in a solver reduction";
    case BSM_ETIMEOUT: return "bounded device wait timed out";
    default: return "unknown status";
  }
}

const char* bsm_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"
