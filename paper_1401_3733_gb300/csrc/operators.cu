// operators.cu -- Wilson operators from hop launches (Sec. II-B).
#include "operators.cuh"

namespace bsm {

int launch_hop_f64(int d, bool real, const HopArgs& A, cudaStream_t s);
int launch_hop_f32(int d, bool real, const HopArgs& A, cudaStream_t s);
int launch_hop_df64(int d, bool real, const HopArgs& A, cudaStream_t s);
int launch_hop_bf16(int d, bool real, const HopArgs& A, cudaStream_t s);
int launch_hop_f32r12(int d, bool real, const HopArgs& A, cudaStream_t s);

int launch_hop(int prec, int d, bool real, const HopArgs& A, cudaStream_t s) {
  switch (prec) {
    case BSM_F64: return launch_hop_f64(d, real, A, s);
    case BSM_F32: return launch_hop_f32(d, real, A, s);
    case BSM_DF64: return launch_hop_df64(d, real, A, s);
    case BSM_BF16: return launch_hop_bf16(d, real, A, s);
    case BSM_F32R12: return launch_hop_f32r12(d, real, A, s);
    default: return -1;
  }
}

OpCtx make_ctx(const bsm_lattice& L, const void* links, int prec, cudaStream_t s) {
  OpCtx c;
  c.g = make_geom(L);
  const RepInfo ri = rep_info(L.N, L.rep);
  c.d = ri.d;
  c.real = ri.real;
  c.prec = prec;
  c.A = 4.0 + L.m0;
  c.links = reinterpret_cast<const char*>(links);
  c.link_block = link_block_bytes(c.g.Vh, c.d, c.real, prec);
  c.half_bytes = half_spinor_bytes(c.g.Vh, c.d, prec);
  c.s = s;
  for (int mu = 0; mu < 4; ++mu) {
    c.ph3[mu][0] = (float)cos(3.0 * L.bc_phase[mu]);
    c.ph3[mu][1] = (float)sin(3.0 * L.bc_phase[mu]);
  }
  return c;
}

namespace {
HopArgs hop_args(const OpCtx& c, int p, const void* in, void* out, int dagger, const void* x, double a, double b,
                 double* partials, const int* done) {
  HopArgs h{};
  h.links = c.links + (size_t)p * c.link_block;
  h.in = in;
  h.out = out;
  h.x = x;
  h.a = a;
  h.b = b;
  h.partials = partials;
  h.done = done;
  h.g = c.g;
  h.p = p;
  h.dagger = dagger;
  for (int mu = 0; mu < 4; ++mu) {
    h.ph3[mu][0] = c.ph3[mu][0];
    h.ph3[mu][1] = c.ph3[mu][1];
  }
  return h;
}
}  // namespace

int op_hop(const OpCtx& c, int p, const void* in, void* out, int dagger, const void* x, double a, double b,
           double* partials, const int* done) {
  const int blocks = launch_hop(c.prec, c.d, c.real, hop_args(c, p, in, out, dagger, x, a, b, partials, done), c.s);
  if (blocks < 0) return BSM_EUNSUPPORTED;
  return partials != nullptr ? blocks : 0;
}

int op_dhat_dag_cg(const OpCtx& c, const void* u, void* tmp_o, void* r, void* x, const void* p, const float* alpha,
                   double* partials, const int* done) {
  int n = op_hop(c, 1, u, tmp_o, 1, nullptr, 0.0, 1.0, nullptr, done);
  if (n < 0) return n;
  HopArgs h = hop_args(c, 0, tmp_o, nullptr, 1, u, c.A, -1.0 / (4.0 * c.A), partials, done);
  h.cg_r = r;
  h.cg_x = x;
  h.cg_p = p;
  h.cg_alpha = alpha;
  const int blocks = launch_hop(c.prec, c.d, c.real, h, c.s);
  if (blocks < 0) return BSM_EUNSUPPORTED;
  return blocks;
}

int op_dhat(const OpCtx& c, const void* in_e, void* out_e, void* tmp_o, int dagger, double* partials,
            const int* done) {
  // tmp_o = H_oe in_e ; out_e = A in_e - 1/(4A) H_eo tmp_o
  int r = op_hop(c, 1, in_e, tmp_o, dagger, nullptr, 0.0, 1.0, nullptr, done);
  if (r < 0) return r;
  return op_hop(c, 0, tmp_o, out_e, dagger, in_e, c.A, -1.0 / (4.0 * c.A), partials, done);
}

int op_dirac(const OpCtx& c, const void* in, void* out, int dagger, double* partials, const int* done) {
  const char* ie = reinterpret_cast<const char*>(in);
  const char* io = ie + c.half_bytes;
  char* oe = reinterpret_cast<char*>(out);
  char* oo = oe + c.half_bytes;
  // out_e = A in_e - 1/2 H_eo in_o ; out_o = A in_o - 1/2 H_oe in_e
  const int n0 = op_hop(c, 0, io, oe, dagger, ie, c.A, -0.5, partials, done);
  if (n0 < 0) return n0;
  const int n1 = op_hop(c, 1, ie, oo, dagger, io, c.A, -0.5, partials ? partials + n0 : nullptr, done);
  if (n1 < 0) return n1;
  return n0 + n1;
}

}  // namespace bsm
