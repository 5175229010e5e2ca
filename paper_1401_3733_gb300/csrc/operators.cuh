// operators.cuh -- the Wilson operators of Sec. II-B assembled from hop
// launches: the parity block H_{p,1-p}, the full D = A - H/2 and the even-odd
// Schur operator Dhat = A - 1/(4A) H_eo H_oe (adjoints through the dagger
// flag, H^+ = g5 H g5).
#pragma once

#include "bsm_internal.cuh"

namespace bsm {

struct OpCtx {
  Geom g;
  int d;
  bool real;
  int prec;
  double A;              // 4 + m0
  const char* links;     // device-layout links; block p at links + p * link_block
  size_t link_block;
  size_t half_bytes;     // one parity of a spinor at `prec`
  cudaStream_t s;
  float ph3[4][2];       // (cos, sin) of 3 phi_mu (two-row links)
};

// fills ctx from a validated lattice; links may be null for size queries
OpCtx make_ctx(const bsm_lattice& L, const void* links, int prec, cudaStream_t s);

// out_p = a*x + b*H_{p,1-p} in  (x may be null: out_p = b*H in); returns the
// number of partials written (0 when partials is null), or <0 on error
int op_hop(const OpCtx& c, int p, const void* in, void* out, int dagger, const void* x, double a, double b,
           double* partials, const int* done);

// the second factor of Dhat^+ Dhat fused with a CG step (FP32 vectors):
// tmp_o = H^+_oe u, then Ap = A u - 1/(4A) H^+_eo tmp_o is not stored but
// applied, r -= alpha Ap and x += alpha p (alpha = *alpha, device); writes
// the partials of |r|^2 and returns their count, or < 0 on error
int op_dhat_dag_cg(const OpCtx& c, const void* u, void* tmp_o, void* r, void* x, const void* p, const float* alpha,
                   double* partials, const int* done);

// out_e = Dhat in_e (or Dhat^+); tmp_o: one half spinor; partials of |out|^2
int op_dhat(const OpCtx& c, const void* in_e, void* out_e, void* tmp_o, int dagger, double* partials,
            const int* done);

// out = D in (or D^+) on full spinors; partials (2 blocks' worth) of |out|^2
int op_dirac(const OpCtx& c, const void* in, void* out, int dagger, double* partials, const int* done);

}  // namespace bsm
