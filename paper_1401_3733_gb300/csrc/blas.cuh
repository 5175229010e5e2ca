// blas.cuh -- vector kernels and deterministic reductions for CG (Sec. II-B
// inversion by CG; Sec. III "elementary vector operations").
#pragma once

#include "bsm_internal.cuh"

namespace bsm {

// CG scalars kept on the device; kernels read alpha/beta from here so that
// an iteration needs no host round trip.
struct CgState {
  double rr;        // |r|^2 of the current residual
  double rr_prev;   // |r|^2 before the last beta step
  double pAp;       // <p, M p> = |Dhat p|^2
  double alpha, beta;
  float alpha_f;    // alpha rounded to FP32 (the fused FP32 CG step reads it)
  double stop2;     // tol^2 |rhs|^2
  double rr_max;    // max |r|^2 since the last reliable update
  double delta2;    // reliable-update trigger, squared
  double aux[4];    // scratch scalars (reductions outside the iteration)
  int iter, max_iter;
  int done;         // 0 running, 1 iterated residual converged, 2 breakdown, 3 NaN/Inf, 4 max_iter
  int want_update;  // mixed precision: |r|^2 < delta2 * rr_max
};

enum { kDoneRunning = 0, kDoneConverged = 1, kDoneBreakdown = 2, kDoneNaN = 3, kDoneMaxIter = 4 };

constexpr int kBlasThreads = 256;
constexpr int kBlasMaxBlocks = 152 * 8;  // grid-stride loops over a whole-GPU grid
inline int blas_blocks(size_t n16) {
  size_t b = (n16 + kBlasThreads - 1) / kBlasThreads;
  return (int)(b < (size_t)kBlasMaxBlocks ? (b == 0 ? 1 : b) : kBlasMaxBlocks);
}

// --- host launchers (blas.cu); n16 counts 16-byte vector elements ----------
// sum partials[0..n) in a fixed order into *out
void reduce_launch(const double* partials, int n, double* out, cudaStream_t s);
// CG iteration pieces (prec = precision of x, r, p, Ap)
void cg_alpha_launch(CgState* st, const double* partials, int n, cudaStream_t s);
void cg_beta_launch(CgState* st, const double* partials, int n, cudaStream_t s);
int cg_xr_update_launch(int prec, void* x, void* r, const void* p, const void* Ap, size_t n16, CgState* st,
                        double* partials, cudaStream_t s);
void cg_p_update_launch(int prec, void* p, const void* r, size_t n16, const CgState* st, cudaStream_t s);
// generic: partials of Re<a, b> (a == b gives |a|^2); returns block count
int dot_launch(int prec, const void* a, const void* b, size_t n16, double* partials, cudaStream_t s);
// y = a*x + b*y elementwise on FP64 or DF64 vectors; returns blocks;
// optional |y|^2 partials
int axpby_launch(int prec, double a, const void* x, double b, void* y, size_t n16, double* partials, cudaStream_t s);
// y_outer += x32 (widened), then x32 = 0, over `halves` half spinors of
// n32_half float4 elements each (the outer/FP32 component pairing is handled
// here); prec_outer is BSM_F64 or BSM_DF64
void accumulate32_launch(int prec_outer, void* y, void* x32, size_t n32_half, int halves, cudaStream_t s);
// y32 = nearest FP32 of x_outer, same shape convention
void convert_to32_launch(int prec_outer, void* y32, const void* x, size_t n32_half, int halves, cudaStream_t s);
// FP64 <-> DF64 vectors (n16 complex elements)
void f64_df64_launch(void* dst, const void* src, size_t n16, bool to_df64, cudaStream_t s);
// y -= (*num / *den) * x   (FP32 vectors, device scalars)
void axpy_ratio32_launch(void* y, const void* x, size_t n16, const double* num, const double* den, cudaStream_t s);

}  // namespace bsm
