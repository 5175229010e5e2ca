// blas.cu -- vector kernels and deterministic reductions for CG.
//
// Reductions: each thread accumulates its grid-stride share in FP64 (for
// FP32 vectors the four products of one 16-byte element are summed in FP32
// first, for DF64 vectors the two products of one complex element in
// double-float, then added in FP64), a fixed shuffle tree gives one partial
// per block, and a single-block finalize kernel sums the partials in a fixed
// order.  The result is therefore bit-reproducible for a given problem size.
// DF64 vector updates run in double-float arithmetic on the FP32 units.
#include "blas.cuh"

namespace bsm {

namespace {

__device__ __forceinline__ double edot(const double2& a, const double2& b) { return fma(a.x, b.x, a.y * b.y); }
__device__ __forceinline__ double edot(const float4& a, const float4& b) {
  return (double)fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}
__device__ __forceinline__ double2 eaxpy(double a, const double2& x, const double2& y) {
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ float4 eaxpy(double a, const float4& x, const float4& y) {
  const float f = (float)a;
  return make_float4(fmaf(f, x.x, y.x), fmaf(f, x.y, y.y), fmaf(f, x.z, y.z), fmaf(f, x.w, y.w));
}
// x + b y
__device__ __forceinline__ double2 expay(const double2& x, double b, const double2& y) {
  return make_double2(fma(b, y.x, x.x), fma(b, y.y, x.y));
}
__device__ __forceinline__ float4 expay(const float4& x, double b, const float4& y) {
  const float f = (float)b;
  return make_float4(fmaf(f, y.x, x.x), fmaf(f, y.y, x.y), fmaf(f, y.z, x.z), fmaf(f, y.w, x.w));
}

// DF64 element: one complex number as (re.hi, re.lo, im.hi, im.lo)
struct dfc {
  float4 v;
};
__device__ __forceinline__ df dre(const dfc& a) { return df(a.v.x, a.v.y); }
__device__ __forceinline__ df dim(const dfc& a) { return df(a.v.z, a.v.w); }
__device__ __forceinline__ dfc dmake(df re, df im) {
  re = df_norm(re);
  im = df_norm(im);
  dfc c;
  c.v = make_float4(re.hi, re.lo, im.hi, im.lo);
  return c;
}
__device__ __forceinline__ double edot(const dfc& a, const dfc& b) {
  return (double)fma(dim(a), dim(b), dre(a) * dre(b));
}
__device__ __forceinline__ dfc eaxpy(double a, const dfc& x, const dfc& y) {
  const df al(a);
  return dmake(fma(al, dre(x), dre(y)), fma(al, dim(x), dim(y)));
}
__device__ __forceinline__ dfc expay(const dfc& x, double b, const dfc& y) {
  const df be(b);
  return dmake(fma(be, dre(y), dre(x)), fma(be, dim(y), dim(x)));
}
// a x + b y
__device__ __forceinline__ double2 eaxpby(double a, const double2& x, double b, const double2& y) {
  return make_double2(fma(a, x.x, b * y.x), fma(a, x.y, b * y.y));
}
__device__ __forceinline__ dfc eaxpby(double a, const dfc& x, double b, const dfc& y) {
  const df al(a), be(b);
  return dmake(fma(al, dre(x), be * dre(y)), fma(al, dim(x), be * dim(y)));
}

template <typename E>
struct ElemOf;
template <>
struct ElemOf<F64> {
  using T = double2;
};
template <>
struct ElemOf<F32> {
  using T = float4;
};
template <>
struct ElemOf<DF64> {
  using T = dfc;
};

// Second stage of the deterministic reductions: the sum of n FP64 block
// partials by one block of kTotalThreads, in a fixed order.  Thread t adds
// partials t, t + 1024, ... with eight loads in flight per step (pairwise),
// then each warp folds its 32 sums with shuffles and warp 0 folds the 32
// warp sums.  The value is valid in thread 0.
constexpr int kTotalThreads = 1024;

__device__ double block_total(const double* __restrict__ partials, int n) {
  double s = 0.0;
  int k = threadIdx.x;
  for (; k + 7 * kTotalThreads < n; k += 8 * kTotalThreads) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = partials[k + j * kTotalThreads];
    s += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
  }
  for (; k < n; k += kTotalThreads) s += partials[k];
  __shared__ double warp_sums[kTotalThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) warp_sums[warp] = s;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = warp_sums[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

__global__ void __launch_bounds__(kTotalThreads) reduce_kernel(const double* __restrict__ partials, int n,
                                                               double* out) {
  const double s = block_total(partials, n);
  if (threadIdx.x == 0) *out = s;
}

// alpha = rr / <p, M p>
__global__ void __launch_bounds__(kTotalThreads) cg_alpha_kernel(CgState* st, const double* __restrict__ partials,
                                                                 int n) {
  if (st->done) return;
  const double pAp = block_total(partials, n);
  if (threadIdx.x != 0) return;
  st->pAp = pAp;
  if (!isfinite(pAp)) {
    st->done = kDoneNaN;
    st->alpha = 0.0;
  } else if (!(pAp > 0.0)) {
    st->done = kDoneBreakdown;
    st->alpha = 0.0;
  } else {
    st->alpha = st->rr / pAp;
  }
  st->alpha_f = (float)st->alpha;
}

// beta = |r_new|^2 / |r|^2, convergence and reliable-update flags
__global__ void __launch_bounds__(kTotalThreads) cg_beta_kernel(CgState* st, const double* __restrict__ partials,
                                                                int n) {
  if (st->done) return;
  const double rr_new = block_total(partials, n);
  if (threadIdx.x != 0) return;
  st->iter += 1;
  st->rr_prev = st->rr;
  st->beta = rr_new / st->rr;
  st->rr = rr_new;
  if (!isfinite(rr_new)) {
    st->done = kDoneNaN;
    return;
  }
  if (rr_new > st->rr_max) st->rr_max = rr_new;
  if (rr_new < st->delta2 * st->rr_max) st->want_update = 1;
  if (rr_new <= st->stop2) st->done = kDoneConverged;
  else if (st->iter >= st->max_iter) st->done = kDoneMaxIter;
}

// x += alpha p ; r -= alpha Ap ; partials of |r|^2
template <typename P>
__global__ void __launch_bounds__(kBlasThreads) cg_xr_kernel(typename ElemOf<P>::T* __restrict__ x,
                                                             typename ElemOf<P>::T* __restrict__ r,
                                                             const typename ElemOf<P>::T* __restrict__ p,
                                                             const typename ElemOf<P>::T* __restrict__ Ap,
                                                             size_t n, const CgState* st, double* partials) {
  if (st->done) return;
  const double alpha = st->alpha;
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    x[k] = eaxpy(alpha, p[k], x[k]);
    const auto rk = eaxpy(-alpha, Ap[k], r[k]);
    r[k] = rk;
    acc += edot(rk, rk);
  }
  block_sum_store_wide<kBlasThreads>(acc, partials);
}

// p = r + beta p
template <typename P>
__global__ void __launch_bounds__(kBlasThreads) cg_p_kernel(typename ElemOf<P>::T* __restrict__ p,
                                                            const typename ElemOf<P>::T* __restrict__ r, size_t n,
                                                            const CgState* st) {
  if (st->done) return;
  const double beta = st->beta;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads)
    p[k] = expay(r[k], beta, p[k]);
}

template <typename P>
__global__ void __launch_bounds__(kBlasThreads) dot_kernel(const typename ElemOf<P>::T* __restrict__ a,
                                                           const typename ElemOf<P>::T* __restrict__ b, size_t n,
                                                           double* partials) {
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads)
    acc += edot(a[k], b[k]);
  block_sum_store_wide<kBlasThreads>(acc, partials);
}

template <typename P>
__global__ void __launch_bounds__(kBlasThreads) axpby_kernel(double a, const typename ElemOf<P>::T* __restrict__ x,
                                                             double b, typename ElemOf<P>::T* __restrict__ y,
                                                             size_t n, double* partials) {
  double acc = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const auto v = eaxpby(a, x[k], b, y[k]);
    y[k] = v;
    acc += edot(v, v);
  }
  if (partials != nullptr) block_sum_store_wide<kBlasThreads>(acc, partials);
}

// FP64/DF64 and FP32 half spinors pair their components differently: FP32
// element k of a half (float4) holds the spin-0/1 complex component at outer
// element k and the spin-2/3 component at outer element k + n32, n32 = float4
// elements per half.
__device__ __forceinline__ void add_float2(double2& y, float re, float im) {
  y.x += re;
  y.y += im;
}
__device__ __forceinline__ void add_float2(dfc& y, float re, float im) {
  y = dmake(dre(y) + df(re, 0.f), dim(y) + df(im, 0.f));
}
__device__ __forceinline__ float2 round_float2(const double2& x) {
  return make_float2(__double2float_rn(x.x), __double2float_rn(x.y));
}
__device__ __forceinline__ float2 round_float2(const dfc& x) {
  return make_float2(__fadd_rn(x.v.x, x.v.y), __fadd_rn(x.v.z, x.v.w));  // nearest float to hi + lo
}

// y_outer += widen(x32); x32 = 0
template <typename P>
__global__ void __launch_bounds__(kBlasThreads) acc32_kernel(typename ElemOf<P>::T* __restrict__ y,
                                                             float4* __restrict__ x, size_t n32, size_t n) {
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const size_t h = k / n32, kk = k - h * n32;
    auto* yh = y + h * 2 * n32;
    const float4 v = x[k];
    auto a = yh[kk], b = yh[kk + n32];
    add_float2(a, v.x, v.y);
    add_float2(b, v.z, v.w);
    yh[kk] = a;
    yh[kk + n32] = b;
    x[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// y32 = nearest FP32 of x_outer
template <typename P>
__global__ void __launch_bounds__(kBlasThreads) conv32_kernel(float4* __restrict__ y,
                                                              const typename ElemOf<P>::T* __restrict__ x,
                                                              size_t n32, size_t n) {
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const size_t h = k / n32, kk = k - h * n32;
    const auto* xh = x + h * 2 * n32;
    const float2 a = round_float2(xh[kk]), b = round_float2(xh[kk + n32]);
    y[k] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// FP64 <-> DF64, elementwise (same component order)
__global__ void __launch_bounds__(kBlasThreads) f64_to_df64_kernel(dfc* __restrict__ y, const double2* __restrict__ x,
                                                                   size_t n) {
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const df re(x[k].x), im(x[k].y);
    dfc c;
    c.v = make_float4(re.hi, re.lo, im.hi, im.lo);
    y[k] = c;
  }
}
__global__ void __launch_bounds__(kBlasThreads) df64_to_f64_kernel(double2* __restrict__ y, const dfc* __restrict__ x,
                                                                   size_t n) {
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads)
    y[k] = make_double2((double)dre(x[k]), (double)dim(x[k]));
}

__global__ void __launch_bounds__(kBlasThreads) axpy_ratio32_kernel(float4* __restrict__ y,
                                                                    const float4* __restrict__ x, size_t n,
                                                                    const double* num, const double* den) {
  const double c = -(*num) / (*den);
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads)
    y[k] = eaxpy(c, x[k], y[k]);
}

}  // namespace

void reduce_launch(const double* partials, int n, double* out, cudaStream_t s) {
  reduce_kernel<<<1, kTotalThreads, 0, s>>>(partials, n, out);
}
void cg_alpha_launch(CgState* st, const double* partials, int n, cudaStream_t s) {
  cg_alpha_kernel<<<1, kTotalThreads, 0, s>>>(st, partials, n);
}
void cg_beta_launch(CgState* st, const double* partials, int n, cudaStream_t s) {
  cg_beta_kernel<<<1, kTotalThreads, 0, s>>>(st, partials, n);
}

template <typename P>
using E = typename ElemOf<P>::T;

int cg_xr_update_launch(int prec, void* x, void* r, const void* p, const void* Ap, size_t n16, CgState* st,
                        double* partials, cudaStream_t s) {
  const int b = blas_blocks(n16);
  switch (prec) {
    case BSM_F64:
      cg_xr_kernel<F64><<<b, kBlasThreads, 0, s>>>((E<F64>*)x, (E<F64>*)r, (const E<F64>*)p, (const E<F64>*)Ap, n16,
                                                    st, partials);
      break;
    case BSM_F32:
      cg_xr_kernel<F32><<<b, kBlasThreads, 0, s>>>((E<F32>*)x, (E<F32>*)r, (const E<F32>*)p, (const E<F32>*)Ap, n16,
                                                    st, partials);
      break;
    default:
      cg_xr_kernel<DF64><<<b, kBlasThreads, 0, s>>>((E<DF64>*)x, (E<DF64>*)r, (const E<DF64>*)p,
                                                     (const E<DF64>*)Ap, n16, st, partials);
      break;
  }
  return b;
}

void cg_p_update_launch(int prec, void* p, const void* r, size_t n16, const CgState* st, cudaStream_t s) {
  const int b = blas_blocks(n16);
  switch (prec) {
    case BSM_F64: cg_p_kernel<F64><<<b, kBlasThreads, 0, s>>>((E<F64>*)p, (const E<F64>*)r, n16, st); break;
    case BSM_F32: cg_p_kernel<F32><<<b, kBlasThreads, 0, s>>>((E<F32>*)p, (const E<F32>*)r, n16, st); break;
    default: cg_p_kernel<DF64><<<b, kBlasThreads, 0, s>>>((E<DF64>*)p, (const E<DF64>*)r, n16, st); break;
  }
}

int dot_launch(int prec, const void* a, const void* b, size_t n16, double* partials, cudaStream_t s) {
  const int nb = blas_blocks(n16);
  switch (prec) {
    case BSM_F64:
      dot_kernel<F64><<<nb, kBlasThreads, 0, s>>>((const E<F64>*)a, (const E<F64>*)b, n16, partials);
      break;
    case BSM_F32:
      dot_kernel<F32><<<nb, kBlasThreads, 0, s>>>((const E<F32>*)a, (const E<F32>*)b, n16, partials);
      break;
    default:
      dot_kernel<DF64><<<nb, kBlasThreads, 0, s>>>((const E<DF64>*)a, (const E<DF64>*)b, n16, partials);
      break;
  }
  return nb;
}

int axpby_launch(int prec, double a, const void* x, double b, void* y, size_t n16, double* partials, cudaStream_t s) {
  const int nb = blas_blocks(n16);
  switch (prec) {
    case BSM_F64:
      axpby_kernel<F64><<<nb, kBlasThreads, 0, s>>>(a, (const E<F64>*)x, b, (E<F64>*)y, n16, partials);
      break;
    default:
      axpby_kernel<DF64><<<nb, kBlasThreads, 0, s>>>(a, (const E<DF64>*)x, b, (E<DF64>*)y, n16, partials);
      break;
  }
  return nb;
}

void accumulate32_launch(int prec_outer, void* y, void* x32, size_t n32_half, int halves, cudaStream_t s) {
  const size_t n = n32_half * halves;
  if (prec_outer == BSM_F64)
    acc32_kernel<F64><<<blas_blocks(n), kBlasThreads, 0, s>>>((E<F64>*)y, (float4*)x32, n32_half, n);
  else
    acc32_kernel<DF64><<<blas_blocks(n), kBlasThreads, 0, s>>>((E<DF64>*)y, (float4*)x32, n32_half, n);
}

void convert_to32_launch(int prec_outer, void* y32, const void* x, size_t n32_half, int halves, cudaStream_t s) {
  const size_t n = n32_half * halves;
  if (prec_outer == BSM_F64)
    conv32_kernel<F64><<<blas_blocks(n), kBlasThreads, 0, s>>>((float4*)y32, (const E<F64>*)x, n32_half, n);
  else
    conv32_kernel<DF64><<<blas_blocks(n), kBlasThreads, 0, s>>>((float4*)y32, (const E<DF64>*)x, n32_half, n);
}

void f64_df64_launch(void* dst, const void* src, size_t n16, bool to_df64, cudaStream_t s) {
  if (to_df64)
    f64_to_df64_kernel<<<blas_blocks(n16), kBlasThreads, 0, s>>>((dfc*)dst, (const double2*)src, n16);
  else
    df64_to_f64_kernel<<<blas_blocks(n16), kBlasThreads, 0, s>>>((double2*)dst, (const dfc*)src, n16);
}

void axpy_ratio32_launch(void* y, const void* x, size_t n16, const double* num, const double* den, cudaStream_t s) {
  axpy_ratio32_kernel<<<blas_blocks(n16), kBlasThreads, 0, s>>>((float4*)y, (const float4*)x, n16, num, den);
}

}  // namespace bsm
