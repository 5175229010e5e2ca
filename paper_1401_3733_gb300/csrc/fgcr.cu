// fgcr.cu -- flexible GCR on the full Wilson operator D x = b (FP64), with
// either no preconditioner or the learned parallel-transport preconditioner,
// in FP64 throughout or in FP32 restart cycles with the residual recomputed
// in FP64 after each cycle (defect correction: x += e, r = b - D x).
//
// Flexible GCR (Notay 2000): z = M(r), w = A z; w and z are orthogonalised
// against the stored w_j (beta_j = <w_j, w>/|w_j|^2, w -= beta_j w_j,
// z -= beta_j z_j), then alpha = <w, r>/|w|^2, x += alpha z, r -= alpha w;
// after `restart` directions the basis is dropped.  A is the full operator D,
// or the even-site Schur operator Dhat (even-odd option).
// Because the preconditioner may change from step to step (a network in
// reduced precision is not exactly linear in the rounding), GCR's flexible
// form is needed rather than CG on the normal equations.
//
// The complex scalars stay on the device; the host reads |r|^2 once per
// iteration to decide convergence.  Reductions are deterministic (fixed
// block partials summed in a fixed order).
#include <chrono>

#include "blas.cuh"
#include "operators.cuh"

namespace bsm {

size_t ptc_workspace_bytes(const bsm_lattice& L, int C, int nb, bool train);
int ptc_pack(const bsm_lattice& L, const double* psi, void* F, bool unpack, bool even_only, cudaStream_t s);
int ptc_pack32(const bsm_lattice& L, const float* psi, void* F, bool unpack, int even_only, cudaStream_t s);
bool ptc_fused_supported(int C);
int ptc_apply(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* in,
              void* out, int nb, int prec, void* ws, cudaStream_t s, bool even_only = false, bool reset_err = true);

namespace {

// Element arithmetic at the vector's own precision (FP32 for the FP32
// cycles: GB300's FP64 units are far slower than its FP32 units); each
// thread's partial sums are handed to the block reductions in FP64.
template <typename T> struct Arith;
template <> struct Arith<double2> { using R = double; };
template <> struct Arith<float2> { using R = float; };

// a coefficient (FP64) in the vectors' precision: converted once, outside
// the element loops (a conversion from FP64 issues at GB300's FP64 rate)
template <typename T>
__device__ __forceinline__ T coef_as(double2 c) {
  using R = typename Arith<T>::R;
  T t;
  t.x = (R)c.x;
  t.y = (R)c.y;
  return t;
}

template <typename T>
__device__ __forceinline__ T csub_mul(T x, T c, T a) {  // x - c a
  x.x -= c.x * a.x - c.y * a.y;
  x.y -= c.x * a.y + c.y * a.x;
  return x;
}

template <typename T>
__device__ __forceinline__ T cadd_mul(T x, T c, T a) {  // x + c a
  x.x += c.x * a.x - c.y * a.y;
  x.y += c.x * a.y + c.y * a.x;
  return x;
}

// per-thread sums -> block partials at out[j * stride + blockIdx.x]
template <int NV>
__device__ __forceinline__ void store_sums(float (&v)[NV], double* out, size_t stride) {
  block_sums_store_f32<kBlasThreads, NV>(v, out, stride);
}
template <int NV>
__device__ __forceinline__ void store_sums(double (&v)[NV], double* out, size_t stride) {
#pragma unroll
  for (int j = 0; j < NV; ++j) block_sum_store_wide<kBlasThreads>(v[j], out + j * stride);
}

constexpr int kDotChunk = 8;  // directions per dot launch (accumulators in registers)

// partials of <w_j, v> = sum conj(w_j) v for j = j0 .. j0 + CNT - 1, w_j at
// basis + j * stride: re of j at [(2 (j - j0)) G + blk], im at [(2 (j - j0) + 1) G + blk].
// CNT is a template constant so that all CNT + 1 loads of an element issue together.
template <typename T, int CNT>
__global__ void __launch_bounds__(kBlasThreads) multi_dot_kernel(const T* __restrict__ basis, size_t stride, int j0,
                                                                 const T* __restrict__ v, size_t n,
                                                                 double* partials) {
  using R = typename Arith<T>::R;
  R re[CNT], im[CNT];
#pragma unroll
  for (int j = 0; j < CNT; ++j) re[j] = im[j] = 0;
  const T* b0 = basis + (size_t)j0 * stride;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const T y = v[k];
    T x[CNT];
#pragma unroll
    for (int j = 0; j < CNT; ++j) x[j] = b0[(size_t)j * stride + k];
#pragma unroll
    for (int j = 0; j < CNT; ++j) {
      re[j] += x[j].x * y.x + x[j].y * y.y;
      im[j] += x[j].x * y.y - x[j].y * y.x;
    }
  }
  R sums[2 * CNT];
#pragma unroll
  for (int j = 0; j < CNT; ++j) {
    sums[2 * j] = re[j];
    sums[2 * j + 1] = im[j];
  }
  store_sums<2 * CNT>(sums, partials, gridDim.x);
}

template <typename T>
void multi_dot_launch(int G, const T* basis, size_t stride, int j0, int cnt, const T* v, size_t n, double* part,
                      cudaStream_t s) {
  switch (cnt) {
#define BSM_MD(C) \
  case C: multi_dot_kernel<T, C><<<G, kBlasThreads, 0, s>>>(basis, stride, j0, v, n, part); break;
    BSM_MD(1) BSM_MD(2) BSM_MD(3) BSM_MD(4) BSM_MD(5) BSM_MD(6) BSM_MD(7) BSM_MD(8)
#undef BSM_MD
    default: break;
  }
}

__device__ double sum_partials(const double* __restrict__ p, int n) {
  __shared__ double buf[kBlasThreads];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += kBlasThreads) s += p[k];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int o = kBlasThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) buf[threadIdx.x] += buf[threadIdx.x + o];
    __syncthreads();
  }
  const double r = buf[0];
  __syncthreads();
  return r;
}

// coef_j = <w_j, w> / |w_j|^2 for j = j0 + blockIdx.x (one block per direction)
__global__ void gs_coef_kernel(const double* __restrict__ partials, int nblk, int j0,
                               const double* __restrict__ norm2, double2* coef) {
  const int j = blockIdx.x;
  const double re = sum_partials(partials + (size_t)(2 * j) * nblk, nblk);
  const double im = sum_partials(partials + (size_t)(2 * j + 1) * nblk, nblk);
  if (threadIdx.x == 0) {
    const double nn = norm2[j0 + j];
    coef[j0 + j] = nn > 0.0 ? make_double2(re / nn, im / nn) : make_double2(0.0, 0.0);
  }
}

// w -= sum_j coef_j w_j  (j < k <= 64; w_j at wb + j * stride)
template <typename T>
__global__ void __launch_bounds__(kBlasThreads) gs_update_kernel(T* __restrict__ w, const T* __restrict__ wb,
                                                                 size_t stride, int k, size_t n,
                                                                 const double2* __restrict__ coef) {
  __shared__ T c[64];
  for (int j = threadIdx.x; j < k; j += kBlasThreads) c[j] = coef_as<T>(coef[j]);
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kBlasThreads) {
    T x = w[e];
#pragma unroll 4
    for (int j = 0; j < k; ++j) x = csub_mul(x, c[j], wb[(size_t)j * stride + e]);
    w[e] = x;
  }
}

// x += sum_j gamma_j z_j  (j < K <= 64; z_j at zb + j * stride)
template <typename T>
__global__ void __launch_bounds__(kBlasThreads) x_update_kernel(T* __restrict__ x, const T* __restrict__ zb,
                                                                size_t stride, int K, size_t n,
                                                                const double2* __restrict__ gamma) {
  __shared__ T c[64];
  for (int j = threadIdx.x; j < K; j += kBlasThreads) c[j] = coef_as<T>(gamma[j]);
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kBlasThreads) {
    T v = x[e];
#pragma unroll 4
    for (int j = 0; j < K; ++j) v = cadd_mul(v, c[j], zb[(size_t)j * stride + e]);
    x[e] = v;
  }
}

// The cycle's solution update in the stored (not orthogonalised) directions:
// with zhat_k = z_k - sum_{j<k} beta_jk zhat_j (A zhat_k = the orthogonalised
// w_k), sum_k alpha_k zhat_k = sum_j gamma_j z_j, gamma by back substitution
// (k from K-1 down: gamma_k = a_k, then a_j -= gamma_k beta_jk for j < k;
// a = alpha at the start).  beta_jk at bmat[k * ld + j].  One block of 64.
__global__ void __launch_bounds__(64) backsolve_kernel(const double2* __restrict__ alpha,
                                                       const double2* __restrict__ bmat, int ld, int K,
                                                       double2* __restrict__ gamma) {
  __shared__ double2 a[64];
  const int j = threadIdx.x;
  if (j < K) a[j] = alpha[j];
  __syncthreads();
  for (int k = K - 1; k >= 1; --k) {
    const double2 g = a[k];
    if (j < k) {
      const double2 b = bmat[(size_t)k * ld + j];
      a[j] = make_double2(a[j].x - (g.x * b.x - g.y * b.y), a[j].y - (g.x * b.y + g.y * b.x));
    }
    __syncthreads();
  }
  if (j < K) gamma[j] = a[j];
}

// partials of |w|^2 [blk], Re<w, r> [G + blk], Im<w, r> [2G + blk]
template <typename T>
__global__ void __launch_bounds__(kBlasThreads) wr_kernel(const T* __restrict__ w, const T* __restrict__ r, size_t n,
                                                          double* partials) {
  using R = typename Arith<T>::R;
  R ww = 0, re = 0, im = 0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const T x = w[k], y = r[k];
    ww += x.x * x.x + x.y * x.y;
    re += x.x * y.x + x.y * y.y;
    im += x.x * y.y - x.y * y.x;
  }
  R sums[3] = {ww, re, im};
  store_sums<3>(sums, partials, gridDim.x);
}

// norm2_k = |w|^2, alpha = <w, r> / |w|^2 (one block)
__global__ void alpha_kernel(const double* __restrict__ partials, int nblk, double* norm2_k, double2* alpha) {
  const double ww = sum_partials(partials, nblk);
  const double re = sum_partials(partials + nblk, nblk);
  const double im = sum_partials(partials + 2 * nblk, nblk);
  if (threadIdx.x == 0) {
    *norm2_k = ww;
    *alpha = ww > 0.0 ? make_double2(re / ww, im / ww) : make_double2(0.0, 0.0);
  }
}

// r -= alpha w ; partials of |r|^2
template <typename T>
__global__ void __launch_bounds__(kBlasThreads) r_update_kernel(T* __restrict__ r, const T* __restrict__ w, size_t n,
                                                                const double2* __restrict__ alpha, double* partials) {
  using R = typename Arith<T>::R;
  const T a = coef_as<T>(*alpha);
  R rr = 0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const T q = csub_mul(r[k], a, w[k]);
    r[k] = q;
    rr += q.x * q.x + q.y * q.y;
  }
  R sums[1] = {rr};
  store_sums<1>(sums, partials, gridDim.x);
}

// partials of |a - b|^2 (b may be null: |a|^2); with out != null also out = a - b
__global__ void __launch_bounds__(kBlasThreads) diff2_kernel(const double2* __restrict__ a, const double2* b,
                                                             double2* out, size_t n, double* partials) {
  double s = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    double2 v = a[k];
    if (b != nullptr) {
      v.x -= b[k].x;
      v.y -= b[k].y;
    }
    if (out != nullptr) out[k] = v;
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  block_sum_store_wide<kBlasThreads>(s, partials);
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct FgcrLayout {
  size_t r, bhat, tmp, x32, r32, basis, scal, part, F_in, F_out, ptc, dfi, dfo, total;
};

// Vectors are full spinors, or even half spinors with opts.eo.  Mixed: the
// cycle vectors (x32, r32, basis) are FP32 next to the FP64 residual r.
FgcrLayout fgcr_layout(const bsm_lattice& L, const bsm_fgcr_opts& o) {
  const Geom g = make_geom(L);
  const int d = rep_info(L.N, L.rep).d;
  const bool mixed = o.prec_inner == BSM_F32;
  const int parts = o.eo ? 1 : 2;
  const size_t v64 = parts * half_spinor_bytes(g.Vh, d, BSM_F64);
  const size_t vc = parts * half_spinor_bytes(g.Vh, d, mixed ? BSM_F32 : BSM_F64);
  FgcrLayout y{};
  size_t p = 0;
  y.r = p; p = al(p + 2 * half_spinor_bytes(g.Vh, d, BSM_F64));  // full: also holds D x at the end
  if (o.eo) {
    y.bhat = p; p = al(p + v64);
    y.tmp = p; p = al(p + half_spinor_bytes(g.Vh, d, BSM_F64));   // odd temporary of Dhat
  }
  if (mixed) {
    y.x32 = p; p = al(p + vc);
    y.r32 = p; p = al(p + vc);
  }
  y.basis = p; p = al(p + vc * 2 * (size_t)o.restart);  // z_0 .. z_{m-1}, w_0 .. w_{m-1}
  y.scal = p; p = al(p + sizeof(double) * ((size_t)o.restart + 2 * (size_t)o.restart * (o.restart + 2) + 8));
  y.part = p; p = al(p + sizeof(double) * 2 * kDotChunk * kBlasMaxBlocks);
  if (o.precond == BSM_FGCR_PTC) {
    const size_t f = (size_t)2 * g.Vh * d * 4 * sizeof(float2);
    y.F_in = p; p = al(p + f);
    y.F_out = p; p = al(p + f);
    y.ptc = p; p = al(p + ptc_workspace_bytes(L, o.channels, 1, false));
  }
  if (o.prec_outer == BSM_DF64) {  // double-float copies of the outer operator's input and output
    y.dfi = p; p = al(p + 2 * half_spinor_bytes(g.Vh, d, BSM_F64));
    y.dfo = p; p = al(p + 2 * half_spinor_bytes(g.Vh, d, BSM_F64));
  }
  y.total = p;
  return y;
}

struct Fgcr {
  const bsm_lattice& L;
  const bsm_fgcr_opts& o;
  const void *U32, *W1, *W2;
  FgcrLayout y;
  char* w;
  cudaStream_t s;
  double* norm2;   // [restart]
  double2* bmat;   // [restart][restart]: column k holds beta_jk, j < k
  double2* alpha;  // [restart]
  double2* gamma;  // [restart]
  double* scalar;
  double* part;
  int G = 0;

  int host_read(double* dptr, double* out) const {
    if (cudaMemcpyAsync(out, dptr, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BSM_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? BSM_OK : BSM_ECUDA;
  }

  // the network's error word (the first word of its workspace: set when an
  // MMA-completion wait of the fused kernel gave up): BSM_ETIMEOUT if set
  int network_status() const {
    if (o.precond != BSM_FGCR_PTC) return BSM_OK;
    int err = 0;
    if (cudaMemcpyAsync(&err, w + y.ptc, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return BSM_ECUDA;
    return err ? BSM_ETIMEOUT : BSM_OK;
  }

  // out = D in (full) or Dhat in (even half; odd temporary in tmp)
  int apply(const OpCtx& c, const void* in, void* out) const {
    const int rc = o.eo ? op_dhat(c, in, out, w + y.tmp, 0, nullptr, nullptr) : op_dirac(c, in, out, 0, nullptr, nullptr);
    return rc < 0 ? rc : BSM_OK;
  }

  // apply() with the outer context on FP64 vectors: with prec_outer
  // BSM_DF64 through double-float copies (same element count and order)
  int apply64(const OpCtx& c, const void* in, void* out) const {
    if (o.prec_outer != BSM_DF64) return apply(c, in, out);
    const size_t n = (o.eo ? 1 : 2) * c.half_bytes / 16;
    f64_df64_launch(w + y.dfi, in, n, true, s);
    const int rc = apply(c, w + y.dfi, w + y.dfo);
    if (rc != BSM_OK) return rc;
    f64_df64_launch(out, w + y.dfo, n, false, s);
    return BSM_OK;
  }

  // z = M(r) at the cycle precision T; with eo the network acts on the field
  // that is r on the even sites and zero on the odd ones, and z keeps the even part
  template <typename T>
  int precondition(const T* r, T* z, size_t bytes) const {
    if (o.precond != BSM_FGCR_PTC)
      return cudaMemcpyAsync(z, r, bytes, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? BSM_OK : BSM_ECUDA;
    int rc;
    const bool f32 = sizeof(T) == sizeof(float2);
    // the fused BF16 network never reads the odd rows of an even-only input
    const bool odd_unread = o.eo && o.ptc_prec == BSM_BF16 && ptc_fused_supported(o.channels);
    rc = f32 ? ptc_pack32(L, reinterpret_cast<const float*>(r), w + y.F_in, false, o.eo ? (odd_unread ? 2 : 1) : 0, s)
             : ptc_pack(L, reinterpret_cast<const double*>(r), w + y.F_in, false, o.eo != 0, s);
    if (rc != BSM_OK) return rc;
    if ((rc = ptc_apply(L, U32, W1, W2, o.channels, w + y.F_in, w + y.F_out, 1, o.ptc_prec, w + y.ptc, s,
                        o.eo != 0, false)) != BSM_OK)
      return rc;
    return f32 ? ptc_pack32(L, reinterpret_cast<const float*>(z), w + y.F_out, true, o.eo ? 1 : 0, s)
               : ptc_pack(L, reinterpret_cast<const double*>(z), w + y.F_out, true, o.eo != 0, s);
  }

  // One restart cycle of FGCR on A x = r at precision T (x, r updated in
  // place): up to `restart` directions, at most `budget` iterations; stops
  // early once |r|^2 <= stop2.  Each new w = A z is orthogonalised against
  // the cycle's earlier ones in one pass (classical Gram-Schmidt: the dots
  // <w_j, w> of all j at once, then w -= sum_j beta_j w_j).  In exact
  // arithmetic this equals modified Gram-Schmidt; in floating point, and
  // above all in the FP32 cycles, classical Gram-Schmidt loses orthogonality
  // faster when w is nearly in the span of the w_j, which can cost extra
  // inner steps near the critical mass.  The iterates stay consistent either
  // way (x and r are updated with the same beta), and the FP64 residual
  // recomputed after each FP32 cycle is the stopping test, so the lost
  // orthogonality shows up as iterations, not as error.  Then r -= alpha w.  The preconditioned directions z are stored as they
  // come; the solution update that the orthogonalised directions imply is
  // formed once at the cycle's end from the stored beta and alpha (the
  // deferred update of GCR: half the basis traffic per step, and x is not
  // touched inside the cycle).  Returns the iterations, or < 0 on error;
  // *rr = the last |r|^2.
  template <typename T>
  int cycle(const OpCtx& c, T* x, T* r, size_t bytes, double stop2, int budget, double* rr) const {
    const size_t n = bytes / sizeof(T), stride = bytes / sizeof(T);
    T* zb = reinterpret_cast<T*>(w + y.basis);
    T* wb = zb + stride * o.restart;
    const int check = o.check_every > 0 ? o.check_every : 1;
    int it = 0, rc;
    int K = 0;  // directions of this cycle
    for (int k = 0; k < o.restart && it < budget; ++k) {
      T* z = zb + stride * k;
      T* wv = wb + stride * k;
      if ((rc = precondition<T>(r, z, bytes)) != BSM_OK) return rc;
      if ((rc = apply(c, z, wv)) != BSM_OK) return rc;
      double2* beta = bmat + (size_t)k * o.restart;
      if (k > 0) {
        for (int j0 = 0; j0 < k; j0 += kDotChunk) {
          const int cnt = k - j0 < kDotChunk ? k - j0 : kDotChunk;
          multi_dot_launch<T>(G, wb, stride, j0, cnt, wv, n, part, s);
          gs_coef_kernel<<<cnt, kBlasThreads, 0, s>>>(part, G, j0, norm2, beta);
        }
        gs_update_kernel<T><<<G, kBlasThreads, 0, s>>>(wv, wb, stride, k, n, beta);
      }
      wr_kernel<T><<<G, kBlasThreads, 0, s>>>(wv, r, n, part);
      alpha_kernel<<<1, kBlasThreads, 0, s>>>(part, G, norm2 + k, alpha + k);
      r_update_kernel<T><<<G, kBlasThreads, 0, s>>>(r, wv, n, alpha + k, part);
      reduce_launch(part, G, scalar, s);
      ++it;
      K = k + 1;
      // the host reads |r|^2 every check_every steps (and at the cycle's end):
      // fewer round trips, at most check_every - 1 steps past convergence
      if (it % check == 0 || k == o.restart - 1 || it == budget) {
        if ((rc = host_read(scalar, rr)) != BSM_OK) return rc;
        if (!isfinite(*rr) || *rr <= stop2) break;
      }
    }
    // x += sum_k alpha_k zhat_k, in the stored directions
    if (K > 0) {
      backsolve_kernel<<<1, 64, 0, s>>>(alpha, bmat, o.restart, K, gamma);
      x_update_kernel<T><<<G, kBlasThreads, 0, s>>>(x, zb, stride, K, n, gamma);
    }
    return it;
  }
};

}  // namespace

size_t fgcr_workspace_bytes(const bsm_lattice& L, const bsm_fgcr_opts& o) { return fgcr_layout(L, o).total; }

// validated by the caller
int fgcr_solve(const bsm_lattice& L, const void* U64, const void* U32, const void* W1, const void* W2,
               const void* b, void* x, const bsm_fgcr_opts& o, bsm_fgcr_stats* stats, void* ws, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const bool mixed = o.prec_inner == BSM_F32;
  const bool eo = o.eo != 0;
  const bool df = o.prec_outer == BSM_DF64;  // outer operator in double-float (only with FP32 cycles)
  const OpCtx c64 = make_ctx(L, U64, df ? BSM_DF64 : BSM_F64, s);
  const OpCtx c32 = make_ctx(L, mixed ? U32 : U64, mixed ? BSM_F32 : BSM_F64, s);
  Fgcr F{L, o, U32, W1, W2, fgcr_layout(L, o), reinterpret_cast<char*>(ws), s};
  char* w = F.w;
  // the 16-byte arrays first, so that each stays 16-byte aligned for any restart
  F.bmat = reinterpret_cast<double2*>(w + F.y.scal);
  F.alpha = F.bmat + (size_t)o.restart * o.restart;
  F.gamma = F.alpha + o.restart;
  F.norm2 = reinterpret_cast<double*>(F.gamma + o.restart);
  F.scalar = F.norm2 + o.restart;
  F.part = reinterpret_cast<double*>(w + F.y.part);
  const size_t h64 = c64.half_bytes, full64 = 2 * h64;
  const size_t v64 = eo ? h64 : full64, nv64 = v64 / sizeof(double2);
  F.G = blas_blocks(full64 / sizeof(double2));
  const char* bc = reinterpret_cast<const char*>(b);
  char* xc = reinterpret_cast<char*>(x);
  double2* r = reinterpret_cast<double2*>(w + F.y.r);
  int rc;

  // |b|^2 (full), the system's right-hand side rhs (b, or bhat_e = b_e + H_eo b_o / (2A)), r = rhs, x = 0
  diff2_kernel<<<F.G, kBlasThreads, 0, s>>>(reinterpret_cast<const double2*>(b), nullptr, nullptr,
                                            full64 / sizeof(double2), F.part);
  reduce_launch(F.part, F.G, F.scalar, s);
  double bb = 0.0;
  if ((rc = F.host_read(F.scalar, &bb)) != BSM_OK) return rc;
  if (!(bb > 0.0)) {
    cudaMemsetAsync(x, 0, full64, s);
    if (stats) *stats = bsm_fgcr_stats{0, 0, 0.0, 0.0};
    return isfinite(bb) ? BSM_OK : BSM_ENAN;
  }
  const double2* rhs = reinterpret_cast<const double2*>(b);
  if (eo) {
    if (df) {  // bhat_e from double-float copies of b_e, b_o
      f64_df64_launch(w + F.y.dfi, b, full64 / 16, true, s);
      if ((rc = op_hop(c64, 0, w + F.y.dfi + h64, w + F.y.dfo, 0, w + F.y.dfi, 1.0, 1.0 / (2.0 * c64.A), nullptr,
                       nullptr)) < 0)
        return rc;
      f64_df64_launch(w + F.y.bhat, w + F.y.dfo, h64 / 16, false, s);
    } else if ((rc = op_hop(c64, 0, bc + h64, w + F.y.bhat, 0, bc, 1.0, 1.0 / (2.0 * c64.A), nullptr, nullptr)) < 0) {
      return rc;
    }
    rhs = reinterpret_cast<const double2*>(w + F.y.bhat);
  }
  cudaMemsetAsync(x, 0, full64, s);
  cudaMemcpyAsync(r, rhs, v64, cudaMemcpyDeviceToDevice, s);
  // stop on |rhs - A x| <= tol |b|: with eo the full residual of the
  // reconstructed solution equals the even-site Schur residual
  const double stop2 = o.tol * o.tol * bb;
  double rr = 0.0;
  diff2_kernel<<<F.G, kBlasThreads, 0, s>>>(r, nullptr, nullptr, nv64, F.part);
  reduce_launch(F.part, F.G, F.scalar, s);
  if ((rc = F.host_read(F.scalar, &rr)) != BSM_OK) return rc;
  double2* xv = reinterpret_cast<double2*>(x);
  if (o.precond == BSM_FGCR_PTC && cudaMemsetAsync(w + F.y.ptc, 0, sizeof(int), s) != cudaSuccess) return BSM_ECUDA;
  int it = 0, cycles = 0, status = BSM_OK;
  while (rr > stop2) {
    if (it >= o.max_iter) {
      status = BSM_ENOCONV;
      break;
    }
    int k;
    if (!mixed) {
      k = F.cycle<double2>(c64, xv, r, v64, stop2, o.max_iter - it, &rr);
    } else {
      // FP32 cycle on A e = r from e = 0, to |r32| <= inner_tol |r|, then
      // x += e and r = rhs - A x in FP64
      const size_t v32 = eo ? c32.half_bytes : 2 * c32.half_bytes, nh = c32.half_bytes / 16;
      float2* x32 = reinterpret_cast<float2*>(w + F.y.x32);
      float2* r32 = reinterpret_cast<float2*>(w + F.y.r32);
      cudaMemsetAsync(x32, 0, v32, s);
      convert_to32_launch(BSM_F64, r32, r, nh, eo ? 1 : 2, s);
      const double inner = o.inner_tol > 0.0 ? o.inner_tol : 0.1;
      double rr32 = 0.0;
      k = F.cycle<float2>(c32, x32, r32, v32, fmax(inner * inner * rr, stop2), o.max_iter - it, &rr32);
      if (k >= 0) {
        accumulate32_launch(BSM_F64, x, x32, nh, eo ? 1 : 2, s);
        if ((rc = F.apply64(c64, x, r)) != BSM_OK) return rc;
        diff2_kernel<<<F.G, kBlasThreads, 0, s>>>(rhs, r, r, nv64, F.part);
        reduce_launch(F.part, F.G, F.scalar, s);
        if ((rc = F.host_read(F.scalar, &rr)) != BSM_OK) return rc;
        if (!isfinite(rr32)) rr = rr32;
      }
    }
    if (k < 0) return k;
    it += k;
    ++cycles;
    if ((rc = F.network_status()) != BSM_OK) {  // the network's tensor-core waits gave up
      status = rc;
      break;
    }
    if (!isfinite(rr)) {
      status = BSM_ENAN;
      break;
    }
  }
  // eo: x_o = (b_o + H_oe x_e / 2) / A
  if (eo && df) {  // from double-float copies of x_e and b_o
    f64_df64_launch(w + F.y.dfi, xc, h64 / 16, true, s);
    f64_df64_launch(w + F.y.dfi + h64, bc + h64, h64 / 16, true, s);
    if ((rc = op_hop(c64, 1, w + F.y.dfi, w + F.y.dfo + h64, 0, w + F.y.dfi + h64, 1.0 / c64.A, 1.0 / (2.0 * c64.A),
                     nullptr, nullptr)) < 0)
      return rc;
    f64_df64_launch(xc + h64, w + F.y.dfo + h64, h64 / 16, false, s);
  } else if (eo && (rc = op_hop(c64, 1, xc, xc + h64, 0, bc + h64, 1.0 / c64.A, 1.0 / (2.0 * c64.A), nullptr,
                                nullptr)) < 0) {
    return rc;
  }
  // true residual |b - D x| / |b| (D x into r)
  if (df) {
    f64_df64_launch(w + F.y.dfi, x, full64 / 16, true, s);
    if ((rc = op_dirac(c64, w + F.y.dfi, w + F.y.dfo, 0, nullptr, nullptr)) < 0) return rc;
    f64_df64_launch(r, w + F.y.dfo, full64 / 16, false, s);
  } else if ((rc = op_dirac(c64, x, r, 0, nullptr, nullptr)) < 0) {
    return rc;
  }
  diff2_kernel<<<F.G, kBlasThreads, 0, s>>>(reinterpret_cast<const double2*>(b), r, nullptr,
                                            full64 / sizeof(double2), F.part);
  reduce_launch(F.part, F.G, F.scalar, s);
  double res2 = 0.0;
  if ((rc = F.host_read(F.scalar, &res2)) != BSM_OK) return rc;
  if (stats) {
    stats->iters = it;
    stats->cycles = cycles;
    stats->true_res = sqrt(res2 / bb);
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status == BSM_OK && !isfinite(res2)) status = BSM_ENAN;
  return status;
}

}  // namespace bsm
