// fgcr.cu -- flexible GCR on the full Wilson operator D x = b (FP64), with
// either no preconditioner or the learned parallel-transport preconditioner,
// in FP64 throughout or in FP32 restart cycles with the residual recomputed
// in FP64 after each cycle (defect correction: x += e, r = b - D x).
//
// Flexible GCR (Notay 2000): z = M(r), w = D z; w and z are orthogonalised
// against the stored w_j by modified Gram-Schmidt (beta_j = <w_j, w>/|w_j|^2,
// w -= beta_j w_j, z -= beta_j z_j), then alpha = <w, r>/|w|^2,
// x += alpha z, r -= alpha w; after `restart` directions the basis is dropped.
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
int ptc_pack(const bsm_lattice& L, const double* psi, void* F, bool unpack, cudaStream_t s);
int ptc_pack32(const bsm_lattice& L, const float* psi, void* F, bool unpack, cudaStream_t s);
int ptc_apply(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* in,
              void* out, int nb, int prec, void* ws, cudaStream_t s);

namespace {

// complex elements as (x, y) pairs; accumulation always in FP64
template <typename T> __device__ __forceinline__ double2 ld2(const T* p, size_t k) {
  const T v = p[k];
  return make_double2(v.x, v.y);
}
template <typename T> __device__ __forceinline__ void st2(T* p, size_t k, double2 v);
template <> __device__ __forceinline__ void st2<double2>(double2* p, size_t k, double2 v) { p[k] = v; }
template <> __device__ __forceinline__ void st2<float2>(float2* p, size_t k, double2 v) {
  p[k] = make_float2((float)v.x, (float)v.y);
}

// partials of <a, b> = sum conj(a) b: re at [blk], im at [gridDim + blk]
template <typename T>
__global__ void __launch_bounds__(kBlasThreads) cdot_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                            size_t n, double* partials) {
  double re = 0.0, im = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const double2 x = ld2(a, k), y = ld2(b, k);
    re = fma(x.x, y.x, fma(x.y, y.y, re));
    im = fma(x.x, y.y, fma(-x.y, y.x, im));
  }
  block_sum_store<kBlasThreads>(re, partials);
  __syncthreads();
  block_sum_store<kBlasThreads>(im, partials + gridDim.x);
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

// coef = <w_j, w> / |w_j|^2 (one block)
__global__ void mgs_coef_kernel(const double* __restrict__ partials, int nblk, const double* __restrict__ norm2_j,
                                double2* coef) {
  const double re = sum_partials(partials, nblk);
  const double im = sum_partials(partials + nblk, nblk);
  if (threadIdx.x == 0) {
    const double n = *norm2_j;
    *coef = n > 0.0 ? make_double2(re / n, im / n) : make_double2(0.0, 0.0);
  }
}

// w -= coef w_j ; z -= coef z_j
template <typename T>
__global__ void __launch_bounds__(kBlasThreads) mgs_update_kernel(T* __restrict__ w, const T* __restrict__ wj,
                                                                  T* __restrict__ z, const T* __restrict__ zj,
                                                                  size_t n, const double2* __restrict__ coef) {
  const double2 c = *coef;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const double2 a = ld2(wj, k), b = ld2(zj, k);
    double2 x = ld2(w, k), y = ld2(z, k);
    x.x -= c.x * a.x - c.y * a.y;
    x.y -= c.x * a.y + c.y * a.x;
    y.x -= c.x * b.x - c.y * b.y;
    y.y -= c.x * b.y + c.y * b.x;
    st2(w, k, x);
    st2(z, k, y);
  }
}

// partials of |w|^2 [blk], Re<w, r> [G + blk], Im<w, r> [2G + blk]
template <typename T>
__global__ void __launch_bounds__(kBlasThreads) wr_kernel(const T* __restrict__ w, const T* __restrict__ r, size_t n,
                                                          double* partials) {
  double ww = 0.0, re = 0.0, im = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const double2 x = ld2(w, k), y = ld2(r, k);
    ww = fma(x.x, x.x, fma(x.y, x.y, ww));
    re = fma(x.x, y.x, fma(x.y, y.y, re));
    im = fma(x.x, y.y, fma(-x.y, y.x, im));
  }
  block_sum_store<kBlasThreads>(ww, partials);
  __syncthreads();
  block_sum_store<kBlasThreads>(re, partials + gridDim.x);
  __syncthreads();
  block_sum_store<kBlasThreads>(im, partials + 2 * gridDim.x);
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

// x += alpha z ; r -= alpha w ; partials of |r|^2
template <typename T>
__global__ void __launch_bounds__(kBlasThreads) xr_kernel(T* __restrict__ x, T* __restrict__ r,
                                                          const T* __restrict__ z, const T* __restrict__ w, size_t n,
                                                          const double2* __restrict__ alpha, double* partials) {
  const double2 a = *alpha;
  double rr = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const double2 zz = ld2(z, k), ww = ld2(w, k);
    double2 xx = ld2(x, k), q = ld2(r, k);
    xx.x += a.x * zz.x - a.y * zz.y;
    xx.y += a.x * zz.y + a.y * zz.x;
    q.x -= a.x * ww.x - a.y * ww.y;
    q.y -= a.x * ww.y + a.y * ww.x;
    st2(x, k, xx);
    st2(r, k, q);
    const double2 qs = ld2(r, k);  // the stored (rounded) residual
    rr = fma(qs.x, qs.x, fma(qs.y, qs.y, rr));
  }
  block_sum_store<kBlasThreads>(rr, partials);
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
  block_sum_store<kBlasThreads>(s, partials);
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct FgcrLayout {
  size_t r, x32, r32, basis, scal, part, F_in, F_out, ptc, total;
};

// mixed: FP32 cycle vectors (x32, r32, basis) next to the FP64 residual r
FgcrLayout fgcr_layout(const bsm_lattice& L, const bsm_fgcr_opts& o) {
  const Geom g = make_geom(L);
  const int d = rep_info(L.N, L.rep).d;
  const bool mixed = o.prec_inner == BSM_F32;
  const size_t full = 2 * half_spinor_bytes(g.Vh, d, mixed ? BSM_F32 : BSM_F64);
  FgcrLayout y{};
  size_t p = 0;
  y.r = p; p = al(p + 2 * half_spinor_bytes(g.Vh, d, BSM_F64));
  if (mixed) {
    y.x32 = p; p = al(p + full);
    y.r32 = p; p = al(p + full);
  }
  y.basis = p; p = al(p + full * 2 * (size_t)o.restart);  // z_0 .. z_{m-1}, w_0 .. w_{m-1}
  y.scal = p; p = al(p + sizeof(double) * ((size_t)o.restart + 8));
  y.part = p; p = al(p + sizeof(double) * 3 * kBlasMaxBlocks);
  if (o.precond == BSM_FGCR_PTC) {
    const size_t f = (size_t)2 * g.Vh * d * 4 * sizeof(float2);
    y.F_in = p; p = al(p + f);
    y.F_out = p; p = al(p + f);
    y.ptc = p; p = al(p + ptc_workspace_bytes(L, o.channels, 1, false));
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
  double* norm2;
  double2 *coef, *alpha;
  double* scalar;
  double* part;
  int G = 0;

  int host_read(double* dptr, double* out) const {
    if (cudaMemcpyAsync(out, dptr, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BSM_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? BSM_OK : BSM_ECUDA;
  }

  // z = M(r) at the cycle precision T
  template <typename T>
  int precondition(const T* r, T* z, size_t full) const {
    if (o.precond != BSM_FGCR_PTC) return cudaMemcpyAsync(z, r, full, cudaMemcpyDeviceToDevice, s) == cudaSuccess
                                              ? BSM_OK : BSM_ECUDA;
    int rc;
    const bool f32 = sizeof(T) == sizeof(float2);
    rc = f32 ? ptc_pack32(L, reinterpret_cast<const float*>(r), w + y.F_in, false, s)
             : ptc_pack(L, reinterpret_cast<const double*>(r), w + y.F_in, false, s);
    if (rc != BSM_OK) return rc;
    if ((rc = ptc_apply(L, U32, W1, W2, o.channels, w + y.F_in, w + y.F_out, 1, o.ptc_prec, w + y.ptc, s)) != BSM_OK)
      return rc;
    return f32 ? ptc_pack32(L, reinterpret_cast<const float*>(z), w + y.F_out, true, s)
               : ptc_pack(L, reinterpret_cast<const double*>(z), w + y.F_out, true, s);
  }

  // One restart cycle of FGCR on D x = r at precision T (x, r updated in
  // place): up to `restart` directions, at most `budget` iterations; stops
  // early once |r|^2 <= stop2.  Returns the iterations, or < 0 on error;
  // *rr receives the last |r|^2.
  template <typename T>
  int cycle(const OpCtx& c, T* x, T* r, size_t full, double stop2, int budget, double* rr) const {
    const size_t n = full / sizeof(T);
    auto Z = [&](int j) { return reinterpret_cast<T*>(w + y.basis + full * j); };
    auto Wb = [&](int j) { return reinterpret_cast<T*>(w + y.basis + full * (o.restart + j)); };
    int it = 0, rc;
    for (int k = 0; k < o.restart && it < budget; ++k) {
      T* z = Z(k);
      T* wv = Wb(k);
      if ((rc = precondition<T>(r, z, full)) != BSM_OK) return rc;
      if ((rc = op_dirac(c, z, wv, 0, nullptr, nullptr)) < 0) return rc;
      for (int j = 0; j < k; ++j) {
        cdot_kernel<T><<<G, kBlasThreads, 0, s>>>(Wb(j), wv, n, part);
        mgs_coef_kernel<<<1, kBlasThreads, 0, s>>>(part, G, norm2 + j, coef);
        mgs_update_kernel<T><<<G, kBlasThreads, 0, s>>>(wv, Wb(j), z, Z(j), n, coef);
      }
      wr_kernel<T><<<G, kBlasThreads, 0, s>>>(wv, r, n, part);
      alpha_kernel<<<1, kBlasThreads, 0, s>>>(part, G, norm2 + k, alpha);
      xr_kernel<T><<<G, kBlasThreads, 0, s>>>(x, r, z, wv, n, alpha, part);
      reduce_launch(part, G, scalar, s);
      if ((rc = host_read(scalar, rr)) != BSM_OK) return rc;
      ++it;
      if (!isfinite(*rr) || *rr <= stop2) break;
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
  const OpCtx c64 = make_ctx(L, U64, BSM_F64, s);
  const OpCtx c32 = make_ctx(L, mixed ? U32 : U64, mixed ? BSM_F32 : BSM_F64, s);
  Fgcr F{L, o, U32, W1, W2, fgcr_layout(L, o), reinterpret_cast<char*>(ws), s};
  char* w = F.w;
  F.norm2 = reinterpret_cast<double*>(w + F.y.scal);   // [restart]
  F.coef = reinterpret_cast<double2*>(F.norm2 + o.restart);
  F.alpha = F.coef + 1;
  F.scalar = reinterpret_cast<double*>(F.alpha + 1);
  F.part = reinterpret_cast<double*>(w + F.y.part);
  const size_t full64 = 2 * c64.half_bytes, n64 = full64 / sizeof(double2);
  F.G = blas_blocks(n64);
  double2* r = reinterpret_cast<double2*>(w + F.y.r);
  double2* xv = reinterpret_cast<double2*>(x);
  const double2* bv = reinterpret_cast<const double2*>(b);

  // x = 0, r = b
  cudaMemsetAsync(x, 0, full64, s);
  cudaMemcpyAsync(r, b, full64, cudaMemcpyDeviceToDevice, s);
  diff2_kernel<<<F.G, kBlasThreads, 0, s>>>(bv, nullptr, nullptr, n64, F.part);
  reduce_launch(F.part, F.G, F.scalar, s);
  double bb = 0.0;
  int rc = F.host_read(F.scalar, &bb);
  if (rc != BSM_OK) return rc;
  if (!(bb > 0.0)) {
    if (stats) *stats = bsm_fgcr_stats{0, 0, 0.0, 0.0};
    return isfinite(bb) ? BSM_OK : BSM_ENAN;
  }
  const double stop2 = o.tol * o.tol * bb;
  double rr = bb;
  int it = 0, cycles = 0, status = BSM_OK;
  while (rr > stop2) {
    if (it >= o.max_iter) {
      status = BSM_ENOCONV;
      break;
    }
    int k;
    if (!mixed) {
      k = F.cycle<double2>(c64, xv, r, full64, stop2, o.max_iter - it, &rr);
    } else {
      // FP32 cycle on D e = r from e = 0, to |r32| <= inner_tol |r|, then
      // x += e and the residual recomputed in FP64
      const size_t full32 = 2 * c32.half_bytes, nh = c32.half_bytes / 16;
      float2* x32 = reinterpret_cast<float2*>(w + F.y.x32);
      float2* r32 = reinterpret_cast<float2*>(w + F.y.r32);
      cudaMemsetAsync(x32, 0, full32, s);
      convert_to32_launch(BSM_F64, r32, r, nh, 2, s);
      const double inner = o.inner_tol > 0.0 ? o.inner_tol : 0.1;
      double rr32 = 0.0;
      k = F.cycle<float2>(c32, x32, r32, full32, fmax(inner * inner * rr, stop2), o.max_iter - it, &rr32);
      if (k >= 0) {
        accumulate32_launch(BSM_F64, x, x32, nh, 2, s);
        if ((rc = op_dirac(c64, x, r, 0, nullptr, nullptr)) < 0) return rc;
        diff2_kernel<<<F.G, kBlasThreads, 0, s>>>(bv, r, r, n64, F.part);
        reduce_launch(F.part, F.G, F.scalar, s);
        if ((rc = F.host_read(F.scalar, &rr)) != BSM_OK) return rc;
        if (!isfinite(rr32)) rr = rr32;
      }
    }
    if (k < 0) return k;
    it += k;
    ++cycles;
    if (!isfinite(rr)) {
      status = BSM_ENAN;
      break;
    }
  }
  // true residual |b - D x| / |b| (into r)
  if ((rc = op_dirac(c64, x, r, 0, nullptr, nullptr)) < 0) return rc;
  diff2_kernel<<<F.G, kBlasThreads, 0, s>>>(bv, r, nullptr, n64, F.part);
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
