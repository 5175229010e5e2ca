// fgcr.cu -- flexible GCR on the full Wilson operator D x = b (FP64), with
// either no preconditioner or the learned parallel-transport preconditioner.
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
int ptc_apply(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* in,
              void* out, int nb, int prec, void* ws, cudaStream_t s);

namespace {

// partials of <a, b> = sum conj(a) b: re at [blk], im at [gridDim + blk]
__global__ void __launch_bounds__(kBlasThreads) cdot_kernel(const double2* __restrict__ a,
                                                            const double2* __restrict__ b, size_t n,
                                                            double* partials) {
  double re = 0.0, im = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const double2 x = a[k], y = b[k];
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
__global__ void __launch_bounds__(kBlasThreads) mgs_update_kernel(double2* __restrict__ w,
                                                                  const double2* __restrict__ wj,
                                                                  double2* __restrict__ z,
                                                                  const double2* __restrict__ zj, size_t n,
                                                                  const double2* __restrict__ coef) {
  const double2 c = *coef;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const double2 a = wj[k], b = zj[k];
    double2 x = w[k], y = z[k];
    x.x -= c.x * a.x - c.y * a.y;
    x.y -= c.x * a.y + c.y * a.x;
    y.x -= c.x * b.x - c.y * b.y;
    y.y -= c.x * b.y + c.y * b.x;
    w[k] = x;
    z[k] = y;
  }
}

// partials of |w|^2 [blk], Re<w, r> [G + blk], Im<w, r> [2G + blk]
__global__ void __launch_bounds__(kBlasThreads) wr_kernel(const double2* __restrict__ w,
                                                          const double2* __restrict__ r, size_t n,
                                                          double* partials) {
  double ww = 0.0, re = 0.0, im = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const double2 x = w[k], y = r[k];
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
__global__ void __launch_bounds__(kBlasThreads) xr_kernel(double2* __restrict__ x, double2* __restrict__ r,
                                                          const double2* __restrict__ z,
                                                          const double2* __restrict__ w, size_t n,
                                                          const double2* __restrict__ alpha, double* partials) {
  const double2 a = *alpha;
  double rr = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    const double2 zz = z[k], ww = w[k];
    double2 xx = x[k], q = r[k];
    xx.x += a.x * zz.x - a.y * zz.y;
    xx.y += a.x * zz.y + a.y * zz.x;
    q.x -= a.x * ww.x - a.y * ww.y;
    q.y -= a.x * ww.y + a.y * ww.x;
    x[k] = xx;
    r[k] = q;
    rr = fma(q.x, q.x, fma(q.y, q.y, rr));
  }
  block_sum_store<kBlasThreads>(rr, partials);
}

// partials of |a - b|^2 (b may be null: |a|^2)
__global__ void __launch_bounds__(kBlasThreads) diff2_kernel(const double2* __restrict__ a,
                                                             const double2* __restrict__ b, size_t n,
                                                             double* partials) {
  double s = 0.0;
  for (size_t k = blockIdx.x * (size_t)kBlasThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kBlasThreads) {
    double2 v = a[k];
    if (b != nullptr) {
      v.x -= b[k].x;
      v.y -= b[k].y;
    }
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  block_sum_store<kBlasThreads>(s, partials);
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct FgcrLayout {
  size_t r, basis, scal, part, F_in, F_out, ptc, total;
};

FgcrLayout fgcr_layout(const bsm_lattice& L, const bsm_fgcr_opts& o) {
  const Geom g = make_geom(L);
  const int d = rep_info(L.N, L.rep).d;
  const size_t full = 2 * half_spinor_bytes(g.Vh, d, BSM_F64);
  FgcrLayout y{};
  size_t p = 0;
  y.r = p; p = al(p + full);
  y.basis = p; p = al(p + full * 2 * (size_t)o.restart);  // z_0 .. z_{m-1}, w_0 .. w_{m-1}
  y.scal = p; p = al(p + sizeof(double) * ((size_t)o.restart + 8));
  y.part = p; p = al(p + sizeof(double) * 3 * kBlasMaxBlocks);
  y.F_in = y.F_out = y.ptc = 0;
  if (o.precond == BSM_FGCR_PTC) {
    const size_t f = (size_t)2 * g.Vh * d * 4 * sizeof(float2);
    y.F_in = p; p = al(p + f);
    y.F_out = p; p = al(p + f);
    y.ptc = p; p = al(p + ptc_workspace_bytes(L, o.channels, 1, false));
  }
  y.total = p;
  return y;
}

}  // namespace

size_t fgcr_workspace_bytes(const bsm_lattice& L, const bsm_fgcr_opts& o) { return fgcr_layout(L, o).total; }

// validated by the caller
int fgcr_solve(const bsm_lattice& L, const void* U64, const void* U32, const void* W1, const void* W2,
               const void* b, void* x, const bsm_fgcr_opts& o, bsm_fgcr_stats* stats, void* ws, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const OpCtx c = make_ctx(L, U64, BSM_F64, s);
  const FgcrLayout y = fgcr_layout(L, o);
  char* w = reinterpret_cast<char*>(ws);
  const size_t full = 2 * c.half_bytes, n = full / sizeof(double2);
  const int m = o.restart;
  double2* r = reinterpret_cast<double2*>(w + y.r);
  double2* xv = reinterpret_cast<double2*>(x);
  const double2* bv = reinterpret_cast<const double2*>(b);
  auto Z = [&](int j) { return reinterpret_cast<double2*>(w + y.basis + full * j); };
  auto Wb = [&](int j) { return reinterpret_cast<double2*>(w + y.basis + full * (m + j)); };
  double* norm2 = reinterpret_cast<double*>(w + y.scal);                 // [m]
  double2* coef = reinterpret_cast<double2*>(norm2 + m);                 // 2 doubles
  double2* alpha = coef + 1;                                             // 2 doubles
  double* scalar = reinterpret_cast<double*>(alpha + 1);                 // reductions read by the host
  double* part = reinterpret_cast<double*>(w + y.part);
  const int G = blas_blocks(n);

  auto host_read = [&](double* dptr, double* out) -> int {
    if (cudaMemcpyAsync(out, dptr, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BSM_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? BSM_OK : BSM_ECUDA;
  };

  // x = 0, r = b
  cudaMemsetAsync(x, 0, full, s);
  cudaMemcpyAsync(r, b, full, cudaMemcpyDeviceToDevice, s);
  diff2_kernel<<<G, kBlasThreads, 0, s>>>(bv, nullptr, n, part);
  reduce_launch(part, G, scalar, s);
  double bb = 0.0, rr = 0.0;
  int rc = host_read(scalar, &bb);
  if (rc != BSM_OK) return rc;
  rr = bb;
  const double stop2 = o.tol * o.tol * bb;
  int it = 0, k = 0, status = BSM_OK;
  if (!(bb > 0.0)) {
    if (stats) *stats = bsm_fgcr_stats{0, 0.0, 0.0};
    return isfinite(bb) ? BSM_OK : BSM_ENAN;
  }
  while (rr > stop2) {
    if (it >= o.max_iter) {
      status = BSM_ENOCONV;
      break;
    }
    double2* z = Z(k);
    double2* wv = Wb(k);
    // z = M(r)
    if (o.precond == BSM_FGCR_PTC) {
      if ((rc = ptc_pack(L, reinterpret_cast<const double*>(r), w + y.F_in, false, s)) != BSM_OK) return rc;
      if ((rc = ptc_apply(L, U32, W1, W2, o.channels, w + y.F_in, w + y.F_out, 1, o.ptc_prec, w + y.ptc, s)) !=
          BSM_OK)
        return rc;
      if ((rc = ptc_pack(L, reinterpret_cast<const double*>(z), w + y.F_out, true, s)) != BSM_OK) return rc;
    } else {
      cudaMemcpyAsync(z, r, full, cudaMemcpyDeviceToDevice, s);
    }
    // w = D z
    if ((rc = op_dirac(c, z, wv, 0, nullptr, nullptr)) < 0) return rc;
    for (int j = 0; j < k; ++j) {
      cdot_kernel<<<G, kBlasThreads, 0, s>>>(Wb(j), wv, n, part);
      mgs_coef_kernel<<<1, kBlasThreads, 0, s>>>(part, G, norm2 + j, coef);
      mgs_update_kernel<<<G, kBlasThreads, 0, s>>>(wv, Wb(j), z, Z(j), n, coef);
    }
    wr_kernel<<<G, kBlasThreads, 0, s>>>(wv, r, n, part);
    alpha_kernel<<<1, kBlasThreads, 0, s>>>(part, G, norm2 + k, alpha);
    xr_kernel<<<G, kBlasThreads, 0, s>>>(xv, r, z, wv, n, alpha, part);
    reduce_launch(part, G, scalar, s);
    if ((rc = host_read(scalar, &rr)) != BSM_OK) return rc;
    ++it;
    if (!isfinite(rr)) {
      status = BSM_ENAN;
      break;
    }
    if (++k == m) k = 0;
  }
  // true residual |b - D x| / |b| (into r)
  if ((rc = op_dirac(c, x, r, 0, nullptr, nullptr)) < 0) return rc;
  diff2_kernel<<<G, kBlasThreads, 0, s>>>(bv, r, n, part);
  reduce_launch(part, G, scalar, s);
  double res2 = 0.0;
  if ((rc = host_read(scalar, &res2)) != BSM_OK) return rc;
  if (stats) {
    stats->iters = it;
    stats->true_res = sqrt(res2 / bb);
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status == BSM_OK && !isfinite(res2)) status = BSM_ENAN;
  return status;
}

}  // namespace bsm
