// cg_batch.cu -- mixed-precision CG on the even-odd normal equations
// Dhat^+ Dhat x_e = Dhat^+ bhat_e (Sec. II-B) of many systems at once: a batch
// of lattices of uneven size (SU(2) / SU(3) fundamental), each with nrhs
// right-hand sides sharing its gauge field.
//
// Every iteration treats all systems together:
//   p = r + beta_s p                  one launch over all systems
//   Mp = Dhat^+ Dhat p               one persistent cooperative launch of four
//                                    hop phases over all lattices and RHS
//                                    (batch.cu), each link read once per site
//                                    for all RHS of its lattice
//   pAp_s = |Dhat p|^2, alpha_s      a reduction launch and a scalar launch
//   x += alpha_s p, r -= alpha_s Mp, |r|^2, beta_s    two more launches
// in FP32 with per-system FP64 scalars kept on the device, so that the
// iterations between two host checks are captured once as a CUDA graph and
// replayed.  Reductions are deterministic: fixed per-block partials per
// system, summed in a fixed order.
// At each host check, every system whose residual has fallen by delta (or
// below the stopping bound) gets a reliable update (Clark et al. 2010) in the
// outer precision (FP64 or double-float): x_e += x32, r = bp - M x_e
// recomputed, the FP32 residual restarted from it and p re-projected against
// it.  A system stops, frozen with zero steps, once that recomputed residual
// is <= tol |bp|; the solve ends when every system has stopped.
// FP32 vectors use the multi-RHS layout of each lattice (RHS innermost);
// b, x and the outer vectors are ordinary FP64 device-layout spinors.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "batch.cuh"
#include "blas.cuh"
#include "operators.cuh"

namespace bsm {
namespace {

constexpr int kMaxItems = 32;
constexpr int kMaxRhs = 16;               // nrhs in {1, 2, 4, 8, 16}: divides the block ranges below
constexpr int kBtThreads = 256;
constexpr int kBtBlockElems = kBtThreads * 8;  // float4 elements per block of a vector kernel

struct SysState {
  double rr, rr_max, rr_prev, pAp, alpha, beta, stop2, rhs2;
  double rr_true;   // |bp - M x|^2 of the last reliable update
  double res_full;  // |b - D x|^2 at the end
  float alpha_f, beta_f;
  int active;       // 1: iterating; 0: stopped (zero steps)
  int want_update;  // the residual fell by delta or below the stop: reliable update at the next host check
  int nan;
  int iters;        // iterations taken while active
  int updates;      // reliable updates
  int stop_iter;    // iterations when it stopped
};

struct BtItem {
  float4 *x, *r, *p, *u, *Mp;
  long long n;      // float4 elements per vector: 2 d V_h nrhs
  int nrhs, sys0, blk0, nblk;
};
struct BtTable {
  BtItem it[kMaxItems];
  int count;
};

__device__ __forceinline__ int bt_item(const BtTable& T, int b) {
  int k = 0;
  while (k + 1 < T.count && b >= T.it[k + 1].blk0) ++k;
  return k;
}

// one double per (block, rhs): thread t holds the sum of RHS t % nrhs; the
// threads t < nrhs add the 256 / nrhs per-thread sums of their RHS in order
__device__ __forceinline__ void bt_block_partials(float v, int nrhs, double* out) {
  __shared__ double buf[kBtThreads];
  buf[threadIdx.x] = (double)v;
  __syncthreads();
  if ((int)threadIdx.x < nrhs) {
    double s = 0.0;
    for (int k = threadIdx.x; k < kBtThreads; k += nrhs) s += buf[k];
    out[threadIdx.x] = s;
  }
}

__device__ __forceinline__ float sq4(float4 a) { return fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, a.w * a.w))); }
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// p = r + beta_s p
__global__ void __launch_bounds__(kBtThreads) bt_p_kernel(const __grid_constant__ BtTable T, const SysState* st) {
  const BtItem& I = T.it[bt_item(T, blockIdx.x)];
  const long long e0 = (long long)(blockIdx.x - I.blk0) * kBtBlockElems + threadIdx.x;
  const float beta = st[I.sys0 + (int)(threadIdx.x % I.nrhs)].beta_f;
  for (long long e = e0; e < I.n && e < e0 - threadIdx.x + kBtBlockElems; e += kBtThreads)
    I.p[e] = axpy4(beta, I.p[e], I.r[e]);
}

// partials of |u|^2 per system
__global__ void __launch_bounds__(kBtThreads) bt_norm_u_kernel(const __grid_constant__ BtTable T, double* part) {
  const BtItem& I = T.it[bt_item(T, blockIdx.x)];
  const long long e0 = (long long)(blockIdx.x - I.blk0) * kBtBlockElems + threadIdx.x;
  float acc = 0.f;
  for (long long e = e0; e < I.n && e < e0 - threadIdx.x + kBtBlockElems; e += kBtThreads) acc += sq4(I.u[e]);
  bt_block_partials(acc, I.nrhs, part + (size_t)blockIdx.x * kMaxRhs);
}

// x += alpha_s p, r -= alpha_s Mp; partials of |r|^2 per system
__global__ void __launch_bounds__(kBtThreads) bt_xr_kernel(const __grid_constant__ BtTable T, const SysState* st,
                                                           double* part) {
  const BtItem& I = T.it[bt_item(T, blockIdx.x)];
  const long long e0 = (long long)(blockIdx.x - I.blk0) * kBtBlockElems + threadIdx.x;
  const float al = st[I.sys0 + (int)(threadIdx.x % I.nrhs)].alpha_f;
  float acc = 0.f;
  for (long long e = e0; e < I.n && e < e0 - threadIdx.x + kBtBlockElems; e += kBtThreads) {
    I.x[e] = axpy4(al, I.p[e], I.x[e]);
    const float4 r = axpy4(-al, I.Mp[e], I.r[e]);
    I.r[e] = r;
    acc += sq4(r);
  }
  bt_block_partials(acc, I.nrhs, part + (size_t)blockIdx.x * kMaxRhs);
}

constexpr int kSumThreads = 128;  // threads that sum one system's block partials

// sum over the item's blocks of one system's partials, in a fixed order:
// thread t adds blocks t, t + 128, ..., then a fixed shuffle and warp tree;
// the result is valid in thread 0
__device__ double bt_sum(const BtTable& T, const double* part, int k, int r) {
  const BtItem& I = T.it[k];
  double s = 0.0;
  for (int b = threadIdx.x; b < I.nblk; b += kSumThreads) s += part[(size_t)(I.blk0 + b) * kMaxRhs + r];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double w[kSumThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int j = 0; j < kSumThreads / 32; ++j) t += w[j];
  return t;
}

// fixed-order sum of part[0..n) by one block of kSumThreads threads; valid in thread 0
__device__ double block_sum_fixed(const double* part, int n) {
  double s = 0.0;
  for (int b = threadIdx.x; b < n; b += kSumThreads) s += part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double w[kSumThreads / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int j = 0; j < kSumThreads / 32; ++j) t += w[j];
  __syncthreads();
  return t;
}

// one block per system (grid: items x 16): alpha_s = |r|^2 / |Dhat p|^2 (zero for a stopped system)
__global__ void __launch_bounds__(kSumThreads) bt_alpha_kernel(const __grid_constant__ BtTable T, SysState* st,
                                                               const double* part) {
  const int k = blockIdx.x, r = blockIdx.y;
  if (r >= T.it[k].nrhs) return;
  const double pAp = bt_sum(T, part, k, r);
  if (threadIdx.x != 0) return;
  SysState& S = st[T.it[k].sys0 + r];
  S.pAp = pAp;
  double a = 0.0;
  if (!isfinite(pAp)) S.nan = 1;
  else if (S.active && pAp > 0.0) a = S.rr / pAp;
  S.alpha = a;
  S.alpha_f = (float)a;
}

// one block per system: the new |r|^2, beta_s, the reliable-update trigger
__global__ void __launch_bounds__(kSumThreads) bt_beta_kernel(const __grid_constant__ BtTable T, SysState* st,
                                                              const double* part, double delta2) {
  const int k = blockIdx.x, r = blockIdx.y;
  if (r >= T.it[k].nrhs) return;
  const double rr = bt_sum(T, part, k, r);
  if (threadIdx.x != 0) return;
  SysState& S = st[T.it[k].sys0 + r];
  if (!S.active) {
    S.beta = 0.0;
    S.beta_f = 0.f;
    return;
  }
  if (!isfinite(rr)) {
    S.nan = 1;
    S.active = 0;
    S.beta = 0.0;
    S.beta_f = 0.f;
    return;
  }
  const double b = S.rr > 0.0 ? rr / S.rr : 0.0;
  S.beta = b;
  S.beta_f = (float)b;
  S.rr_prev = S.rr;
  S.rr = rr;
  if (rr > S.rr_max) S.rr_max = rr;
  if (rr < delta2 * S.rr_max || rr <= S.stop2) S.want_update = 1;
  ++S.iters;
}

// --- one system's slot (RHS r of an item) against its FP64 outer vectors ---
// FP32 element (plane q = s d + c, site i) of a half spinor holds spins s and
// s + 2 of colour c; FP64 element k holds one complex number, spin s at
// plane q and spin s + 2 at plane q + 2d (n32 = 2 d V_h elements apart).
// The FP32 vectors hold all RHS in the site-major multi-RHS layout: element
// k = q V_h + i of a single-RHS half spinor is element (i 2d + q) n_rhs + r.
__device__ __forceinline__ long long slot_at(long long k, unsigned vh, long long n32, int nrhs, int r) {
  const unsigned q = (unsigned)k / vh, i = (unsigned)k - q * vh;
  return ((long long)i * (n32 / vh) + q) * nrhs + r;
}

// y64 += x32[slot], x32[slot] = 0
__global__ void __launch_bounds__(kBtThreads) slot_acc_kernel(double2* y, float4* x, long long n32, unsigned vh,
                                                              int nrhs, int r) {
  for (long long k = blockIdx.x * (long long)kBtThreads + threadIdx.x; k < n32; k += (long long)gridDim.x * kBtThreads) {
    float4* xp = x + slot_at(k, vh, n32, nrhs, r);
    const float4 v = *xp;
    double2 a = y[k], b = y[k + n32];
    a.x += v.x, a.y += v.y, b.x += v.z, b.y += v.w;
    y[k] = a;
    y[k + n32] = b;
    *xp = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// y32[slot] = nearest FP32 of x64
__global__ void __launch_bounds__(kBtThreads) slot_conv_kernel(float4* y, const double2* x, long long n32, unsigned vh,
                                                               int nrhs, int r) {
  for (long long k = blockIdx.x * (long long)kBtThreads + threadIdx.x; k < n32; k += (long long)gridDim.x * kBtThreads) {
    const double2 a = x[k], b = x[k + n32];
    y[slot_at(k, vh, n32, nrhs, r)] =
        make_float4(__double2float_rn(a.x), __double2float_rn(a.y), __double2float_rn(b.x), __double2float_rn(b.y));
  }
}

// partials of Re<r, p> and |r|^2 of one slot
__global__ void __launch_bounds__(kBtThreads) slot_dots_kernel(const float4* rv, const float4* pv, long long n32,
                                                               unsigned vh, int nrhs, int r, double* part) {
  float rp = 0.f, rr = 0.f;
  for (long long k = blockIdx.x * (long long)kBtThreads + threadIdx.x; k < n32; k += (long long)gridDim.x * kBtThreads) {
    const long long e = slot_at(k, vh, n32, nrhs, r);
    const float4 a = rv[e], b = pv[e];
    rp = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, rp))));
    rr += sq4(a);
  }
  float v[2] = {rp, rr};
  block_sums_store_f32<kBtThreads, 2>(v, part, gridDim.x);
}

// c = -<r, p> / <r, r> from the slot_dots partials (one thread, fixed order)
__global__ void __launch_bounds__(kSumThreads) slot_coef_kernel(const double* part, int nb, float* c) {
  const double rp = block_sum_fixed(part, nb);
  const double rr = block_sum_fixed(part + nb, nb);
  if (threadIdx.x == 0) *c = rr > 0.0 ? (float)(-rp / rr) : 0.f;
}

// p[slot] += c r[slot]
__global__ void __launch_bounds__(kBtThreads) slot_project_kernel(float4* pv, const float4* rv, long long n32, unsigned vh,
                                                                  int nrhs, int r, const float* cp) {
  const float c = *cp;
  for (long long k = blockIdx.x * (long long)kBtThreads + threadIdx.x; k < n32; k += (long long)gridDim.x * kBtThreads) {
    const long long e = slot_at(k, vh, n32, nrhs, r);
    pv[e] = axpy4(c, rv[e], pv[e]);
  }
}

// the reliable update's outcome for one system, on the device: stop once the
// recomputed residual (summed from the partials in a fixed order) is below
// the bound, else continue from it (beta from the last iterated residual)
__global__ void __launch_bounds__(kSumThreads) sys_update_kernel(SysState* st, int sys, const double* part, int nb) {
  const double rr = block_sum_fixed(part, nb);
  if (threadIdx.x != 0) return;
  SysState& S = st[sys];
  S.rr_true = rr;
  ++S.updates;
  S.want_update = 0;
  if (!isfinite(rr)) {
    S.nan = 1;
    S.active = 0;
    return;
  }
  if (rr <= S.stop2) {
    S.active = 0;
    S.rr = rr;
    S.stop_iter = S.iters;
    return;
  }
  S.beta = S.rr_prev > 0.0 ? rr / S.rr_prev : 0.0;
  S.beta_f = (float)S.beta;
  S.rr = S.rr_max = rr;
}

// the true residual of a system at the end (partials of |bp - M x|^2 and |b - D x|^2)
__global__ void __launch_bounds__(kSumThreads) sys_final_kernel(SysState* st, int sys, const double* part_n, int nn,
                                                                const double* part_f, int nf) {
  const double a = block_sum_fixed(part_n, nn);
  const double b = block_sum_fixed(part_f, nf);
  if (threadIdx.x != 0) return;
  SysState& S = st[sys];
  S.rr_true = a;
  S.res_full = b;
  if (S.active) S.stop_iter = S.iters;
}

int slot_blocks(long long n) {
  const long long b = (n + kBtThreads - 1) / kBtThreads;
  return (int)(b < kBlasMaxBlocks ? (b < 1 ? 1 : b) : kBlasMaxBlocks);
}

struct ItemPlan {
  OpCtx c32, co;        // FP32 inner and outer (F64 / DF64) operator contexts
  size_t half32, half64;  // one RHS's even half: FP32 and FP64 bytes
  float4 *x32, *r32, *p32, *u32, *Mp32, *t32;
  std::vector<double2*> bp;  // per RHS: Dhat^+ bhat_e, FP64
};

struct Layout {
  size_t ctl, st, part, scal, opart, items, bp, tmp, total;
  size_t max_half64;
  int nblocks, nsys;
};

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

Layout layout(const bsm_cg_batch_item* items, int count) {
  Layout y{};
  size_t o = 0;
  y.ctl = o; o += al256(batch_control_bytes());
  int nsys = 0, nblocks = 0;
  size_t vec32 = 0, bp = 0;
  for (int k = 0; k < count; ++k) {
    const Geom g = make_geom(items[k].lat);
    const int d = items[k].lat.N;
    const long long n = (long long)2 * d * g.Vh * items[k].nrhs;
    nblocks += (int)((n + kBtBlockElems - 1) / kBtBlockElems);
    nsys += items[k].nrhs;
    vec32 += 6 * al256(half_spinor_bytes(g.Vh, d, BSM_F32) * items[k].nrhs);
    const size_t h64 = half_spinor_bytes(g.Vh, d, BSM_F64);
    bp += items[k].nrhs * al256(h64);
    y.max_half64 = h64 > y.max_half64 ? h64 : y.max_half64;
  }
  y.nsys = nsys;
  y.nblocks = nblocks;
  y.st = o; o += al256(sizeof(SysState) * nsys);
  y.part = o; o += al256(sizeof(double) * kMaxRhs * (size_t)nblocks);
  y.scal = o; o += al256(sizeof(double) * 16);
  y.opart = o; o += al256(sizeof(double) * 2 * kBlasMaxBlocks);
  y.items = o; o += vec32;
  y.bp = o; o += bp;
  // outer temporaries, sized for the largest lattice: two full spinors and
  // three halves (outer precision; DF64 takes the bytes of FP64)
  y.tmp = o; o += 2 * al256(2 * y.max_half64) + 3 * al256(y.max_half64);
  y.total = o;
  return y;
}

struct BatchSolver {
  const bsm_cg_batch_item* items;
  int count;
  const bsm_cg_opts& o;
  cudaStream_t s;
  char* w;
  Layout y;
  std::vector<ItemPlan> plan;
  BtTable T;
  std::vector<BatchNormalItem> nitems;
  SysState* st;
  double *part, *scal, *opart;
  char *tfa, *tfb, *tha, *thb, *thc;  // outer temporaries: full a, full b, halves a, b, c
  int po;

  BatchSolver(const bsm_cg_batch_item* it, int n, const bsm_cg_opts& opts, void* ws, cudaStream_t st_)
      : items(it), count(n), o(opts), s(st_), w(reinterpret_cast<char*>(ws)), y(layout(it, n)), po(opts.prec_outer) {
    st = reinterpret_cast<SysState*>(w + y.st);
    part = reinterpret_cast<double*>(w + y.part);
    scal = reinterpret_cast<double*>(w + y.scal);
    opart = reinterpret_cast<double*>(w + y.opart);
    tfa = w + y.tmp;
    tfb = tfa + al256(2 * y.max_half64);
    tha = tfb + al256(2 * y.max_half64);
    thb = tha + al256(y.max_half64);
    thc = thb + al256(y.max_half64);
    memset(&T, 0, sizeof(T));
    T.count = count;
    size_t off = y.items, boff = y.bp;
    int sys0 = 0, blk0 = 0;
    plan.resize(count);
    for (int k = 0; k < count; ++k) {
      ItemPlan& P = plan[k];
      const bsm_cg_batch_item& I = items[k];
      P.c32 = make_ctx(I.lat, I.U_rep32, BSM_F32, s);
      P.co = make_ctx(I.lat, I.U_rep64, po, s);
      P.half32 = P.c32.half_bytes;
      P.half64 = half_spinor_bytes(P.c32.g.Vh, P.c32.d, BSM_F64);
      const size_t v = al256(P.half32 * I.nrhs);
      float4** vecs[6] = {&P.x32, &P.r32, &P.p32, &P.u32, &P.Mp32, &P.t32};
      for (float4** q : vecs) {
        *q = reinterpret_cast<float4*>(w + off);
        off += v;
      }
      for (int r = 0; r < I.nrhs; ++r) {
        P.bp.push_back(reinterpret_cast<double2*>(w + boff));
        boff += al256(P.half64);
      }
      BtItem& B = T.it[k];
      B.x = P.x32, B.r = P.r32, B.p = P.p32, B.u = P.u32, B.Mp = P.Mp32;
      B.n = (long long)(P.half32 / 16) * I.nrhs;
      B.nrhs = I.nrhs;
      B.sys0 = sys0;
      B.blk0 = blk0;
      B.nblk = (int)((B.n + kBtBlockElems - 1) / kBtBlockElems);
      sys0 += I.nrhs;
      blk0 += B.nblk;
      BatchNormalItem N;
      N.lat = I.lat;
      N.U32 = I.U_rep32;
      N.p = P.p32;
      N.u = P.u32;
      N.t = P.t32;
      N.Mp = P.Mp32;
      N.nrhs = I.nrhs;
      nitems.push_back(N);
    }
  }

  const char* b_of(int k, int r) const {
    return reinterpret_cast<const char*>(items[k].b) + (size_t)r * 2 * plan[k].half64;
  }
  char* x_of(int k, int r) const { return reinterpret_cast<char*>(items[k].x) + (size_t)r * 2 * plan[k].half64; }

  int host_scalar(const double* dev, double* h) {
    cudaError_t e = cudaMemcpyAsync(h, dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return BSM_ECUDA;
    }
    return BSM_OK;
  }

  // outer operator on FP64 vectors: out_half = M in_half (M = Dhat^+ Dhat at
  // the outer precision; double-float through copies)
  int apply_normal_outer(int k, const void* in_e, void* out_e) {
    const ItemPlan& P = plan[k];
    const size_t n16 = P.half64 / 16;
    int rc;
    if (po == BSM_DF64) {
      f64_df64_launch(tfa, in_e, n16, true, s);
      if ((rc = op_dhat(P.co, tfa, tfb, thb, 0, nullptr, nullptr)) < 0) return rc;
      if ((rc = op_dhat(P.co, tfb, tha, thb, 1, nullptr, nullptr)) < 0) return rc;
      f64_df64_launch(out_e, tha, n16, false, s);
    } else {
      if ((rc = op_dhat(P.co, in_e, tha, thb, 0, nullptr, nullptr)) < 0) return rc;
      if ((rc = op_dhat(P.co, tha, out_e, thb, 1, nullptr, nullptr)) < 0) return rc;
    }
    return BSM_OK;
  }

  // bp = Dhat^+ (b_e + H_eo b_o / (2A)) of system (k, r); |bp|^2 and |b|^2 -> scal[0], scal[1]
  int prepare(int k, int r) {
    const ItemPlan& P = plan[k];
    const size_t h = P.half64;
    const char* b = b_of(k, r);
    double2* bp = P.bp[r];
    int rc;
    if (po == BSM_DF64) {
      f64_df64_launch(tfa, b, 2 * h / 16, true, s);
      if ((rc = op_hop(P.co, 0, tfa + h, tfb, 0, tfa, 1.0, 1.0 / (2.0 * P.co.A), nullptr, nullptr)) < 0) return rc;
      if ((rc = op_dhat(P.co, tfb, tha, thb, 1, nullptr, nullptr)) < 0) return rc;
      f64_df64_launch(bp, tha, h / 16, false, s);
    } else {
      if ((rc = op_hop(P.co, 0, b + h, tfb, 0, b, 1.0, 1.0 / (2.0 * P.co.A), nullptr, nullptr)) < 0) return rc;
      if ((rc = op_dhat(P.co, tfb, bp, thb, 1, nullptr, nullptr)) < 0) return rc;
    }
    const int n1 = dot_launch(BSM_F64, bp, bp, h / 16, opart, s);
    reduce_launch(opart, n1, scal, s);
    const int n2 = dot_launch(BSM_F64, b, b, 2 * h / 16, opart + kBlasMaxBlocks, s);
    reduce_launch(opart + kBlasMaxBlocks, n2, scal + 1, s);
    return BSM_OK;
  }

  // r64 (in thc) = bp - M x_e of system (k, r); partials of |r64|^2 in
  // part_out; returns their count (or < 0)
  int true_residual(int k, int r, double* part_out) {
    const ItemPlan& P = plan[k];
    int rc = apply_normal_outer(k, x_of(k, r), thc);
    if (rc != BSM_OK) return rc;
    return axpby_launch(BSM_F64, 1.0, P.bp[r], -1.0, thc, P.half64 / 16, part_out, s);
  }

  // restart the FP32 residual of (k, r) from r64 (thc) and re-project p against it
  void restart_slot(int k, int r) {
    const ItemPlan& P = plan[k];
    const long long n32 = (long long)(P.half32 / 16);
    const int nr = items[k].nrhs, nb = slot_blocks(n32);
    const unsigned vh = (unsigned)P.c32.g.Vh;
    slot_conv_kernel<<<nb, kBtThreads, 0, s>>>(P.r32, reinterpret_cast<const double2*>(thc), n32, vh, nr, r);
    slot_dots_kernel<<<nb, kBtThreads, 0, s>>>(P.r32, P.p32, n32, vh, nr, r, opart);
    float* c = reinterpret_cast<float*>(scal + 8);
    slot_coef_kernel<<<1, kSumThreads, 0, s>>>(opart, nb, c);
    slot_project_kernel<<<nb, kBtThreads, 0, s>>>(P.p32, P.r32, n32, vh, nr, r, c);
  }

  // one iteration of every system
  int iterate() {
    const int nb = y.nblocks;
    bt_p_kernel<<<nb, kBtThreads, 0, s>>>(T, st);
    int rc = batch_normal_launch(nitems.data(), count, w + y.ctl, 1.0, s);
    if (rc != BSM_OK) return rc;
    bt_norm_u_kernel<<<nb, kBtThreads, 0, s>>>(T, part);
    bt_alpha_kernel<<<dim3(count, kMaxRhs), kSumThreads, 0, s>>>(T, st, part);
    bt_xr_kernel<<<nb, kBtThreads, 0, s>>>(T, st, part);
    const double delta = o.delta > 0 ? o.delta : 0.1;
    bt_beta_kernel<<<dim3(count, kMaxRhs), kSumThreads, 0, s>>>(T, st, part, delta * delta);
    return BSM_OK;
  }
};

}  // namespace

size_t cg_batch_workspace_bytes(const bsm_cg_batch_item* items, int count) { return layout(items, count).total; }

// validated by the caller: mixed precision (FP32 inner), even-odd, nrhs in {1, 2, 4, 8, 16}
int cg_solve_batch(const bsm_cg_batch_item* items, int count, const bsm_cg_opts& o, bsm_cg_stats* stats, void* ws,
                   cudaStream_t s) {
  if (cudaStreamSynchronize(s) != cudaSuccess) return BSM_ECUDA;
  const auto t0 = std::chrono::steady_clock::now();
  BatchSolver B(items, count, o, ws, s);
  const int nsys = B.y.nsys;
  const int check = o.check_every > 0 ? o.check_every : 8;
  std::vector<SysState> hs(nsys);
  std::vector<double> b2(nsys, 0.0);
  int rc = BSM_OK;

  // right-hand sides, x = 0, r = bp, p = 0
  for (int k = 0, sys = 0; k < count; ++k) {
    const ItemPlan& P = B.plan[k];
    const size_t v32 = P.half32 * items[k].nrhs;
    cudaMemsetAsync(P.x32, 0, v32, s);
    cudaMemsetAsync(P.p32, 0, v32, s);
    for (int r = 0; r < items[k].nrhs; ++r, ++sys) {
      if ((rc = B.prepare(k, r)) != BSM_OK) return rc;
      double h2[2];
      const cudaError_t e = cudaMemcpyAsync(h2, B.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return BSM_ECUDA;
      SysState& S = hs[sys];
      memset(&S, 0, sizeof(S));
      S.rhs2 = h2[0];
      b2[sys] = h2[1];
      if (!isfinite(S.rhs2) || !isfinite(b2[sys])) return BSM_ENAN;
      S.rr = S.rr_max = S.rr_prev = S.rhs2;
      S.stop2 = o.tol * o.tol * S.rhs2;
      S.active = S.rhs2 > 0.0;
      cudaMemsetAsync(B.x_of(k, r), 0, 2 * P.half64, s);
      slot_conv_kernel<<<slot_blocks((long long)(P.half32 / 16)), kBtThreads, 0, s>>>(
          P.r32, P.bp[r], (long long)(P.half32 / 16), (unsigned)P.c32.g.Vh, items[k].nrhs, r);
    }
  }
  cudaMemcpyAsync(B.st, hs.data(), sizeof(SysState) * nsys, cudaMemcpyHostToDevice, s);

  // one application of the batch operator before any capture: its first
  // call per batch shape tunes the launch configuration (p is zero here, and
  // u, t, Mp are recomputed by the first iteration)
  if ((rc = batch_normal_launch(B.nitems.data(), count, B.w + B.y.ctl, 1.0, s)) != BSM_OK ||
      (rc = batch_status(B.w + B.y.ctl, s)) != BSM_OK)
    return rc;

  // the iterations between host checks, captured once (not on the legacy default stream)
  cudaGraphExec_t exec = nullptr;
  const bool graph = o.use_graph != 0 && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
  if (graph) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return BSM_ECUDA;
    for (int j = 0; j < check && rc >= 0; ++j) rc = B.iterate();
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc != BSM_OK) return rc;
    if (e != cudaSuccess || cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return BSM_ECUDA;
    }
    cudaGraphDestroy(g);
  }

  int status = BSM_OK, iter = 0;
  auto read_states = [&]() -> int {
    cudaMemcpyAsync(hs.data(), B.st, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, s);
    return cudaStreamSynchronize(s) == cudaSuccess ? BSM_OK : BSM_ECUDA;
  };
  for (;;) {
    int running = 0;
    for (const SysState& S : hs) running += S.active;
    if (running == 0) break;
    if (iter >= o.max_iter) {
      status = BSM_ENOCONV;
      break;
    }
    if (graph) {
      if (cudaGraphLaunch(exec, s) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return BSM_ECUDA;
      }
    } else {
      for (int j = 0; j < check; ++j)
        if ((rc = B.iterate()) != BSM_OK) return rc;
    }
    iter += check;
    if ((rc = batch_status(B.w + B.y.ctl, s)) != BSM_OK || (rc = read_states()) != BSM_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      return rc;
    }
    // reliable updates of the systems that asked for one, queued without a
    // host round trip (the outcome is decided on the device)
    int queued = 0;
    for (int k = 0, sys = 0; k < count; ++k)
      for (int r = 0; r < items[k].nrhs; ++r, ++sys) {
        const SysState& S = hs[sys];
        if (S.nan) status = BSM_ENAN;
        if (!S.active || !S.want_update || S.nan) continue;
        const ItemPlan& P = B.plan[k];
        const long long n32 = (long long)(P.half32 / 16);
        slot_acc_kernel<<<slot_blocks(n32), kBtThreads, 0, s>>>(reinterpret_cast<double2*>(B.x_of(k, r)), P.x32, n32,
                                                               (unsigned)P.c32.g.Vh, items[k].nrhs, r);
        const int n = B.true_residual(k, r, B.opart + kBlasMaxBlocks);
        if (n < 0) return n;
        B.restart_slot(k, r);
        sys_update_kernel<<<1, kSumThreads, 0, s>>>(B.st, sys, B.opart + kBlasMaxBlocks, n);
        ++queued;
      }
    if (status == BSM_ENAN) break;
    if (queued && (rc = read_states()) != BSM_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      return rc;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);

  // odd sites x_o = (b_o + H_oe x_e / 2) / A and the residuals, at the outer precision
  for (int k = 0, sys = 0; k < count; ++k) {
    const ItemPlan& P = B.plan[k];
    const size_t h = P.half64;
    for (int r = 0; r < items[k].nrhs; ++r, ++sys) {
      if (hs[sys].active) {  // not stopped: fold in the last FP32 steps
        const long long n32 = (long long)(P.half32 / 16);
        slot_acc_kernel<<<slot_blocks(n32), kBtThreads, 0, s>>>(reinterpret_cast<double2*>(B.x_of(k, r)), P.x32,
                                                               n32, (unsigned)P.c32.g.Vh, items[k].nrhs, r);
      }
      const int nn = B.true_residual(k, r, B.opart);
      if (nn < 0) return nn;
      char* x = B.x_of(k, r);
      const char* b = B.b_of(k, r);
      if (B.po == BSM_DF64) {
        f64_df64_launch(B.tfa, x, h / 16, true, s);
        f64_df64_launch(B.tfa + h, b + h, h / 16, true, s);
        if ((rc = op_hop(P.co, 1, B.tfa, B.tfb, 0, B.tfa + h, 1.0 / P.co.A, 1.0 / (2.0 * P.co.A), nullptr,
                         nullptr)) < 0)
          return rc;
        f64_df64_launch(x + h, B.tfb, h / 16, false, s);
        f64_df64_launch(B.tfa, x, 2 * h / 16, true, s);
        if ((rc = op_dirac(P.co, B.tfa, B.tfb, 0, nullptr, nullptr)) < 0) return rc;
        f64_df64_launch(B.tfa, B.tfb, 2 * h / 16, false, s);
      } else {
        if ((rc = op_hop(P.co, 1, x, x + h, 0, b + h, 1.0 / P.co.A, 1.0 / (2.0 * P.co.A), nullptr, nullptr)) < 0)
          return rc;
        if ((rc = op_dirac(P.co, x, B.tfa, 0, nullptr, nullptr)) < 0) return rc;
      }
      const int nf = axpby_launch(BSM_F64, -1.0, b, 1.0, B.tfa, 2 * h / 16, B.opart + kBlasMaxBlocks, s);
      sys_final_kernel<<<1, kSumThreads, 0, s>>>(B.st, sys, B.opart, nn, B.opart + kBlasMaxBlocks, nf);
    }
  }
  cudaMemcpyAsync(hs.data(), B.st, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return BSM_ECUDA;
  for (int sys = 0; sys < nsys; ++sys) {
    const SysState& S = hs[sys];
    if (stats) {
      bsm_cg_stats& Q = stats[sys];
      Q.iters = S.stop_iter;
      Q.reliable_updates = S.updates;
      Q.true_res_normal = S.rhs2 > 0 ? sqrt(S.rr_true / S.rhs2) : 0.0;
      Q.true_res_full = b2[sys] > 0 ? sqrt(S.res_full / b2[sys]) : 0.0;
    }
    if (status == BSM_OK && !(S.rhs2 == 0.0 || S.rr_true <= o.tol * o.tol * S.rhs2)) status = BSM_ENOCONV;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats)
    for (int k = 0; k < nsys; ++k) stats[k].seconds = secs;
  return status;
}

}  // namespace bsm
