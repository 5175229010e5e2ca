// hop_df64.cu -- DF64 (double-float) instantiations of the hopping block (Sec. II-B).
//
// The double-float hop costs about 9k FP32 operations per site against 1536
// bytes of traffic, so unlike the FP32 hop it is bound by the FP32 pipe and by
// instruction issue, not by HBM.  For complex representations with d <= 3
// (the SU(2)/SU(3) fundamental and SU(3) two-index ones) a dedicated kernel
// attacks both:
//  - issue: the link matrix-vector products and the spin reconstruction run
//    on packed FP32 pairs (f32x2.cuh), the two lanes being the two projected
//    spin components h0, h1 that every link multiplies, so one instruction
//    does the work of two;
//  - latency: the links and the neighbour spinor of the next direction-sense
//    are copied into shared memory (cp.async, two stages per thread) while
//    the current one is computed.
// Every lane operation is the scalar double-float operation of df64.cuh in
// the same order, so its results equal the generic kernel's bit for bit.
// The other DF64 cases use the generic hop_kernel of hop.cuh.
#include "f32x2.cuh"
#include "hop.cuh"

namespace bsm {
namespace {

constexpr int kDfThreads = 64;    // threads (sites) per block of the staged kernel
constexpr int kDfMinBlocks = 4;   // resident blocks per SM: 166 registers, 43 KB shared (d = 3)

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most one committed group of this thread is still in flight
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// per-thread shared-memory slots of one stage: the d^2 link elements and the
// 4d spin-colour components of the neighbour spinor, each one float4
template <int D>
struct DfStage {
  static constexpr int links = D * D, psi = 4 * D, slots = links + psi;
  static constexpr size_t bytes = (size_t)2 * slots * kDfThreads * sizeof(float4);
};

// neighbour of direction-sense k = 2 mu + fb without indexing a local array
__device__ __forceinline__ int neighbour_of(int k, const int (&nf)[4], const int (&nb)[4]) {
  int n = nf[0];
  n = k == 1 ? nb[0] : n;
  n = k == 2 ? nf[1] : n;
  n = k == 3 ? nb[1] : n;
  n = k == 4 ? nf[2] : n;
  n = k == 5 ? nb[2] : n;
  n = k == 6 ? nf[3] : n;
  n = k == 7 ? nb[3] : n;
  return n;
}

// Spin reconstruction of direction MU from W = (w0, w1) (lanes = the two
// projected spin components; chain form with negated low parts) into the
// upper accumulators a01 = (acc0, acc1) and the lower ones a23 = (acc2, acc3):
// acc0,1 += w0,1 and acc2,3 += sg B_mu^+ (w0, w1), B_mu^+ acting as a lane
// swap and the signs of +-1 / +-i.
template <int MU, int D>
__device__ __forceinline__ void reconstruct_pairs(dfp2 (&a01re)[D], dfp2 (&a01im)[D], dfp2 (&a23re)[D],
                                                  dfp2 (&a23im)[D], const dfn2 (&Wre)[D], const dfn2 (&Wim)[D],
                                                  float sg) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    padd(a01re[a], Wre[a].hi, Wre[a].nlo);
    padd(a01im[a], Wim[a].hi, Wim[a].nlo);
    f32x2 cr_h, cr_n, ci_h, ci_n, sr, si;  // (c0, c1) before the lane signs sr, si
    if (MU == 0) {         // (c0, c1) = (w0, w1)
      cr_h = Wre[a].hi, cr_n = Wre[a].nlo, ci_h = Wim[a].hi, ci_n = Wim[a].nlo;
      sr = si = pk2(sg, sg);
    } else if (MU == 1) {  // (i w1, i w0)
      cr_h = swap2(Wim[a].hi), cr_n = swap2(Wim[a].nlo), ci_h = swap2(Wre[a].hi), ci_n = swap2(Wre[a].nlo);
      sr = pk2(-sg, -sg);
      si = pk2(sg, sg);
    } else if (MU == 2) {  // (w1, -w0)
      cr_h = swap2(Wre[a].hi), cr_n = swap2(Wre[a].nlo), ci_h = swap2(Wim[a].hi), ci_n = swap2(Wim[a].nlo);
      sr = si = pk2(sg, -sg);
    } else {               // (i w0, -i w1)
      cr_h = Wim[a].hi, cr_n = Wim[a].nlo, ci_h = Wre[a].hi, ci_n = Wre[a].nlo;
      sr = pk2(-sg, sg);
      si = pk2(sg, -sg);
    }
    padd(a23re[a], mul2(cr_h, sr), mul2(cr_n, sr));
    padd(a23im[a], mul2(ci_h, si), mul2(ci_n, si));
  }
}

// PARTIALS: the launch writes block partials of |out|^2.  It is a template
// parameter because merely compiling the norm and block reduction into the
// kernel slows the hop without partials by 11 % (357 against 320 us per
// launch on the 32^3 x 64 workload): the hop gets its own instantiation.
template <int D, bool PARTIALS>
__global__ void __launch_bounds__(kDfThreads, kDfMinBlocks) hop_df64_staged_kernel(const HopArgs A) {
  using S = DfStage<D>;
  extern __shared__ float4 stage_mem[];  // [stage 2][slot][thread]
  if (A.done != nullptr && *A.done != 0) return;  // uniform over the grid
  const int t = threadIdx.x;
  const int i = blockIdx.x * kDfThreads + t;
  const bool active = i < A.g.Vh;
  const size_t Vh = (size_t)A.g.Vh;
  int nf[4] = {0, 0, 0, 0}, nb[4] = {0, 0, 0, 0};
  const float4* lt = nullptr;
  if (active) {
    eo_neighbours(A.g, i, A.p, nf, nb);
    lt = LinkIO<DF64, D, false>::tile_ptr(A.links, i);
  }
  const float4* in = reinterpret_cast<const float4*>(A.in);
  // copies for direction-sense k (links planes k d^2 .. k d^2 + d^2 - 1 of the
  // site's tile, then the 4d planes of the neighbour spinor) into stage k & 1
  auto issue = [&](int k) {
    if (active && k < 8) {
      const int n = neighbour_of(k, nf, nb);
      float4* dst = stage_mem + (size_t)(k & 1) * S::slots * kDfThreads + t;
      const float4* ls = lt + (size_t)(k * S::links) * kLinkTile;
#pragma unroll
      for (int q = 0; q < S::psi; ++q) cp_async16(dst + (S::links + q) * kDfThreads, in + (size_t)q * Vh + n);
#pragma unroll
      for (int c = 0; c < S::links; ++c) cp_async16(dst + c * kDfThreads, ls + c * kLinkTile);
    }
    cp_async_commit();  // every thread commits, so the group count stays uniform
  };
  issue(0);
  issue(1);

  const df sg = A.dagger ? df(1.f, 0.f) : df(-1.f, 0.f);  // forward sense; backward is -sg
  const f32x2 m1 = pk2(-1.f, -1.f), z2 = pk2(0.f, 0.f);
  dfp2 a01re[D], a01im[D], a23re[D], a23im[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    a01re[a].hi = a01re[a].lo = z2;
    a01im[a] = a23re[a] = a23im[a] = a01re[a];
  }
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    cp_async_wait_all_but_one();  // this thread's copies for sense k have landed
    const float4* st = stage_mem + (size_t)(k & 1) * S::slots * kDfThreads + t;
    const int mu = k >> 1;
    const df s = (k & 1) ? -sg : sg;
    // spin projection h = u + s B_mu l (scalar), then the pairs (h0, h1) with their negations
    dfv2 Hre[D], Him[D];
    {
      cx<df> psi[4][D], h[2][D];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const float4 v = st[(S::links + sp * D + a) * kDfThreads];
          psi[sp][a] = cmake(df(v.x, v.y), df(v.z, v.w));
        }
      switch (mu) {
        case 0: spin_project<0>(psi, s, h); break;
        case 1: spin_project<1>(psi, s, h); break;
        case 2: spin_project<2>(psi, s, h); break;
        default: spin_project<3>(psi, s, h); break;
      }
#pragma unroll
      for (int b = 0; b < D; ++b) {
        Hre[b].hi = pk2(h[0][b].re.hi, h[1][b].re.hi);
        Hre[b].lo = pk2(h[0][b].re.lo, h[1][b].re.lo);
        Him[b].hi = pk2(h[0][b].im.hi, h[1][b].im.hi);
        Him[b].lo = pk2(h[0][b].im.lo, h[1][b].im.lo);
        Hre[b].nhi = mul2(Hre[b].hi, m1);
        Hre[b].nlo = mul2(Hre[b].lo, m1);
        Him[b].nhi = mul2(Him[b].hi, m1);
        Him[b].nlo = mul2(Him[b].lo, m1);
      }
    }
    // W[a] = sum_b U[a][b] H[b]: w.re = u.re h.re - u.im h.im, w.im = u.re h.im + u.im h.re
    // in the order of cmac, the first term of each chain started without a sum
    dfn2 Wre[D], Wim[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const float4 v = st[(a * D + b) * kDfThreads];
        const f32x2 rh = pk2(v.x, v.x), rl = pk2(v.y, v.y), ih = pk2(v.z, v.z), il = pk2(v.w, v.w);
        dfv2 nHim;  // -h.im and its negation: -u.im h.im = u.im (-h.im)
        nHim.hi = Him[b].nhi;
        nHim.lo = Him[b].nlo;
        nHim.nhi = Him[b].hi;
        nHim.nlo = Him[b].lo;
        if (b == 0) {
          Wre[a] = prod2(rh, rl, Hre[b]);
          Wim[a] = prod2(rh, rl, Him[b]);
        } else {
          fmacc2(rh, rl, Hre[b], Wre[a]);
          fmacc2(rh, rl, Him[b], Wim[a]);
        }
        fmacc2(ih, il, nHim, Wre[a]);
        fmacc2(ih, il, Hre[b], Wim[a]);
      }
    }
    switch (mu) {
      case 0: reconstruct_pairs<0, D>(a01re, a01im, a23re, a23im, Wre, Wim, s.hi); break;
      case 1: reconstruct_pairs<1, D>(a01re, a01im, a23re, a23im, Wre, Wim, s.hi); break;
      case 2: reconstruct_pairs<2, D>(a01re, a01im, a23re, a23im, Wre, Wim, s.hi); break;
      default: reconstruct_pairs<3, D>(a01re, a01im, a23re, a23im, Wre, Wim, s.hi); break;
    }
    issue(k + 2);  // stage k & 1 has been read: refill it with sense k + 2
  }

  double nrm = 0.0;
  if (active) {
    cx<df> acc[4][D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float x0, x1, y0, y1;
      up2(a01re[a].hi, x0, x1), up2(a01re[a].lo, y0, y1);
      acc[0][a].re = df(x0, y0), acc[1][a].re = df(x1, y1);
      up2(a01im[a].hi, x0, x1), up2(a01im[a].lo, y0, y1);
      acc[0][a].im = df(x0, y0), acc[1][a].im = df(x1, y1);
      up2(a23re[a].hi, x0, x1), up2(a23re[a].lo, y0, y1);
      acc[2][a].re = df(x0, y0), acc[3][a].re = df(x1, y1);
      up2(a23im[a].hi, x0, x1), up2(a23im[a].lo, y0, y1);
      acc[2][a].im = df(x0, y0), acc[3][a].im = df(x1, y1);
    }
    // epilogue as in hop_kernel: out = a x + b H in, or b H in
    const df bb = epi_b<df>(A);
    if (A.x != nullptr) {
      const df aa = epi_a<df>(A);
      cx<df> xs[4][D];
      SpinorIO<DF64, D>::load(A.x, Vh, i, xs);
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < D; ++c)
          acc[sp][c] = cmake(fma(aa, xs[sp][c].re, bb * acc[sp][c].re), fma(aa, xs[sp][c].im, bb * acc[sp][c].im));
    } else if (!A.b_one) {
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < D; ++c) acc[sp][c] = cmake(bb * acc[sp][c].re, bb * acc[sp][c].im);
    }
    SpinorIO<DF64, D>::store(A.out, Vh, i, acc);
    if constexpr (PARTIALS) {
      df n = df(0.f, 0.f);
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < D; ++c) n = fma(acc[sp][c].re, acc[sp][c].re, fma(acc[sp][c].im, acc[sp][c].im, n));
      nrm = (double)n;
    }
  }
  if constexpr (PARTIALS) block_sum_store<kDfThreads>(nrm, A.partials);
}

template <int D>
int launch_staged(const HopArgs& A, cudaStream_t s) {
  static_assert(DfStage<D>::bytes <= 48 * 1024, "stage fits the default dynamic shared memory limit");
  const int blocks = (A.g.Vh + kDfThreads - 1) / kDfThreads;
  if (A.partials != nullptr)
    hop_df64_staged_kernel<D, true><<<blocks, kDfThreads, DfStage<D>::bytes, s>>>(with_f32_scalars(A));
  else
    hop_df64_staged_kernel<D, false><<<blocks, kDfThreads, DfStage<D>::bytes, s>>>(with_f32_scalars(A));
  return blocks;
}

}  // namespace

int hop_partials_df64(int Vh) { return (Vh + kDfThreads - 1) / kDfThreads; }

int launch_hop_df64(int d, bool real, const HopArgs& A, cudaStream_t s) {
  if (real) {
    switch (d) {
      case 3: return launch_hop_t<DF64, 3, true>(A, s);
      case 8: return launch_hop_t<DF64, 8, true>(A, s);
      default: return -1;
    }
  }
  switch (d) {
    case 2: return launch_staged<2>(A, s);
    case 3: return launch_staged<3>(A, s);
    case 4: return launch_hop_t<DF64, 4, false>(A, s);
    case 6: return launch_hop_t<DF64, 6, false>(A, s);
    case 8: return launch_hop_t<DF64, 8, false>(A, s);
    default: return -1;
  }
}

}  // namespace bsm
