// mrhs.cuh -- the hopping block for many right-hand sides at once (the N_f
// fermion flavours of Sec. II-A share one gauge field): every link is read
// from memory once per site and applied to all RHS, which raises the
// arithmetic intensity from ~1 to ~n_rhs/2 flop per byte.
//
// Multi-RHS spinor layout (site-major): the 2d planes of the single-RHS
// FP32/BF16 layout with the RHS index innermost, element (plane, site, rhs)
// at (site*2d + plane)*n_rhs + rhs, so that a site's spinors of all RHS are
// one contiguous block of 2d*n_rhs elements, which SpinorIO addresses as a
// field of n_rhs "sites" (mrhs_block).  One thread owns one output site and
// a block of RB consecutive RHS; the RB spinors live in registers and each
// link element, loaded once through L1 (the other RHS blocks of the same site
// reuse it from there), multiplies all of them.
#pragma once

#include <type_traits>

#include "f32x2.cuh"
#include "hop.cuh"

namespace bsm {

struct MrhsArgs {
  const void* links;  // link block of output parity p
  const void* in;     // multi-RHS half spinor of parity 1-p
  void* out;          // multi-RHS half spinor of parity p
  const void* x;      // optional same-parity input: out = a*x + b*H in
  double a, b;
  Geom g;
  int p;
  int dagger;
  int nrhs;
  float af, bf;       // a, b in FP32 and b == 1 (with_f32_scalars at launch)
  int b_one;
};

template <>
__device__ __forceinline__ float epi_a<float, MrhsArgs>(const MrhsArgs& A) { return A.af; }
template <>
__device__ __forceinline__ float epi_b<float, MrhsArgs>(const MrhsArgs& A) { return A.bf; }

// site n's block of a multi-RHS FP32 (float4 elements) or BF16 (uint2)
// half spinor: 2d planes of n_rhs elements
template <typename P, int D>
__device__ __forceinline__ const void* mrhs_block(const void* base, int n, size_t nr) {
  constexpr size_t elem = std::is_same<P, BF16>::value ? sizeof(uint2) : sizeof(float4);
  return static_cast<const char*>(base) + (size_t)(unsigned)n * (2 * D) * nr * elem;
}
template <typename P, int D>
__device__ __forceinline__ void* mrhs_block(void* base, int n, size_t nr) {
  return const_cast<void*>(mrhs_block<P, D>(static_cast<const void*>(base), n, nr));
}

template <int MU, int FB, typename P, int D, bool REAL, int RB, bool L2IN = false>
__device__ __forceinline__ void mrhs_sense(const MrhsArgs& A, const typename LinkIO<P, D, REAL>::vec* lt, int n,
                                           int r0, typename P::R sg, cx<typename P::R> (&acc)[RB][4][D]) {
  using R = typename P::R;
  using L = LinkIO<P, D, REAL>;
  const size_t nr = (size_t)A.nrhs;
  const void* blk = mrhs_block<P, D>(A.in, n, nr);
  cx<R> h[RB][2][D];
#pragma unroll
  for (int j = 0; j < RB; ++j) {
    cx<R> psi[4][D];
    if constexpr (L2IN) SpinorIO<P, D>::template load<true>(blk, nr, r0 + j, psi);
    else SpinorIO<P, D>::load(blk, nr, r0 + j, psi);
    spin_project<MU>(psi, sg, h[j]);
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<R> w[RB][2];
#pragma unroll
    for (int j = 0; j < RB; ++j) w[j][0] = w[j][1] = cmake(R(0), R(0));
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const typename L::elem u = L::template load_one<FB, true>(lt, MU, a * D + b);
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        link_mac(w[j][0], u, h[j][0][b]);
        link_mac(w[j][1], u, h[j][1][b]);
      }
    }
#pragma unroll
    for (int j = 0; j < RB; ++j) spin_reconstruct<MU>(acc[j], a, w[j][0], w[j][1], sg);
  }
}

template <int MU, typename P, int D, bool REAL, int RB, bool L2IN = false>
__device__ __forceinline__ void mrhs_direction(const MrhsArgs& A, const typename LinkIO<P, D, REAL>::vec* lt,
                                               int nf, int nb, int r0, typename P::R sg,
                                               cx<typename P::R> (&acc)[RB][4][D]) {
  mrhs_sense<MU, 0, P, D, REAL, RB, L2IN>(A, lt, nf, r0, sg, acc);
  mrhs_sense<MU, 1, P, D, REAL, RB, L2IN>(A, lt, nb, r0, -sg, acc);
}

// Minimum resident blocks (register budget) per RHS block: measured on the
// 24^4, 12-RHS workload, one RHS per thread wants about 168 registers (3
// blocks per SM) at d = 6 and 128 (4 blocks per SM) at d = 3, two RHS per
// thread at d = 6 about 255 (2 blocks per SM); tighter budgets spill or lose.
template <int D, int RB>
struct MrhsOccupancy {
  static constexpr int min_blocks = D <= 2 ? 1 : (RB == 1 && D == 3) ? 4 : RB == 1 ? 3 : (RB == 2 && D >= 6) ? 2 : 1;
};

// the output of site i, RHS r0 .. r0+RB-1 (one thread); L2IN reads the
// input spinor through L2 only (it was written earlier in the same kernel)
template <typename P, int D, bool REAL, int RB, bool L2IN = false>
__device__ __forceinline__ void mrhs_site(const MrhsArgs& A, int i, int r0) {
  using R = typename P::R;
  int nf[4], nb[4];
  eo_neighbours(A.g, i, A.p, nf, nb);
  const auto* lt = LinkIO<P, D, REAL>::tile_ptr(A.links, i);
  const R sg = A.dagger ? R(1) : R(-1);  // forward sign; backward is -sg
  cx<R> acc[RB][4][D];
#pragma unroll
  for (int j = 0; j < RB; ++j)
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int a = 0; a < D; ++a) acc[j][s][a] = cmake(R(0), R(0));
  mrhs_direction<0, P, D, REAL, RB, L2IN>(A, lt, nf[0], nb[0], r0, sg, acc);
  mrhs_direction<1, P, D, REAL, RB, L2IN>(A, lt, nf[1], nb[1], r0, sg, acc);
  mrhs_direction<2, P, D, REAL, RB, L2IN>(A, lt, nf[2], nb[2], r0, sg, acc);
  mrhs_direction<3, P, D, REAL, RB, L2IN>(A, lt, nf[3], nb[3], r0, sg, acc);

  const size_t nr = (size_t)A.nrhs;
  const R b = epi_b<R>(A);
#pragma unroll
  for (int j = 0; j < RB; ++j) {
    const int e = r0 + j;
    if (A.x != nullptr) {
      const R a = epi_a<R>(A);
      cx<R> xs[4][D];
      SpinorIO<P, D>::load(mrhs_block<P, D>(A.x, i, nr), nr, e, xs);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c)
          acc[j][s][c] = cmake(fma(a, xs[s][c].re, b * acc[j][s][c].re), fma(a, xs[s][c].im, b * acc[j][s][c].im));
    } else if (!A.b_one) {
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c) acc[j][s][c] = cmake(b * acc[j][s][c].re, b * acc[j][s][c].im);
    }
    SpinorIO<P, D>::store(mrhs_block<P, D>(A.out, i, nr), nr, e, acc[j]);
  }
}

template <typename P, int D, bool REAL, int RB>
__global__ void __launch_bounds__(kHopThreads, MrhsOccupancy<D, RB>::min_blocks) hop_mrhs_kernel(const MrhsArgs A) {
  const int nblk = A.nrhs / RB;
  const long long t = blockIdx.x * (long long)kHopThreads + threadIdx.x;
  if (t >= (long long)A.g.Vh * nblk) return;
  const int i = (int)(t / nblk);
  mrhs_site<P, D, REAL, RB>(A, i, (int)(t - (long long)i * nblk) * RB);
}

// ---------------------------------------------------------------------------
// Paired RHS: two right-hand sides in the two lanes of packed FP32 pairs
// (f32x2.cuh).  The link element is broadcast to both lanes and every
// multiply-add and sum of the link products and the spin reconstruction
// serves two RHS with one instruction: the same lane operations as the scalar
// kernel in the same order (bit-identical results), about two thirds of its
// issue slots.  The spin projection stays scalar per RHS.
// ---------------------------------------------------------------------------
struct cxp {
  f32x2 re, im;
};

template <int MU, int NP, int D>
__device__ __forceinline__ void reconstruct_paired(cxp (&acc)[NP][4][D], int a, const cxp (&W)[NP][2], float sg) {
  const f32x2 ps = pk2(sg, sg), ns = pk2(-sg, -sg);
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const cxp w0 = W[j][0], w1 = W[j][1];
    acc[j][0][a].re = add2(acc[j][0][a].re, w0.re);
    acc[j][0][a].im = add2(acc[j][0][a].im, w0.im);
    acc[j][1][a].re = add2(acc[j][1][a].re, w1.re);
    acc[j][1][a].im = add2(acc[j][1][a].im, w1.im);
    // acc2 += sg c0, acc3 += sg c1 with (c0, c1) = B_mu^+ (w0, w1)
    if (MU == 0) {         // (w0, w1)
      acc[j][2][a].re = fma2(ps, w0.re, acc[j][2][a].re);
      acc[j][2][a].im = fma2(ps, w0.im, acc[j][2][a].im);
      acc[j][3][a].re = fma2(ps, w1.re, acc[j][3][a].re);
      acc[j][3][a].im = fma2(ps, w1.im, acc[j][3][a].im);
    } else if (MU == 1) {  // (i w1, i w0): c0 = (-w1.im, w1.re), c1 = (-w0.im, w0.re)
      acc[j][2][a].re = fma2(ns, w1.im, acc[j][2][a].re);
      acc[j][2][a].im = fma2(ps, w1.re, acc[j][2][a].im);
      acc[j][3][a].re = fma2(ns, w0.im, acc[j][3][a].re);
      acc[j][3][a].im = fma2(ps, w0.re, acc[j][3][a].im);
    } else if (MU == 2) {  // (w1, -w0)
      acc[j][2][a].re = fma2(ps, w1.re, acc[j][2][a].re);
      acc[j][2][a].im = fma2(ps, w1.im, acc[j][2][a].im);
      acc[j][3][a].re = fma2(ns, w0.re, acc[j][3][a].re);
      acc[j][3][a].im = fma2(ns, w0.im, acc[j][3][a].im);
    } else {               // (i w0, -i w1): c0 = (-w0.im, w0.re), c1 = (w1.im, -w1.re)
      acc[j][2][a].re = fma2(ns, w0.im, acc[j][2][a].re);
      acc[j][2][a].im = fma2(ps, w0.re, acc[j][2][a].im);
      acc[j][3][a].re = fma2(ps, w1.im, acc[j][3][a].re);
      acc[j][3][a].im = fma2(ns, w1.re, acc[j][3][a].im);
    }
  }
}

template <int MU, int FB, typename P, int D, bool REAL, int NP, bool L2IN>
__device__ __forceinline__ void mrhs_sense_paired(const MrhsArgs& A, const typename LinkIO<P, D, REAL>::vec* lt, int n,
                                                  int r0, float sg, cxp (&acc)[NP][4][D]) {
  using L = LinkIO<P, D, REAL>;
  const size_t nr = (size_t)A.nrhs;
  const void* blk = mrhs_block<P, D>(A.in, n, nr);
  cxp H[NP][2][D];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    cx<float> h[2][2][D];  // [lane][half][colour]
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      cx<float> psi[4][D];
      const int e = r0 + 2 * j + l;
      if constexpr (L2IN) SpinorIO<P, D>::template load<true>(blk, nr, e, psi);
      else SpinorIO<P, D>::load(blk, nr, e, psi);
      spin_project<MU>(psi, sg, h[l]);
    }
#pragma unroll
    for (int hf = 0; hf < 2; ++hf)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        H[j][hf][b].re = pk2(h[0][hf][b].re, h[1][hf][b].re);
        H[j][hf][b].im = pk2(h[0][hf][b].im, h[1][hf][b].im);
      }
  }
  const f32x2 z = pk2(0.f, 0.f);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cxp W[NP][2];
#pragma unroll
    for (int j = 0; j < NP; ++j) W[j][0].re = W[j][0].im = W[j][1].re = W[j][1].im = z;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const typename L::elem u = L::template load_one<FB, true>(lt, MU, a * D + b);
      if constexpr (REAL) {
        const f32x2 uu = pk2(u, u);
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            W[j][hf].re = fma2(uu, H[j][hf][b].re, W[j][hf].re);
            W[j][hf].im = fma2(uu, H[j][hf][b].im, W[j][hf].im);
          }
      } else {
        const f32x2 ur = pk2(u.re, u.re), ui = pk2(u.im, u.im), nui = pk2(-u.im, -u.im);
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            W[j][hf].re = fma2(ur, H[j][hf][b].re, W[j][hf].re);
            W[j][hf].re = fma2(nui, H[j][hf][b].im, W[j][hf].re);
            W[j][hf].im = fma2(ur, H[j][hf][b].im, W[j][hf].im);
            W[j][hf].im = fma2(ui, H[j][hf][b].re, W[j][hf].im);
          }
      }
    }
    reconstruct_paired<MU, NP, D>(acc, a, W, sg);
  }
}

// NP pairs (2 NP RHS from r0) of site i: the paired counterpart of mrhs_site
template <typename P, int D, bool REAL, int NP, bool L2IN = false>
__device__ __forceinline__ void mrhs_site_paired(const MrhsArgs& A, int i, int r0) {
  int nf[4], nb[4];
  eo_neighbours(A.g, i, A.p, nf, nb);
  const auto* lt = LinkIO<P, D, REAL>::tile_ptr(A.links, i);
  const float sg = A.dagger ? 1.f : -1.f;  // forward sign; backward is -sg
  cxp acc[NP][4][D];
  const f32x2 z = pk2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < NP; ++j)
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a) acc[j][sp][a].re = acc[j][sp][a].im = z;
  mrhs_sense_paired<0, 0, P, D, REAL, NP, L2IN>(A, lt, nf[0], r0, sg, acc);
  mrhs_sense_paired<0, 1, P, D, REAL, NP, L2IN>(A, lt, nb[0], r0, -sg, acc);
  mrhs_sense_paired<1, 0, P, D, REAL, NP, L2IN>(A, lt, nf[1], r0, sg, acc);
  mrhs_sense_paired<1, 1, P, D, REAL, NP, L2IN>(A, lt, nb[1], r0, -sg, acc);
  mrhs_sense_paired<2, 0, P, D, REAL, NP, L2IN>(A, lt, nf[2], r0, sg, acc);
  mrhs_sense_paired<2, 1, P, D, REAL, NP, L2IN>(A, lt, nb[2], r0, -sg, acc);
  mrhs_sense_paired<3, 0, P, D, REAL, NP, L2IN>(A, lt, nf[3], r0, sg, acc);
  mrhs_sense_paired<3, 1, P, D, REAL, NP, L2IN>(A, lt, nb[3], r0, -sg, acc);

  const size_t nr = (size_t)A.nrhs;
  const float b = epi_b<float>(A);
#pragma unroll
  for (int j = 0; j < NP; ++j)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      cx<float> o[4][D];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float r0v, r1v, i0v, i1v;
          up2(acc[j][sp][a].re, r0v, r1v);
          up2(acc[j][sp][a].im, i0v, i1v);
          o[sp][a] = l == 0 ? cmake(r0v, i0v) : cmake(r1v, i1v);
        }
      const int e = r0 + 2 * j + l;
      if (A.x != nullptr) {
        const float a = epi_a<float>(A);
        cx<float> xs[4][D];
        SpinorIO<P, D>::load(mrhs_block<P, D>(A.x, i, nr), nr, e, xs);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < D; ++c)
            o[sp][c] = cmake(fmaf(a, xs[sp][c].re, b * o[sp][c].re), fmaf(a, xs[sp][c].im, b * o[sp][c].im));
      } else if (!A.b_one) {
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int c = 0; c < D; ++c) o[sp][c] = cmake(b * o[sp][c].re, b * o[sp][c].im);
      }
      SpinorIO<P, D>::store(mrhs_block<P, D>(A.out, i, nr), nr, e, o);
    }
}

template <typename P, int D, bool REAL, int NP>
__global__ void __launch_bounds__(kHopThreads, MrhsOccupancy<D, 2 * NP>::min_blocks) hop_mrhs_paired_kernel(
    const MrhsArgs A) {
  const int nblk = A.nrhs / (2 * NP);
  const long long t = blockIdx.x * (long long)kHopThreads + threadIdx.x;
  if (t >= (long long)A.g.Vh * nblk) return;
  const int i = (int)(t / nblk);
  mrhs_site_paired<P, D, REAL, NP>(A, i, (int)(t - (long long)i * nblk) * 2 * NP);
}

// paired candidates of the tuner: 2 NP RHS per thread, code kPairedBlock + 2 NP
constexpr int kPairedBlock = 100;

template <typename P, int D, bool REAL, int NP>
inline void launch_mrhs_paired_t(const MrhsArgs& A, cudaStream_t s) {
  const long long n = (long long)A.g.Vh * (A.nrhs / (2 * NP));
  const int blocks = (int)((n + kHopThreads - 1) / kHopThreads);
  hop_mrhs_paired_kernel<P, D, REAL, NP><<<blocks, kHopThreads, 0, s>>>(with_f32_scalars(A));
}

// RHS blocks compiled for colour dimension D (register budget: the RB
// accumulators hold 8*D*RB reals)
template <int D>
struct MrhsBlocks {
  static constexpr int max_rb = D <= 3 ? 4 : 2;
};

template <typename P, int D, bool REAL, int RB>
inline void launch_mrhs_t(const MrhsArgs& A, cudaStream_t s) {
  const long long n = (long long)A.g.Vh * (A.nrhs / RB);
  const int blocks = (int)((n + kHopThreads - 1) / kHopThreads);
  hop_mrhs_kernel<P, D, REAL, RB><<<blocks, kHopThreads, 0, s>>>(with_f32_scalars(A));
}

// dispatch on RB for one (P, D, REAL); false if RB is not compiled for D
template <typename P, int D, bool REAL>
inline bool launch_mrhs_rb(int rb, const MrhsArgs& A, cudaStream_t s) {
  switch (rb) {
    case kPairedBlock + 2: launch_mrhs_paired_t<P, D, REAL, 1>(A, s); return true;
    case kPairedBlock + 4:
      if constexpr (MrhsBlocks<D>::max_rb >= 4) { launch_mrhs_paired_t<P, D, REAL, 2>(A, s); return true; }
      return false;
    case 1: launch_mrhs_t<P, D, REAL, 1>(A, s); return true;
    case 2: launch_mrhs_t<P, D, REAL, 2>(A, s); return true;
    case 3:
      if constexpr (MrhsBlocks<D>::max_rb >= 3) { launch_mrhs_t<P, D, REAL, 3>(A, s); return true; }
      return false;
    case 4:
      if constexpr (MrhsBlocks<D>::max_rb >= 4) { launch_mrhs_t<P, D, REAL, 4>(A, s); return true; }
      return false;
    default: return false;
  }
}

}  // namespace bsm
