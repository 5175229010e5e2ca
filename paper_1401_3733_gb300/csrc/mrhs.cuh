// mrhs.cuh -- the hopping block for many right-hand sides at once (the N_f
// fermion flavours of Sec. II-A share one gauge field): every link is read
// from memory once per site and applied to all RHS, which raises the
// arithmetic intensity from ~1 to ~n_rhs/2 flop per byte.
//
// Multi-RHS spinor layout: the single-RHS layout with the RHS index
// innermost, element (plane, site, rhs) at (plane*V_h + site)*n_rhs + rhs, so
// SpinorIO addresses it as a field of V_h*n_rhs "sites".  One thread owns one
// output site and a block of RB consecutive RHS; the RB spinors live in
// registers and each link element, loaded once through L1 (the other RHS
// blocks of the same site reuse it from there), multiplies all of them.
#pragma once

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

template <int MU, int FB, typename P, int D, bool REAL, int RB, bool L2IN = false>
__device__ __forceinline__ void mrhs_sense(const MrhsArgs& A, const typename LinkIO<P, D, REAL>::vec* lt, int n,
                                           int r0, typename P::R sg, cx<typename P::R> (&acc)[RB][4][D]) {
  using R = typename P::R;
  using L = LinkIO<P, D, REAL>;
  const size_t nr = (size_t)A.nrhs;
  const size_t Vn = (size_t)A.g.Vh * nr;
  cx<R> h[RB][2][D];
#pragma unroll
  for (int j = 0; j < RB; ++j) {
    cx<R> psi[4][D];
    if constexpr (L2IN) SpinorIO<P, D>::template load<true>(A.in, Vn, (int)((size_t)n * nr + r0 + j), psi);
    else SpinorIO<P, D>::load(A.in, Vn, (int)((size_t)n * nr + r0 + j), psi);
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
  const size_t Vn = (size_t)A.g.Vh * nr;
  const R b = epi_b<R>(A);
#pragma unroll
  for (int j = 0; j < RB; ++j) {
    const int e = (int)((size_t)i * nr + r0 + j);
    if (A.x != nullptr) {
      const R a = epi_a<R>(A);
      cx<R> xs[4][D];
      SpinorIO<P, D>::load(A.x, Vn, e, xs);
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
    SpinorIO<P, D>::store(A.out, Vn, e, acc[j]);
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
