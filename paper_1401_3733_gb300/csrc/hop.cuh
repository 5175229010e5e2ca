// hop.cuh -- the Wilson hopping block H_{p,1-p} (Sec. II-B "Dphi"), one
// thread per output site of parity p.
//
// For each direction mu the two neighbour spinors are spin-projected to two
// colour vectors (chiral basis, g_mu = [[0, B_mu], [B_mu^+, 0]] with B_0 = 1,
// B_k = -i sigma_k):
//     (1 + sg g_mu) psi = ( h , sg B_mu^+ h ),   h = u + sg B_mu l,
// where u, l are the upper and lower spin pairs and sg = -1 for the forward
// term (1 - g_mu) U(x) psi(x+mu), sg = +1 for the backward term
// (1 + g_mu) U(x-mu)^+ psi(x-mu); the adjoint H^+ = g5 H g5 flips sg.  The
// link then multiplies the two colour vectors, one row at a time, and the
// row is reconstructed into the four spin components of the accumulator.
// The forward and backward links of mu share one 16-byte load (FP32) or sit
// in neighbouring planes (FP64) of the site's link tile, so a warp reads its
// links from one contiguous region; links are read with the streaming cache hint
// because each is used once per hop, neighbour spinors through the read-only
// path because each is used by 8 output sites.
#pragma once

#include "bsm_internal.cuh"

namespace bsm {

// h = u + sg * B_mu l
template <int MU, typename R, int D>
__device__ __forceinline__ void spin_project(const cx<R> (&s)[4][D], R sg, cx<R> (&h)[2][D]) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const cx<R> u0 = s[0][a], u1 = s[1][a], l0 = s[2][a], l1 = s[3][a];
    cx<R> b0, b1;  // B_mu l
    if (MU == 0) {
      b0 = l0;
      b1 = l1;
    } else if (MU == 1) {  // (-i l1, -i l0)
      b0 = cmake(l1.im, -l1.re);
      b1 = cmake(l0.im, -l0.re);
    } else if (MU == 2) {  // (-l1, l0)
      b0 = cmake(-l1.re, -l1.im);
      b1 = l0;
    } else {               // (-i l0, i l1)
      b0 = cmake(l0.im, -l0.re);
      b1 = cmake(-l1.im, l1.re);
    }
    h[0][a] = cmake(fma(sg, b0.re, u0.re), fma(sg, b0.im, u0.im));
    h[1][a] = cmake(fma(sg, b1.re, u1.re), fma(sg, b1.im, u1.im));
  }
}

// acc[0,1][a] += w ; acc[2,3][a] += sg * B_mu^+ w
template <int MU, typename R, int D>
__device__ __forceinline__ void spin_reconstruct(cx<R> (&acc)[4][D], int a, const cx<R>& w0,
                                                 const cx<R>& w1, R sg) {
  acc[0][a].re += w0.re;
  acc[0][a].im += w0.im;
  acc[1][a].re += w1.re;
  acc[1][a].im += w1.im;
  cx<R> c0, c1;  // B_mu^+ w
  if (MU == 0) {
    c0 = w0;
    c1 = w1;
  } else if (MU == 1) {  // (i w1, i w0)
    c0 = cmake(-w1.im, w1.re);
    c1 = cmake(-w0.im, w0.re);
  } else if (MU == 2) {  // (w1, -w0)
    c0 = w1;
    c1 = cmake(-w0.re, -w0.im);
  } else {               // (i w0, -i w1)
    c0 = cmake(-w0.im, w0.re);
    c1 = cmake(w1.im, -w1.re);
  }
  acc[2][a].re = fma(sg, c0.re, acc[2][a].re);
  acc[2][a].im = fma(sg, c0.im, acc[2][a].im);
  acc[3][a].re = fma(sg, c1.re, acc[3][a].re);
  acc[3][a].im = fma(sg, c1.im, acc[3][a].im);
}

// Double-float specialisations: the projector and reconstruction signs are
// exactly +-1, so they are folded into the operands (a sign flip) instead of
// costing a double-float multiply-add.
__device__ __forceinline__ df signed_df(float s, df x) { return df(s * x.hi, s * x.lo); }

template <int MU, int D>
__device__ __forceinline__ void spin_project(const cx<df> (&s)[4][D], df sgd, cx<df> (&h)[2][D]) {
  const float sg = sgd.hi;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const cx<df> u0 = s[0][a], u1 = s[1][a], l0 = s[2][a], l1 = s[3][a];
    cx<df> b0, b1;
    if (MU == 0) {
      b0 = l0;
      b1 = l1;
    } else if (MU == 1) {
      b0 = cmake(l1.im, -l1.re);
      b1 = cmake(l0.im, -l0.re);
    } else if (MU == 2) {
      b0 = cmake(-l1.re, -l1.im);
      b1 = l0;
    } else {
      b0 = cmake(l0.im, -l0.re);
      b1 = cmake(-l1.im, l1.re);
    }
    h[0][a] = cmake(u0.re + signed_df(sg, b0.re), u0.im + signed_df(sg, b0.im));
    h[1][a] = cmake(u1.re + signed_df(sg, b1.re), u1.im + signed_df(sg, b1.im));
  }
}

template <int MU, int D>
__device__ __forceinline__ void spin_reconstruct(cx<df> (&acc)[4][D], int a, const cx<df>& w0, const cx<df>& w1,
                                                 df sgd) {
  const float sg = sgd.hi;
  acc[0][a].re += w0.re;
  acc[0][a].im += w0.im;
  acc[1][a].re += w1.re;
  acc[1][a].im += w1.im;
  cx<df> c0, c1;
  if (MU == 0) {
    c0 = w0;
    c1 = w1;
  } else if (MU == 1) {
    c0 = cmake(-w1.im, w1.re);
    c1 = cmake(-w0.im, w0.re);
  } else if (MU == 2) {
    c0 = w1;
    c1 = cmake(-w0.re, -w0.im);
  } else {
    c0 = cmake(-w0.im, w0.re);
    c1 = cmake(w1.im, -w1.re);
  }
  acc[2][a].re += signed_df(sg, c0.re);
  acc[2][a].im += signed_df(sg, c0.im);
  acc[3][a].re += signed_df(sg, c1.re);
  acc[3][a].im += signed_df(sg, c1.im);
}

template <typename R>
__device__ __forceinline__ void link_mac(cx<R>& w, const cx<R>& u, const cx<R>& h) { cmac(w, u, h); }
template <typename R>
__device__ __forceinline__ void link_mac(cx<R>& w, R u, const cx<R>& h) { rmac(w, u, h); }

// One sense (FB = 0 forward, 1 backward) of direction mu: used where the two
// senses are processed one after the other to halve the live registers
// (double-float, whose dependent chains need occupancy more than load
// batching).
template <int MU, int FB, typename P, int D, bool REAL>
__device__ __forceinline__ void hop_sense(const HopArgs& A, size_t Vh, const typename LinkIO<P, D, REAL>::vec* lt,
                                          int n, typename P::R sg, cx<typename P::R> (&acc)[4][D]) {
  using R = typename P::R;
  using L = LinkIO<P, D, REAL>;
  cx<R> h[2][D];
  {
    cx<R> psi[4][D];
    SpinorIO<P, D>::load(A.in, Vh, n, psi);
    spin_project<MU>(psi, sg, h);
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<R> w0 = cmake(R(0), R(0)), w1 = w0;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const typename L::elem u = L::template load_one<FB>(lt, MU, a * D + b);
      link_mac(w0, u, h[0][b]);
      link_mac(w1, u, h[1][b]);
    }
    spin_reconstruct<MU>(acc, a, w0, w1, sg);
  }
}

// The same with (mu, sense) chosen at run time, for a loop over the 8
// direction-senses that is not unrolled: the link matrix-vector code then
// appears once in the kernel instead of eight times (double-float: fully
// unrolled, the kernel outgrows the instruction cache and warps stall on
// instruction fetch).  Only the cheap spin projection and reconstruction
// are specialised per direction.
template <typename P, int D, bool REAL>
__device__ __forceinline__ void hop_sense_rt(const HopArgs& A, size_t Vh,
                                             const typename LinkIO<P, D, REAL>::vec* lt, int mu, int fb, int n,
                                             typename P::R sg, cx<typename P::R> (&acc)[4][D]) {
  using R = typename P::R;
  using L = LinkIO<P, D, REAL>;
  cx<R> h[2][D];
  {
    cx<R> psi[4][D];
    SpinorIO<P, D>::load(A.in, Vh, n, psi);
    switch (mu) {
      case 0: spin_project<0>(psi, sg, h); break;
      case 1: spin_project<1>(psi, sg, h); break;
      case 2: spin_project<2>(psi, sg, h); break;
      default: spin_project<3>(psi, sg, h); break;
    }
  }
  // complex links: sense fb of direction mu sits fb planes-of-D^2 after the
  // forward planes; real links: both senses share each plane (select the half)
  const auto* lf = REAL ? lt : lt + (size_t)fb * D * D * kLinkTile;
  cx<R> w0[D], w1[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    w0[a] = cmake(R(0), R(0));
    w1[a] = w0[a];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const typename L::elem u = (REAL && fb) ? L::template load_one<1>(lf, mu, a * D + b)
                                              : L::template load_one<0>(lf, mu, a * D + b);
      link_mac(w0[a], u, h[0][b]);
      link_mac(w1[a], u, h[1][b]);
    }
  }
  switch (mu) {
    case 0:
#pragma unroll
      for (int a = 0; a < D; ++a) spin_reconstruct<0>(acc, a, w0[a], w1[a], sg);
      break;
    case 1:
#pragma unroll
      for (int a = 0; a < D; ++a) spin_reconstruct<1>(acc, a, w0[a], w1[a], sg);
      break;
    case 2:
#pragma unroll
      for (int a = 0; a < D; ++a) spin_reconstruct<2>(acc, a, w0[a], w1[a], sg);
      break;
    default:
#pragma unroll
      for (int a = 0; a < D; ++a) spin_reconstruct<3>(acc, a, w0[a], w1[a], sg);
      break;
  }
}

template <typename P>
struct HopSplitSenses {
  static constexpr bool value = P::prec == BSM_DF64;
};

// Two-row SU(3) links (F32R12): each sense's full matrix is rebuilt in
// registers (third row from the first two, times the boundary factor when
// the hop crosses the lattice edge), then applied as in the FP32 kernel.
template <int MU, int D>
__device__ __forceinline__ void hop_direction_r12(const HopArgs& A, size_t Vh, const float4* lt, int nf, int nb,
                                                  float sgf, float sgb, cx<float> (&acc)[4][D], unsigned edges) {
  using L = LinkIO<F32R12, D, false>;
  cx<float> hf[2][D], hb[2][D];
  {
    cx<float> psi[4][D];
    SpinorIO<F32R12, D>::load(A.in, Vh, nf, psi);
    spin_project<MU>(psi, sgf, hf);
    SpinorIO<F32R12, D>::load(A.in, Vh, nb, psi);
    spin_project<MU>(psi, sgb, hb);
  }
  const cx<float> one = cmake(1.f, 0.f);
  const cx<float> phf = ((edges >> MU) & 1u) ? cmake(A.ph3[MU][0], A.ph3[MU][1]) : one;
  const cx<float> phb = ((edges >> (4 + MU)) & 1u) ? cmake(A.ph3[MU][0], -A.ph3[MU][1]) : one;
  cx<float> U[3][3];
  L::template load_matrix<0>(lt, MU, phf, U);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<float> w0 = cmake(0.f, 0.f), w1 = w0;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      cmac(w0, U[a][b], hf[0][b]);
      cmac(w1, U[a][b], hf[1][b]);
    }
    spin_reconstruct<MU>(acc, a, w0, w1, sgf);
  }
  L::template load_matrix<1>(lt, MU, phb, U);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<float> w0 = cmake(0.f, 0.f), w1 = w0;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      cmac(w0, U[a][b], hb[0][b]);
      cmac(w1, U[a][b], hb[1][b]);
    }
    spin_reconstruct<MU>(acc, a, w0, w1, sgb);
  }
}

template <int MU, typename P, int D, bool REAL>
__device__ __forceinline__ void hop_direction(const HopArgs& A, size_t Vh, const typename LinkIO<P, D, REAL>::vec* lt,
                                              int nf, int nb, typename P::R sgf, typename P::R sgb,
                                              cx<typename P::R> (&acc)[4][D], unsigned edges) {
  using R = typename P::R;
  using L = LinkIO<P, D, REAL>;
  if constexpr (P::prec == BSM_F32R12) {
    hop_direction_r12<MU, D>(A, Vh, lt, nf, nb, sgf, sgb, acc, edges);
  } else if constexpr (HopSplitSenses<P>::value) {
    hop_sense<MU, 0, P, D, REAL>(A, Vh, lt, nf, sgf, acc);
    hop_sense<MU, 1, P, D, REAL>(A, Vh, lt, nb, sgb, acc);
  } else {
    cx<R> hf[2][D], hb[2][D];
    {
      cx<R> psi[4][D];
      SpinorIO<P, D>::load(A.in, Vh, nf, psi);
      spin_project<MU>(psi, sgf, hf);
      SpinorIO<P, D>::load(A.in, Vh, nb, psi);
      spin_project<MU>(psi, sgb, hb);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      cx<R> wf0 = cmake(R(0), R(0)), wf1 = wf0, wb0 = wf0, wb1 = wf0;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        typename L::elem uf, ub;
        L::load(lt, MU, a * D + b, uf, ub);
        link_mac(wf0, uf, hf[0][b]);
        link_mac(wf1, uf, hf[1][b]);
        link_mac(wb0, ub, hb[0][b]);
        link_mac(wb1, ub, hb[1][b]);
      }
      spin_reconstruct<MU>(acc, a, wf0, wf1, sgf);
      spin_reconstruct<MU>(acc, a, wb0, wb1, sgb);
    }
  }
}

// Minimum resident blocks per SM (register budget) of each instantiation: the
// FP32 kernels are bound by memory latency and want about 128 registers so
// that each thread keeps a direction's loads in flight; the double-float
// kernels are bound by dependent FP32 chains and want occupancy; larger d
// need more registers.
template <typename P, int D>
struct HopOccupancy {
  static constexpr int min_blocks = P::prec == BSM_F64 ? (D <= 2 ? 4 : D == 3 ? 2 : 1)
                                                       : (D <= 3 ? 4 : D == 4 ? 3 : D == 6 ? 2 : 1);
};

// EPI = 1 (FP32 vectors only): the output is the CG product Ap of this
// site; instead of storing it the epilogue completes the CG step,
// r -= alpha Ap and x += alpha p, and the partials are those of |r|^2
template <typename P, int D, bool REAL, int EPI = 0>
__global__ void __launch_bounds__(kHopThreads, HopOccupancy<P, D>::min_blocks) hop_kernel(const HopArgs A) {
  using R = typename P::R;
  if (A.done != nullptr && *A.done != 0) return;  // uniform over the grid
  const int i = blockIdx.x * kHopThreads + threadIdx.x;
  double nrm = 0.0;
  if (i < A.g.Vh) {
    const size_t Vh = (size_t)A.g.Vh;
    int nf[4], nb[4];
    eo_neighbours(A.g, i, A.p, nf, nb);
    const auto* lt = LinkIO<P, D, REAL>::tile_ptr(A.links, i);
    const R sg = A.dagger ? R(1) : R(-1);  // forward sign; backward is -sg
    const unsigned edges = P::prec == BSM_F32R12 ? eo_edges(A.g, i, A.p) : 0u;
    cx<R> acc[4][D];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int a = 0; a < D; ++a) acc[s][a] = cmake(R(0), R(0));
    if constexpr (HopSplitSenses<P>::value) {
#pragma unroll 1
      for (int k = 0; k < 8; ++k) {
        const int mu = k >> 1, fb = k & 1;
        hop_sense_rt<P, D, REAL>(A, Vh, lt, mu, fb, fb ? nb[mu] : nf[mu], fb ? -sg : sg, acc);
      }
    } else {
      hop_direction<0, P, D, REAL>(A, Vh, lt, nf[0], nb[0], sg, -sg, acc, edges);
      hop_direction<1, P, D, REAL>(A, Vh, lt, nf[1], nb[1], sg, -sg, acc, edges);
      hop_direction<2, P, D, REAL>(A, Vh, lt, nf[2], nb[2], sg, -sg, acc, edges);
      hop_direction<3, P, D, REAL>(A, Vh, lt, nf[3], nb[3], sg, -sg, acc, edges);
    }

    const R b = epi_b<R>(A);
    if (A.x != nullptr) {
      const R a = epi_a<R>(A);
      cx<R> xs[4][D];
      SpinorIO<P, D>::load(A.x, Vh, i, xs);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c)
          acc[s][c] = cmake(fma(a, xs[s][c].re, b * acc[s][c].re), fma(a, xs[s][c].im, b * acc[s][c].im));
    } else if (!A.b_one) {
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c) acc[s][c] = cmake(b * acc[s][c].re, b * acc[s][c].im);
    }
    if constexpr (EPI == 1) {
      // rows written only by this thread: read through L2 (not the read-only path)
      const R al = *A.cg_alpha;
      cx<R> v[4][D], w[4][D];
      SpinorIO<P, D>::template load<true>(A.cg_r, Vh, i, v);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          acc[s][c] = cmake(fma(-al, acc[s][c].re, v[s][c].re), fma(-al, acc[s][c].im, v[s][c].im));  // r
        }
      SpinorIO<P, D>::store(A.cg_r, Vh, i, acc);
      SpinorIO<P, D>::template load<true>(A.cg_x, Vh, i, v);
      SpinorIO<P, D>::template load<true>(A.cg_p, Vh, i, w);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c)
          v[s][c] = cmake(fma(al, w[s][c].re, v[s][c].re), fma(al, w[s][c].im, v[s][c].im));
      SpinorIO<P, D>::store(A.cg_x, Vh, i, v);
    } else {
      SpinorIO<P, D>::store(A.out, Vh, i, acc);
    }
    if (A.partials != nullptr) {
      if constexpr (sizeof(R) == sizeof(float)) {
        // FP32 kernels: the 2d squares of one spin summed in FP32, the four
        // spin sums converted and added in FP64 (the thread's partial is
        // FP64; an FP64 operation per square would cost 24 FP64-pipe
        // instructions per site on this part)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          float n = 0.f;
#pragma unroll
          for (int c = 0; c < D; ++c) n = fmaf(acc[s][c].re, acc[s][c].re, fmaf(acc[s][c].im, acc[s][c].im, n));
          nrm += (double)n;
        }
      } else {
        R n = R(0);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < D; ++c) n = fma(acc[s][c].re, acc[s][c].re, fma(acc[s][c].im, acc[s][c].im, n));
        nrm = (double)n;
      }
    }
  }
  if (A.partials != nullptr) block_sum_store<kHopThreads>(nrm, A.partials);
}

template <typename P, int D, bool REAL>
inline int launch_hop_t(const HopArgs& A, cudaStream_t s) {
  const int blocks = hop_blocks(A.g.Vh);
  if constexpr (P::prec == BSM_F32 || P::prec == BSM_F32R12) {
    if (A.cg_r != nullptr) {
      hop_kernel<P, D, REAL, 1><<<blocks, kHopThreads, 0, s>>>(with_f32_scalars(A));
      return blocks;
    }
  }
  hop_kernel<P, D, REAL><<<blocks, kHopThreads, 0, s>>>(with_f32_scalars(A));
  return blocks;
}

}  // namespace bsm
