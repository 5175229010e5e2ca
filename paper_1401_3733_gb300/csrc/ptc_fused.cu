// ptc_fused.cu -- BF16 inference of the parallel-transport preconditioner
// with the two channel-mixing GEMMs fused into the transport kernel.
//
// A tile is 128 consecutive eo sites of one parity (128 d rows of the PTC
// field).  Stage 1: two threads per site compute the 9 transports of the
// one-channel input (T_0, and U_mu(x) F(x+mu), U_mu(x-mu)^+ F(x-mu) for two
// directions each) in FP32 and store them, rounded to BF16 and realified
// (re, im interleaved), as the A tile X1 (rows x 72, padded to 80) in shared
// memory.  Stage 2: each warp takes 16-row tiles through
//     Y1 = X1 W1  (72 -> 8C reals)   and   Z2 = Y1 W2p  (8C -> 72 reals)
// as mma.sync.m16n8k16 (BF16 x BF16 -> FP32).  The FP32 accumulator
// fragments of two adjacent 8-column tiles of Y1 are, element for element,
// the A fragment of one 16-deep k-step of the second GEMM, so Y1 is rounded
// to BF16 in registers and never stored.  Z2 (rows x 36 complex, BF16) is the
// only intermediate written to memory, slot-major (Z2[k][row][spin]) so that
// the stencil kernel, which forms out = sum_k T_k Z2_k, reads each
// neighbour's slot as whole, contiguous 16-byte groups.  The weights come
// realified and transposed ([n][k], k padded) so that B fragments are
// conflict-free 32-bit shared loads.
//
// The kernel is persistent (one 512-thread block per SM, weights staged in
// shared memory once) and warp-specialised: 8 producer warps run stage 1 for
// the next tile while 8 consumer warps run stage 2 on the previous one, with
// two X1 buffers handed over through hardware named barriers, so that the
// gathers from HBM overlap the tensor-core work.
#include <cuda_bf16.h>

#include "bsm_internal.cuh"

namespace bsm {

namespace {

constexpr int kFusedSites = 128;   // eo sites per block (two threads per site in the transport stage)
constexpr int kFusedThreads = 256;
constexpr int kXStride = 88;        // bf16 per X1 row in shared memory (72 used, 80 for the MMA k-steps)

template <int C>
struct FusedShape {
  static constexpr int N1 = 8 * C;           // Y1 reals per row
  static constexpr int W1Stride = kXStride;  // W1T row (one Y1 column): 80 k + 8 pad
  static constexpr int W2Stride = N1 + 8;    // W2T row (one Z2 column): 8C k + 8 pad
  static constexpr int W1Elems = N1 * W1Stride;
  static constexpr int W2Elems = 72 * W2Stride;
};

__device__ __forceinline__ unsigned pack_bf2(float lo, float hi) { return f2_to_bf2(lo, hi); }

__device__ __forceinline__ void mma16816(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// realified, transposed, padded weights (bf16): W1T[n][k] = W1r[k][n], W2T[n][k] = W2pr[k][n]
template <int C>
__global__ void fused_prep_kernel(const float2* __restrict__ W1, const float2* __restrict__ W2p,
                                  __nv_bfloat16* __restrict__ W1T, __nv_bfloat16* __restrict__ W2T) {
  using S = FusedShape<C>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // realified entry (k, n) of a complex K x N matrix M: [[Re, Im], [-Im, Re]] blocks
  auto real_of = [](const float2* M, int N, int k, int n) {
    const float2 w = M[(k >> 1) * N + (n >> 1)];
    if ((k & 1) == 0) return (n & 1) ? w.y : w.x;
    return (n & 1) ? w.x : -w.y;
  };
  if (t < S::W1Elems) {
    const int n = t / S::W1Stride, k = t % S::W1Stride;
    W1T[t] = __float2bfloat16_rn(k < 72 ? real_of(W1, 4 * C, k, n) : 0.f);
  } else if (t < S::W1Elems + S::W2Elems) {
    const int u = t - S::W1Elems;
    const int n = u / S::W2Stride, k = u % S::W2Stride;
    W2T[u] = __float2bfloat16_rn(k < S::N1 ? real_of(W2p, 36, k, n) : 0.f);
  }
}

// hardware named barriers (ids 1..4; 0 is __syncthreads) between the
// producer and the consumer warps.  bar.arrive signals without waiting,
// bar.sync waits until `count` threads have arrived or synced; both order
// the executing thread's earlier shared-memory accesses before the barrier.
__device__ __forceinline__ void named_sync(int id, int count) {
  __syncwarp();
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
  __syncwarp();
  asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}
constexpr int kBarFull = 1, kBarEmpty = 3;  // + buffer index

struct FusedTile {
  int p, i0;
  long long prow0, orow0;  // first site row of this (sample, parity) and of the other parity
};

__device__ __forceinline__ FusedTile fused_tile(const Geom& g, int t, int bpp) {
  FusedTile f;
  const int b = t / (2 * bpp);
  f.p = (t / bpp) % 2;
  f.i0 = (t % bpp) * kFusedSites;
  f.prow0 = ((long long)b * 2 + f.p) * g.Vh;
  f.orow0 = ((long long)b * 2 + 1 - f.p) * g.Vh;
  return f;
}

// stage 1 (producer thread tid in [0, 256)): the 9 transports of the
// one-channel input for site i0 + (tid mod 128), directions 2 half .. 2 half + 1,
// into the X1 tile (bf16, realified) in shared memory
template <int D, bool EO>
__device__ __forceinline__ void transport_tile(const char* __restrict__ links, size_t link_block,
                                               const float2* __restrict__ F, const Geom& g, const FusedTile& f,
                                               __nv_bfloat16* sX, int tid) {
  // EO (even-only input): the input vanishes on odd sites, so an even site
  // has only its own term (X1 slot 0) and an odd site only the transports of
  // its neighbours (slots 1..8); the even-only stencil then reads slot 0 of
  // Z2 on even rows and slots 1..8 on odd rows, so only those are computed.
  const bool self_only = EO && f.p == 0, no_self = EO && f.p == 1;
  const int sl = tid & (kFusedSites - 1), half = tid / kFusedSites;
  const int i = f.i0 + sl;
  unsigned* xr[D];
#pragma unroll
  for (int c = 0; c < D; ++c) xr[c] = reinterpret_cast<unsigned*>(sX + (sl * D + c) * kXStride);
  if (i < g.Vh && self_only) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (half == 0) {
        const float4* q = reinterpret_cast<const float4*>(F + ((f.prow0 + i) * D + c) * 4);
        const float4 v0 = __ldg(q), v1 = __ldg(q + 1);
        xr[c][0] = pack_bf2(v0.x, v0.y);
        xr[c][1] = pack_bf2(v0.z, v0.w);
        xr[c][2] = pack_bf2(v1.x, v1.y);
        xr[c][3] = pack_bf2(v1.z, v1.w);
      }
      for (int e = 4 + half; e < 36; e += 2) xr[c][e] = 0u;
    }
  } else if (i < g.Vh) {
    int nf[4], nb_[4];
    eo_neighbours(g, i, f.p, nf, nb_);
    using L = LinkIO<F32, D, false>;
    const auto* lt = L::tile_ptr(links + (size_t)f.p * link_block, i);
    if (half == 0 && no_self) {
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) xr[c][e] = 0u;
    } else if (half == 0) {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float4* q = reinterpret_cast<const float4*>(F + ((f.prow0 + i) * D + c) * 4);
        const float4 v0 = __ldg(q), v1 = __ldg(q + 1);
        xr[c][0] = pack_bf2(v0.x, v0.y);
        xr[c][1] = pack_bf2(v0.z, v0.w);
        xr[c][2] = pack_bf2(v1.x, v1.y);
        xr[c][3] = pack_bf2(v1.z, v1.w);
      }
    }
#pragma unroll
    for (int m2 = 0; m2 < 2; ++m2) {
      const int mu = 2 * half + m2;
      cx<float> Uf[D][D], Ub[D][D];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) L::load(lt, mu, a * D + bb, Uf[a][bb], Ub[a][bb]);
#pragma unroll
      for (int fb = 0; fb < 2; ++fb) {
        const int n = fb ? nb_[mu] : nf[mu];
        cx<float> in[4][D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const float4* q = reinterpret_cast<const float4*>(F + ((f.orow0 + n) * D + c) * 4);
          const float4 v0 = __ldg(q), v1 = __ldg(q + 1);
          in[0][c] = cmake(v0.x, v0.y);
          in[1][c] = cmake(v0.z, v0.w);
          in[2][c] = cmake(v1.x, v1.y);
          in[3][c] = cmake(v1.z, v1.w);
        }
        const int k = 1 + 2 * mu + fb;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            cx<float> w = cmake(0.f, 0.f);
#pragma unroll
            for (int bb = 0; bb < D; ++bb) cmac(w, fb ? Ub[a][bb] : Uf[a][bb], in[s][bb]);
            xr[a][k * 4 + s] = pack_bf2(w.re, w.im);
          }
      }
    }
  } else {
    // rows of sites past the end of the parity block: zero (their outputs are not stored)
#pragma unroll
    for (int c = 0; c < D; ++c)
      for (int e = half; e < 36; e += 2) xr[c][e] = 0u;
  }
  if (half == 1) {
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int e = 36; e < 40; ++e) xr[c][e] = 0u;  // k padding 72..79
  }
}

// stage 2, rows r0 .. r0 + 31 of the tile (a pair of 16-row tiles) through
// both GEMMs, Z2 to global memory.  Each B fragment read from shared memory
// feeds the MMAs of both row tiles.  Y1 = X1 W1 is formed in two column
// chunks and Z2 = Y1 W2p in three groups of three 8-column tiles, bounding
// the live accumulators.
template <int D, int C, bool EO>
__device__ __forceinline__ void mix_pair(const unsigned* X32, const unsigned* W132, const unsigned* W232,
                                         unsigned* __restrict__ Z, long long zrows, const FusedTile& f,
                                         int valid_rows, int r0, int lane) {
  using S = FusedShape<C>;
  constexpr int NM = 2;                // row tiles
  constexpr int NCH = C >= 4 ? 2 : 1;  // column chunks of Y1, each an even number of 8-column tiles
  constexpr int NC = C / NCH;
  constexpr int GS = 3;                // Z2 8-column tiles per group
  const bool self_only = EO && f.p == 0, no_self = EO && f.p == 1;
  const int gq = lane >> 2, q = lane & 3;
  constexpr int xs = kXStride / 2, w1s = S::W1Stride / 2, w2s = S::W2Stride / 2;
  // Y1 accumulators -> A fragments of the second GEMM (two 8-column tiles per 16-deep k-step)
  unsigned a2[NM][C / 2][4];
#pragma unroll
  for (int h = 0; h < NCH; ++h) {
    float acc[NM][NC][4];
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
      for (int n = 0; n < NC; ++n) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 5; ++kk) {
      if (self_only && kk > 0) break;  // X1 beyond slot 0 is zero
      unsigned a[NM][4];
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const int rr = r0 + m * 16 + gq;
        a[m][0] = X32[rr * xs + kk * 8 + q];
        a[m][1] = X32[(rr + 8) * xs + kk * 8 + q];
        a[m][2] = X32[rr * xs + kk * 8 + 4 + q];
        a[m][3] = X32[(rr + 8) * xs + kk * 8 + 4 + q];
      }
#pragma unroll
      for (int nn = 0; nn < NC; ++nn) {
        const int n = h * NC + nn;
        const unsigned b0 = W132[(n * 8 + gq) * w1s + kk * 8 + q];
        const unsigned b1 = W132[(n * 8 + gq) * w1s + kk * 8 + 4 + q];
#pragma unroll
        for (int m = 0; m < NM; ++m) mma16816(acc[m][nn], a[m], b0, b1);
      }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
      for (int tt = 0; tt < NC / 2; ++tt) {
        const int t = h * (NC / 2) + tt;
        a2[m][t][0] = pack_bf2(acc[m][2 * tt][0], acc[m][2 * tt][1]);
        a2[m][t][1] = pack_bf2(acc[m][2 * tt][2], acc[m][2 * tt][3]);
        a2[m][t][2] = pack_bf2(acc[m][2 * tt + 1][0], acc[m][2 * tt + 1][1]);
        a2[m][t][3] = pack_bf2(acc[m][2 * tt + 1][2], acc[m][2 * tt + 1][3]);
      }
  }
  // Z2 row (prow0 + i0) * D + local row; the 8-column tile n is slot k = n, column pair q is spin q
  const long long zr = (f.prow0 + f.i0) * D + r0;
#pragma unroll
  for (int gp = 0; gp < 9 / GS; ++gp) {
    if (self_only && gp > 0) break;  // only slot 0 is read
    float acc2[NM][GS][4];
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
      for (int n = 0; n < GS; ++n) acc2[m][n][0] = acc2[m][n][1] = acc2[m][n][2] = acc2[m][n][3] = 0.f;
#pragma unroll
    for (int t = 0; t < C / 2; ++t)
#pragma unroll
      for (int nn = 0; nn < GS; ++nn) {
        const int n = gp * GS + nn;
        if ((self_only && n > 0) || (no_self && n == 0)) continue;  // Z2 slots nobody reads
        const unsigned b0 = W232[(n * 8 + gq) * w2s + t * 8 + q];
        const unsigned b1 = W232[(n * 8 + gq) * w2s + t * 8 + 4 + q];
#pragma unroll
        for (int m = 0; m < NM; ++m) mma16816(acc2[m][nn], a2[m][t], b0, b1);
      }
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const int rr = r0 + m * 16 + gq;
#pragma unroll
      for (int nn = 0; nn < GS; ++nn) {
        const int n = gp * GS + nn;
        if ((self_only && n > 0) || (no_self && n == 0)) continue;
        if (rr < valid_rows) Z[(n * zrows + zr + m * 16 + gq) * 4 + q] = pack_bf2(acc2[m][nn][0], acc2[m][nn][1]);
        if (rr + 8 < valid_rows)
          Z[(n * zrows + zr + m * 16 + gq + 8) * 4 + q] = pack_bf2(acc2[m][nn][2], acc2[m][nn][3]);
      }
    }
  }
}

// stage 2 (consumer warp w in [0, 8)) of the block's it-th tile: the tile's
// 4 D pairs of 16-row tiles are dealt to the warps round-robin, continuing
// from the previous tile (tile it starts at pair index 4 D it), so that with
// 12 pairs per tile (D = 3) the warps that take two pairs alternate from one
// tile to the next
template <int D, int C, bool EO>
__device__ __forceinline__ void mix_tile(const __nv_bfloat16* sX, const __nv_bfloat16* sW1,
                                         const __nv_bfloat16* sW2, unsigned* __restrict__ Z, long long zrows,
                                         const Geom& g, const FusedTile& f, int w, int lane, int it) {
  static_assert(D == 2 || D == 3, "the fused kernel takes d = 2 or 3");
  const unsigned* X32 = reinterpret_cast<const unsigned*>(sX);
  const unsigned* W132 = reinterpret_cast<const unsigned*>(sW1);
  const unsigned* W232 = reinterpret_cast<const unsigned*>(sW2);
  const int valid_rows = (g.Vh - f.i0 < kFusedSites ? g.Vh - f.i0 : kFusedSites) * D;
  const int first = (w + 8 - (4 * D * it) % 8) % 8;
#pragma unroll 1
  for (int pr = first; pr < 4 * D; pr += 8) mix_pair<D, C, EO>(X32, W132, W232, Z, zrows, f, valid_rows, pr * 32, lane);
}

// L2 prefetch of a contiguous range (16-byte aligned address and size); a
// hint with no completion to wait for
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// the links (one contiguous range of 32-site link tiles) and the own-parity
// input rows of tile t into L2, by producer threads 0..4
template <int D>
__device__ __forceinline__ void prefetch_tile(const char* links, size_t link_block, const float2* F, const Geom& g,
                                              int t, int bpp, int tid) {
  const FusedTile f = fused_tile(g, t, bpp);
  constexpr unsigned kLinkTileBytes = kLinkTile * 4 * D * D * 16;  // 4 D^2 float4 planes per 32 sites
  if (tid < kFusedSites / kLinkTile) {
    const int lt = f.i0 / kLinkTile + tid;
    if (lt * kLinkTile < g.Vh)  // link tiles exist up to ceil(Vh / 32)
      prefetch_l2(links + (size_t)f.p * link_block + (size_t)lt * kLinkTileBytes, kLinkTileBytes);
  } else if (tid == kFusedSites / kLinkTile) {
    const int n = g.Vh - f.i0 < kFusedSites ? g.Vh - f.i0 : kFusedSites;
    prefetch_l2(F + (f.prow0 + f.i0) * D * 4, (unsigned)n * D * 32);
  }
}

// Persistent and warp-specialised: one block per SM walks the tiles
// t = blockIdx.x, + gridDim.x, ...  Warps 0-7 (producers) transport tile t
// into X1 buffer (iteration & 1) while warps 8-15 (consumers) run the GEMMs
// of the previous tile from the other buffer, so the gathers from HBM and
// the tensor-core work overlap.  Buffer hand-over: producers arrive on
// FULL[b] after filling b, consumers sync on it; consumers arrive on
// EMPTY[b] after reading b when the block has a tile two iterations later,
// and producers sync on EMPTY[b] before refilling b from their third
// iteration on.  Both sides walk the same tile sequence, so every barrier
// sees exactly kFusedThreads arrivals and kFusedThreads waiters.
template <int D, int C, bool EO>
__global__ void __launch_bounds__(2 * kFusedThreads, 1)
    fused_kernel(const char* __restrict__ links, size_t link_block, const float2* __restrict__ F,
                 const __nv_bfloat16* __restrict__ W1T, const __nv_bfloat16* __restrict__ W2T,
                 unsigned* __restrict__ Z, long long zrows, Geom g, int bpp, int ntiles) {
  using S = FusedShape<C>;
  constexpr int kRows = kFusedSites * D;
  constexpr int kAll = 2 * kFusedThreads;
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* sX0 = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* sW1 = sX0 + 2 * kRows * kXStride;
  __nv_bfloat16* sW2 = sW1 + S::W1Elems;

  // weights into shared memory once per block (16-byte copies; both sizes are multiples of 16 bytes)
  {
    const uint4* s1 = reinterpret_cast<const uint4*>(W1T);
    uint4* d1 = reinterpret_cast<uint4*>(sW1);
    for (int k = threadIdx.x; k < S::W1Elems / 8; k += kAll) d1[k] = s1[k];
    const uint4* s2 = reinterpret_cast<const uint4*>(W2T);
    uint4* d2 = reinterpret_cast<uint4*>(sW2);
    for (int k = threadIdx.x; k < S::W2Elems / 8; k += kAll) d2[k] = s2[k];
  }
  __syncthreads();

  if (threadIdx.x < kFusedThreads) {
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int buf = it & 1;
      if (t + (int)gridDim.x < ntiles) prefetch_tile<D>(links, link_block, F, g, t + gridDim.x, bpp, threadIdx.x);
      if (it >= 2) named_sync(kBarEmpty + buf, kAll);
      transport_tile<D, EO>(links, link_block, F, g, fused_tile(g, t, bpp), sX0 + buf * kRows * kXStride,
                            threadIdx.x);
      named_arrive(kBarFull + buf, kAll);
    }
  } else {
    const int w = (threadIdx.x - kFusedThreads) >> 5, lane = threadIdx.x & 31;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int buf = it & 1;
      named_sync(kBarFull + buf, kAll);
      mix_tile<D, C, EO>(sX0 + buf * kRows * kXStride, sW1, sW2, Z, zrows, g, fused_tile(g, t, bpp), w, lane, it);
      if (t + 2 * gridDim.x < ntiles) named_arrive(kBarEmpty + buf, kAll);
    }
  }
}

// out(x)[s] = sum_k (T_k Z_k)(x)[s] with Z in BF16, slot-major: Z[k][row] = 4 spins (16 bytes)
// (even_only: output parity 0 only, one thread per even site)
template <int D>
__global__ void __launch_bounds__(128) stencil_bf16_kernel(const char* __restrict__ links, size_t link_block,
                                                           const uint4* __restrict__ Z, long long zrows,
                                                           float2* __restrict__ out, Geom g, int nb,
                                                           int even_only) {
  const long long t = blockIdx.x * 128LL + threadIdx.x;
  const int np = even_only ? 1 : 2;
  if (t >= (long long)nb * np * g.Vh) return;
  const int i = (int)(t % g.Vh);
  const int p = (int)((t / g.Vh) % np);
  const int b = (int)(t / ((long long)np * g.Vh));
  const long long prow = ((long long)b * 2 + p) * g.Vh, orow = ((long long)b * 2 + 1 - p) * g.Vh;
  int nf[4], nb_[4];
  eo_neighbours(g, i, p, nf, nb_);
  using L = LinkIO<F32, D, false>;
  const auto* lt = L::tile_ptr(links + (size_t)p * link_block, i);
  auto unpack = [](unsigned u) {
    const float2 f = bf2_to_f2(u);
    return cmake(f.x, f.y);
  };
  cx<float> acc[4][D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const uint4 v = __ldg(Z + (prow + i) * D + c);
    acc[0][c] = unpack(v.x);
    acc[1][c] = unpack(v.y);
    acc[2][c] = unpack(v.z);
    acc[3][c] = unpack(v.w);
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    cx<float> Uf[D][D], Ub[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = 0; bb < D; ++bb) L::load(lt, mu, a * D + bb, Uf[a][bb], Ub[a][bb]);
#pragma unroll
    for (int fb = 0; fb < 2; ++fb) {
      const int n = fb ? nb_[mu] : nf[mu];
      const int k = 1 + 2 * mu + fb;
      cx<float> in[4][D];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const uint4 v = __ldg(Z + k * zrows + (orow + n) * D + c);
        in[0][c] = unpack(v.x);
        in[1][c] = unpack(v.y);
        in[2][c] = unpack(v.z);
        in[3][c] = unpack(v.w);
      }
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int bb = 0; bb < D; ++bb) cmac(acc[s][a], fb ? Ub[a][bb] : Uf[a][bb], in[s][bb]);
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    float4* o = reinterpret_cast<float4*>(out + ((prow + i) * D + c) * 4);
    o[0] = make_float4(acc[0][c].re, acc[0][c].im, acc[1][c].re, acc[1][c].im);
    o[1] = make_float4(acc[2][c].re, acc[2][c].im, acc[3][c].re, acc[3][c].im);
  }
}

template <int D, int C>
size_t fused_smem() {
  return (size_t)(2 * kFusedSites * D * kXStride + FusedShape<C>::W1Elems + FusedShape<C>::W2Elems) * 2;
}

template <int D, int C>
int fused_launch(const char* links, size_t link_block, const void* F, const void* W1, const void* W2p, void* W1T,
                 void* W2T, void* Z, void* out, const Geom& g, int nb, bool even_only, cudaStream_t s) {
  using S = FusedShape<C>;
  const int n = S::W1Elems + S::W2Elems;
  fused_prep_kernel<C><<<(n + 255) / 256, 256, 0, s>>>(reinterpret_cast<const float2*>(W1),
                                                       reinterpret_cast<const float2*>(W2p),
                                                       reinterpret_cast<__nv_bfloat16*>(W1T),
                                                       reinterpret_cast<__nv_bfloat16*>(W2T));
  const size_t smem = fused_smem<D, C>();
  auto kern = even_only ? fused_kernel<D, C, true> : fused_kernel<D, C, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return BSM_ECUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                               cudaSuccess || sms <= 0)
    return BSM_ECUDA;
  const int bpp = (g.Vh + kFusedSites - 1) / kFusedSites;
  const int ntiles = nb * 2 * bpp;
  const long long sites = (long long)nb * 2 * g.Vh, zrows = sites * D;
  kern<<<ntiles < sms ? ntiles : sms, 2 * kFusedThreads, smem, s>>>(
      links, link_block, reinterpret_cast<const float2*>(F), reinterpret_cast<const __nv_bfloat16*>(W1T),
      reinterpret_cast<const __nv_bfloat16*>(W2T), reinterpret_cast<unsigned*>(Z), zrows, g, bpp, ntiles);
  const long long outs = even_only ? sites / 2 : sites;
  stencil_bf16_kernel<D><<<(int)((outs + 127) / 128), 128, 0, s>>>(
      links, link_block, reinterpret_cast<const uint4*>(Z), zrows, reinterpret_cast<float2*>(out), g, nb,
      even_only ? 1 : 0);
  return BSM_OK;
}

template <int D>
int fused_dispatch_c(int C, const char* links, size_t lb, const void* F, const void* W1, const void* W2p, void* W1T,
                     void* W2T, void* Z, void* out, const Geom& g, int nb, bool eo, cudaStream_t s) {
  switch (C) {
    case 2: return fused_launch<D, 2>(links, lb, F, W1, W2p, W1T, W2T, Z, out, g, nb, eo, s);
    case 4: return fused_launch<D, 4>(links, lb, F, W1, W2p, W1T, W2T, Z, out, g, nb, eo, s);
    case 8: return fused_launch<D, 8>(links, lb, F, W1, W2p, W1T, W2T, Z, out, g, nb, eo, s);
    case 12: return fused_launch<D, 12>(links, lb, F, W1, W2p, W1T, W2T, Z, out, g, nb, eo, s);
    default: return BSM_EUNSUPPORTED;
  }
}

}  // namespace

// hidden-channel counts with a fused BF16 kernel
bool ptc_fused_supported(int C) { return C == 2 || C == 4 || C == 8 || C == 12; }

// bytes of the realified weights W1T + W2T (bf16) for C channels
size_t ptc_fused_weight_bytes(int C) { return (size_t)(8 * C * kXStride + 72 * (8 * C + 8)) * 2; }

// Z: 9 x rows x 4 BF16 complex (4 bytes each), slot-major; W1T/W2T: ptc_fused_weight_bytes(C), 16-byte aligned
int ptc_fused_apply(const char* links, size_t link_block, int d, int C, const void* F, const void* W1,
                    const void* W2p, void* Wt, void* Z, void* out, const Geom& g, int nb, bool even_only,
                    cudaStream_t s) {
  void* W1T = Wt;
  void* W2T = reinterpret_cast<char*>(Wt) + (size_t)8 * C * kXStride * 2;
  if (d == 2) return fused_dispatch_c<2>(C, links, link_block, F, W1, W2p, W1T, W2T, Z, out, g, nb, even_only, s);
  if (d == 3) return fused_dispatch_c<3>(C, links, link_block, F, W1, W2p, W1T, W2T, Z, out, g, nb, even_only, s);
  return BSM_EUNSUPPORTED;
}

}  // namespace bsm
