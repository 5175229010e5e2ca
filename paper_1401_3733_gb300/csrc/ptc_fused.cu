// ptc_fused.cu -- BF16 inference of the parallel-transport preconditioner
// with the two channel-mixing GEMMs fused into the transport kernel, on the
// tcgen05 tensor cores.
//
// A tile is 128 consecutive eo sites of one parity (128 d rows of the PTC
// field).  Stage 1 (producer warps): four threads per site, one direction
// mu each, compute the 9 transports of the one-channel input (T_0, and
// U_mu(x) F(x+mu), U_mu(x-mu)^+ F(x-mu)) in FP32 and store them, rounded to
// BF16 and realified (re, im interleaved), as the tile X1 (rows x 72 reals,
// padded to 80) in shared memory.  Stage 2 (consumer
// warps), per block of 128 rows:
//     Y1 = X1 W1  (80 -> 8C reals)   and   Z2 = Y1 W2p  (8C -> 72 reals)
// as tcgen05.mma (BF16 x BF16 -> FP32, M = 128) issued by one thread, with
// the accumulators in tensor memory.  The consumer warps read Y1 back
// (tcgen05.ld, one TMEM lane = one row per thread), round it to BF16 into
// shared memory as the A operand of the second MMA, and read Z2 back into
// global memory.  Z2 (rows x 36 complex, BF16) is the only intermediate
// written to memory, slot-major (Z2[k][row][spin]) so that the stencil
// kernel, which forms out = sum_k T_k Z2_k, reads each neighbour's slot as
// whole, contiguous 16-byte groups.
//
// All MMA operands sit in shared memory in the tensor core's no-swizzle,
// K-major layout: 8 x 8 BF16 core matrices of 128 contiguous bytes (16 B
// per row), K-adjacent cores 128 B apart (the descriptor's leading byte
// offset), 8-row groups kcores * 128 B apart (its stride byte offset).  A
// transport result (one row, one slot: 4 spins x re, im) is exactly one core
// row, so the producers store it as one 16-byte word.
//
// The kernel is persistent (one block per SM, weights staged once) and
// warp-specialised: 16 producer warps run stage 1 for the next tile while 4
// consumer warps run stage 2 on the previous one, with two X1 buffers
// handed over through hardware named barriers, so that the gathers from HBM
// overlap the tensor-core work.
#include <cuda_bf16.h>
#include <stdlib.h>

#include "bsm_internal.cuh"

namespace bsm {

namespace {

constexpr int kFusedSites = 128;                      // eo sites per tile
constexpr int kProducers = 512;                       // 16 warps, four threads per site (one direction each)
constexpr int kConsumers = 128;                       // 4 warps, one per TMEM lane quarter
constexpr int kFusedThreads = kProducers + kConsumers;
constexpr int kK1 = 80;                               // GEMM1 depth: 72 transport reals + 8 zero
constexpr int kN2 = 80;                               // GEMM2 width: 72 Z2 reals + 8 zero columns
constexpr int kTmemCols = 512;                        // Y1 accumulators at column 128 rb, Z2 at kD2Col
constexpr int kD2Col = 384;
constexpr unsigned kWaitCap = 1u << 20;               // polls of an MMA-completion barrier before giving up

template <int C>
struct FusedShape {
  static constexpr int N1 = 8 * C;              // Y1 reals per row: GEMM1 width, GEMM2 depth
  static constexpr int W1Bytes = N1 * kK1 * 2;  // GEMM1 B operand (N1 rows of K = 80)
  static constexpr int W2Bytes = kN2 * N1 * 2;  // GEMM2 B operand (80 rows of K = N1)
  static constexpr int Y1Bytes = 128 * N1 * 2;  // GEMM2 A operand of one 128-row block
};

// byte offset of element (r, k) of a K-major operand of `kcores` 8-wide
// core columns, in the no-swizzle core-matrix layout
__host__ __device__ constexpr int core_off(int r, int k, int kcores) {
  return (r >> 3) * (kcores * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ unsigned pack_bf2(float lo, float hi) { return f2_to_bf2(lo, hi); }

// realified, transposed weights in the core-matrix layout (bf16): GEMM1's B
// is W1T[n][k] = W1r[k][n] (n < 8C, k < 80, zero for k >= 72), GEMM2's B is
// W2T[n][k] = W2pr[k][n] (n < 80, zero for n >= 72, k < 8C)
template <int C>
__global__ void fused_prep_kernel(const float2* __restrict__ W1, const float2* __restrict__ W2p,
                                  unsigned char* __restrict__ Wt) {
  using S = FusedShape<C>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // realified entry (k, n) of a complex K x N matrix M: [[Re, Im], [-Im, Re]] blocks
  auto real_of = [](const float2* M, int N, int k, int n) {
    const float2 w = M[(k >> 1) * N + (n >> 1)];
    if ((k & 1) == 0) return (n & 1) ? w.y : w.x;
    return (n & 1) ? w.x : -w.y;
  };
  if (t < S::N1 * kK1) {
    const int n = t / kK1, k = t % kK1;
    *reinterpret_cast<__nv_bfloat16*>(Wt + core_off(n, k, kK1 / 8)) =
        __float2bfloat16_rn(k < 72 ? real_of(W1, 4 * C, k, n) : 0.f);
  } else if (t < S::N1 * kK1 + kN2 * S::N1) {
    const int u = t - S::N1 * kK1;
    const int n = u / S::N1, k = u % S::N1;
    *reinterpret_cast<__nv_bfloat16*>(Wt + S::W1Bytes + core_off(n, k, C)) =
        __float2bfloat16_rn(n < 72 ? real_of(W2p, 36, k, n) : 0.f);
  }
}

// hardware named barriers (ids 1..5; 0 is __syncthreads) between the
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
constexpr int kBarConsumers = 5;            // the consumer warps alone

// ---- tcgen05 helpers -------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading byte offset 128
// (K-adjacent core matrices), stride byte offset `sbo` (8-row groups),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
         (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t umma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on `mbar` once every MMA issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
// bounded wait for the completion of phase `parity` of `mbar`; false after `polls` polls
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, unsigned polls = kWaitCap) {
  for (unsigned n = 0; n < polls; ++n) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 8 / 16 consecutive FP32 columns of this thread's TMEM lane into r[0..];
// the values are defined only after tmem_wait
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// wait for this thread's outstanding tcgen05.ld; the empty statements after
// it tie r[0..N) to the wait, so that no use of them is scheduled earlier
template <int N>
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[N]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < N; ++j) asm volatile("" : "+r"(r[j]));
}
// 8 FP32 values (4 spins x re, im) -> one 16-byte group of 4 packed BF16 pairs
__device__ __forceinline__ uint4 pack8(const uint32_t* r) {
  return make_uint4(pack_bf2(__uint_as_float(r[0]), __uint_as_float(r[1])),
                    pack_bf2(__uint_as_float(r[2]), __uint_as_float(r[3])),
                    pack_bf2(__uint_as_float(r[4]), __uint_as_float(r[5])),
                    pack_bf2(__uint_as_float(r[6]), __uint_as_float(r[7])));
}

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

// stage 1 (producer thread tid in [0, 512)): for site i0 + (tid mod 128) and
// direction mu = tid / 128, the transports of the one-channel input from
// x + mu and x - mu (slots 1 + 2 mu, 2 + 2 mu), and for mu = 0 also the
// site's own value (slot 0), into the X1 tile (bf16, realified, core-matrix
// layout) in shared memory.
// Slot k of row r is the 16-byte core row at core_off(r, 8 k, 10); core
// column 9 (k = 72..79) stays zero from the kernel's start.
template <int D, bool EO>
__device__ __forceinline__ void transport_tile(const char* __restrict__ links, size_t link_block,
                                               const float2* __restrict__ F, const Geom& g, const FusedTile& f,
                                               unsigned char* sX, int tid) {
  // EO (even-only input): the input vanishes on odd sites, so an even site
  // has only its own term (X1 slot 0) and an odd site only the transports of
  // its neighbours (slots 1..8); the even-only stencil then reads slot 0 of
  // Z2 on even rows and slots 1..8 on odd rows, so only those are computed.
  const bool self_only = EO && f.p == 0, no_self = EO && f.p == 1;
  const int sl = tid & (kFusedSites - 1), mu = tid / kFusedSites;
  const int i = f.i0 + sl;
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  auto put = [&](int c, int k, const uint4& v) {
    *reinterpret_cast<uint4*>(sX + core_off(sl * D + c, 8 * k, kK1 / 8)) = v;
  };
  auto own = [&](int c) {
    const float4* q = reinterpret_cast<const float4*>(F + ((f.prow0 + i) * D + c) * 4);
    const float4 v0 = __ldg(q), v1 = __ldg(q + 1);
    return make_uint4(pack_bf2(v0.x, v0.y), pack_bf2(v0.z, v0.w), pack_bf2(v1.x, v1.y), pack_bf2(v1.z, v1.w));
  };
  if (i < g.Vh && !self_only) {
    int nf[4], nb_[4];
    eo_neighbours(g, i, f.p, nf, nb_);
    using L = LinkIO<F32, D, false>;
    const auto* lt = L::tile_ptr(links + (size_t)f.p * link_block, i);
    if (mu == 0) {
#pragma unroll
      for (int c = 0; c < D; ++c) put(c, 0, no_self ? zero : own(c));
    }
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
      for (int a = 0; a < D; ++a) {
        unsigned v[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          cx<float> w = cmake(0.f, 0.f);
#pragma unroll
          for (int bb = 0; bb < D; ++bb) cmac(w, fb ? Ub[a][bb] : Uf[a][bb], in[s][bb]);
          v[s] = pack_bf2(w.re, w.im);
        }
        put(a, k, make_uint4(v[0], v[1], v[2], v[3]));
      }
    }
  } else {
    // an even site of an even-only input (its own term only), or a row past
    // the end of the parity block (zero; its outputs are not stored)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (mu == 0) put(c, 0, (i < g.Vh) ? own(c) : zero);
      put(c, 1 + 2 * mu, zero);
      put(c, 2 + 2 * mu, zero);
    }
  }
}

// L2 prefetch of a contiguous range (16-byte aligned address and size); a
// hint with no completion to wait for
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// the links (one contiguous range of 32-site link tiles) and the own-parity
// input rows of tile t into L2, by producer threads 0..4; an even tile of an
// even-only input reads no links
template <int D, bool EO>
__device__ __forceinline__ void prefetch_tile(const char* links, size_t link_block, const float2* F, const Geom& g,
                                              int t, int bpp, int tid) {
  const FusedTile f = fused_tile(g, t, bpp);
  constexpr unsigned kLinkTileBytes = kLinkTile * 4 * D * D * 16;  // 4 D^2 float4 planes per 32 sites
  if (tid < kFusedSites / kLinkTile) {
    if (EO && f.p == 0) return;
    const int lt = f.i0 / kLinkTile + tid;
    if (lt * kLinkTile < g.Vh)  // link tiles exist up to ceil(Vh / 32)
      prefetch_l2(links + (size_t)f.p * link_block + (size_t)lt * kLinkTileBytes, kLinkTileBytes);
  } else if (tid == kFusedSites / kLinkTile) {
    const int n = g.Vh - f.i0 < kFusedSites ? g.Vh - f.i0 : kFusedSites;
    prefetch_l2(F + (f.prow0 + f.i0) * D * 4, (unsigned)n * D * 32);
  }
}

// An MMA-completion wait that gives up (after `polls` polls) is followed by
// a second wait of kWaitCap polls for the same MMAs, so that nothing the
// tensor core may still write is read or reused; the thread then records the
// failure in the block's `failed` flag and the launch's error word `err`.
// From the next MMA on, the block issues no more MMAs and waits for none:
// its remaining tiles keep the buffer hand-over with the producers and store
// their Z2 rows as NaN.
__device__ __forceinline__ bool mma_wait(uint32_t mbar, uint32_t parity, unsigned polls, int* failed,
                                         int* __restrict__ err) {
  if (mbar_wait(mbar, parity, polls)) return true;
  mbar_wait(mbar, parity, kWaitCap);
  *reinterpret_cast<volatile int*>(failed) = 1;
  atomicExch(err, 1);
  return false;
}

// stage 2 (consumer thread c in [0, 128) = TMEM lane c) for one tile:
// GEMM1 for all D row blocks, then per row block the Y1 read-back, GEMM2 and
// the Z2 read-back.  Returns false if an MMA-completion wait gave up or the
// block had already given up (the tile's Z2 rows are then stored as NaN).
template <int D, int C, bool EO>
__device__ __forceinline__ bool mix_tile(const unsigned char* sX, const unsigned char* sW1,
                                         const unsigned char* sW2, unsigned char* sY1, uint64_t* mbar,
                                         uint32_t tmem, uint4* __restrict__ Z, long long zrows, const Geom& g,
                                         const FusedTile& f, int c, int it, bool more, unsigned polls,
                                         int* failed, int* __restrict__ err) {
  using S = FusedShape<C>;
  constexpr int kY1Batch = S::N1 % 48 == 0 ? 48 : S::N1 % 32 == 0 ? 32 : 16;  // Y1 columns per TMEM wait
  const bool self_only = EO && f.p == 0, no_self = EO && f.p == 1;
  const int buf = it & 1;
  // read after the FULL barrier, which every consumer passed after any earlier failure was recorded
  const bool skip1 = *reinterpret_cast<volatile int*>(failed) != 0;
  bool ok = !skip1;
  if (c == 0 && !skip1) {
    const uint32_t xa = smem_u32(sX), wa = smem_u32(sW1);
    for (int rb = 0; rb < D; ++rb)
      for (int kk = 0; kk < (self_only ? 1 : kK1 / 16); ++kk)  // self_only: X1 beyond slot 1 is zero
        umma(tmem + rb * S::N1, umma_desc(xa + rb * (128 * kK1 * 2) + kk * 256, kK1 / 8 * 128),
             umma_desc(wa + kk * 256, kK1 / 8 * 128), umma_idesc(S::N1), kk);
    umma_commit(smem_u32(mbar));
  }
  if (!skip1) ok &= mma_wait(smem_u32(mbar), it & 1, polls, failed, err);
  tc_fence_after();
  if (more) named_arrive(kBarEmpty + buf, kFusedThreads);  // X1[buf] has been read
  const uint32_t lane = tmem + ((uint32_t)((c >> 5) * 32) << 16);
  const int valid_rows = (g.Vh - f.i0 < kFusedSites ? g.Vh - f.i0 : kFusedSites) * D;
#pragma unroll 1
  for (int rb = 0; rb < D; ++rb) {
    // Y1 rows of this block: TMEM -> BF16 -> shared memory (GEMM2's A
    // operand), in batches of up to 48 columns per wait
#pragma unroll
    for (int c0 = 0; c0 < S::N1; c0 += kY1Batch) {
      uint32_t r[kY1Batch];
#pragma unroll
      for (int j = 0; j < kY1Batch; j += 16) tmem_ld16(lane + rb * S::N1 + c0 + j, &r[j]);
      tmem_wait(r);
#pragma unroll
      for (int j = 0; j < kY1Batch; j += 8) *reinterpret_cast<uint4*>(sY1 + core_off(c, c0 + j, C)) = pack8(&r[j]);
    }
    fence_async_smem();
    tc_fence_before();
    named_sync(kBarConsumers, kConsumers);
    tc_fence_after();
    // every consumer's GEMM1 (or previous GEMM2) wait is recorded before this barrier
    const bool skip2 = *reinterpret_cast<volatile int*>(failed) != 0;
    if (skip2) ok = false;
    if (c == 0 && !skip2) {
      const uint32_t ya = smem_u32(sY1), wb = smem_u32(sW2);
      for (int kk = 0; kk < C / 2; ++kk)
        umma(tmem + kD2Col, umma_desc(ya + kk * 256, C * 128), umma_desc(wb + kk * 256, C * 128), umma_idesc(kN2),
             kk);
      umma_commit(smem_u32(mbar + 1));
    }
    if (!skip2) ok &= mma_wait(smem_u32(mbar + 1), (it * D + rb) & 1, polls, failed, err);
    tc_fence_after();
    // Z2 rows of this block: TMEM -> BF16 -> global, one 16-byte group (4
    // spins) per slot; slots 0..3 and 4..8 in one wait each
    const int row = rb * 128 + c;
    const long long zrow = (f.prow0 + f.i0) * D + row;
    const bool store = row < valid_rows;
    auto put = [&](int n, const uint32_t* r) {
      uint4 v = pack8(r);
      if (!ok) v = make_uint4(0x7fc07fc0u, 0x7fc07fc0u, 0x7fc07fc0u, 0x7fc07fc0u);  // BF16 NaN
      if (store) Z[n * zrows + zrow] = v;
    };
    if (self_only) {  // only slot 0 is read
      uint32_t r[8];
      tmem_ld8(lane + kD2Col, r);
      tmem_wait(r);
      put(0, r);
    } else {
      {
        uint32_t r[32];
        tmem_ld16(lane + kD2Col, &r[0]);
        tmem_ld16(lane + kD2Col + 16, &r[16]);
        tmem_wait(r);
#pragma unroll
        for (int n = 0; n < 4; ++n)
          if (!(no_self && n == 0)) put(n, &r[8 * n]);
      }
      {
        uint32_t r[40];
        tmem_ld16(lane + kD2Col + 32, &r[0]);
        tmem_ld16(lane + kD2Col + 48, &r[16]);
        tmem_ld8(lane + kD2Col + 64, &r[32]);
        tmem_wait(r);
#pragma unroll
        for (int n = 4; n < 9; ++n) put(n, &r[8 * (n - 4)]);
      }
    }
    tc_fence_before();
  }
  return ok;
}

// Persistent and warp-specialised: one block per SM walks the tiles
// t = blockIdx.x, + gridDim.x, ...  Warps 0-15 (producers) transport tile t
// into X1 buffer (iteration & 1) while warps 16-19 (consumers) run the MMAs
// of the previous tile from the other buffer.  Buffer hand-over: producers
// arrive on FULL[b] after filling b, consumers sync on it; consumers arrive
// on EMPTY[b] once GEMM1 has read b, when the block has a tile two
// iterations later, and producers sync on EMPTY[b] before refilling b from
// their third iteration on.  Both sides walk the same tile sequence, so
// every barrier sees exactly its expected arrivals and waiters.
template <int D, int C, bool EO>
__global__ void __launch_bounds__(kFusedThreads, 1)
    fused_kernel(const char* __restrict__ links, size_t link_block, const float2* __restrict__ F,
                 const unsigned char* __restrict__ Wt, uint4* __restrict__ Z, long long zrows, Geom g, int bpp,
                 int ntiles, int* __restrict__ err, unsigned polls) {
  using S = FusedShape<C>;
  constexpr int kRows = kFusedSites * D;
  constexpr int kX1Bytes = kRows * kK1 * 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sX = smem;  // two X1 buffers
  unsigned char* sW1 = smem + 2 * kX1Bytes;
  unsigned char* sW2 = sW1 + S::W1Bytes;
  unsigned char* sY1 = sW2 + S::W2Bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sY1 + S::Y1Bytes);  // [0] GEMM1 done, [1] GEMM2 done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  int* failed = reinterpret_cast<int*>(tslot + 1);  // an MMA-completion wait of this block gave up
  const int tid = threadIdx.x;
  if (tid == 0) *failed = 0;

  // weights into shared memory once; zero core column 9 of both X1 buffers;
  // barriers; tensor memory
  for (int k = tid; k < (S::W1Bytes + S::W2Bytes) / 16; k += kFusedThreads)
    reinterpret_cast<uint4*>(sW1)[k] = reinterpret_cast<const uint4*>(Wt)[k];
  for (int r = tid; r < 2 * kRows; r += kFusedThreads)
    *reinterpret_cast<uint4*>(sX + (r / kRows) * kX1Bytes + core_off(r % kRows, 72, kK1 / 8)) =
        make_uint4(0u, 0u, 0u, 0u);
  if (tid == kProducers) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)));
  }
  if (tid >= kProducers && tid < kProducers + 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (tid < kProducers) {
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int buf = it & 1;
      if (t + (int)gridDim.x < ntiles) prefetch_tile<D, EO>(links, link_block, F, g, t + gridDim.x, bpp, tid);
      if (it >= 2) named_sync(kBarEmpty + buf, kFusedThreads);
      transport_tile<D, EO>(links, link_block, F, g, fused_tile(g, t, bpp), sX + buf * kX1Bytes, tid);
      fence_async_smem();  // X1 writes -> visible to the tensor core
      named_arrive(kBarFull + buf, kFusedThreads);
    }
  } else {
    const int c = tid - kProducers;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int buf = it & 1;
      named_sync(kBarFull + buf, kFusedThreads);
      tc_fence_after();
      mix_tile<D, C, EO>(sX + buf * kX1Bytes, sW1, sW2, sY1, mbar, tmem, Z, zrows, g, fused_tile(g, t, bpp), c, it,
                         t + 2 * (int)gridDim.x < ntiles, polls, failed, err);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid >= kProducers && tid < kProducers + 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
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
  using S = FusedShape<C>;
  return (size_t)2 * kFusedSites * D * kK1 * 2 + S::W1Bytes + S::W2Bytes + S::Y1Bytes + 32;
}

template <int D, int C>
int fused_launch(const char* links, size_t link_block, const void* F, const void* W1, const void* W2p, void* Wt,
                 void* Z, void* out, const Geom& g, int nb, bool even_only, int* err, unsigned polls, cudaStream_t s) {
  using S = FusedShape<C>;
  const int n = S::N1 * kK1 + kN2 * S::N1;
  fused_prep_kernel<C><<<(n + 255) / 256, 256, 0, s>>>(reinterpret_cast<const float2*>(W1),
                                                       reinterpret_cast<const float2*>(W2p),
                                                       reinterpret_cast<unsigned char*>(Wt));
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
  kern<<<ntiles < sms ? ntiles : sms, kFusedThreads, smem, s>>>(
      links, link_block, reinterpret_cast<const float2*>(F), reinterpret_cast<const unsigned char*>(Wt),
      reinterpret_cast<uint4*>(Z), zrows, g, bpp, ntiles, err, polls);
  const long long outs = even_only ? sites / 2 : sites;
  stencil_bf16_kernel<D><<<(int)((outs + 127) / 128), 128, 0, s>>>(
      links, link_block, reinterpret_cast<const uint4*>(Z), zrows, reinterpret_cast<float2*>(out), g, nb,
      even_only ? 1 : 0);
  return BSM_OK;
}

template <int D>
int fused_dispatch_c(int C, const char* links, size_t lb, const void* F, const void* W1, const void* W2p, void* Wt,
                     void* Z, void* out, const Geom& g, int nb, bool eo, int* err, unsigned polls, cudaStream_t s) {
  switch (C) {
    case 2: return fused_launch<D, 2>(links, lb, F, W1, W2p, Wt, Z, out, g, nb, eo, err, polls, s);
    case 4: return fused_launch<D, 4>(links, lb, F, W1, W2p, Wt, Z, out, g, nb, eo, err, polls, s);
    case 8: return fused_launch<D, 8>(links, lb, F, W1, W2p, Wt, Z, out, g, nb, eo, err, polls, s);
    case 12: return fused_launch<D, 12>(links, lb, F, W1, W2p, Wt, Z, out, g, nb, eo, err, polls, s);
    default: return BSM_EUNSUPPORTED;
  }
}

// polls of an MMA-completion wait before it gives up: kWaitCap, or the value
// of BSM_PTC_WAIT_POLLS (0 makes every first wait give up at once, which is
// how the tests reach the error path)
unsigned wait_polls() {
  const char* env = getenv("BSM_PTC_WAIT_POLLS");
  if (env == nullptr || *env == '\0') return kWaitCap;
  char* end = nullptr;
  const unsigned long v = strtoul(env, &end, 10);
  return (end != nullptr && *end == '\0' && v <= kWaitCap) ? (unsigned)v : kWaitCap;
}

}  // namespace

// hidden-channel counts with a fused BF16 kernel
bool ptc_fused_supported(int C) { return C == 2 || C == 4 || C == 8 || C == 12; }

// bytes of the realified weights in the core-matrix layout (bf16): GEMM1's B (8C x 80) and GEMM2's B (80 x 8C)
size_t ptc_fused_weight_bytes(int C) { return (size_t)2 * (8 * C) * 80 * 2; }

// Z: 9 x rows x 4 BF16 complex (4 bytes each), slot-major; Wt: ptc_fused_weight_bytes(C), 16-byte aligned;
// err: a device word the kernel sets to 1 when an MMA-completion wait gives up (never cleared here)
int ptc_fused_apply(const char* links, size_t link_block, int d, int C, const void* F, const void* W1,
                    const void* W2p, void* Wt, void* Z, void* out, const Geom& g, int nb, bool even_only, int* err,
                    cudaStream_t s) {
  const unsigned polls = wait_polls();
  if (d == 2) return fused_dispatch_c<2>(C, links, link_block, F, W1, W2p, Wt, Z, out, g, nb, even_only, err, polls, s);
  if (d == 3) return fused_dispatch_c<3>(C, links, link_block, F, W1, W2p, Wt, Z, out, g, nb, even_only, err, polls, s);
  return BSM_EUNSUPPORTED;
}

}  // namespace bsm
