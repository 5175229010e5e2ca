// mrhs_tc.cu -- multi-RHS hopping block on the tensor cores (BF16 storage,
// FP32 accumulation) for the larger colour dimensions d = 4, 6, 8.
//
// For one site and one of its 8 direction-senses the hop is a small dense
// contraction: W = U h, with U the d x d link and h the d x (2 spins x n_rhs)
// block of spin-projected neighbour spinors.  In real form, with the real
// parts of the colours in K rows 0..7 and the imaginary parts in rows 8..15,
//     [Wr; Wi] = [[Ur, -Ui], [Ui, Ur]] [hr; hi]
// is an M = K = 16, N = 2 n_rhs GEMM: one mma.sync.m16n8k16 (bf16 x bf16 ->
// f32) per 8 columns.  The lower spin components of the term are
// sg B_mu^+ (U h) = U (sg B_mu^+ h), a second B operand that is a sign flip
// and re/im exchange of the first one's registers, so both spin halves
// accumulate in the MMA accumulators across all 8 direction-senses and no
// reconstruction runs per direction.  Each site has its own link, so no A
// operand is shared across sites (tcgen05 needs M >= 64 rows with one A):
// one warp owns one site at a time.
//
// Operands are built in registers.  Lane (g, t) = (lane / 4, lane % 4) of
// the warp holds, in the mma.sync fragment layouts,
//   A: link elements U[g][t], U[g][t + d/2] (real and imaginary pairs);
//   B: colours t and t + d/2 of column n = g of each 8-column tile,
// i.e. the K index runs over the colours in the order (0, d/2, 1, d/2+1, ...);
// this pairing puts the lanes t of one shared-memory read on different banks.
// Columns are assigned so that one lane holds both spins of one RHS: tile
// 2k has spin 0 and tile 2k+1 spin 1 of RHS r = 8k + g; for n_rhs = 4 or 12
// the last tile holds RHS 8k + (g & 3), spin g >> 2.  A lane therefore reads
// four (psi0, psi2) / (psi1, psi3) words per RHS, projects them with packed
// bf16x2 FMAs (u + s l, s = +-1 or +-i: one rounding to BF16, as storing an
// FP32 projection would give) and packs the real and imaginary pairs.
//
// Data movement: a block of 4 warps works on 4 consecutive sites at a time
// (one per warp), whose links share the 32-byte sectors of the tiled link
// layout; the block copies the next 4 sites' links into a double buffer of
// per-site link blocks (cp.async, 8 bytes per element) while it computes the
// current ones.  Every warp runs through its site's 8 direction-senses as a
// stream of items and copies item j + S - 2 (the neighbour's multi-RHS spinor
// block, 2d plane rows of n_rhs words, one contiguous run in the site-major
// multi-RHS layout, as 16-byte cp.async pieces of the lanes) into an S-stage
// ring of its shared memory while it computes item j; the same-site input of
// the a x + b H form is copied the same way during the site.  The grid is
// persistent.  The copies bound the kernel: on 24^4 x 12 RHS at d = 6 it
// takes 0.50 ms per D, against 0.56 ms when each block was 2d rows 16 MB
// apart (plane-major), where the copies alone took 0.48 ms and the arithmetic
// alone 0.40 ms.  (In that layout, moving half or all of each item by TMA
// tile copies, completing on mbarriers, measured slower: 0.73 and 0.66 ms; so
// did copying the 4 sites' neighbour blocks as one slab per block, 0.57 ms,
// and staging only their z neighbours once per block, 5 blocks in place of
// 8, 0.561 ms.)
#include "mrhs.cuh"

namespace bsm {

namespace {

constexpr int kTcWarps = 4;        // warps (sites) per block
constexpr int kTcBlocksPerSm = 4;  // register budget: 128 per thread
constexpr unsigned kSign2 = 0x80008000u;

template <int D, int NR>
struct TcLayout {
  // a site's block in shared memory: 2d plane rows of n_rhs words; rows are
  // padded by 32 bytes when n_rhs is a multiple of 8, so that the row pitch is
  // 8 or 24 words mod 32 and the lanes t of one read (rows t, t + d/2, ...
  // apart) fall on different banks
  static constexpr int pitch = NR * 8 + (NR % 8 == 0 ? 32 : 0);
  static constexpr int spin_bytes = 2 * D * pitch;
  // per-site link block: 4 d^2 (fwd, bwd) pairs; the stride is 16 words mod
  // 32 so that the copies of two sites (lanes 0-7, 8-15) use different banks
  static constexpr int link_site = 4 * D * D * 8 + ((4 * D * D * 8 / 4) % 32 == 16 ? 0 : 64);
  static constexpr int link_buf = kTcWarps * link_site;
  static constexpr int S = 4;  // ring depth: two items in flight (8 stages measured no faster: the copies are bandwidth-bound)
  static constexpr int warp_bytes = (S + 1) * spin_bytes;  // S stages, then the x block
  static constexpr int links_off = kTcWarps * warp_bytes;  // two link buffers
  static constexpr int block_bytes = links_off + 2 * link_buf;
  static constexpr int link_elems = kTcWarps * 4 * D * D;  // elements of a quad's links
  static constexpr int row_chunks = NR / 2;                // 16-byte pieces of a plane row
  static constexpr int block_src = 2 * D * NR * 8;         // a site's block in memory: 2d rows, unpadded
  static constexpr int chunks = 2 * D * row_chunks;        // pieces of a block
  static constexpr int per_lane = (chunks + 31) / 32;
  static constexpr int NT = NR / 4;                        // 8-column tiles
  static constexpr int NGF = NR / 8;                       // RHS groups filling two tiles
  static constexpr bool HALF = (NR % 8) != 0;              // a last tile of 4 RHS x 2 spins
  static_assert(NR % 4 == 0 && NR <= 16, "n_rhs in {4, 8, 12, 16}");
  static_assert(spin_bytes % 16 == 0 && link_site % 16 == 0, "aligned areas");
  static_assert((4 * D * D) % 8 == 0 && D % 2 == 0 && S - 2 <= 7, "copy mappings");
};

__device__ __forceinline__ void cp_async8_ca(unsigned s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16_cg(unsigned s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint2 lds64(unsigned a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ uint4 lds128(unsigned a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}

// d = a * b + c on bf16x2, rounded once
__device__ __forceinline__ unsigned hfma2(unsigned a, unsigned b, unsigned c) {
  unsigned d;
  asm("fma.rn.bf16x2 %0, %1, %2, %3;\n" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// unsigned division n / d for n < 2^31 by a multiply and a shift:
// m = ceil(2^(31 + l) / d), l = ceil(log2 d) (Granlund and Montgomery 1994)
struct FastDiv {
  unsigned m;
  int sh;  // l - 1, or -1 for d = 1
  __device__ __forceinline__ void init(unsigned dv) {
    if (dv <= 1) {
      m = 0;
      sh = -1;
      return;
    }
    const int l = 32 - __clz(dv - 1);
    m = (unsigned)(((1ull << (31 + l)) + dv - 1) / dv);
    sh = l - 1;
  }
  __device__ __forceinline__ unsigned div(unsigned n) const { return sh < 0 ? n : __umulhi(n, m) >> sh; }
};

// the 8 neighbours (forward, backward per direction) of eo site i of parity
// p, as eo_neighbours computes them, with the divisions by multiplications
struct TcGeom {
  FastDiv zh, y, x;
  __device__ __forceinline__ void init(const Geom& g) {
    zh.init((unsigned)g.Zh);
    y.init((unsigned)g.Y);
    x.init((unsigned)g.X);
  }
  __device__ __forceinline__ void neighbours(const Geom& g, int i, int p, int (&nb8)[8]) const {
    const int row = (int)zh.div((unsigned)i), k = i - row * g.Zh;
    const int r2 = (int)y.div((unsigned)row), yy = row - r2 * g.Y;
    const int t = (int)x.div((unsigned)r2), xx = r2 - t * g.X;
    const int z = 2 * k + ((t + xx + yy + p) & 1);
    nb8[0] = (t == g.T - 1) ? i - (g.T - 1) * g.st : i + g.st;
    nb8[1] = (t == 0) ? i + (g.T - 1) * g.st : i - g.st;
    nb8[2] = (xx == g.X - 1) ? i - (g.X - 1) * g.sx : i + g.sx;
    nb8[3] = (xx == 0) ? i + (g.X - 1) * g.sx : i - g.sx;
    nb8[4] = (yy == g.Y - 1) ? i - (g.Y - 1) * g.sy : i + g.sy;
    nb8[5] = (yy == 0) ? i + (g.Y - 1) * g.sy : i - g.sy;
    const int Z = 2 * g.Zh;
    const int zf = (z == Z - 1) ? 0 : z + 1;
    const int zb = (z == 0) ? Z - 1 : z - 1;
    nb8[6] = row * g.Zh + (zf >> 1);
    nb8[7] = row * g.Zh + (zb >> 1);
  }
};

// bf16x2 (re, im) factors: +1 = 0x3f80, -1 = 0xbf80 in each half
constexpr unsigned kPP = 0x3f803f80u, kPM = 0xbf803f80u, kMM = 0xbf80bf80u, kMP = 0x3f80bf80u;

// B-operand registers of one spin: (Re h[c], Re h[c']) and (Im h[c], Im h[c'])
struct Bfrag {
  unsigned re, im;
};

// The projected spins of one RHS for direction MU, colours c, c' of this
// lane, from the staged words w[0..3] = planes c, c', D+c, D+c', each
// (low word, high word) = (psi0, psi2) or (psi1, psi3) as bf16x2 (re, im):
//   h0 = u0 + s b0, h1 = u1 + s b1, (b0, b1) = B_mu (l0, l1)   (u = psi0,1, l = psi2,3)
// with MU = 0: (l0, l1); 1: (-i l1, -i l0); 2: (-l1, l0); 3: (-i l0, i l1);
// SM is the sign bits of s = -+1.
template <int MU, unsigned SM>
__device__ __forceinline__ void tc_project(const uint2 (&w)[4], Bfrag& b0, Bfrag& b1) {
  const unsigned l0c = w[0].y, l0d = w[1].y, l1c = w[2].y, l1d = w[3].y;
  unsigned s0c, s0d, s1c, s1d;
  constexpr unsigned f0 = (MU == 0 ? kPP : MU == 2 ? kMM : kPM) ^ SM;
  constexpr unsigned f1 = (MU == 0 || MU == 2 ? kPP : MU == 1 ? kPM : kMP) ^ SM;
  if constexpr (MU == 0) {
    s0c = l0c, s0d = l0d, s1c = l1c, s1d = l1d;
  } else if constexpr (MU == 1) {  // -i (x + iy) = y - ix: exchange re/im, then (1, -1)
    s0c = __byte_perm(l1c, 0, 0x1032), s0d = __byte_perm(l1d, 0, 0x1032);
    s1c = __byte_perm(l0c, 0, 0x1032), s1d = __byte_perm(l0d, 0, 0x1032);
  } else if constexpr (MU == 2) {
    s0c = l1c, s0d = l1d, s1c = l0c, s1d = l0d;
  } else {  // -i l0 and i l1 = (-y, x)
    s0c = __byte_perm(l0c, 0, 0x1032), s0d = __byte_perm(l0d, 0, 0x1032);
    s1c = __byte_perm(l1c, 0, 0x1032), s1d = __byte_perm(l1d, 0, 0x1032);
  }
  const unsigned h0c = hfma2(f0, s0c, w[0].x), h0d = hfma2(f0, s0d, w[1].x);
  const unsigned h1c = hfma2(f1, s1c, w[2].x), h1d = hfma2(f1, s1d, w[3].x);
  b0.re = __byte_perm(h0c, h0d, 0x5410);
  b0.im = __byte_perm(h0c, h0d, 0x7632);
  b1.re = __byte_perm(h1c, h1d, 0x5410);
  b1.im = __byte_perm(h1c, h1d, 0x7632);
}

// The lower-spin operands s q, q = B_mu^+ h: MU = 0: (h0, h1); 1: (i h1, i h0);
// 2: (h1, -h0); 3: (i h0, -i h1).  Multiplying by +-1 or +-i only flips signs
// and exchanges the real and imaginary registers, so these are exact.
template <int MU, unsigned M>
__device__ __forceinline__ void tc_lower(const Bfrag& h0, const Bfrag& h1, Bfrag& q0, Bfrag& q1) {
  constexpr unsigned N = kSign2;
  if constexpr (MU == 0) {
    q0 = {h0.re ^ M, h0.im ^ M};
    q1 = {h1.re ^ M, h1.im ^ M};
  } else if constexpr (MU == 1) {
    q0 = {h1.im ^ (N ^ M), h1.re ^ M};
    q1 = {h0.im ^ (N ^ M), h0.re ^ M};
  } else if constexpr (MU == 2) {
    q0 = {h1.re ^ M, h1.im ^ M};
    q1 = {h0.re ^ (N ^ M), h0.im ^ (N ^ M)};
  } else {
    q0 = {h0.im ^ (N ^ M), h0.re ^ M};
    q1 = {h1.im ^ M, h1.re ^ (N ^ M)};
  }
}

// A fragments of a link: lane (g, t) holds rows g, g + 8 and K columns 2t,
// 2t+1, 2t+8, 2t+9 of [[Ur, -Ui], [Ui, Ur]], i.e. colours c = t and c' = t + d/2,
// from elements e0 = U[g][c], e1 = U[g][c']; `mask` is zero for lanes whose
// columns lie outside the d x d block
__device__ __forceinline__ void tc_afrag(unsigned e0, unsigned e1, unsigned mask, unsigned (&a)[4]) {
  a[0] = __byte_perm(e0, e1, 0x5410) & mask;  // Ur
  a[1] = __byte_perm(e0, e1, 0x7632) & mask;  // Ui
  a[2] = a[1] ^ kSign2;                       // -Ui
  a[3] = a[0];                                // Ur
}

// per-lane constant offsets
template <int D, int NR>
struct TcLane {
  using L = TcLayout<D, NR>;
  unsigned rd[4];  // planes c, c', D+c, D+c' (c = t, c' = t + d/2) at RHS g; colours 0, d/2 for idle lanes
  unsigned rdh;    // to RHS 8 NGF + (g & 3) instead of g
  unsigned la;     // link element (g, c) within a site's link block; (g, c') is d/2 elements on
  unsigned amask;
  unsigned src[L::per_lane];  // cp.async piece k of a site's block (bytes from its start)
  unsigned dst[L::per_lane];
  __device__ __forceinline__ void init(int lane) {
#pragma unroll
    for (int k = 0; k < L::per_lane; ++k) {
      const int cc = min(lane + 32 * k, L::chunks - 1);
      const int plane = cc / L::row_chunks, w = cc % L::row_chunks;
      src[k] = (unsigned)cc * 16;  // the site's block is contiguous
      dst[k] = (unsigned)(plane * L::pitch + w * 16);
    }
    const int g = lane >> 2, t = lane & 3;
    const int c = t < D / 2 ? t : 0;
    const int planes[4] = {c, c + D / 2, D + c, D + c + D / 2};
#pragma unroll
    for (int m = 0; m < 4; ++m) rd[m] = (unsigned)(planes[m] * L::pitch + g * 8);
    rdh = (unsigned)(8 * (8 * L::NGF + (g & 3)) - 8 * g);
    la = (unsigned)((min(g, D - 1) * D + c) * 8);
    amask = t < D / 2 ? ~0u : 0u;
  }
};

// one direction-sense (MU, FB) of the warp's current site from its stage
template <int MU, int FB, bool DAG, int D, int NR>
__device__ __forceinline__ void tc_item(unsigned stage, unsigned lsite, const TcLane<D, NR>& ln, unsigned (&abwd)[4],
                                        float (&cu)[NR / 4][4], float (&cl)[NR / 4][4], int g) {
  using L = TcLayout<D, NR>;
  // sg = -1 (+1 for the adjoint) on forward senses, -sg on backward ones
  constexpr unsigned SM = ((DAG ? 0u : kSign2) ^ (FB ? kSign2 : 0u));
  unsigned a[4];
  if constexpr (FB == 0) {
    const uint2 v0 = lds64(lsite + ln.la + MU * D * D * 8);            // (fwd, bwd) of U[g][c]
    const uint2 v1 = lds64(lsite + ln.la + (MU * D * D + D / 2) * 8);  // and of U[g][c + d/2]
    tc_afrag(v0.x, v1.x, ln.amask, a);
    tc_afrag(v0.y, v1.y, ln.amask, abwd);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = abwd[q];
  }
#pragma unroll
  for (int k = 0; k < L::NGF; ++k) {
    uint2 w[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) w[m] = lds64(stage + ln.rd[m] + 64 * k);
    Bfrag h0, h1, q0, q1;
    tc_project<MU, SM>(w, h0, h1);
    tc_lower<MU, SM>(h0, h1, q0, q1);
    mma_bf16(cu[2 * k], a, h0.re, h0.im);
    mma_bf16(cu[2 * k + 1], a, h1.re, h1.im);
    mma_bf16(cl[2 * k], a, q0.re, q0.im);
    mma_bf16(cl[2 * k + 1], a, q1.re, q1.im);
  }
  if constexpr (L::HALF) {
    uint2 w[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) w[m] = lds64(stage + ln.rd[m] + ln.rdh);
    Bfrag h0, h1, q0, q1;
    tc_project<MU, SM>(w, h0, h1);
    tc_lower<MU, SM>(h0, h1, q0, q1);
    const bool s1 = g >= 4;  // this lane's column holds spin 1
    mma_bf16(cu[2 * L::NGF], a, s1 ? h1.re : h0.re, s1 ? h1.im : h0.im);
    mma_bf16(cl[2 * L::NGF], a, s1 ? q1.re : q0.re, s1 ? q1.im : q0.im);
  }
}

// output words of one lane: plane, RHS r and r + 1, from upper (spin s) and
// lower (spin s + 2) accumulators -> (psi_s, psi_s+2) pairs, optionally
// a x + b W with x from the staged same-site block
__device__ __forceinline__ void tc_store(const MrhsArgs& A, char* out, size_t off, bool with_x, unsigned xs,
                                         const float (&u)[4], const float (&l)[4]) {
  float v[8] = {u[0], u[2], l[0], l[2], u[1], u[3], l[1], l[3]};  // (re, im) of psi_s(r), psi_s+2(r), ... r + 1
  if (with_x) {
    const uint4 xv = lds128(xs);
    const unsigned xw[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = bf2_to_f2(xw[q]);
      v[2 * q] = fmaf(A.af, f.x, A.bf * v[2 * q]);
      v[2 * q + 1] = fmaf(A.af, f.y, A.bf * v[2 * q + 1]);
    }
  } else if (!A.b_one) {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] *= A.bf;
  }
  *reinterpret_cast<uint4*>(out + off) =
      make_uint4(f2_to_bf2(v[0], v[1]), f2_to_bf2(v[2], v[3]), f2_to_bf2(v[4], v[5]), f2_to_bf2(v[6], v[7]));
}

template <int D, int NR, bool DAG>
__global__ void __launch_bounds__(32 * kTcWarps, kTcBlocksPerSm) hop_mrhs_tc_kernel(const MrhsArgs A) {
  using L = TcLayout<D, NR>;
  constexpr int S = L::S;
  extern __shared__ __align__(128) unsigned char tc_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int Vh = A.g.Vh;
  const int nq = (Vh + kTcWarps - 1) / kTcWarps;  // quads of consecutive sites
  int q = blockIdx.x;
  if (q >= nq) return;  // uniform over the block, before any barrier

  const unsigned base = (unsigned)__cvta_generic_to_shared(tc_smem);
  const unsigned ring = base + warp * L::warp_bytes;
  const unsigned xbuf = ring + S * L::spin_bytes;
  const unsigned links = base + L::links_off;
  TcLane<D, NR> ln;
  ln.init(lane);
  TcGeom geo;
  geo.init(A.g);
  __syncthreads();

  const bool with_x = A.x != nullptr;
  char* out = static_cast<char*>(A.out);
  const char* in = static_cast<const char*>(A.in);
  const char* xin = static_cast<const char*>(A.x);

  // the links of quad qq (sites 4 qq .. 4 qq + 3, one link tile) into buffer b
  auto fetch_links = [&](int qq, int b) {
    const uint2* lt = LinkIO<BF16, D, false>::tile_ptr(A.links, kTcWarps * qq);
    for (int idx = threadIdx.x; idx < L::link_elems; idx += 32 * kTcWarps) {
      const int s = (idx >> 3) & 3, P = ((idx >> 5) << 3) | (idx & 7);
      if (kTcWarps * qq + s < Vh)
        cp_async8_ca(links + b * L::link_buf + s * L::link_site + P * 8, lt + (size_t)P * kLinkTile + s);
    }
  };

  int site = kTcWarps * q + warp;
  int nb8[8];
  // Every step commits one cp.async group (its item's pieces; at step 0 also
  // the next quad's links, at step 1 the site's x block), so the group of
  // item j is complete once at most S - 2 newer groups are pending.
  auto issue = [&](unsigned st, const char* field, int n) {  // site n's block of `field` into st
    const char* src = field + (size_t)(unsigned)n * L::block_src;
#pragma unroll
    for (int c = 0; c < L::per_lane; ++c)
      if (L::chunks % 32 == 0 || lane + 32 * c < L::chunks) cp_async16_cg(st + ln.dst[c], src + ln.src[c]);
  };
  fetch_links(q, 0);
  if (site < Vh) geo.neighbours(A.g, site, A.p, nb8);
#pragma unroll
  for (int j = 0; j < S - 2; ++j) {
    if (site < Vh) issue(ring + j * L::spin_bytes, in, nb8[j]);
    cp_commit();
  }

  for (int k = 0; q < nq; ++k) {
    const int qn = q + gridDim.x;
    const int next = kTcWarps * qn + warp;
    const bool active = site < Vh, next_active = qn < nq && next < Vh;
    // quad q's links: in the prologue's groups (k = 0) or in step 0's group of
    // the previous iteration, seven groups back
    if (k == 0) cp_wait<0>();
    else cp_wait<7>();
    __syncthreads();  // the links are in buffer k & 1 for every warp; buffer (k + 1) & 1 is free
    const unsigned lsite = links + (k & 1) * L::link_buf + warp * L::link_site;

    if (active) {
      float cu[L::NT][4], cl[L::NT][4];
#pragma unroll
      for (int j = 0; j < L::NT; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) cu[j][c] = cl[j][c] = 0.f;
      unsigned abwd[4];
      auto step = [&](auto ds_c) {
        constexpr int ds = decltype(ds_c)::value;
        constexpr int fj = ds + S - 2;  // item to copy: the next site's from fj = 8 on
        constexpr int fds = fj % 8;
        if constexpr (ds == 10 - S) {  // the current site's last copy went out in the step before
          if (next_active) geo.neighbours(A.g, next, A.p, nb8);
        }
        if (fj < 8 || next_active) issue(ring + (fj % S) * L::spin_bytes, in, nb8[fds]);
        if constexpr (ds == 0) {
          if (qn < nq) fetch_links(qn, (k + 1) & 1);
        }
        if constexpr (ds == 1) {  // this site's own input for a x + b H, read in the epilogue
          if (with_x) issue(xbuf, xin, site);
        }
        cp_commit();
        cp_wait<S - 2>();  // this lane's pieces of item ds
        __syncwarp();      // every lane's pieces of item ds are visible; the stage read two steps ago is free
        tc_item<ds / 2, ds % 2, DAG, D, NR>(ring + (ds % S) * L::spin_bytes, lsite, ln, abwd, cu, cl, g);
      };
      step(std::integral_constant<int, 0>{});
      step(std::integral_constant<int, 1>{});
      step(std::integral_constant<int, 2>{});
      step(std::integral_constant<int, 3>{});
      step(std::integral_constant<int, 4>{});
      step(std::integral_constant<int, 5>{});
      step(std::integral_constant<int, 6>{});
      step(std::integral_constant<int, 7>{});

      // epilogue: lane (g, t) holds colour g (rows g, g + 8) of columns 2t, 2t+1 of every tile
      if (g < D) {
#pragma unroll
        for (int kk = 0; kk < L::NGF; ++kk) {
          const int r = 8 * kk + 2 * t;
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const int plane = s * D + g;
            const size_t off = (size_t)(unsigned)site * L::block_src + (size_t)(plane * NR + r) * 8;
            const unsigned xs = xbuf + (unsigned)(plane * L::pitch + r * 8);
            tc_store(A, out, off, with_x, xs, cu[2 * kk + s], cl[2 * kk + s]);
          }
        }
        if constexpr (L::HALF) {
          const int r = 8 * L::NGF + 2 * (t & 1), plane = (t >> 1) * D + g;
          const size_t off = (size_t)(unsigned)site * L::block_src + (size_t)(plane * NR + r) * 8;
          const unsigned xs = xbuf + (unsigned)(plane * L::pitch + r * 8);
          tc_store(A, out, off, with_x, xs, cu[2 * L::NGF], cl[2 * L::NGF]);
        }
      }
      __syncwarp();  // the x block and the stages are read before later copies refill them
    }
    q = qn;
    site = next;
  }
  cp_wait<0>();
}

// launch shape per device: the shared-memory opt-in and the occupancy are
// per device, so they are set up once for each device the kernel runs on
constexpr int kTcMaxDevices = 64;

template <int D, int NR, bool DAG>
bool launch_tc_dag(const MrhsArgs& A, cudaStream_t s) {
  using L = TcLayout<D, NR>;
  const size_t smem = (size_t)L::block_bytes;
  static int grid_cap[kTcMaxDevices];  // SMs x resident blocks, 0 until set up
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTcMaxDevices) return false;
  if (grid_cap[dev] == 0) {
    if (smem > 48 * 1024 && cudaFuncSetAttribute(hop_mrhs_tc_kernel<D, NR, DAG>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return false;
    int sms = 0, b = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return false;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, hop_mrhs_tc_kernel<D, NR, DAG>, 32 * kTcWarps, smem) !=
            cudaSuccess ||
        b <= 0)
      return false;
    grid_cap[dev] = sms * b;
  }
  const int nq = (A.g.Vh + kTcWarps - 1) / kTcWarps;
  hop_mrhs_tc_kernel<D, NR, DAG><<<std::min(nq, grid_cap[dev]), 32 * kTcWarps, smem, s>>>(with_f32_scalars(A));
  return true;
}

template <int D, int NR>
bool launch_tc_t(const MrhsArgs& A, cudaStream_t s) {
  return A.dagger ? launch_tc_dag<D, NR, true>(A, s) : launch_tc_dag<D, NR, false>(A, s);
}

template <int D>
bool launch_tc_nt(const MrhsArgs& A, cudaStream_t s) {
  switch (A.nrhs) {
    case 4: return launch_tc_t<D, 4>(A, s);
    case 8: return launch_tc_t<D, 8>(A, s);
    case 12: return launch_tc_t<D, 12>(A, s);
    case 16: return launch_tc_t<D, 16>(A, s);
    default: return false;
  }
}

}  // namespace

// tensor-core path: BF16 storage, complex representation, d in {4, 6, 8},
// n_rhs in {4, 8, 12, 16}; false when it does not apply
bool launch_mrhs_tc(int prec, int d, bool real, const MrhsArgs& A, cudaStream_t s) {
  if (prec != BSM_BF16 || real) return false;
  switch (d) {
    case 4: return launch_tc_nt<4>(A, s);
    case 6: return launch_tc_nt<6>(A, s);
    case 8: return launch_tc_nt<8>(A, s);
    default: return false;
  }
}

}  // namespace bsm
