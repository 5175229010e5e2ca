// bsm_internal.cuh -- shared device-side building blocks of the GB300 library:
// complex arithmetic, precision policies, the device field layouts declared
// in include/bsm.h, and the even-odd lattice geometry (Sec. II-A).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bsm.h"
#include "df64.cuh"

namespace bsm {

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <typename R>
struct cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ cx<R> cmake(R re, R im) {
  cx<R> c;
  c.re = re;
  c.im = im;
  return c;
}

// w += u * h (4 fused multiply-adds)
template <typename R>
__device__ __forceinline__ void cmac(cx<R>& w, const cx<R>& u, const cx<R>& h) {
  w.re = fma(u.re, h.re, w.re);
  w.re = fma(-u.im, h.im, w.re);
  w.im = fma(u.re, h.im, w.im);
  w.im = fma(u.im, h.re, w.im);
}

// w += u * h for a real u
template <typename R>
__device__ __forceinline__ void rmac(cx<R>& w, R u, const cx<R>& h) {
  w.re = fma(u, h.re, w.re);
  w.im = fma(u, h.im, w.im);
}

// ---------------------------------------------------------------------------
// precision policies
// ---------------------------------------------------------------------------
struct F64 {
  using R = double;
  static constexpr int prec = BSM_F64;
};
struct F32 {
  using R = float;
  static constexpr int prec = BSM_F32;
};
struct DF64 {
  using R = df;
  static constexpr int prec = BSM_DF64;
};
// bfloat16 storage, FP32 arithmetic
struct BF16 {
  using R = float;
  static constexpr int prec = BSM_BF16;
};
// FP32 with SU(3) links stored as their first two rows (third rebuilt)
struct F32R12 {
  using R = float;
  static constexpr int prec = BSM_F32R12;
};

// bytes per real number of a precision (DF64 stores two floats)
inline size_t real_bytes(int prec) {
  return (prec == BSM_F32 || prec == BSM_F32R12) ? 4 : prec == BSM_BF16 ? 2 : 8;
}
// precision of the vectors (spinors) that go with links at `prec`
__host__ __device__ inline int vector_prec(int prec) { return prec == BSM_F32R12 ? BSM_F32 : prec; }

// load through L1 (data shared by several threads) or with the streaming hint
template <bool L1, typename T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (L1) return __ldg(p);
  else return __ldcs(p);
}
__device__ __forceinline__ float2 bf2_to_f2(unsigned int v) {
  __nv_bfloat162 b;
  memcpy(&b, &v, 4);
  return __bfloat1622float2(b);
}
__device__ __forceinline__ unsigned int f2_to_bf2(float x, float y) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(x, y);
  unsigned int v;
  memcpy(&v, &b, 4);
  return v;
}

// bytes of one parity block of a spinor with d colours
inline size_t half_spinor_bytes(int64_t Vh, int d, int prec) { return (size_t)Vh * 8 * d * real_bytes(prec); }
// Links are tiled: the sites of one parity are grouped in tiles of
// kLinkTile consecutive eo indices, and a tile stores all its link planes
// contiguously ([tile][plane][kLinkTile]), so a warp reads its 8 links per
// site from one contiguous region.  V_h is padded up to a whole tile.
constexpr int kLinkTile = 32;
inline size_t padded_sites(int64_t Vh) { return (size_t)((Vh + kLinkTile - 1) / kLinkTile) * kLinkTile; }
// bytes of the links of one output parity
inline size_t link_block_bytes(int64_t Vh, int d, bool real, int prec) {
  if (prec == BSM_F32R12) return padded_sites(Vh) * 8 * 12 * 4;  // two rows of SU(3): 12 floats per link
  return padded_sites(Vh) * 8 * d * d * real_bytes(prec) * (real ? 1 : 2);
}
// element offset of (plane, site i) in a tiled link block of `planes` planes
__host__ __device__ __forceinline__ size_t link_index(int planes, int plane, int i) {
  return ((size_t)(i / kLinkTile) * planes + plane) * kLinkTile + (i % kLinkTile);
}

// ---------------------------------------------------------------------------
// even-odd geometry: dims {T, X, Y, Z}, Z even; a site of parity p with index
// i in its parity block has z = 2k + ((t+x+y+p) & 1), i = ((t*X+x)*Y+y)*Z/2 + k
// ---------------------------------------------------------------------------
struct Geom {
  int T, X, Y, Zh;   // Zh = Z/2
  int sy, sx, st;    // eo-index strides of a step in y, x, t
  int Vh;
};

inline Geom make_geom(const bsm_lattice& L) {
  Geom g;
  g.T = L.dims[0];
  g.X = L.dims[1];
  g.Y = L.dims[2];
  g.Zh = L.dims[3] / 2;
  g.sy = g.Zh;
  g.sx = g.Y * g.Zh;
  g.st = g.X * g.Y * g.Zh;
  g.Vh = g.T * g.st;
  return g;
}

// indices (in the other parity block) of the 8 neighbours of eo site i of
// parity p: nf[mu] = x + mu, nb[mu] = x - mu
__device__ __forceinline__ void eo_neighbours(const Geom& g, int i, int p, int nf[4], int nb[4]) {
  const int k = i % g.Zh;
  const int row = i / g.Zh;
  const int y = row % g.Y;
  const int r2 = row / g.Y;
  const int x = r2 % g.X;
  const int t = r2 / g.X;
  const int z = 2 * k + ((t + x + y + p) & 1);
  nf[0] = (t == g.T - 1) ? i - (g.T - 1) * g.st : i + g.st;
  nb[0] = (t == 0) ? i + (g.T - 1) * g.st : i - g.st;
  nf[1] = (x == g.X - 1) ? i - (g.X - 1) * g.sx : i + g.sx;
  nb[1] = (x == 0) ? i + (g.X - 1) * g.sx : i - g.sx;
  nf[2] = (y == g.Y - 1) ? i - (g.Y - 1) * g.sy : i + g.sy;
  nb[2] = (y == 0) ? i + (g.Y - 1) * g.sy : i - g.sy;
  const int Z = 2 * g.Zh;
  const int zf = (z == Z - 1) ? 0 : z + 1;
  const int zb = (z == 0) ? Z - 1 : z - 1;
  nf[3] = row * g.Zh + (zf >> 1);
  nb[3] = row * g.Zh + (zb >> 1);
}

// boundary crossings of eo site i of parity p: bit mu set when its forward
// neighbour wraps (x_mu = L_mu - 1), bit 4 + mu when its backward one does (x_mu = 0)
__device__ __forceinline__ unsigned eo_edges(const Geom& g, int i, int p) {
  const int k = i % g.Zh;
  const int row = i / g.Zh;
  const int y = row % g.Y;
  const int r2 = row / g.Y;
  const int x = r2 % g.X;
  const int t = r2 / g.X;
  const int z = 2 * k + ((t + x + y + p) & 1);
  const int c[4] = {t, x, y, z}, L[4] = {g.T, g.X, g.Y, 2 * g.Zh};
  unsigned m = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    if (c[mu] == L[mu] - 1) m |= 1u << mu;
    if (c[mu] == 0) m |= 1u << (4 + mu);
  }
  return m;
}

// ---------------------------------------------------------------------------
// spinor layout access
// ---------------------------------------------------------------------------
template <typename P, int D>
struct SpinorIO;

template <int D>
struct SpinorIO<F64, D> {
  // 4D planes of double2, plane = spin*D + colour
  __device__ __forceinline__ static void load(const void* base, size_t Vh, int i, cx<double> (&s)[4][D]) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const double2 v = __ldg(b + (size_t)(sp * D + a) * Vh + i);
        s[sp][a] = cmake(v.x, v.y);
      }
  }
  __device__ __forceinline__ static void store(void* base, size_t Vh, int i, const cx<double> (&s)[4][D]) {
    double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a) b[(size_t)(sp * D + a) * Vh + i] = make_double2(s[sp][a].re, s[sp][a].im);
  }
};

template <int D>
struct SpinorIO<F32, D>;
template <int D>
struct SpinorIO<F32R12, D>;

template <int D>
struct SpinorIO<F32, D> {
  // 2D planes of float4, plane = s*D + colour, (psi[s][c], psi[s+2][c]).
  // L2ONLY loads bypass L1 (for data written earlier in the same kernel).
  template <bool L2ONLY = false>
  __device__ __forceinline__ static void load(const void* base, size_t Vh, int i, cx<float> (&s)[4][D]) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const float4* q = b + (size_t)(sp * D + a) * Vh + i;
        const float4 v = L2ONLY ? __ldcg(q) : __ldg(q);
        s[sp][a] = cmake(v.x, v.y);
        s[sp + 2][a] = cmake(v.z, v.w);
      }
  }
  __device__ __forceinline__ static void store(void* base, size_t Vh, int i, const cx<float> (&s)[4][D]) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a)
        b[(size_t)(sp * D + a) * Vh + i] = make_float4(s[sp][a].re, s[sp][a].im, s[sp + 2][a].re, s[sp + 2][a].im);
  }
};

// F32R12 stores its spinors exactly as F32 does
template <int D>
struct SpinorIO<F32R12, D> : SpinorIO<F32, D> {};

template <int D>
struct SpinorIO<BF16, D> {
  // as FP32 with bfloat16 values: 2D planes of uint2 = (psi[s][c], psi[s+2][c])
  __device__ __forceinline__ static void load(const void* base, size_t Vh, int i, cx<float> (&s)[4][D]) {
    const uint2* b = reinterpret_cast<const uint2*>(base);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const uint2 v = __ldg(b + (size_t)(sp * D + a) * Vh + i);
        const float2 u = bf2_to_f2(v.x), l = bf2_to_f2(v.y);
        s[sp][a] = cmake(u.x, u.y);
        s[sp + 2][a] = cmake(l.x, l.y);
      }
  }
  __device__ __forceinline__ static void store(void* base, size_t Vh, int i, const cx<float> (&s)[4][D]) {
    uint2* b = reinterpret_cast<uint2*>(base);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a)
        b[(size_t)(sp * D + a) * Vh + i] =
            make_uint2(f2_to_bf2(s[sp][a].re, s[sp][a].im), f2_to_bf2(s[sp + 2][a].re, s[sp + 2][a].im));
  }
};

template <int D>
struct SpinorIO<DF64, D> {
  // 4D planes of float4 (re.hi, re.lo, im.hi, im.lo), plane = spin*D + colour
  __device__ __forceinline__ static void load(const void* base, size_t Vh, int i, cx<df> (&s)[4][D]) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const float4 v = __ldg(b + (size_t)(sp * D + a) * Vh + i);
        s[sp][a] = cmake(df(v.x, v.y), df(v.z, v.w));
      }
  }
  __device__ __forceinline__ static void store(void* base, size_t Vh, int i, const cx<df> (&s)[4][D]) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const df re = df_norm(s[sp][a].re), im = df_norm(s[sp][a].im);
        b[(size_t)(sp * D + a) * Vh + i] = make_float4(re.hi, re.lo, im.hi, im.lo);
      }
  }
};

// ---------------------------------------------------------------------------
// link layout access: forward link U(x) and backward link U(x-mu)^+ of
// direction mu, element c, for the thread's site.  `tile` points at the
// site's column of its tile (tile_ptr); planes are kLinkTile elements apart.
// ---------------------------------------------------------------------------
template <typename P, int D, bool REAL>
struct LinkIO;

template <int D>
struct LinkIO<F64, D, false> {
  using elem = cx<double>;
  using vec = double2;
  static constexpr int planes = 8 * D * D;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  __device__ __forceinline__ static void load(const vec* t, int mu, int c, elem& f, elem& b) {
    const double2 vf = __ldcs(t + ((2 * mu) * D * D + c) * kLinkTile);
    const double2 vb = __ldcs(t + ((2 * mu + 1) * D * D + c) * kLinkTile);
    f = cmake(vf.x, vf.y);
    b = cmake(vb.x, vb.y);
  }
  template <int FB, bool L1 = false>
  __device__ __forceinline__ static elem load_one(const vec* t, int mu, int c) {
    const double2 v = ldx<L1>(t + ((2 * mu + FB) * D * D + c) * kLinkTile);
    return cmake(v.x, v.y);
  }
};

template <int D>
struct LinkIO<F32, D, false> {
  using elem = cx<float>;
  using vec = float4;
  static constexpr int planes = 4 * D * D;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  __device__ __forceinline__ static void load(const vec* t, int mu, int c, elem& f, elem& b) {
    const float4 v = __ldcs(t + (mu * D * D + c) * kLinkTile);
    f = cmake(v.x, v.y);
    b = cmake(v.z, v.w);
  }
  template <int FB, bool L1 = false>
  __device__ __forceinline__ static elem load_one(const vec* t, int mu, int c) {
    const float4 v = ldx<L1>(t + (mu * D * D + c) * kLinkTile);
    return FB == 0 ? cmake(v.x, v.y) : cmake(v.z, v.w);
  }
};

template <int D>
struct LinkIO<F64, D, true> {
  using elem = double;
  using vec = double2;
  static constexpr int planes = 4 * D * D;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  __device__ __forceinline__ static void load(const vec* t, int mu, int c, elem& f, elem& b) {
    const double2 v = __ldcs(t + (mu * D * D + c) * kLinkTile);
    f = v.x;
    b = v.y;
  }
  template <int FB, bool L1 = false>
  __device__ __forceinline__ static elem load_one(const vec* t, int mu, int c) {
    const double2 v = ldx<L1>(t + (mu * D * D + c) * kLinkTile);
    return FB == 0 ? v.x : v.y;
  }
};

template <int D>
struct LinkIO<F32, D, true> {
  using elem = float;
  using vec = float2;
  static constexpr int planes = 4 * D * D;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  __device__ __forceinline__ static void load(const vec* t, int mu, int c, elem& f, elem& b) {
    const float2 v = __ldcs(t + (mu * D * D + c) * kLinkTile);
    f = v.x;
    b = v.y;
  }
  template <int FB, bool L1 = false>
  __device__ __forceinline__ static elem load_one(const vec* t, int mu, int c) {
    const float2 v = ldx<L1>(t + (mu * D * D + c) * kLinkTile);
    return FB == 0 ? v.x : v.y;
  }
};

// SU(3) links as two rows (12 floats = 3 float4 per link): plane
// mu * 6 + fb * 3 + q holds elements 2q, 2q + 1 of the row-major first two
// rows of the forward (fb = 0) or backward (fb = 1) link.  The third row of
// an SU(3) matrix is the complex conjugate of the cross product of the first
// two; a link multiplied by the boundary phase c needs the factor c^3 (c*^3
// for the stored backward link U^+) on it.
template <int D, bool REAL>
struct LinkIO<F32R12, D, REAL> {
  static_assert(D == 3 && !REAL, "two-row links are SU(3) fundamental only");
  using vec = float4;
  static constexpr int planes = 24;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  // the full matrix of sense FB of direction mu; ph = the third row's phase factor
  template <int FB>
  __device__ __forceinline__ static void load_matrix(const vec* t, int mu, cx<float> ph, cx<float> (&U)[3][3]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 v = __ldcs(t + (mu * 6 + FB * 3 + q) * kLinkTile);
      U[(2 * q) / 3][(2 * q) % 3] = cmake(v.x, v.y);
      U[(2 * q + 1) / 3][(2 * q + 1) % 3] = cmake(v.z, v.w);
    }
    // row 2 = ph * conj(row 0 x row 1)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a = (c + 1) % 3, b = (c + 2) % 3;
      const cx<float> p = U[0][a], q = U[1][b], r = U[0][b], u = U[1][a];
      // x = p q - r u, then w = conj(x)
      const float xr = fmaf(p.re, q.re, fmaf(-p.im, q.im, fmaf(-r.re, u.re, r.im * u.im)));
      const float xi = fmaf(p.re, q.im, fmaf(p.im, q.re, fmaf(-r.re, u.im, -(r.im * u.re))));
      U[2][c] = cmake(fmaf(ph.re, xr, ph.im * xi), fmaf(ph.im, xr, -(ph.re * xi)));
    }
  }
};

template <int D>
struct LinkIO<DF64, D, false> {
  using elem = cx<df>;
  using vec = float4;
  static constexpr int planes = 8 * D * D;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  __device__ __forceinline__ static void load(const vec* t, int mu, int c, elem& f, elem& b) {
    const float4 vf = __ldcs(t + ((2 * mu) * D * D + c) * kLinkTile);
    const float4 vb = __ldcs(t + ((2 * mu + 1) * D * D + c) * kLinkTile);
    f = cmake(df(vf.x, vf.y), df(vf.z, vf.w));
    b = cmake(df(vb.x, vb.y), df(vb.z, vb.w));
  }
  template <int FB, bool L1 = false>
  __device__ __forceinline__ static elem load_one(const vec* t, int mu, int c) {
    const float4 v = ldx<L1>(t + ((2 * mu + FB) * D * D + c) * kLinkTile);
    return cmake(df(v.x, v.y), df(v.z, v.w));
  }
};

template <int D>
struct LinkIO<DF64, D, true> {
  using elem = df;
  using vec = float4;
  static constexpr int planes = 4 * D * D;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  __device__ __forceinline__ static void load(const vec* t, int mu, int c, elem& f, elem& b) {
    const float4 v = __ldcs(t + (mu * D * D + c) * kLinkTile);
    f = df(v.x, v.y);
    b = df(v.z, v.w);
  }
  template <int FB, bool L1 = false>
  __device__ __forceinline__ static elem load_one(const vec* t, int mu, int c) {
    const float4 v = ldx<L1>(t + (mu * D * D + c) * kLinkTile);
    return FB == 0 ? df(v.x, v.y) : df(v.z, v.w);
  }
};

template <int D>
struct LinkIO<BF16, D, false> {
  using elem = cx<float>;
  using vec = uint2;  // (forward re/im, backward re/im) as two bfloat16 pairs
  static constexpr int planes = 4 * D * D;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  __device__ __forceinline__ static void load(const vec* t, int mu, int c, elem& f, elem& b) {
    const uint2 v = __ldcs(t + (mu * D * D + c) * kLinkTile);
    const float2 x = bf2_to_f2(v.x), y = bf2_to_f2(v.y);
    f = cmake(x.x, x.y);
    b = cmake(y.x, y.y);
  }
  template <int FB, bool L1 = false>
  __device__ __forceinline__ static elem load_one(const vec* t, int mu, int c) {
    const uint2 v = ldx<L1>(t + (mu * D * D + c) * kLinkTile);
    const float2 x = bf2_to_f2(FB == 0 ? v.x : v.y);
    return cmake(x.x, x.y);
  }
};

template <int D>
struct LinkIO<BF16, D, true> {
  using elem = float;
  using vec = unsigned int;  // (forward, backward) bfloat16 pair
  static constexpr int planes = 4 * D * D;
  __device__ __forceinline__ static const vec* tile_ptr(const void* base, int i) {
    return reinterpret_cast<const vec*>(base) + link_index(planes, 0, i);
  }
  __device__ __forceinline__ static void load(const vec* t, int mu, int c, elem& f, elem& b) {
    const float2 x = bf2_to_f2(__ldcs(t + (mu * D * D + c) * kLinkTile));
    f = x.x;
    b = x.y;
  }
  template <int FB, bool L1 = false>
  __device__ __forceinline__ static elem load_one(const vec* t, int mu, int c) {
    const float2 x = bf2_to_f2(ldx<L1>(t + (mu * D * D + c) * kLinkTile));
    return FB == 0 ? x.x : x.y;
  }
};

// ---------------------------------------------------------------------------
// block reductions -> one FP64 partial per block, in a fixed order (so the
// sum is deterministic for a fixed launch shape).  Every thread of the block
// must reach them.  GB300 issues an FP64 warp instruction only every ~16
// cycles per SM, so the cost of a reduction is counted in FP64 warp
// instructions:
//  - block_sum_store: a shuffle tree in every warp, then one warp over the
//    per-warp sums (5 (W + 1) FP64 adds for W warps, W doubles of shared
//    memory); for kernels whose own FP64 work dwarfs it;
//  - block_sum_store_wide: the values go to shared memory and one warp adds
//    them (W - 1 + 5 adds, THREADS doubles of shared memory); for short
//    memory-bound vector kernels;
//  - block_sums_store_f32 (below): FP32 shuffle trees, then W FP64 adds per
//    value; for kernels whose per-thread sums are FP32.
// ---------------------------------------------------------------------------
template <int THREADS>
__device__ __forceinline__ void block_sum_store(double v, double* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ double warp_sums[THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_sums[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < THREADS / 32 ? warp_sums[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[blockIdx.x] = s;
  }
}

template <int THREADS>
__device__ __forceinline__ void block_sum_store_wide(double v, double* out) {
  __shared__ double buf[THREADS];
  buf[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = buf[threadIdx.x];
#pragma unroll
    for (int k = threadIdx.x + 32; k < THREADS; k += 32) s += buf[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
  }
  __syncthreads();  // buf may be reused by the next call
}

// NV FP32 accumulators per thread -> NV FP64 block partials at
// out[j * stride + blockIdx.x]: FP32 shuffle trees within each warp, then
// the per-warp sums added in FP64 by NV threads (for FP32 vector kernels,
// whose per-thread sums are FP32 already)
template <int THREADS, int NV>
__device__ __forceinline__ void block_sums_store_f32(float (&v)[NV], double* out, size_t stride) {
  constexpr int W = THREADS / 32;
  __shared__ double buf[NV][W];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) buf[j][threadIdx.x >> 5] = (double)x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < W; ++w) s += buf[threadIdx.x][w];
    out[threadIdx.x * stride + blockIdx.x] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// host-side helpers shared by the translation units
// ---------------------------------------------------------------------------
struct RepInfo {
  int d;
  bool real;
};
// d and realness of a supported (N, rep); d < 0 if unsupported
RepInfo rep_info(int N, int rep);

// parameters of one hop launch (Sec. II-B hopping block H_{p,1-p})
struct HopArgs {
  const void* links;   // link block of output parity p
  const void* in;      // half spinor of parity 1-p
  void* out;           // half spinor of parity p
  const void* x;       // optional same-parity input: out = a*x + b*H in
  double a, b;
  double* partials;    // optional per-block partial sums of |out|^2
  const int* done;     // optional early-exit flag (CG): skip when *done != 0
  Geom g;
  int p;               // output parity
  int dagger;          // apply H^+ = g5 H g5
  float ph3[4][2];     // (cos, sin) of 3 phi_mu: two-row links' boundary factor
  float af, bf;        // a, b rounded to FP32, and b == 1 (set at launch: FP32
  int b_one;           // kernels avoid per-thread FP64 conversions and compares)
  // fused CG step (FP32 vectors; cg_r != nullptr): out is not written, the
  // epilogue does r -= alpha out, x += alpha p with alpha = *cg_alpha
  void* cg_r;
  void* cg_x;
  const void* cg_p;
  const float* cg_alpha;
};

// the epilogue scalars at the kernel's arithmetic precision: FP32 kernels
// take the FP32 copies (GB300 issues FP64 instructions at a small fraction
// of the FP32 rate, so a per-thread FP64 convert or compare is not free)
template <typename R, typename Args>
__device__ __forceinline__ R epi_a(const Args& A) { return (R)A.a; }
template <typename R, typename Args>
__device__ __forceinline__ R epi_b(const Args& A) { return (R)A.b; }
template <>
__device__ __forceinline__ float epi_a<float, HopArgs>(const HopArgs& A) { return A.af; }
template <>
__device__ __forceinline__ float epi_b<float, HopArgs>(const HopArgs& A) { return A.bf; }

template <typename Args>
inline Args with_f32_scalars(Args A) {
  A.af = (float)A.a;
  A.bf = (float)A.b;
  A.b_one = A.b == 1.0;
  return A;
}

// launch the hop for (prec, d, real); returns the number of blocks (the
// number of partials written when args.partials != nullptr), or -1
int launch_hop(int prec, int d, bool real, const HopArgs& args, cudaStream_t s);

constexpr int kHopThreads = 128;
inline int hop_blocks(int Vh) { return (Vh + kHopThreads - 1) / kHopThreads; }
// block partials written by one DF64 hop launch (its staged kernel runs
// smaller blocks than kHopThreads)
int hop_partials_df64(int Vh);
// the most block partials one hop launch of any precision writes
inline int hop_partials_max(int Vh) { return hop_blocks(Vh) > hop_partials_df64(Vh) ? hop_blocks(Vh) : hop_partials_df64(Vh); }

void set_cuda_error(cudaError_t e);

// argument checks shared by the entry points (defined in api.cu): every
// field of the lattice (BSM_OK, BSM_EINVAL or BSM_EUNSUPPORTED); precisions
// a lattice's operators accept; 16-byte alignment; intersecting byte ranges
int check_lattice(const bsm_lattice* L);
bool prec_lat_ok(const bsm_lattice* L, int prec);
bool aligned(const void* p);
bool overlap(const void* a, size_t na, const void* b, size_t nb);

}  // namespace bsm
