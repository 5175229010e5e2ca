// mrhs_tc.cu -- multi-RHS hopping block on the tensor cores (BF16 storage,
// FP32 accumulation) for the larger colour dimensions d = 4, 6, 8.
//
// For one site and one of its 8 direction-senses the hop is a small dense
// contraction: W = U h, with U the d x d link and h the d x (2 spins x n_rhs)
// block of spin-projected neighbour spinors.  In real form
//     [Wr; Wi] = [[Ur, -Ui], [Ui, Ur]] [hr; hi]
// is an M = K = 2d (padded to 16), N = 2 n_rhs GEMM, i.e. one
// mma.sync.m16n8k16 (bf16 x bf16 -> f32) per 8 columns.  The lower spin
// components of the term are sg B_mu^+ (U h) = U (sg B_mu^+ h): a second
// B operand h' built from the same spinors, so both halves of the spinor
// accumulate inside the MMA accumulators across all 8 direction-senses.
// Each site has its own link, so the contraction cannot share an A operand
// across sites (tcgen05 needs M >= 64 rows with one A); one warp owns one
// site and issues 2 * n_rhs / 4 MMAs per direction-sense.
//
// Per warp and direction-sense: the link (d^2 bf16 pairs) is staged in
// shared memory, each lane builds its A-fragment registers from it, the
// lanes build h^T and h'^T (n x 16 bf16, K rows 2d..15 kept zero) from the
// neighbour spinors, and the MMAs run.  The epilogue writes the FP32
// accumulators to shared memory, reassembles complex spinor components per
// (RHS, colour), applies the optional a*x + b*H form and stores BF16.
#include "mrhs.cuh"

namespace bsm {

namespace {

constexpr int kTcWarps = 4;  // warps (sites) per block

__device__ __forceinline__ unsigned short bf16_bits(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  unsigned short u;
  memcpy(&u, &b, 2);
  return u;
}
__device__ __forceinline__ float bits_bf16(unsigned short u) {
  __nv_bfloat16 b;
  memcpy(&b, &u, 2);
  return __bfloat162float(b);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int D, int NT>
struct TcShared {
  unsigned link[D * D];                 // bf16 (re, im) pairs of the link
  unsigned short h[2][8 * NT][16];      // h^T and h'^T: [column n][K row]
  float c[2][16][8 * NT];               // accumulators for the epilogue
};

// value of the realified, padded link at (row r, column k) for this lane's
// fragment slot: 0 = zero, else 1 + element index * 4 + part * 2 + negate
__device__ __forceinline__ int a_code(int D, int r, int k) {
  if (r >= 2 * D || k >= 2 * D) return 0;
  const int rb = r / D, kb = k / D, e = (r % D) * D + (k % D);
  const int part = rb == kb ? 0 : 1;       // Ur on the diagonal blocks, Ui off it
  const int neg = (rb == 0 && kb == 1) ? 1 : 0;  // -Ui in the upper right block
  return 1 + e * 4 + part * 2 + neg;
}

__device__ __forceinline__ unsigned short a_value(const unsigned* link, int code) {
  if (code == 0) return 0;
  const int c = code - 1, e = c >> 2, part = (c >> 1) & 1, neg = c & 1;
  const unsigned v = link[e];
  const unsigned short u = part ? (unsigned short)(v >> 16) : (unsigned short)(v & 0xffffu);
  return neg ? (unsigned short)(u ^ 0x8000u) : u;
}

template <int MU, int FB, int D, int NT>
__device__ __forceinline__ void tc_sense(const MrhsArgs& A, TcShared<D, NT>& sh, const uint2* lt, int n, float sg,
                                         const int (&acode)[8], float (&cu)[NT][4], float (&cl)[NT][4]) {
  const int lane = threadIdx.x & 31;
  const int nr = 4 * NT;
  // stage the link
  for (int e = lane; e < D * D; e += 32) {
    const uint2 v = __ldg(lt + (MU * D * D + e) * kLinkTile);
    sh.link[e] = FB == 0 ? v.x : v.y;
  }
  // h and h' columns n = 2 r + s, K rows (colour c: re at c, im at c + d)
  const uint2* in = reinterpret_cast<const uint2*>(A.in);
  const size_t Vn = (size_t)A.g.Vh * nr;
  for (int idx = lane; idx < nr * D; idx += 32) {
    const int r = idx / D, c = idx - r * D;
    const size_t e = (size_t)n * nr + r;
    const uint2 v0 = __ldg(in + (size_t)c * Vn + e);        // (psi0, psi2)
    const uint2 v1 = __ldg(in + (size_t)(D + c) * Vn + e);  // (psi1, psi3)
    const float2 p0 = bf2_to_f2(v0.x), p2 = bf2_to_f2(v0.y), p1 = bf2_to_f2(v1.x), p3 = bf2_to_f2(v1.y);
    const cx<float> u0 = cmake(p0.x, p0.y), u1 = cmake(p1.x, p1.y), l0 = cmake(p2.x, p2.y), l1 = cmake(p3.x, p3.y);
    cx<float> b0, b1;  // B_mu l
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
    const cx<float> h0 = cmake(fmaf(sg, b0.re, u0.re), fmaf(sg, b0.im, u0.im));
    const cx<float> h1 = cmake(fmaf(sg, b1.re, u1.re), fmaf(sg, b1.im, u1.im));
    cx<float> q0, q1;  // B_mu^+ h
    if (MU == 0) {
      q0 = h0;
      q1 = h1;
    } else if (MU == 1) {
      q0 = cmake(-h1.im, h1.re);
      q1 = cmake(-h0.im, h0.re);
    } else if (MU == 2) {
      q0 = h1;
      q1 = cmake(-h0.re, -h0.im);
    } else {
      q0 = cmake(-h0.im, h0.re);
      q1 = cmake(h1.im, -h1.re);
    }
    sh.h[0][2 * r][c] = bf16_bits(h0.re);
    sh.h[0][2 * r][D + c] = bf16_bits(h0.im);
    sh.h[0][2 * r + 1][c] = bf16_bits(h1.re);
    sh.h[0][2 * r + 1][D + c] = bf16_bits(h1.im);
    sh.h[1][2 * r][c] = bf16_bits(sg * q0.re);
    sh.h[1][2 * r][D + c] = bf16_bits(sg * q0.im);
    sh.h[1][2 * r + 1][c] = bf16_bits(sg * q1.re);
    sh.h[1][2 * r + 1][D + c] = bf16_bits(sg * q1.im);
  }
  __syncwarp();
  // A fragment of the realified link
  unsigned a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    a[q] = (unsigned)a_value(sh.link, acode[2 * q]) | ((unsigned)a_value(sh.link, acode[2 * q + 1]) << 16);
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const unsigned* hu = reinterpret_cast<const unsigned*>(sh.h[0][8 * j + g]);
    const unsigned* hl = reinterpret_cast<const unsigned*>(sh.h[1][8 * j + g]);
    mma_bf16(cu[j], a, hu[t], hu[t + 4]);
    mma_bf16(cl[j], a, hl[t], hl[t + 4]);
  }
  __syncwarp();
}

template <int MU, int D, int NT>
__device__ __forceinline__ void tc_direction(const MrhsArgs& A, TcShared<D, NT>& sh, const uint2* lt, int nf, int nb,
                                             float sg, const int (&acode)[8], float (&cu)[NT][4],
                                             float (&cl)[NT][4]) {
  tc_sense<MU, 0, D, NT>(A, sh, lt, nf, sg, acode, cu, cl);
  tc_sense<MU, 1, D, NT>(A, sh, lt, nb, -sg, acode, cu, cl);
}

template <int D, int NT>
__global__ void __launch_bounds__(32 * kTcWarps) hop_mrhs_tc_kernel(const MrhsArgs A) {
  __shared__ TcShared<D, NT> shared_all[kTcWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kTcWarps + warp;  // this warp's output site
  if (i >= A.g.Vh) return;                     // uniform over the warp
  TcShared<D, NT>& sh = shared_all[warp];
  // K rows 2d..15 of h^T, h'^T stay zero
  for (int e = lane; e < 2 * 8 * NT * 16; e += 32) (&sh.h[0][0][0])[e] = 0;
  const int g = lane >> 2, t = lane & 3;
  int acode[8];  // fragment slots: (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)
  acode[0] = a_code(D, g, 2 * t);
  acode[1] = a_code(D, g, 2 * t + 1);
  acode[2] = a_code(D, g + 8, 2 * t);
  acode[3] = a_code(D, g + 8, 2 * t + 1);
  acode[4] = a_code(D, g, 2 * t + 8);
  acode[5] = a_code(D, g, 2 * t + 9);
  acode[6] = a_code(D, g + 8, 2 * t + 8);
  acode[7] = a_code(D, g + 8, 2 * t + 9);
  __syncwarp();

  int nf[4], nb[4];
  eo_neighbours(A.g, i, A.p, nf, nb);
  const uint2* lt = LinkIO<BF16, D, false>::tile_ptr(A.links, i);
  const float sg = A.dagger ? 1.f : -1.f;
  float cu[NT][4], cl[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) cu[j][q] = cl[j][q] = 0.f;
  tc_direction<0, D, NT>(A, sh, lt, nf[0], nb[0], sg, acode, cu, cl);
  tc_direction<1, D, NT>(A, sh, lt, nf[1], nb[1], sg, acode, cu, cl);
  tc_direction<2, D, NT>(A, sh, lt, nf[2], nb[2], sg, acode, cu, cl);
  tc_direction<3, D, NT>(A, sh, lt, nf[3], nb[3], sg, acode, cu, cl);

  // epilogue: accumulators -> shared (rows = re/im of colours, columns = (rhs, spin))
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int col = 8 * j + 2 * t;
    sh.c[0][g][col] = cu[j][0];
    sh.c[0][g][col + 1] = cu[j][1];
    sh.c[0][g + 8][col] = cu[j][2];
    sh.c[0][g + 8][col + 1] = cu[j][3];
    sh.c[1][g][col] = cl[j][0];
    sh.c[1][g][col + 1] = cl[j][1];
    sh.c[1][g + 8][col] = cl[j][2];
    sh.c[1][g + 8][col + 1] = cl[j][3];
  }
  __syncwarp();
  const int nr = 4 * NT;
  const size_t Vn = (size_t)A.g.Vh * nr;
  uint2* out = reinterpret_cast<uint2*>(A.out);
  const uint2* xin = reinterpret_cast<const uint2*>(A.x);
  const float a = A.af, b = A.bf;
  for (int idx = lane; idx < nr * D; idx += 32) {
    const int r = idx / D, c = idx - r * D;
    float s[4][2];  // spin, re/im
    for (int sp = 0; sp < 2; ++sp) {
      s[sp][0] = sh.c[0][c][2 * r + sp];
      s[sp][1] = sh.c[0][D + c][2 * r + sp];
      s[sp + 2][0] = sh.c[1][c][2 * r + sp];
      s[sp + 2][1] = sh.c[1][D + c][2 * r + sp];
    }
    const size_t e = (size_t)i * nr + r;
    if (xin != nullptr) {
      const uint2 x0 = __ldg(xin + (size_t)c * Vn + e), x1 = __ldg(xin + (size_t)(D + c) * Vn + e);
      const float2 xs[4] = {bf2_to_f2(x0.x), bf2_to_f2(x1.x), bf2_to_f2(x0.y), bf2_to_f2(x1.y)};
      for (int sp = 0; sp < 4; ++sp) {
        s[sp][0] = fmaf(a, xs[sp].x, b * s[sp][0]);
        s[sp][1] = fmaf(a, xs[sp].y, b * s[sp][1]);
      }
    } else if (b != 1.f) {
      for (int sp = 0; sp < 4; ++sp) {
        s[sp][0] *= b;
        s[sp][1] *= b;
      }
    }
    out[(size_t)c * Vn + e] = make_uint2(f2_to_bf2(s[0][0], s[0][1]), f2_to_bf2(s[2][0], s[2][1]));
    out[(size_t)(D + c) * Vn + e] = make_uint2(f2_to_bf2(s[1][0], s[1][1]), f2_to_bf2(s[3][0], s[3][1]));
  }
}

template <int D, int NT>
void launch_tc_t(const MrhsArgs& A, cudaStream_t s) {
  const int blocks = (A.g.Vh + kTcWarps - 1) / kTcWarps;
  hop_mrhs_tc_kernel<D, NT><<<blocks, 32 * kTcWarps, 0, s>>>(with_f32_scalars(A));
}

template <int D>
bool launch_tc_nt(const MrhsArgs& A, cudaStream_t s) {
  switch (A.nrhs) {
    case 4: launch_tc_t<D, 1>(A, s); return true;
    case 8: launch_tc_t<D, 2>(A, s); return true;
    case 12: launch_tc_t<D, 3>(A, s); return true;
    case 16: launch_tc_t<D, 4>(A, s); return true;
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
