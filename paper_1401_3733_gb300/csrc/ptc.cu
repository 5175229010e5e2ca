// ptc.cu -- a learned, gauge-equivariant preconditioner: two linear
// parallel-transport convolution (PTC) layers, 1 -> C -> 1 channels.
//
// Layer (a linear map, as a preconditioner should be):
//   out_o(x)[s'] = sum_{k, i, s} (T_k phi_i)(x)[s] W[(k, i, s), (o, s')]
// with the transports T_0 = 1, T_{+mu} phi(x) = U_mu(x) phi(x+mu),
// T_{-mu} phi(x) = U_mu(x-mu)^+ phi(x-mu) (k = 1 + 2 mu, 2 + 2 mu), the FP32
// representation links of the Dirac operator (boundary phases included).
// The weights act on channel and spin only, so the layer is gauge equivariant.
//
// PTC field layout: rows (batch, parity, eo site, colour), each row holding C
// channels x 4 spins complex FP32, so that one layer is a transport kernel
// writing X (rows x 9 C 4 complex: the 9 transported copies of every channel)
// followed by a dense GEMM Y = X W (K = 9 C 4, N = C_out 4) that every site
// shares: a genuine dense contraction, run by the tall-skinny kernels of
// ptc_gemm.cu (complex FP32 for training; realified BF16 with FP32
// accumulation for inference).  Training: the complex gradients
// G_W = X^H G_Y (split over the rows), G_X = G_Y W^H and the adjoint
// transport G_phi(y) = G_0(y) + sum_mu [U_mu(y-mu)^+ G_{+mu}(y-mu) +
// U_mu(y) G_{-mu}(y+mu)] (below), then Adam.
#include <math.h>

#include "blas.cuh"
#include "operators.cuh"

namespace bsm {

bool ptc_fused_supported(int C);
int ptc_crow_gemm(const void* A, const void* B, void* C, long long rows, int K, int N, bool b_herm, cudaStream_t s);
int ptc_cred_gemm(const void* A, const void* B, void* C, long long rows, int M, int N, void* scratch,
                  cudaStream_t s);
int ptc_brow_gemm(const void* A, const void* B, void* C, long long rows, int K, int N, bool out_bf16,
                  cudaStream_t s);
size_t ptc_fused_weight_bytes(int C);
int ptc_fused_apply(const char* links, size_t link_block, int d, int C, const void* F, const void* W1,
                    const void* W2p, void* Wt, void* Z, void* out, const Geom& g, int nb, bool even_only, int* err,
                    cudaStream_t s);

namespace {

constexpr int kPtcThreads = 128;

struct PtcGeom {
  Geom g;
  int d;
  long long rows;  // nbatch * V * d
  int nb;
};

__device__ __forceinline__ long long ptc_row(const Geom& g, int b, int p, int i, int d, int c) {
  return (((long long)b * 2 + p) * g.Vh + i) * d + c;
}

// X[row(x, c)][(k C + ch) 4 + s] = (T_k F_ch)(x)[s][c]; thread per (b, p, i, ch).
// ADJ: the adjoint transports instead, T_{+mu}^+ F(x) = U_mu(x-mu)^+ F(x-mu)
// in slot 1 + 2 mu and T_{-mu}^+ F(x) = U_mu(x) F(x+mu) in slot 2 + 2 mu.
template <int D, bool BF, bool ADJ>
__global__ void __launch_bounds__(kPtcThreads) ptc_transport_kernel(const char* __restrict__ links,
                                                                    size_t link_block, const float2* __restrict__ F,
                                                                    void* __restrict__ X, Geom g, int nb, int C) {
  const long long t = blockIdx.x * (long long)kPtcThreads + threadIdx.x;
  const long long total = (long long)nb * 2 * g.Vh * C;
  if (t >= total) return;
  const int ch = (int)(t % C);
  const long long site = t / C;
  const int i = (int)(site % g.Vh);
  const int p = (int)((site / g.Vh) % 2);
  const int b = (int)(site / (2LL * g.Vh));
  int nf[4], nb_[4];
  eo_neighbours(g, i, p, nf, nb_);
  using L = LinkIO<F32, D, false>;
  const auto* lt = L::tile_ptr(links + (size_t)p * link_block, i);
  const int rowF = C * 4, rowX = 9 * C * 4;
  auto put = [&](int k, int c, int s, cx<float> v) {
    const long long e = ptc_row(g, b, p, i, D, c) * rowX + (k * C + ch) * 4 + s;
    if (BF) reinterpret_cast<unsigned int*>(X)[e] = f2_to_bf2(v.re, v.im);
    else reinterpret_cast<float2*>(X)[e] = make_float2(v.re, v.im);
  };
  for (int c = 0; c < D; ++c)
    for (int s = 0; s < 4; ++s) {
      const float2 v = F[ptc_row(g, b, p, i, D, c) * rowF + ch * 4 + s];
      put(0, c, s, cmake(v.x, v.y));
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
      const bool back = ADJ ? fb == 0 : fb == 1;  // through Ub from x - mu, else through Uf from x + mu
      const int n = back ? nb_[mu] : nf[mu];
      cx<float> in[4][D];
      for (int c = 0; c < D; ++c)
        for (int s = 0; s < 4; ++s) {
          const float2 v = F[ptc_row(g, b, 1 - p, n, D, c) * rowF + ch * 4 + s];
          in[s][c] = cmake(v.x, v.y);
        }
      for (int s = 0; s < 4; ++s)
        for (int a = 0; a < D; ++a) {
          cx<float> w = cmake(0.f, 0.f);
          for (int bb = 0; bb < D; ++bb) cmac(w, back ? Ub[a][bb] : Uf[a][bb], in[s][bb]);
          put(1 + 2 * mu + fb, a, s, w);
        }
    }
  }
}

// out(x)[o][s] = sum_k (T_k Z_{k,o})(x)[s] with Z[row][(k Co + o) 4 + s]; thread per (b, p, i, o)
template <int D>
__global__ void __launch_bounds__(kPtcThreads) ptc_stencil_kernel(const char* __restrict__ links,
                                                                  size_t link_block, const float2* __restrict__ Z,
                                                                  float2* __restrict__ out, Geom g, int nb, int Co) {
  const long long t = blockIdx.x * (long long)kPtcThreads + threadIdx.x;
  const long long total = (long long)nb * 2 * g.Vh * Co;
  if (t >= total) return;
  const int o = (int)(t % Co);
  const long long site = t / Co;
  const int i = (int)(site % g.Vh);
  const int p = (int)((site / g.Vh) % 2);
  const int b = (int)(site / (2LL * g.Vh));
  int nf[4], nb_[4];
  eo_neighbours(g, i, p, nf, nb_);
  using L = LinkIO<F32, D, false>;
  const auto* lt = L::tile_ptr(links + (size_t)p * link_block, i);
  const int rowZ = 9 * Co * 4, rowO = Co * 4;
  cx<float> acc[4][D];
  for (int c = 0; c < D; ++c)
    for (int s = 0; s < 4; ++s) {
      const float2 v = Z[ptc_row(g, b, p, i, D, c) * rowZ + o * 4 + s];
      acc[s][c] = cmake(v.x, v.y);
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
      for (int c = 0; c < D; ++c)
        for (int s = 0; s < 4; ++s) {
          const float2 v = Z[ptc_row(g, b, 1 - p, n, D, c) * rowZ + (k * Co + o) * 4 + s];
          in[s][c] = cmake(v.x, v.y);
        }
      for (int s = 0; s < 4; ++s)
        for (int a = 0; a < D; ++a)
          for (int bb = 0; bb < D; ++bb) cmac(acc[s][a], fb ? Ub[a][bb] : Uf[a][bb], in[s][bb]);
    }
  }
  for (int c = 0; c < D; ++c)
    for (int s = 0; s < 4; ++s)
      out[ptc_row(g, b, p, i, D, c) * rowO + o * 4 + s] = make_float2(acc[s][c].re, acc[s][c].im);
}

// W (9 Ci 4 x 4 Co, rows (k, i, s), columns (o, t)) <-> Wp (4 Ci x 9 4 Co, rows (i, s),
// columns (k, o, t)); back = 1 maps Wp to W
__global__ void ptc_permute_kernel(const float2* __restrict__ src, float2* __restrict__ dst, int Ci, int Co,
                                   int back) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = 9 * Ci * 4 * 4 * Co;
  if (e >= n) return;
  const int col = e % (4 * Co), row = e / (4 * Co);  // W coordinates
  const int k = row / (Ci * 4), is = row % (Ci * 4);
  const int ep = is * (9 * 4 * Co) + k * 4 * Co + col;
  if (back) dst[e] = src[ep];
  else dst[ep] = src[e];
}

// FP64 device spinor (one field) <-> PTC one-channel field (FP32); thread per (p, i).
// even_only: psi is the even half alone; the odd rows of F are zero (pack) or ignored (unpack)
__global__ void ptc_pack_kernel(double2* __restrict__ psi, float2* __restrict__ F, Geom g, int d, int unpack,
                                int even_only) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.Vh) return;
  const int p = t / g.Vh, i = t - p * g.Vh;
  float2* f = F + ((size_t)p * g.Vh + i) * d * 4;
  if (even_only && p == 1) {
    if (!unpack)
      for (int e = 0; e < 4 * d; ++e) f[e] = make_float2(0.f, 0.f);
    return;
  }
  double2* blk = psi + (size_t)p * 4 * d * g.Vh;
  for (int c = 0; c < d; ++c)
    for (int s = 0; s < 4; ++s) {
      double2* q = blk + (size_t)(s * d + c) * g.Vh + i;
      if (unpack) *q = make_double2(f[c * 4 + s].x, f[c * 4 + s].y);
      else f[c * 4 + s] = make_float2((float)q->x, (float)q->y);
    }
}

// FP32 device spinor (2d planes of float4 (psi[s][c], psi[s+2][c]), s = 0, 1)
// <-> PTC one-channel field; thread per (p, i); even_only as above
__global__ void ptc_pack32_kernel(float4* __restrict__ psi, float2* __restrict__ F, Geom g, int d, int unpack,
                                  int even_only) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.Vh) return;
  const int p = t / g.Vh, i = t - p * g.Vh;
  float2* f0 = F + ((size_t)p * g.Vh + i) * d * 4;
  if (even_only && p == 1) {
    if (!unpack && even_only == 1)
      for (int e = 0; e < 4 * d; ++e) f0[e] = make_float2(0.f, 0.f);
    return;
  }
  float4* blk = psi + (size_t)p * 2 * d * g.Vh;
  for (int c = 0; c < d; ++c)
    for (int s = 0; s < 2; ++s) {
      float2* f = f0 + c * 4;
      float4* q = blk + (size_t)(s * d + c) * g.Vh + i;
      if (unpack) *q = make_float4(f[s].x, f[s].y, f[s + 2].x, f[s + 2].y);
      else {
        const float4 v = *q;
        f[s] = make_float2(v.x, v.y);
        f[s + 2] = make_float2(v.z, v.w);
      }
    }
}

// G = 2 (Y - E) / |E_b|^2, partial losses (Y, E: rows x 4 complex)
__global__ void __launch_bounds__(kBlasThreads) ptc_loss_kernel(const float2* __restrict__ Y,
                                                                const float2* __restrict__ E,
                                                                float2* __restrict__ G,
                                                                const double* __restrict__ inv_norm2,
                                                                long long per_sample, long long n,
                                                                double* partials) {
  double acc = 0.0;
  for (long long k = blockIdx.x * (long long)kBlasThreads + threadIdx.x; k < n;
       k += (long long)gridDim.x * kBlasThreads) {
    const double w = inv_norm2[k / per_sample];
    const float dx = Y[k].x - E[k].x, dy = Y[k].y - E[k].y;
    G[k] = make_float2((float)(2.0 * w * dx), (float)(2.0 * w * dy));
    acc += w * ((double)dx * dx + (double)dy * dy);
  }
  block_sum_store_wide<kBlasThreads>(acc, partials);
}

// |E_b|^2 per sample -> 1/|E_b|^2 (one block per sample)
__global__ void ptc_inv_norm_kernel(const float2* __restrict__ E, long long per_sample, double* inv_norm2) {
  double acc = 0.0;
  const float2* e = E + blockIdx.x * per_sample;
  for (long long k = threadIdx.x; k < per_sample; k += kBlasThreads) acc += (double)e[k].x * e[k].x + (double)e[k].y * e[k].y;
  __shared__ double buf[kBlasThreads];
  buf[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kBlasThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) buf[threadIdx.x] += buf[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) inv_norm2[blockIdx.x] = buf[0] > 0 ? 1.0 / buf[0] : 0.0;
}

// Adam (Kingma and Ba 2015) on n floats
__global__ void ptc_adam_kernel(float* __restrict__ W, const float* __restrict__ G, float* __restrict__ m,
                                float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                                float c1, float c2) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = G[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  W[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// complex K x N -> realified bf16 2K x 2N: [[Wr, Wi], [-Wi, Wr]] per entry
__global__ void ptc_realify_kernel(const float2* __restrict__ W, __nv_bfloat16* __restrict__ R, int K, int N) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K * N) return;
  const int k = t / N, n = t - k * N;
  const float2 w = W[t];
  R[(size_t)(2 * k) * 2 * N + 2 * n] = __float2bfloat16_rn(w.x);
  R[(size_t)(2 * k) * 2 * N + 2 * n + 1] = __float2bfloat16_rn(w.y);
  R[(size_t)(2 * k + 1) * 2 * N + 2 * n] = __float2bfloat16_rn(-w.y);
  R[(size_t)(2 * k + 1) * 2 * N + 2 * n + 1] = __float2bfloat16_rn(w.x);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int D>
void transport_t(const OpCtx& c, const void* F, void* X, int nb, int C, bool bf16, bool adj, int blocks,
                 cudaStream_t s) {
  const float2* f = reinterpret_cast<const float2*>(F);
  if (adj) ptc_transport_kernel<D, false, true><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, f, X, c.g, nb, C);
  else if (bf16) ptc_transport_kernel<D, true, false><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, f, X, c.g, nb, C);
  else ptc_transport_kernel<D, false, false><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, f, X, c.g, nb, C);
}

// X = the 9 (adjoint) transports of the C-channel field F (FP32, or BF16 output)
void launch_transport(const OpCtx& c, const void* F, void* X, int nb, int C, bool bf16, bool adj, cudaStream_t s) {
  const long long n = (long long)nb * 2 * c.g.Vh * C;
  const int blocks = (int)((n + kPtcThreads - 1) / kPtcThreads);
  if (c.d == 2) transport_t<2>(c, F, X, nb, C, bf16, adj, blocks, s);
  else transport_t<3>(c, F, X, nb, C, bf16, adj, blocks, s);
}

// out = sum_k T_k Z_k (Co channels)
void launch_stencil(const OpCtx& c, const void* Z, void* out, int nb, int Co, cudaStream_t s) {
  const long long n = (long long)nb * 2 * c.g.Vh * Co;
  const int blocks = (int)((n + kPtcThreads - 1) / kPtcThreads);
  const float2* z = reinterpret_cast<const float2*>(Z);
  float2* o = reinterpret_cast<float2*>(out);
  if (c.d == 2) ptc_stencil_kernel<2><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, z, o, c.g, nb, Co);
  else ptc_stencil_kernel<3><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, z, o, c.g, nb, Co);
}

void launch_permute(const void* src, void* dst, int Ci, int Co, bool back, cudaStream_t s) {
  const int n = 9 * Ci * 4 * 4 * Co;
  ptc_permute_kernel<<<(n + 127) / 128, 128, 0, s>>>(reinterpret_cast<const float2*>(src),
                                                      reinterpret_cast<float2*>(dst), Ci, Co, back ? 1 : 0);
}

constexpr size_t kGemmScratch = size_t(32) << 20;  // split-K partials of the weight gradients
size_t al(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// Layer 1 (1 -> C) transports first: X1 = T(in), rows x 36; Y1 = X1 W1, rows x 4C.
// Layer 2 (C -> 1) mixes first: Z2 = Y1 W2p, rows x 36 (W2p: W2 permuted to
// 4C x 36); out = sum_k T_k Z2_k.  Both intermediates of width 9 x 4 are far
// narrower than the 9 x 4C transports of a C-channel field.
struct PtcLayout {
  size_t err, X1, Y1, Z2, W2p, W1r, W2r, Wt, G, GZ2, GY1, GW2p, invn, part, scratch, total;
};

PtcLayout ptc_layout(const bsm_lattice& L, int C, int nb, bool train) {
  const Geom g = make_geom(L);
  const int d = rep_info(L.N, L.rep).d;
  const size_t rows = (size_t)nb * 2 * g.Vh * d;
  const size_t c8 = sizeof(float2);
  PtcLayout y{};
  size_t o = 0;
  y.err = o; o = al(o + sizeof(int));  // error word of the fused kernel (offset 0, read by bsm_ptc_status)
  y.X1 = o; o = al(o + rows * 36 * c8);
  y.Y1 = o; o = al(o + rows * 4 * C * c8);
  y.Z2 = o; o = al(o + rows * 36 * c8);
  y.W2p = o; o = al(o + (size_t)4 * C * 36 * c8);
  y.W1r = o; o = al(o + (size_t)(2 * 36) * (2 * 4 * C) * 2);
  y.W2r = o; o = al(o + (size_t)(2 * 4 * C) * (2 * 36) * 2);
  y.Wt = o; o = al(o + ptc_fused_weight_bytes(C));
  if (train) {
    y.G = o; o = al(o + rows * 4 * c8);
    y.GZ2 = o; o = al(o + rows * 36 * c8);
    y.GY1 = o; o = al(o + rows * 4 * C * c8);
    y.GW2p = o; o = al(o + (size_t)4 * C * 36 * c8);
    y.invn = o; o = al(o + (size_t)(nb + 1) * 8);  // 1/|e_b|^2, then the loss
    y.part = o; o = al(o + (size_t)kBlasMaxBlocks * 8);
  }
  y.scratch = o; o = al(o + kGemmScratch);
  y.total = o;
  return y;
}

size_t ptc_workspace_bytes(const bsm_lattice& L, int C, int nb, bool train) { return ptc_layout(L, C, nb, train).total; }

int ptc_pack(const bsm_lattice& L, const double* psi, void* F, bool unpack, bool even_only, cudaStream_t s) {
  const Geom g = make_geom(L);
  const int d = rep_info(L.N, L.rep).d;
  ptc_pack_kernel<<<(2 * g.Vh + 127) / 128, 128, 0, s>>>(reinterpret_cast<double2*>(const_cast<double*>(psi)),
                                                          reinterpret_cast<float2*>(F), g, d, unpack ? 1 : 0,
                                                          even_only ? 1 : 0);
  return BSM_OK;
}

// even_only: 0 both parities; 1 the even rows, the odd rows of the field
// zeroed (pack) or left (unpack); 2 the even rows only (a consumer that never
// reads the odd rows of the packed field)
int ptc_pack32(const bsm_lattice& L, const float* psi, void* F, bool unpack, int even_only, cudaStream_t s) {
  const Geom g = make_geom(L);
  const int d = rep_info(L.N, L.rep).d;
  ptc_pack32_kernel<<<(2 * g.Vh + 127) / 128, 128, 0, s>>>(reinterpret_cast<float4*>(const_cast<float*>(psi)),
                                                            reinterpret_cast<float2*>(F), g, d, unpack ? 1 : 0,
                                                            even_only);
  return BSM_OK;
}

// out (rows x 4 complex) = layer2(layer1(in)); prec F32 (complex GEMMs) or BF16 (realified GEMMs).
// even_only (BF16 with a fused kernel): `in` vanishes on odd sites and only the
// even rows of `out` are wanted (the even-even block of the network); the odd
// rows of `out` are then left unwritten.
int ptc_apply(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* in,
              void* out, int nb, int prec, void* ws, cudaStream_t s, bool even_only, bool reset_err) {
  const OpCtx c = make_ctx(L, U32, BSM_F32, s);
  const PtcLayout y = ptc_layout(L, C, nb, false);
  char* w = reinterpret_cast<char*>(ws);
  if (reset_err && cudaMemsetAsync(w + y.err, 0, sizeof(int), s) != cudaSuccess) return BSM_ECUDA;
  const int rows = (int)((long long)nb * 2 * c.g.Vh * c.d);
  const bool bf = prec == BSM_BF16;
  launch_permute(W2, w + y.W2p, C, 1, false, s);
  // BF16 with a fused kernel for this C: transports and both GEMMs in one pass (no cuBLAS)
  if (bf && ptc_fused_supported(C))
    return ptc_fused_apply(c.links, c.link_block, c.d, C, in, W1, w + y.W2p, w + y.Wt, w + y.Z2, out, c.g, nb,
                           even_only, reinterpret_cast<int*>(w + y.err), s);
  launch_transport(c, in, w + y.X1, nb, 1, bf, false, s);
  int rc;
  if (!bf) {
    if ((rc = ptc_crow_gemm(w + y.X1, W1, w + y.Y1, rows, 36, 4 * C, false, s)) != BSM_OK ||
        (rc = ptc_crow_gemm(w + y.Y1, w + y.W2p, w + y.Z2, rows, 4 * C, 36, false, s)) != BSM_OK)
      return rc;
  } else {
    __nv_bfloat16* w1r = reinterpret_cast<__nv_bfloat16*>(w + y.W1r);
    __nv_bfloat16* w2r = reinterpret_cast<__nv_bfloat16*>(w + y.W2r);
    ptc_realify_kernel<<<(36 * 4 * C + 127) / 128, 128, 0, s>>>(reinterpret_cast<const float2*>(W1), w1r, 36, 4 * C);
    ptc_realify_kernel<<<(4 * C * 36 + 127) / 128, 128, 0, s>>>(reinterpret_cast<const float2*>(w + y.W2p), w2r,
                                                                4 * C, 36);
    // Y1 in BF16 (it is only an operand of the second GEMM), Z2 in FP32
    if ((rc = ptc_brow_gemm(w + y.X1, w1r, w + y.Y1, rows, 2 * 36, 2 * 4 * C, true, s)) != BSM_OK ||
        (rc = ptc_brow_gemm(w + y.Y1, w2r, w + y.Z2, rows, 2 * 4 * C, 2 * 36, false, s)) != BSM_OK)
      return rc;
  }
  launch_stencil(c, w + y.Z2, out, nb, 1, s);
  return BSM_OK;
}

// loss = sum_b |M(r_b) - e_b|^2 / |e_b|^2 and its gradients G_W1, G_W2 (FP32)
int ptc_loss_grad(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* r,
                  const void* e, int nb, void* GW1, void* GW2, double* loss, void* ws, cudaStream_t s) {
  const OpCtx c = make_ctx(L, U32, BSM_F32, s);
  const PtcLayout y = ptc_layout(L, C, nb, true);
  char* w = reinterpret_cast<char*>(ws);
  const int rows = (int)((long long)nb * 2 * c.g.Vh * c.d);
  double l = 0.0;
  int rc;
  {
    // forward, keeping X1, Y1 and Z2; the output goes to G's slot
    launch_permute(W2, w + y.W2p, C, 1, false, s);
    launch_transport(c, r, w + y.X1, nb, 1, false, false, s);
    if ((rc = ptc_crow_gemm(w + y.X1, W1, w + y.Y1, rows, 36, 4 * C, false, s)) != BSM_OK ||
        (rc = ptc_crow_gemm(w + y.Y1, w + y.W2p, w + y.Z2, rows, 4 * C, 36, false, s)) != BSM_OK)
      return rc;
    launch_stencil(c, w + y.Z2, w + y.G, nb, 1, s);
    // loss and G = dloss/dout (in place)
    const long long per = (long long)rows / nb * 4, n = (long long)rows * 4;
    double* invn = reinterpret_cast<double*>(w + y.invn);
    double* part = reinterpret_cast<double*>(w + y.part);
    ptc_inv_norm_kernel<<<nb, kBlasThreads, 0, s>>>(reinterpret_cast<const float2*>(e), per, invn);
    const int lb = blas_blocks((size_t)n);
    ptc_loss_kernel<<<lb, kBlasThreads, 0, s>>>(reinterpret_cast<const float2*>(w + y.G),
                                                reinterpret_cast<const float2*>(e), reinterpret_cast<float2*>(w + y.G),
                                                invn, per, n, part);
    reduce_launch(part, lb, invn + nb, s);
    // backward: G_Z2 = T^+ G; G_W2p = Y1^H G_Z2; G_Y1 = G_Z2 W2p^H; G_W1 = X1^H G_Y1
    launch_transport(c, w + y.G, w + y.GZ2, nb, 1, false, true, s);
    if ((rc = ptc_cred_gemm(w + y.Y1, w + y.GZ2, w + y.GW2p, rows, 4 * C, 36, w + y.scratch, s)) != BSM_OK ||
        (rc = ptc_crow_gemm(w + y.GZ2, w + y.W2p, w + y.GY1, rows, 36, 4 * C, true, s)) != BSM_OK ||
        (rc = ptc_cred_gemm(w + y.X1, w + y.GY1, GW1, rows, 36, 4 * C, w + y.scratch, s)) != BSM_OK)
      return rc;
    launch_permute(w + y.GW2p, GW2, C, 1, true, s);
    if (cudaMemcpyAsync(&l, invn + nb, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return BSM_ECUDA;
  }
  *loss = l;
  return BSM_OK;
}

int ptc_adam(void* W, const void* G, void* m, void* v, long long nfloat, double lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  ptc_adam_kernel<<<(int)((nfloat + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<float*>(W), reinterpret_cast<const float*>(G), reinterpret_cast<float*>(m),
      reinterpret_cast<float*>(v), nfloat, (float)lr, b1, b2, 1e-8f, c1, c2);
  return BSM_OK;
}

}  // namespace bsm
