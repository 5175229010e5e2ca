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
// shares: a genuine dense contraction, run by cuBLAS (complex FP32 for
// training; realified BF16 with FP32 accumulation for inference).  Training:
// the complex gradients G_W = X^H G_Y, G_X = G_Y W^H (cuBLAS) and the adjoint
// transport G_phi(y) = G_0(y) + sum_mu [U_mu(y-mu)^+ G_{+mu}(y-mu) +
// U_mu(y) G_{-mu}(y+mu)] (below), then Adam.
#include <cublas_v2.h>
#include <math.h>
#include <mutex>

#include "blas.cuh"
#include "operators.cuh"

namespace bsm {

namespace {

constexpr int kPtcThreads = 128;

// ---------------------------------------------------------------------------
// cuBLAS handle per device (created once; cuBLAS's own workspace is set to a
// slice of the caller's workspace on every call)
// ---------------------------------------------------------------------------
std::mutex g_blas_mu;
cublasHandle_t g_blas[64] = {};

cublasHandle_t blas_handle() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (g_blas[dev] == nullptr && cublasCreate(&g_blas[dev]) != CUBLAS_STATUS_SUCCESS) g_blas[dev] = nullptr;
  return g_blas[dev];
}

struct PtcGeom {
  Geom g;
  int d;
  long long rows;  // nbatch * V * d
  int nb;
};

__device__ __forceinline__ long long ptc_row(const Geom& g, int b, int p, int i, int d, int c) {
  return (((long long)b * 2 + p) * g.Vh + i) * d + c;
}

// X[row(x, c)][(k C + ch) 4 + s] = (T_k F_ch)(x)[s][c]; thread per (b, p, i, ch)
template <int D, bool BF>
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
  // k = 0: the field itself
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
      const int n = fb ? nb_[mu] : nf[mu];
      cx<float> in[4][D];
      for (int c = 0; c < D; ++c)
        for (int s = 0; s < 4; ++s) {
          const float2 v = F[ptc_row(g, b, 1 - p, n, D, c) * rowF + ch * 4 + s];
          in[s][c] = cmake(v.x, v.y);
        }
      for (int s = 0; s < 4; ++s)
        for (int a = 0; a < D; ++a) {
          cx<float> w = cmake(0.f, 0.f);
          for (int bb = 0; bb < D; ++bb) cmac(w, fb ? Ub[a][bb] : Uf[a][bb], in[s][bb]);
          put(1 + 2 * mu + fb, a, s, w);
        }
    }
  }
}

// G_F(y) = G_X[y][0] + sum_mu [ Ub(y) G_X[y - mu][1 + 2mu] + Uf(y) G_X[y + mu][2 + 2mu] ]
template <int D>
__global__ void __launch_bounds__(kPtcThreads) ptc_transport_adj_kernel(const char* __restrict__ links,
                                                                        size_t link_block,
                                                                        const float2* __restrict__ GX,
                                                                        float2* __restrict__ GF, Geom g, int nb,
                                                                        int C) {
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
  cx<float> acc[4][D];
  for (int c = 0; c < D; ++c)
    for (int s = 0; s < 4; ++s) {
      const float2 v = GX[ptc_row(g, b, p, i, D, c) * rowX + (0 * C + ch) * 4 + s];
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
      // fb 0: from y - mu with k = 1 + 2 mu through Ub(y); fb 1: from y + mu with k = 2 + 2 mu through Uf(y)
      const int n = fb ? nf[mu] : nb_[mu];
      const int k = 1 + 2 * mu + fb;
      cx<float> in[4][D];
      for (int c = 0; c < D; ++c)
        for (int s = 0; s < 4; ++s) {
          const float2 v = GX[ptc_row(g, b, 1 - p, n, D, c) * rowX + (k * C + ch) * 4 + s];
          in[s][c] = cmake(v.x, v.y);
        }
      for (int s = 0; s < 4; ++s)
        for (int a = 0; a < D; ++a)
          for (int bb = 0; bb < D; ++bb) cmac(acc[s][a], fb ? Uf[a][bb] : Ub[a][bb], in[s][bb]);
    }
  }
  for (int c = 0; c < D; ++c)
    for (int s = 0; s < 4; ++s)
      GF[ptc_row(g, b, p, i, D, c) * rowF + ch * 4 + s] = make_float2(acc[s][c].re, acc[s][c].im);
}

// FP64 device spinor (one field) <-> PTC one-channel field (FP32); thread per (p, i)
__global__ void ptc_pack_kernel(double2* __restrict__ psi, float2* __restrict__ F, Geom g, int d, int unpack) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.Vh) return;
  const int p = t / g.Vh, i = t - p * g.Vh;
  double2* blk = psi + (size_t)p * 4 * d * g.Vh;
  for (int c = 0; c < d; ++c)
    for (int s = 0; s < 4; ++s) {
      float2* f = F + (((size_t)p * g.Vh + i) * d + c) * 4 + s;
      double2* q = blk + (size_t)(s * d + c) * g.Vh + i;
      if (unpack) *q = make_double2(f->x, f->y);
      else *f = make_float2((float)q->x, (float)q->y);
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
  block_sum_store<kBlasThreads>(acc, partials);
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
int launch_transport(const OpCtx& c, const void* F, void* X, int nb, int C, bool bf16, cudaStream_t s) {
  const long long n = (long long)nb * 2 * c.g.Vh * C;
  const int blocks = (int)((n + kPtcThreads - 1) / kPtcThreads);
  const float2* f = reinterpret_cast<const float2*>(F);
#define BSM_PTC_T(DD)                                                                                       \
  if (c.d == DD) {                                                                                          \
    if (bf16) ptc_transport_kernel<DD, true><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, f, X, c.g, nb, C); \
    else ptc_transport_kernel<DD, false><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, f, X, c.g, nb, C);     \
    return BSM_OK;                                                                                          \
  }
  BSM_PTC_T(2)
  BSM_PTC_T(3)
#undef BSM_PTC_T
  return BSM_EUNSUPPORTED;
}

int launch_transport_adj(const OpCtx& c, const void* GX, void* GF, int nb, int C, cudaStream_t s) {
  const long long n = (long long)nb * 2 * c.g.Vh * C;
  const int blocks = (int)((n + kPtcThreads - 1) / kPtcThreads);
  const float2* gx = reinterpret_cast<const float2*>(GX);
  float2* gf = reinterpret_cast<float2*>(GF);
  if (c.d == 2) ptc_transport_adj_kernel<2><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, gx, gf, c.g, nb, C);
  else if (c.d == 3) ptc_transport_adj_kernel<3><<<blocks, kPtcThreads, 0, s>>>(c.links, c.link_block, gx, gf, c.g, nb, C);
  else return BSM_EUNSUPPORTED;
  return BSM_OK;
}

constexpr size_t kBlasWs = size_t(32) << 20;
size_t al(size_t v) { return (v + 255) / 256 * 256; }

// row-major C(MxN) = A(MxK) B(KxN) with optional conjugate-transposes, complex FP32
cublasStatus_t cgemm_rm(cublasHandle_t h, bool ah, bool bh, int M, int N, int K, const void* A, int lda,
                        const void* B, int ldb, void* Cm, int ldc, float beta) {
  // column-major: C^T (N x M) = op(B)^T op(A)^T
  const cuComplex one = make_cuComplex(1.f, 0.f), bt = make_cuComplex(beta, 0.f);
  return cublasCgemm(h, bh ? CUBLAS_OP_C : CUBLAS_OP_N, ah ? CUBLAS_OP_C : CUBLAS_OP_N, N, M, K, &one,
                     reinterpret_cast<const cuComplex*>(B), ldb, reinterpret_cast<const cuComplex*>(A), lda, &bt,
                     reinterpret_cast<cuComplex*>(Cm), ldc);
}

}  // namespace

struct PtcLayout {
  size_t X1, Y1, X2, W1r, W2r, GY2, GX2, GY1, invn, part, blasws, total;
};

PtcLayout ptc_layout(const bsm_lattice& L, int C, int nb, bool train) {
  const Geom g = make_geom(L);
  const int d = rep_info(L.N, L.rep).d;
  const size_t rows = (size_t)nb * 2 * g.Vh * d;
  PtcLayout y{};
  size_t o = 0;
  y.X1 = o; o = al(o + rows * 9 * 4 * 8);
  y.Y1 = o; o = al(o + rows * C * 4 * 8);
  y.X2 = o; o = al(o + rows * 9 * C * 4 * 8);
  y.W1r = o; o = al(o + (size_t)2 * 36 * 2 * C * 4 * 2);
  y.W2r = o; o = al(o + (size_t)2 * 36 * C * 2 * 4 * 2);
  y.GY2 = y.GX2 = y.GY1 = y.invn = y.part = 0;
  if (train) {
    y.GY2 = o; o = al(o + rows * 4 * 8);
    y.GX2 = o; o = al(o + rows * 9 * C * 4 * 8);
    y.GY1 = o; o = al(o + rows * C * 4 * 8);
    y.invn = o; o = al(o + (size_t)(nb + 1) * 8);  // 1/|e_b|^2, then the loss
    y.part = o; o = al(o + (size_t)kBlasMaxBlocks * 8);
  }
  y.blasws = o; o = al(o + kBlasWs);
  y.total = o;
  return y;
}

size_t ptc_workspace_bytes(const bsm_lattice& L, int C, int nb, bool train) { return ptc_layout(L, C, nb, train).total; }

int ptc_pack(const bsm_lattice& L, const double* psi, void* F, bool unpack, cudaStream_t s) {
  const Geom g = make_geom(L);
  const int d = rep_info(L.N, L.rep).d;
  ptc_pack_kernel<<<(2 * g.Vh + 127) / 128, 128, 0, s>>>(reinterpret_cast<double2*>(const_cast<double*>(psi)),
                                                          reinterpret_cast<float2*>(F), g, d, unpack ? 1 : 0);
  return BSM_OK;
}

// out (rows x 4 complex) = layer2(layer1(in)); prec F32 (complex GEMM) or BF16 (realified GEMM)
int ptc_apply(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* in,
              void* out, int nb, int prec, void* ws, cudaStream_t s) {
  const OpCtx c = make_ctx(L, U32, BSM_F32, s);
  if (c.d != 2 && c.d != 3) return BSM_EUNSUPPORTED;
  const PtcLayout y = ptc_layout(L, C, nb, false);
  char* w = reinterpret_cast<char*>(ws);
  const int rows = (int)((long long)nb * 2 * c.g.Vh * c.d);
  std::lock_guard<std::mutex> lock(g_blas_mu);
  cublasHandle_t h = blas_handle();
  if (h == nullptr || cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS ||
      cublasSetWorkspace(h, w + y.blasws, kBlasWs) != CUBLAS_STATUS_SUCCESS)
    return BSM_ECUDA;
  const bool bf = prec == BSM_BF16;
  int rc;
  const int K1 = 36, N1 = 4 * C, K2 = 36 * C, N2 = 4;
  if ((rc = launch_transport(c, in, w + y.X1, nb, 1, bf, s)) != BSM_OK) return rc;
  cublasStatus_t st;
  if (!bf) {
    st = cgemm_rm(h, false, false, rows, N1, K1, w + y.X1, K1, W1, N1, w + y.Y1, N1, 0.f);
    if (st != CUBLAS_STATUS_SUCCESS) return BSM_ECUDA;
    if ((rc = launch_transport(c, w + y.Y1, w + y.X2, nb, C, false, s)) != BSM_OK) return rc;
    st = cgemm_rm(h, false, false, rows, N2, K2, w + y.X2, K2, W2, N2, out, N2, 0.f);
  } else {
    __nv_bfloat16* w1r = reinterpret_cast<__nv_bfloat16*>(w + y.W1r);
    __nv_bfloat16* w2r = reinterpret_cast<__nv_bfloat16*>(w + y.W2r);
    ptc_realify_kernel<<<(K1 * N1 + 127) / 128, 128, 0, s>>>(reinterpret_cast<const float2*>(W1), w1r, K1, N1);
    ptc_realify_kernel<<<(K2 * N2 + 127) / 128, 128, 0, s>>>(reinterpret_cast<const float2*>(W2), w2r, K2, N2);
    const float one = 1.f, zero = 0.f;
    // row-major real C(rows x 2N) = X(rows x 2K) Wr(2K x 2N): column-major C^T = Wr^T X^T
    st = cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, 2 * N1, rows, 2 * K1, &one, w1r, CUDA_R_16BF, 2 * N1, w + y.X1,
                      CUDA_R_16BF, 2 * K1, &zero, w + y.Y1, CUDA_R_32F, 2 * N1, CUBLAS_COMPUTE_32F,
                      CUBLAS_GEMM_DEFAULT);
    if (st != CUBLAS_STATUS_SUCCESS) return BSM_ECUDA;
    if ((rc = launch_transport(c, w + y.Y1, w + y.X2, nb, C, true, s)) != BSM_OK) return rc;
    st = cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, 2 * N2, rows, 2 * K2, &one, w2r, CUDA_R_16BF, 2 * N2, w + y.X2,
                      CUDA_R_16BF, 2 * K2, &zero, out, CUDA_R_32F, 2 * N2, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  }
  return st == CUBLAS_STATUS_SUCCESS ? BSM_OK : BSM_ECUDA;
}

// loss = sum_b |M(r_b) - e_b|^2 / |e_b|^2 and its gradients G_W1, G_W2 (FP32)
int ptc_loss_grad(const bsm_lattice& L, const void* U32, const void* W1, const void* W2, int C, const void* r,
                  const void* e, int nb, void* GW1, void* GW2, double* loss, void* ws, cudaStream_t s) {
  const OpCtx c = make_ctx(L, U32, BSM_F32, s);
  if (c.d != 2 && c.d != 3) return BSM_EUNSUPPORTED;
  const PtcLayout y = ptc_layout(L, C, nb, true);
  char* w = reinterpret_cast<char*>(ws);
  const int rows = (int)((long long)nb * 2 * c.g.Vh * c.d);
  const int K1 = 36, N1 = 4 * C, K2 = 36 * C, N2 = 4;
  int rc;
  {
    std::lock_guard<std::mutex> lock(g_blas_mu);
    cublasHandle_t h = blas_handle();
    if (h == nullptr || cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS ||
        cublasSetWorkspace(h, w + y.blasws, kBlasWs) != CUBLAS_STATUS_SUCCESS)
      return BSM_ECUDA;
    // forward, keeping X1, Y1, X2; Y2 goes to GY2's slot first
    if ((rc = launch_transport(c, r, w + y.X1, nb, 1, false, s)) != BSM_OK) return rc;
    if (cgemm_rm(h, false, false, rows, N1, K1, w + y.X1, K1, W1, N1, w + y.Y1, N1, 0.f) != CUBLAS_STATUS_SUCCESS)
      return BSM_ECUDA;
    if ((rc = launch_transport(c, w + y.Y1, w + y.X2, nb, C, false, s)) != BSM_OK) return rc;
    if (cgemm_rm(h, false, false, rows, N2, K2, w + y.X2, K2, W2, N2, w + y.GY2, N2, 0.f) != CUBLAS_STATUS_SUCCESS)
      return BSM_ECUDA;
    // loss and G_Y2 (in place over Y2)
    const long long per = (long long)rows / nb * 4, n = (long long)rows * 4;
    ptc_inv_norm_kernel<<<nb, kBlasThreads, 0, s>>>(reinterpret_cast<const float2*>(e), per,
                                                     reinterpret_cast<double*>(w + y.invn));
    const int lb = blas_blocks((size_t)n);
    ptc_loss_kernel<<<lb, kBlasThreads, 0, s>>>(reinterpret_cast<const float2*>(w + y.GY2),
                                                reinterpret_cast<const float2*>(e),
                                                reinterpret_cast<float2*>(w + y.GY2),
                                                reinterpret_cast<const double*>(w + y.invn), per, n,
                                                reinterpret_cast<double*>(w + y.part));
    reduce_launch(reinterpret_cast<double*>(w + y.part), lb, reinterpret_cast<double*>(w + y.invn) + nb, s);
    double l = 0.0;
    cudaMemcpyAsync(&l, reinterpret_cast<double*>(w + y.invn) + nb, sizeof(double), cudaMemcpyDeviceToHost, s);
    // backward: G_W2 = X2^H G_Y2, G_X2 = G_Y2 W2^H, G_Y1 = T^+ G_X2, G_W1 = X1^H G_Y1
    if (cgemm_rm(h, true, false, K2, N2, rows, w + y.X2, K2, w + y.GY2, N2, GW2, N2, 0.f) != CUBLAS_STATUS_SUCCESS ||
        cgemm_rm(h, false, true, rows, K2, N2, w + y.GY2, N2, W2, N2, w + y.GX2, K2, 0.f) != CUBLAS_STATUS_SUCCESS)
      return BSM_ECUDA;
    if ((rc = launch_transport_adj(c, w + y.GX2, w + y.GY1, nb, C, s)) != BSM_OK) return rc;
    if (cgemm_rm(h, true, false, K1, N1, rows, w + y.X1, K1, w + y.GY1, N1, GW1, N1, 0.f) != CUBLAS_STATUS_SUCCESS)
      return BSM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BSM_ECUDA;
    if (loss) *loss = l;
  }
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
