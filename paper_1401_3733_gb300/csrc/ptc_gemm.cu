// ptc_gemm.cu -- the dense contractions of the parallel-transport network
// (ptc.cu) as this library's own kernels.
//
// Every GEMM of the network is tall and skinny: the rows are the lattice
// sites x colours (10^5 .. 10^7), the inner and outer widths are 9 x 4 = 36
// and 4 C (C = channels).  Two shapes occur:
//  - row GEMMs, C(rows x N) = A(rows x K) op(B): each row of A meets a small
//    matrix B that every block stages in shared memory (the slice of 16
//    output columns it computes); one thread per row and slice;
//  - reduction GEMMs, C(M x N) = A^H B with A (rows x M), B (rows x N): the
//    weight gradients, a sum over all rows.  Split over the rows: every block
//    accumulates its chunks of rows in registers and writes one partial
//    matrix, and one thread per output element adds the partials in block
//    order (deterministic).
// The complex ones are FP32 (training and the FP32 network); the real BF16
// ones (FP32 accumulation) serve the realified BF16 network for channel
// counts without a fused kernel.
#include <cuda_bf16.h>

#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kGemmThreads = 256;
constexpr int kSlice = 16;            // output columns per thread of a row GEMM
constexpr int kRedRows = 16;          // rows per shared-memory tile of a reduction GEMM
constexpr int kRedMaxOut = 36 * 256;  // M x N of the largest reduction (36 x 4C, C <= 64)
constexpr int kRedOutPerThread = kRedMaxOut / kGemmThreads;

__device__ __forceinline__ float2 cmul_acc(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
// acc += conj(a) b
__device__ __forceinline__ float2 cjmul_acc(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}

// C = A op(B); op(B) = B (K x N, ldb = N) or, with BH, the conjugate
// transpose of B given as N x K (ldb = K).  Grid: (row blocks, N / kSlice).
template <bool BH>
__global__ void __launch_bounds__(kGemmThreads) crow_gemm_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                                 float2* __restrict__ C, long long rows, int K, int N) {
  extern __shared__ float2 bs[];  // [K][kSlice]
  const int n0 = blockIdx.y * kSlice;
  const int nw = N - n0 < kSlice ? N - n0 : kSlice;
  for (int e = threadIdx.x; e < K * kSlice; e += kGemmThreads) {
    const int k = e / kSlice, j = e % kSlice;
    float2 v = make_float2(0.f, 0.f);
    if (j < nw) {
      if (BH) {
        const float2 t = B[(size_t)(n0 + j) * K + k];
        v = make_float2(t.x, -t.y);
      } else {
        v = B[(size_t)k * N + n0 + j];
      }
    }
    bs[e] = v;
  }
  __syncthreads();
  const long long r = blockIdx.x * (long long)kGemmThreads + threadIdx.x;
  if (r >= rows) return;
  float2 acc[kSlice];
#pragma unroll
  for (int j = 0; j < kSlice; ++j) acc[j] = make_float2(0.f, 0.f);
  const float2* a = A + (size_t)r * K;
  for (int k = 0; k < K; ++k) {
    const float2 av = __ldg(a + k);
#pragma unroll
    for (int j = 0; j < kSlice; ++j) acc[j] = cmul_acc(acc[j], av, bs[k * kSlice + j]);
  }
  float2* c = C + (size_t)r * N + n0;
#pragma unroll
  for (int j = 0; j < kSlice; ++j)
    if (j < nw) c[j] = acc[j];
}

// partial[blockIdx.x][m N + n] = sum over this block's rows of conj(A[r][m]) B[r][n]
__global__ void __launch_bounds__(kGemmThreads) cred_gemm_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                                 float2* __restrict__ partial, long long rows, int M,
                                                                 int N) {
  extern __shared__ float2 tiles[];  // A tile [kRedRows][M], then B tile [kRedRows][N]
  float2* as = tiles;
  float2* bt = tiles + kRedRows * M;
  float2 acc[kRedOutPerThread];
#pragma unroll
  for (int j = 0; j < kRedOutPerThread; ++j) acc[j] = make_float2(0.f, 0.f);
  const int MN = M * N;
  for (long long r0 = (long long)blockIdx.x * kRedRows; r0 < rows; r0 += (long long)gridDim.x * kRedRows) {
    const int nr = rows - r0 < kRedRows ? (int)(rows - r0) : kRedRows;
    __syncthreads();
    for (int e = threadIdx.x; e < kRedRows * M; e += kGemmThreads)
      as[e] = e < nr * M ? A[(size_t)r0 * M + e] : make_float2(0.f, 0.f);
    for (int e = threadIdx.x; e < kRedRows * N; e += kGemmThreads)
      bt[e] = e < nr * N ? B[(size_t)r0 * N + e] : make_float2(0.f, 0.f);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRedOutPerThread; ++j) {
      const int o = threadIdx.x + j * kGemmThreads;
      if (o < MN) {
        const int m = o / N, n = o - (o / N) * N;
        float2 s = acc[j];
#pragma unroll
        for (int rr = 0; rr < kRedRows; ++rr) s = cjmul_acc(s, as[rr * M + m], bt[rr * N + n]);
        acc[j] = s;
      }
    }
  }
  float2* p = partial + (size_t)blockIdx.x * MN;
#pragma unroll
  for (int j = 0; j < kRedOutPerThread; ++j) {
    const int o = threadIdx.x + j * kGemmThreads;
    if (o < MN) p[o] = acc[j];
  }
}

// C[o] = sum over the blocks, in block order
__global__ void __launch_bounds__(kGemmThreads) cred_sum_kernel(const float2* __restrict__ partial, int nblk, int MN,
                                                                float2* __restrict__ C) {
  const int o = blockIdx.x * kGemmThreads + threadIdx.x;
  if (o >= MN) return;
  float2 s = make_float2(0.f, 0.f);
  for (int b = 0; b < nblk; ++b) {
    const float2 v = partial[(size_t)b * MN + o];
    s.x += v.x;
    s.y += v.y;
  }
  C[o] = s;
}

__device__ __forceinline__ float bf(const __nv_bfloat16 x) { return __bfloat162float(x); }

// real C(rows x N) = A(rows x K) B(K x N), A and B bfloat16, FP32
// accumulation, C bfloat16 (OUT_BF16) or FP32
template <bool OUT_BF16>
__global__ void __launch_bounds__(kGemmThreads) brow_gemm_kernel(const __nv_bfloat16* __restrict__ A,
                                                                 const __nv_bfloat16* __restrict__ B, void* __restrict__ C,
                                                                 long long rows, int K, int N) {
  extern __shared__ float bsf[];  // [K][kSlice]
  const int n0 = blockIdx.y * kSlice;
  const int nw = N - n0 < kSlice ? N - n0 : kSlice;
  for (int e = threadIdx.x; e < K * kSlice; e += kGemmThreads) {
    const int k = e / kSlice, j = e % kSlice;
    bsf[e] = j < nw ? bf(B[(size_t)k * N + n0 + j]) : 0.f;
  }
  __syncthreads();
  const long long r = blockIdx.x * (long long)kGemmThreads + threadIdx.x;
  if (r >= rows) return;
  float acc[kSlice];
#pragma unroll
  for (int j = 0; j < kSlice; ++j) acc[j] = 0.f;
  const __nv_bfloat16* a = A + (size_t)r * K;
  for (int k = 0; k < K; ++k) {
    const float av = bf(a[k]);
#pragma unroll
    for (int j = 0; j < kSlice; ++j) acc[j] = fmaf(av, bsf[k * kSlice + j], acc[j]);
  }
  if (OUT_BF16) {
    __nv_bfloat16* c = reinterpret_cast<__nv_bfloat16*>(C) + (size_t)r * N + n0;
#pragma unroll
    for (int j = 0; j < kSlice; ++j)
      if (j < nw) c[j] = __float2bfloat16_rn(acc[j]);
  } else {
    float* c = reinterpret_cast<float*>(C) + (size_t)r * N + n0;
#pragma unroll
    for (int j = 0; j < kSlice; ++j)
      if (j < nw) c[j] = acc[j];
  }
}

}  // namespace

// row-major C(rows x N) = A(rows x K) op(B); op(B) = B (K x N) or, with
// b_herm, the conjugate transpose of B stored as N x K; complex FP32
int ptc_crow_gemm(const void* A, const void* B, void* C, long long rows, int K, int N, bool b_herm, cudaStream_t s) {
  const dim3 grid((unsigned)((rows + kGemmThreads - 1) / kGemmThreads), (unsigned)((N + kSlice - 1) / kSlice));
  const size_t smem = (size_t)K * kSlice * sizeof(float2);
  if (smem > 48 * 1024) return BSM_EUNSUPPORTED;
  const float2* a = reinterpret_cast<const float2*>(A);
  const float2* b = reinterpret_cast<const float2*>(B);
  float2* c = reinterpret_cast<float2*>(C);
  if (b_herm) crow_gemm_kernel<true><<<grid, kGemmThreads, smem, s>>>(a, b, c, rows, K, N);
  else crow_gemm_kernel<false><<<grid, kGemmThreads, smem, s>>>(a, b, c, rows, K, N);
  return BSM_OK;
}

// bytes of scratch ptc_cred_gemm needs
size_t ptc_cred_scratch_bytes(int M, int N) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (size_t)2 * sms * M * N * sizeof(float2);
}

// C(M x N) = A^H B with A (rows x M), B (rows x N), complex FP32,
// M N <= 36 x 256 and M + N <= 384; scratch: ptc_cred_scratch_bytes(M, N) bytes
int ptc_cred_gemm(const void* A, const void* B, void* C, long long rows, int M, int N, void* scratch,
                  cudaStream_t s) {
  if (M * N > kRedMaxOut || M + N > 384) return BSM_EUNSUPPORTED;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long chunks = (rows + kRedRows - 1) / kRedRows;
  int nblk = 2 * sms;
  if (chunks < nblk) nblk = (int)(chunks > 0 ? chunks : 1);
  const size_t smem = (size_t)kRedRows * (M + N) * sizeof(float2);
  if (smem > 48 * 1024) return BSM_EUNSUPPORTED;
  float2* part = reinterpret_cast<float2*>(scratch);
  cred_gemm_kernel<<<nblk, kGemmThreads, smem, s>>>(reinterpret_cast<const float2*>(A),
                                                    reinterpret_cast<const float2*>(B), part, rows, M, N);
  const int MN = M * N;
  cred_sum_kernel<<<(MN + kGemmThreads - 1) / kGemmThreads, kGemmThreads, 0, s>>>(part, nblk, MN,
                                                                                  reinterpret_cast<float2*>(C));
  return BSM_OK;
}

// real row-major C(rows x N) = A(rows x K) B(K x N), bfloat16 A and B, FP32
// accumulation, C bfloat16 (out_bf16) or FP32
int ptc_brow_gemm(const void* A, const void* B, void* C, long long rows, int K, int N, bool out_bf16,
                  cudaStream_t s) {
  const dim3 grid((unsigned)((rows + kGemmThreads - 1) / kGemmThreads), (unsigned)((N + kSlice - 1) / kSlice));
  const size_t smem = (size_t)K * kSlice * sizeof(float);
  if (smem > 48 * 1024) return BSM_EUNSUPPORTED;
  const __nv_bfloat16* a = reinterpret_cast<const __nv_bfloat16*>(A);
  const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(B);
  if (out_bf16) brow_gemm_kernel<true><<<grid, kGemmThreads, smem, s>>>(a, b, C, rows, K, N);
  else brow_gemm_kernel<false><<<grid, kGemmThreads, smem, s>>>(a, b, C, rows, K, N);
  return BSM_OK;
}

}  // namespace bsm
