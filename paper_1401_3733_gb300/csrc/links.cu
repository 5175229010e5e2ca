// links.cu -- representation links (Sec. II-A: the fermion transforms under a
// non-trivial representation R of SU(N)) and spinor packing between the
// canonical host order and the device layout.
//
// R(U) is computed in FP64 from closed forms:
//   adjoint     R_ab = 2 Tr(T^a W^b), W^b = U T^b U^+, evaluated entrywise
//               from the sparse generators (2 Re W_ij, -2 Im W_ij, or the
//               Cartan combination of the diagonal);
//   two-index   R_(ij),(kl) = U_ik U_jl -+ U_il U_jk (the 2x2 minors /
//               permanents of U), with factors sqrt2 and 1 on the diagonal
//               pairs of the symmetric representation;
// then multiplied by exp(i phi_mu) on links leaving the last slice of mu,
// rounded once to the target precision (FP32; FP64; or split exactly into a
// DF64 hi/lo pair) and written twice: as the forward
// link of x (block of parity(x)) and, daggered, as the backward link of x+mu
// (block of the other parity).
#include <math.h>

#include "bsm_internal.cuh"

namespace bsm {

namespace {

__host__ __device__ constexpr int rep_dim_c(int N, int REP) {
  return REP == BSM_FUND ? N : REP == BSM_ADJ ? N * N - 1 : REP == BSM_SYM ? N * (N + 1) / 2 : N * (N - 1) / 2;
}

struct LinkGeom {
  int dims[4];
  int V;
  int Vh;
  double cph[4], sph[4];  // cos, sin of the boundary phases
};

__device__ __forceinline__ cx<double> cmul(cx<double> a, cx<double> b) {
  return cmake(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cx<double> cmulc(cx<double> a, cx<double> b) {  // a * conj(b)
  return cmake(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}

template <int N, int REP>
__device__ void rep_of(const cx<double> (&U)[N][N], cx<double> (&R)[rep_dim_c(N, REP)][rep_dim_c(N, REP)]) {
  constexpr int d = rep_dim_c(N, REP);
  if (REP == BSM_FUND) {
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b) R[a][b] = U[a][b];
  } else if (REP == BSM_ADJ) {
    constexpr int noff = N * (N - 1) / 2;
    for (int bcol = 0; bcol < d; ++bcol) {
      // W = U T^b U^+ for generator bcol
      cx<double> W[N][N];
      if (bcol < 2 * noff) {
        int q = bcol < noff ? bcol : bcol - noff, k = 0, l = 1;
        for (int n = 0; n < q; ++n)
          if (++l == N) { ++k; l = k + 1; }
        const bool sym = bcol < noff;
        for (int i = 0; i < N; ++i)
          for (int j = 0; j < N; ++j) {
            const cx<double> p1 = cmulc(U[i][k], U[j][l]);  // U_ik conj(U_jl)
            const cx<double> p2 = cmulc(U[i][l], U[j][k]);  // U_il conj(U_jk)
            if (sym) {
              W[i][j] = cmake(0.5 * (p1.re + p2.re), 0.5 * (p1.im + p2.im));
            } else {  // -i (p1 - p2) / 2
              W[i][j] = cmake(0.5 * (p1.im - p2.im), -0.5 * (p1.re - p2.re));
            }
          }
      } else {
        const int l = bcol - 2 * noff + 1;
        const double nrm = 1.0 / sqrt(2.0 * l * (l + 1));
        for (int i = 0; i < N; ++i)
          for (int j = 0; j < N; ++j) {
            cx<double> s = cmake(0.0, 0.0);
            for (int m = 0; m <= l; ++m) {
              const double Dm = (m < l ? 1.0 : -(double)l) * nrm;
              const cx<double> p = cmulc(U[i][m], U[j][m]);
              s.re += Dm * p.re;
              s.im += Dm * p.im;
            }
            W[i][j] = s;
          }
      }
      // R_ab = 2 Tr(T^a W)
      int a = 0;
      for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j, ++a) {
          R[a][bcol] = cmake(2.0 * W[i][j].re, 0.0);
          R[a + noff][bcol] = cmake(-2.0 * W[i][j].im, 0.0);
        }
      for (int l = 1; l < N; ++l) {
        const double nrm = 1.0 / sqrt(2.0 * l * (l + 1));
        double s = 0.0;
        for (int m = 0; m < l; ++m) s += W[m][m].re;
        s -= l * W[l][l].re;
        R[2 * noff + l - 1][bcol] = cmake(2.0 * nrm * s, 0.0);
      }
    }
  } else {
    constexpr bool sym = REP == BSM_SYM;
    const double r2 = sqrt(2.0);
    int A = 0;
    for (int i = 0; i < N; ++i)
      for (int j = sym ? i : i + 1; j < N; ++j, ++A) {
        int B = 0;
        for (int k = 0; k < N; ++k)
          for (int l = sym ? k : k + 1; l < N; ++l, ++B) {
            const cx<double> t1 = cmul(U[i][k], U[j][l]);
            const cx<double> t2 = cmul(U[i][l], U[j][k]);
            cx<double> v;
            if (!sym) {
              v = cmake(t1.re - t2.re, t1.im - t2.im);
            } else if (i != j && k != l) {
              v = cmake(t1.re + t2.re, t1.im + t2.im);
            } else if (i != j || k != l) {  // one diagonal pair: sqrt2 U_ik U_jl
              v = cmake(r2 * t1.re, r2 * t1.im);
            } else {
              v = t1;
            }
            R[A][B] = v;
          }
      }
  }
}

template <int N, int REP>
__global__ void links_to_rep_kernel(const double2* __restrict__ Uc, void* __restrict__ out, LinkGeom g,
                                    int prec, size_t block_bytes) {
  constexpr int d = rep_dim_c(N, REP);
  constexpr bool real = REP == BSM_ADJ;
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= (int64_t)g.V * 4) return;
  const int s = (int)(l >> 2), mu = (int)(l & 3);
  int c[4];
  {
    int r = s;
    c[3] = r % g.dims[3]; r /= g.dims[3];
    c[2] = r % g.dims[2]; r /= g.dims[2];
    c[1] = r % g.dims[1]; r /= g.dims[1];
    c[0] = r;
  }
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int i = s >> 1;
  int cn[4] = {c[0], c[1], c[2], c[3]};
  cn[mu] = (cn[mu] + 1 == g.dims[mu]) ? 0 : cn[mu] + 1;
  const int sn = ((cn[0] * g.dims[1] + cn[1]) * g.dims[2] + cn[2]) * g.dims[3] + cn[3];
  const int j = sn >> 1;  // neighbour x+mu, parity 1-p

  cx<double> U[N][N];
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      const double2 v = Uc[(size_t)l * N * N + a * N + b];
      U[a][b] = cmake(v.x, v.y);
    }
  cx<double> R[d][d];
  rep_of<N, REP>(U, R);
  if (c[mu] == g.dims[mu] - 1) {  // boundary phase exp(i phi_mu)
    const cx<double> ph = cmake(g.cph[mu], g.sph[mu]);
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) R[a][b] = cmul(ph, R[a][b]);
  }

  char* blk_f = reinterpret_cast<char*>(out) + (size_t)p * block_bytes;
  char* blk_b = reinterpret_cast<char*>(out) + (size_t)(1 - p) * block_bytes;
  if (prec == BSM_F32R12) {
    // SU(3) fundamental: the first two rows of the forward link and of the
    // backward link (R^+), float2 e of row-major element e at plane
    // mu * 6 + fb * 3 + e / 2, half e % 2
    if (d == 3 && !real) {
      float2* P = reinterpret_cast<float2*>(blk_f);
      float2* Q = reinterpret_cast<float2*>(blk_b);
      for (int e = 0; e < 6; ++e) {
        const int a = e / 3, b = e % 3;
        const cx<double> f = R[a][b];
        const cx<double> bw = cmake(R[b][a].re, -R[b][a].im);
        P[2 * link_index(24, mu * 6 + e / 2, i) + (e & 1)] =
            make_float2(__double2float_rn(f.re), __double2float_rn(f.im));
        Q[2 * link_index(24, mu * 6 + 3 + e / 2, j) + (e & 1)] =
            make_float2(__double2float_rn(bw.re), __double2float_rn(bw.im));
      }
    }
    return;
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      const int cc = a * d + b;
      const cx<double> f = R[a][b];
      const cx<double> bw = cmake(R[b][a].re, -R[b][a].im);  // (R^+)_ab
      if (!real && prec == BSM_F64) {
        double2* P = reinterpret_cast<double2*>(blk_f);
        double2* Q = reinterpret_cast<double2*>(blk_b);
        P[link_index(8 * d * d, (2 * mu) * d * d + cc, i)] = make_double2(f.re, f.im);
        Q[link_index(8 * d * d, (2 * mu + 1) * d * d + cc, j)] = make_double2(bw.re, bw.im);
      } else if (!real && prec == BSM_DF64) {
        float4* P = reinterpret_cast<float4*>(blk_f);
        float4* Q = reinterpret_cast<float4*>(blk_b);
        const df fr(f.re), fi(f.im), br(bw.re), bi(bw.im);
        P[link_index(8 * d * d, (2 * mu) * d * d + cc, i)] = make_float4(fr.hi, fr.lo, fi.hi, fi.lo);
        Q[link_index(8 * d * d, (2 * mu + 1) * d * d + cc, j)] = make_float4(br.hi, br.lo, bi.hi, bi.lo);
      } else if (!real && prec == BSM_BF16) {
        // uint2 element (plane, site) = bfloat16 pairs (forward, backward)
        unsigned int* P = reinterpret_cast<unsigned int*>(blk_f);
        unsigned int* Q = reinterpret_cast<unsigned int*>(blk_b);
        P[2 * link_index(4 * d * d, mu * d * d + cc, i)] = f2_to_bf2((float)f.re, (float)f.im);
        Q[2 * link_index(4 * d * d, mu * d * d + cc, j) + 1] = f2_to_bf2((float)bw.re, (float)bw.im);
      } else if (real && prec == BSM_BF16) {
        __nv_bfloat16* P = reinterpret_cast<__nv_bfloat16*>(blk_f);
        __nv_bfloat16* Q = reinterpret_cast<__nv_bfloat16*>(blk_b);
        P[2 * link_index(4 * d * d, mu * d * d + cc, i)] = __double2bfloat16(f.re);
        Q[2 * link_index(4 * d * d, mu * d * d + cc, j) + 1] = __double2bfloat16(bw.re);
      } else if (!real) {
        // float4 element (plane, site) = float2 pair (forward, backward)
        float2* P = reinterpret_cast<float2*>(blk_f);
        float2* Q = reinterpret_cast<float2*>(blk_b);
        P[2 * link_index(4 * d * d, mu * d * d + cc, i)] =
            make_float2(__double2float_rn(f.re), __double2float_rn(f.im));
        Q[2 * link_index(4 * d * d, mu * d * d + cc, j) + 1] =
            make_float2(__double2float_rn(bw.re), __double2float_rn(bw.im));
      } else if (prec == BSM_F64) {
        double* P = reinterpret_cast<double*>(blk_f);
        double* Q = reinterpret_cast<double*>(blk_b);
        P[2 * link_index(4 * d * d, mu * d * d + cc, i)] = f.re;
        Q[2 * link_index(4 * d * d, mu * d * d + cc, j) + 1] = bw.re;
      } else if (prec == BSM_DF64) {
        // float4 element (plane, site) = (forward.hi, forward.lo, backward.hi, backward.lo)
        float2* P = reinterpret_cast<float2*>(blk_f);
        float2* Q = reinterpret_cast<float2*>(blk_b);
        const df a(f.re), b(bw.re);
        P[2 * link_index(4 * d * d, mu * d * d + cc, i)] = make_float2(a.hi, a.lo);
        Q[2 * link_index(4 * d * d, mu * d * d + cc, j) + 1] = make_float2(b.hi, b.lo);
      } else {
        float* P = reinterpret_cast<float*>(blk_f);
        float* Q = reinterpret_cast<float*>(blk_b);
        P[2 * link_index(4 * d * d, mu * d * d + cc, i)] = __double2float_rn(f.re);
        Q[2 * link_index(4 * d * d, mu * d * d + cc, j) + 1] = __double2float_rn(bw.re);
      }
    }
}

// canonical [nrhs][V][4][d] FP64 <-> device layout (RHS index innermost), one
// thread per (RHS, site); plane-major (the single-RHS layout) or site-major
// (the multi-RHS layout, a site's planes of all RHS contiguous)
__global__ void pack_spinor_kernel(const double2* __restrict__ canon, void* __restrict__ dev, int4 dims, int d,
                                   int prec, int unpack, int nrhs, int site_major) {
  const int V = dims.x * dims.y * dims.z * dims.w;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)V * nrhs) return;
  const int rhs = (int)(tid / V);
  const int s = (int)(tid - (long long)rhs * V);
  int r = s;
  const int z = r % dims.w; r /= dims.w;
  const int y = r % dims.z; r /= dims.z;
  const int x = r % dims.y;
  const int t = r / dims.y;
  const int p = (t + x + y + z) & 1;
  // element (plane q of P, eo site, rhs) sits at q * Vh * nrhs + (eo site * nrhs + rhs),
  // or site-major at (eo site * P + q) * nrhs + rhs
  const size_t i = (size_t)(s >> 1) * nrhs + rhs;
  const size_t Vh = (size_t)V / 2 * nrhs;
  auto at = [&](int q, int P) -> size_t {
    return site_major ? ((size_t)(s >> 1) * P + q) * nrhs + rhs : (size_t)q * Vh + i;
  };
  double2* cs = const_cast<double2*>(canon) + ((size_t)rhs * V + s) * 4 * d;
  if (prec == BSM_F64) {
    double2* blk = reinterpret_cast<double2*>(dev) + (size_t)p * 4 * d * Vh;
    for (int q = 0; q < 4 * d; ++q) {
      if (unpack) cs[q] = blk[at(q, 4 * d)];
      else blk[at(q, 4 * d)] = cs[q];
    }
  } else if (prec == BSM_DF64) {
    float4* blk = reinterpret_cast<float4*>(dev) + (size_t)p * 4 * d * Vh;
    for (int q = 0; q < 4 * d; ++q) {
      if (unpack) {
        const float4 v = blk[at(q, 4 * d)];
        cs[q] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
      } else {
        const df re(cs[q].x), im(cs[q].y);
        blk[at(q, 4 * d)] = make_float4(re.hi, re.lo, im.hi, im.lo);
      }
    }
  } else if (prec == BSM_BF16) {
    uint2* blk = reinterpret_cast<uint2*>(dev) + (size_t)p * 2 * d * Vh;
    for (int sp = 0; sp < 2; ++sp)
      for (int a = 0; a < d; ++a) {
        const int q = sp * d + a;
        if (unpack) {
          const uint2 v = blk[at(q, 2 * d)];
          const float2 u = bf2_to_f2(v.x), l = bf2_to_f2(v.y);
          cs[sp * d + a] = make_double2(u.x, u.y);
          cs[(sp + 2) * d + a] = make_double2(l.x, l.y);
        } else {
          const double2 u = cs[sp * d + a], w = cs[(sp + 2) * d + a];
          blk[at(q, 2 * d)] = make_uint2(f2_to_bf2((float)u.x, (float)u.y), f2_to_bf2((float)w.x, (float)w.y));
        }
      }
  } else {
    float4* blk = reinterpret_cast<float4*>(dev) + (size_t)p * 2 * d * Vh;
    for (int sp = 0; sp < 2; ++sp)
      for (int a = 0; a < d; ++a) {
        const int q = sp * d + a;
        if (unpack) {
          const float4 v = blk[at(q, 2 * d)];
          cs[sp * d + a] = make_double2(v.x, v.y);
          cs[(sp + 2) * d + a] = make_double2(v.z, v.w);
        } else {
          const double2 u = cs[sp * d + a], w = cs[(sp + 2) * d + a];
          blk[at(q, 2 * d)] = make_float4(__double2float_rn(u.x), __double2float_rn(u.y), __double2float_rn(w.x),
                                          __double2float_rn(w.y));
        }
      }
  }
}

template <int N, int REP>
void launch_links(const double* U, void* out, const LinkGeom& g, int prec, size_t block_bytes, cudaStream_t s) {
  const int threads = 128;
  const int64_t n = (int64_t)g.V * 4;
  const int blocks = (int)((n + threads - 1) / threads);
  links_to_rep_kernel<N, REP><<<blocks, threads, 0, s>>>(reinterpret_cast<const double2*>(U), out, g, prec,
                                                          block_bytes);
}

}  // namespace

int links_to_rep_launch(const bsm_lattice& L, const double* U, void* out, int prec, cudaStream_t s) {
  const RepInfo ri = rep_info(L.N, L.rep);
  if (ri.d < 0) return BSM_EUNSUPPORTED;
  LinkGeom g;
  for (int m = 0; m < 4; ++m) {
    g.dims[m] = L.dims[m];
    g.cph[m] = cos(L.bc_phase[m]);
    g.sph[m] = sin(L.bc_phase[m]);
  }
  g.V = L.dims[0] * L.dims[1] * L.dims[2] * L.dims[3];
  g.Vh = g.V / 2;
  if (ri.real)
    for (int m = 0; m < 4; ++m) g.sph[m] = 0.0;  // phases are multiples of pi here
  const size_t bb = link_block_bytes(g.Vh, ri.d, ri.real, prec);
#define BSM_LINKS_CASE(NN, RR) \
  if (L.N == NN && L.rep == RR) { launch_links<NN, RR>(U, out, g, prec, bb, s); return BSM_OK; }
  BSM_LINKS_CASE(2, BSM_FUND)
  BSM_LINKS_CASE(3, BSM_FUND)
  BSM_LINKS_CASE(4, BSM_FUND)
  BSM_LINKS_CASE(6, BSM_FUND)
  BSM_LINKS_CASE(8, BSM_FUND)
  BSM_LINKS_CASE(2, BSM_ADJ)
  BSM_LINKS_CASE(3, BSM_ADJ)
  BSM_LINKS_CASE(2, BSM_SYM)
  BSM_LINKS_CASE(3, BSM_SYM)
  BSM_LINKS_CASE(3, BSM_ASYM)
  BSM_LINKS_CASE(4, BSM_ASYM)
#undef BSM_LINKS_CASE
  return BSM_EUNSUPPORTED;
}

void pack_spinor_launch(const bsm_lattice& L, const double* canon, void* dev, int d, int prec, bool unpack,
                        int nrhs, bool site_major, cudaStream_t s) {
  const int4 dims = make_int4(L.dims[0], L.dims[1], L.dims[2], L.dims[3]);
  const long long n = (long long)L.dims[0] * L.dims[1] * L.dims[2] * L.dims[3] * nrhs;
  const int threads = 128;
  pack_spinor_kernel<<<(int)((n + threads - 1) / threads), threads, 0, s>>>(reinterpret_cast<const double2*>(canon),
                                                                            dev, dims, d, prec, unpack ? 1 : 0, nrhs,
                                                                            site_major ? 1 : 0);
}

}  // namespace bsm
