// slab.cu -- domain decomposition of the hop in time (the paper's strong-
// scaling scheme, Sec. II-C: each process owns a block of the lattice and
// exchanges the boundary data of every application of Dphi with its
// neighbours).
//
// A slab is the block of nt time slices [t0, t0 + nt) of the global lattice.
// Its spinors use the device layout of a (nt, X, Y, Z) lattice; t0 and nt are
// even, so a site's local and global parities agree.  The only terms of the
// hop that reach outside the slab are the time-direction terms of its first
// and last slice.  Before the hop each slab sends, for each boundary slice,
// the spin projection that its neighbour needs -- 2 spin x d colour complex
// numbers per site (the "face"), half of the spinor -- and the hop takes
// those two terms from the received faces:
//   forward term of a site on the last slice:   (1 - s g_0) U_0(x) psi(x + 0)
//     psi(x + 0) lies on the first slice of the slab above, which sends
//     h = u + sf B_0 l of it (face side BSM_FACE_LO, sf the forward sign);
//   backward term of a site on the first slice: (1 + s g_0) U_0(x - 0)^+ psi(x - 0)
//     psi(x - 0) lies on the last slice of the slab below, which sends
//     h = u - sf B_0 l of it (side BSM_FACE_HI).
// The receiver multiplies h by its own link (the representation links of the
// global lattice, with the boundary phase folded into the links that cross
// the global time boundary) and reconstructs the lower spins, exactly as for
// an interior neighbour; no phase or link travels with a face.
// Face layout: site f = the site's eo index within its slice, (x Y + y) Z/2 +
// z/2, the same on both sides of the boundary; FP64: 2d planes of double2
// (plane = half * d + colour), FP32: d planes of float4 (h0, h1 of a colour).
#include "hop.cuh"

namespace bsm {
namespace {

constexpr int kSlabThreads = 128;

struct SlabArgs {
  HopArgs h;            // geometry of the slab lattice, links of the global one
  int site_offset;      // t0 * X * Y * Z / 2: a slab site's index in the global parity block
  const void* face_lo;  // received from the slab below (backward terms of slice 0)
  const void* face_hi;  // received from the slab above (forward terms of slice nt - 1)
  int face_sites;       // X * Y * Z / 2
};

template <typename P, int D>
struct FaceIO;

template <int D>
struct FaceIO<F64, D> {
  __device__ __forceinline__ static void load(const void* f, int n, int i, cx<double> (&h)[2][D]) {
    const double2* b = reinterpret_cast<const double2*>(f);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const double2 v = __ldg(b + (size_t)(s * D + a) * n + i);
        h[s][a] = cmake(v.x, v.y);
      }
  }
  __device__ __forceinline__ static void store(void* f, int n, int i, const cx<double> (&h)[2][D]) {
    double2* b = reinterpret_cast<double2*>(f);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < D; ++a) b[(size_t)(s * D + a) * n + i] = make_double2(h[s][a].re, h[s][a].im);
  }
};

template <int D>
struct FaceIO<F32, D> {
  __device__ __forceinline__ static void load(const void* f, int n, int i, cx<float> (&h)[2][D]) {
    const float4* b = reinterpret_cast<const float4*>(f);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float4 v = __ldg(b + (size_t)a * n + i);
      h[0][a] = cmake(v.x, v.y);
      h[1][a] = cmake(v.z, v.w);
    }
  }
  __device__ __forceinline__ static void store(void* f, int n, int i, const cx<float> (&h)[2][D]) {
    float4* b = reinterpret_cast<float4*>(f);
#pragma unroll
    for (int a = 0; a < D; ++a) b[(size_t)a * n + i] = make_float4(h[0][a].re, h[0][a].im, h[1][a].re, h[1][a].im);
  }
};

// the face of one boundary slice of `in` (parity q): h = u + sg B_0 l
template <typename P, int D>
__global__ void __launch_bounds__(kSlabThreads) face_pack_kernel(const void* in, int Vh, int slice_first, int n,
                                                                 typename P::R sg, void* face) {
  using R = typename P::R;
  const int f = blockIdx.x * kSlabThreads + threadIdx.x;
  if (f >= n) return;
  cx<R> psi[4][D], h[2][D];
  SpinorIO<P, D>::load(in, (size_t)Vh, slice_first + f, psi);
  spin_project<0>(psi, sg, h);
  FaceIO<P, D>::store(face, n, f, h);
}

// w = U h for both halves, then the spin reconstruction of direction 0
template <typename P, int D, bool REAL, int FB>
__device__ __forceinline__ void apply_link0(const typename LinkIO<P, D, REAL>::vec* lt, const cx<typename P::R> (&h)[2][D],
                                            typename P::R sg, cx<typename P::R> (&acc)[4][D]) {
  using R = typename P::R;
  using L = LinkIO<P, D, REAL>;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<R> w0 = cmake(R(0), R(0)), w1 = w0;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const typename L::elem u = L::template load_one<FB>(lt, 0, a * D + b);
      link_mac(w0, u, h[0][b]);
      link_mac(w1, u, h[1][b]);
    }
    spin_reconstruct<0>(acc, a, w0, w1, sg);
  }
}

template <typename P, int D, bool REAL>
__global__ void __launch_bounds__(kSlabThreads) slab_hop_kernel(const SlabArgs S) {
  using R = typename P::R;
  const HopArgs& A = S.h;
  const int i = blockIdx.x * kSlabThreads + threadIdx.x;
  if (i >= A.g.Vh) return;
  const size_t Vh = (size_t)A.g.Vh;
  int nf[4], nb[4];
  eo_neighbours(A.g, i, A.p, nf, nb);
  const auto* lt = LinkIO<P, D, REAL>::tile_ptr(A.links, i + S.site_offset);
  const R sg = A.dagger ? R(1) : R(-1);  // forward sign; backward is -sg
  cx<R> acc[4][D];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < D; ++a) acc[s][a] = cmake(R(0), R(0));
  const int t = i / A.g.st, f = i - t * A.g.st;
  // direction 0, forward then backward: from the slab's own spinor, or from a face
  {
    cx<R> h[2][D];
    if (t == A.g.T - 1) {
      FaceIO<P, D>::load(S.face_hi, S.face_sites, f, h);
    } else {
      cx<R> psi[4][D];
      SpinorIO<P, D>::load(A.in, Vh, nf[0], psi);
      spin_project<0>(psi, sg, h);
    }
    apply_link0<P, D, REAL, 0>(lt, h, sg, acc);
    if (t == 0) {
      FaceIO<P, D>::load(S.face_lo, S.face_sites, f, h);
    } else {
      cx<R> psi[4][D];
      SpinorIO<P, D>::load(A.in, Vh, nb[0], psi);
      spin_project<0>(psi, -sg, h);
    }
    apply_link0<P, D, REAL, 1>(lt, h, -sg, acc);
  }
  hop_direction<1, P, D, REAL>(A, Vh, lt, nf[1], nb[1], sg, -sg, acc, 0u);
  hop_direction<2, P, D, REAL>(A, Vh, lt, nf[2], nb[2], sg, -sg, acc, 0u);
  hop_direction<3, P, D, REAL>(A, Vh, lt, nf[3], nb[3], sg, -sg, acc, 0u);
  SpinorIO<P, D>::store(A.out, Vh, i, acc);
}

template <typename P, int D, bool REAL>
void launch_t(const SlabArgs& S, cudaStream_t s) {
  slab_hop_kernel<P, D, REAL><<<(S.h.g.Vh + kSlabThreads - 1) / kSlabThreads, kSlabThreads, 0, s>>>(S);
}

template <typename P>
int launch_slab_prec(int d, bool real, const SlabArgs& S, cudaStream_t s) {
  if (real) {
    switch (d) {
      case 3: launch_t<P, 3, true>(S, s); return BSM_OK;
      case 8: launch_t<P, 8, true>(S, s); return BSM_OK;
      default: return BSM_EUNSUPPORTED;
    }
  }
  switch (d) {
    case 2: launch_t<P, 2, false>(S, s); return BSM_OK;
    case 3: launch_t<P, 3, false>(S, s); return BSM_OK;
    case 4: launch_t<P, 4, false>(S, s); return BSM_OK;
    case 6: launch_t<P, 6, false>(S, s); return BSM_OK;
    case 8: launch_t<P, 8, false>(S, s); return BSM_OK;
    default: return BSM_EUNSUPPORTED;
  }
}

template <typename P>
int launch_face_prec(int d, const void* in, int Vh, int first, int n, double sg, void* face, cudaStream_t s) {
  using R = typename P::R;
  const int blocks = (n + kSlabThreads - 1) / kSlabThreads;
  switch (d) {
    case 2: face_pack_kernel<P, 2><<<blocks, kSlabThreads, 0, s>>>(in, Vh, first, n, (R)sg, face); return BSM_OK;
    case 3: face_pack_kernel<P, 3><<<blocks, kSlabThreads, 0, s>>>(in, Vh, first, n, (R)sg, face); return BSM_OK;
    case 4: face_pack_kernel<P, 4><<<blocks, kSlabThreads, 0, s>>>(in, Vh, first, n, (R)sg, face); return BSM_OK;
    case 6: face_pack_kernel<P, 6><<<blocks, kSlabThreads, 0, s>>>(in, Vh, first, n, (R)sg, face); return BSM_OK;
    case 8: face_pack_kernel<P, 8><<<blocks, kSlabThreads, 0, s>>>(in, Vh, first, n, (R)sg, face); return BSM_OK;
    default: return BSM_EUNSUPPORTED;
  }
}

// the slab's own lattice: the global one with nt time slices
int check_slab(const bsm_slab* S, int prec, bsm_lattice* local) {
  if (S == nullptr) return BSM_EINVAL;
  int rc = check_lattice(&S->global);
  if (rc != BSM_OK) return rc;
  const int T = S->global.dims[0];
  if (S->t0 < 0 || S->nt < 2 || (S->t0 & 1) || (S->nt & 1) || S->t0 + S->nt > T) return BSM_EINVAL;
  if (prec != BSM_F64 && prec != BSM_F32) return BSM_EUNSUPPORTED;
  *local = S->global;
  local->dims[0] = S->nt;
  return BSM_OK;
}

size_t face_sites(const bsm_lattice& L) { return (size_t)L.dims[1] * L.dims[2] * L.dims[3] / 2; }

}  // namespace
}  // namespace bsm

using namespace bsm;

extern "C" size_t bsm_face_bytes(const bsm_slab* slab, int32_t prec) {
  bsm_lattice loc;
  if (check_slab(slab, prec, &loc) != BSM_OK) return 0;
  return face_sites(loc) * 2 * rep_info(loc.N, loc.rep).d * 2 * real_bytes(prec);
}

extern "C" int bsm_face_pack(const bsm_slab* slab, const void* in_slab, void* face, int32_t side, int32_t in_parity,
                             int32_t dagger, int32_t prec, void* stream) {
  bsm_lattice loc;
  int rc = check_slab(slab, prec, &loc);
  if (rc != BSM_OK) return rc;
  if (side != BSM_FACE_LO && side != BSM_FACE_HI) return BSM_EINVAL;
  if (in_parity != BSM_EVEN && in_parity != BSM_ODD) return BSM_EINVAL;
  if (!aligned(in_slab) || !aligned(face)) return BSM_EINVAL;
  const Geom g = make_geom(loc);
  const RepInfo ri = rep_info(loc.N, loc.rep);
  if (overlap(in_slab, half_spinor_bytes(g.Vh, ri.d, prec), face, bsm_face_bytes(slab, prec))) return BSM_EINVAL;
  const int n = g.st;
  const double sf = dagger ? 1.0 : -1.0;  // sign of the forward term
  // LO: the first slice, for the forward terms of the slab below; HI: the
  // last slice, for the backward terms of the slab above
  const int first = side == BSM_FACE_LO ? 0 : (loc.dims[0] - 1) * g.st;
  const double sg = side == BSM_FACE_LO ? sf : -sf;
  (void)in_parity;  // a face is a slice of the given parity block; the parity fixes only which block is passed
  const cudaStream_t s = (cudaStream_t)stream;
  rc = prec == BSM_F64 ? launch_face_prec<F64>(ri.d, in_slab, g.Vh, first, n, sg, face, s)
                       : launch_face_prec<F32>(ri.d, in_slab, g.Vh, first, n, sg, face, s);
  if (rc != BSM_OK) return rc;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return BSM_OK;
}

extern "C" int bsm_dslash_slab(const bsm_slab* slab, const void* U_rep, const void* in_slab, const void* face_lo,
                               const void* face_hi, void* out_slab, int32_t out_parity, int32_t dagger, int32_t prec,
                               void* stream) {
  bsm_lattice loc;
  int rc = check_slab(slab, prec, &loc);
  if (rc != BSM_OK) return rc;
  if (out_parity != BSM_EVEN && out_parity != BSM_ODD) return BSM_EINVAL;
  if (!aligned(U_rep) || !aligned(in_slab) || !aligned(face_lo) || !aligned(face_hi) || !aligned(out_slab))
    return BSM_EINVAL;
  const Geom g = make_geom(loc), gg = make_geom(slab->global);
  const RepInfo ri = rep_info(loc.N, loc.rep);
  const size_t nh = half_spinor_bytes(g.Vh, ri.d, prec), nf = bsm_face_bytes(slab, prec);
  if (overlap(in_slab, nh, out_slab, nh) || overlap(face_lo, nf, out_slab, nh) || overlap(face_hi, nf, out_slab, nh))
    return BSM_EINVAL;
  SlabArgs S{};
  S.h.links = reinterpret_cast<const char*>(U_rep) + (size_t)out_parity * link_block_bytes(gg.Vh, ri.d, ri.real, prec);
  S.h.in = in_slab;
  S.h.out = out_slab;
  S.h.a = 0.0;
  S.h.b = 1.0;
  S.h.g = g;
  S.h.p = out_parity;
  S.h.dagger = dagger != 0;
  S.h = with_f32_scalars(S.h);
  S.site_offset = slab->t0 * g.st;
  S.face_lo = face_lo;
  S.face_hi = face_hi;
  S.face_sites = g.st;
  const cudaStream_t s = (cudaStream_t)stream;
  rc = prec == BSM_F64 ? launch_slab_prec<F64>(ri.d, ri.real, S, s) : launch_slab_prec<F32>(ri.d, ri.real, S, s);
  if (rc != BSM_OK) return rc;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return BSM_ECUDA;
  }
  return BSM_OK;
}
