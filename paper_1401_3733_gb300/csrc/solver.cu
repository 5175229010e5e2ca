// solver.cu -- CG on the normal equations of the Wilson operator (Sec. II-B:
// the Dirac operator is inverted by CG), plain or mixed precision.
//
// Plain: Hestenes-Stiefel CG on M = Dhat^+ Dhat (even-odd, default) or
// M = D^+ D (full lattice), every vector at the outer precision (FP64, or
// FP64-accurate double-float DF64).
//
// Mixed: the same iteration with FP32 hops and FP32 vectors (alpha and beta
// from FP64-accumulated reductions), restarted from "reliable updates" at the
// outer precision (Clark, Babich, Barros, Brower, Rebbi 2010): when the
// iterated residual has dropped by delta since the last update, or has reached
// the tolerance, the FP32 correction is added into the outer solution, the
// residual is recomputed as rhs - M x at the outer precision, copied back to
// FP32, the search direction is re-orthogonalised against it and beta is
// recomputed from the true residual.  The solve ends only when the recomputed
// residual meets the tolerance.
//
// Iteration order (one kernel each, scalars stay on the device):
//   p = r + beta p ; Ap = M p with |Dhat p|^2 fused ; alpha = rr/pAp ;
//   x += alpha p, r -= alpha Ap with |r|^2 fused ; beta = rr_new/rr.
// The host reads the CG state every `check_every` iterations; once the
// device flags completion the remaining queued kernels return immediately.
// Optionally the check_every iterations are captured once as a CUDA graph and
// replayed (all pointers and the device-side scalars are fixed for a solve).
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <chrono>

#include "blas.cuh"
#include "operators.cuh"

namespace bsm {

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct CgLayout {
  size_t state, partA, partB;
  size_t bp, r, p, Ap, u, t;              // outer-precision vectors
  size_t r32, p32, Ap32, u32, t32, x32;   // FP32 vectors (mixed precision)
  size_t bdf, xdf;                        // DF64 copies of b and x (DF64 outer)
  size_t vec64, vec32;                    // bytes of one CG vector
  int npart;
  size_t total;
};

CgLayout cg_layout(const bsm_lattice& L, int prec_inner, int eo, int prec_outer) {
  CgLayout y;
  const Geom g = make_geom(L);
  const RepInfo ri = rep_info(L.N, L.rep);
  const size_t h64 = half_spinor_bytes(g.Vh, ri.d, BSM_F64);  // = DF64 bytes
  const size_t h32 = half_spinor_bytes(g.Vh, ri.d, BSM_F32);
  y.vec64 = eo ? h64 : 2 * h64;
  y.vec32 = eo ? h32 : 2 * h32;
  y.npart = std::max(2 * hop_partials_max(g.Vh), kBlasMaxBlocks);
  size_t o = 0;
  y.state = o; o = align_up(o + sizeof(CgState));
  y.partA = o; o = align_up(o + sizeof(double) * y.npart);
  y.partB = o; o = align_up(o + sizeof(double) * y.npart);
  y.bp = o; o = align_up(o + y.vec64);
  y.r = o; o = align_up(o + y.vec64);
  y.p = o; o = align_up(o + y.vec64);
  y.Ap = o; o = align_up(o + y.vec64);
  // u and t adjacent: together they hold a full outer spinor at the end
  y.u = o; o = align_up(o + (eo ? h64 : 0));
  y.t = o; o = align_up(o + (eo ? h64 : 2 * h64));
  y.r32 = y.p32 = y.Ap32 = y.u32 = y.t32 = y.x32 = 0;
  if (prec_inner == BSM_F32 || prec_inner == BSM_F32R12) {
    y.r32 = o; o = align_up(o + y.vec32);
    y.p32 = o; o = align_up(o + y.vec32);
    y.Ap32 = o; o = align_up(o + y.vec32);
    y.u32 = o; o = align_up(o + (eo ? h32 : 0));
    y.t32 = o; o = align_up(o + (eo ? h32 : 2 * h32));
    y.x32 = o; o = align_up(o + y.vec32);
  }
  y.bdf = y.xdf = 0;
  if (prec_outer == BSM_DF64) {
    y.bdf = o; o = align_up(o + 2 * h64);
    y.xdf = o; o = align_up(o + 2 * h64);
  }
  y.total = o;
  return y;
}

struct Solver {
  OpCtx co, ci;   // outer and inner operator contexts
  CgLayout y;
  char* ws;
  cudaStream_t s;
  int eo;
  CgState* st;
  const int* done;
  double* partA;
  double* partB;

  Solver(const bsm_lattice& L, const void* Uo, const void* U32, int prec_outer, int prec_inner, int eo_, void* ws_,
         cudaStream_t s_)
      : s(s_), eo(eo_) {
    co = make_ctx(L, Uo, prec_outer, s);
    ci = (prec_inner == BSM_F32 || prec_inner == BSM_F32R12) ? make_ctx(L, U32, prec_inner, s) : co;
    y = cg_layout(L, prec_inner, eo, prec_outer);
    ws = reinterpret_cast<char*>(ws_);
    st = reinterpret_cast<CgState*>(ws + y.state);
    done = reinterpret_cast<const int*>(ws + y.state + offsetof(CgState, done));
    partA = reinterpret_cast<double*>(ws + y.partA);
    partB = reinterpret_cast<double*>(ws + y.partB);
  }
  void* at(size_t off) const { return ws + off; }

  // out = M in at the context's precision; partials of |D in|^2 (or Dhat)
  int apply_normal(const OpCtx& c, const void* in, void* out, void* u, void* t, double* parts,
                   const int* dn) const {
    int n;
    if (eo) {
      n = op_dhat(c, in, u, t, 0, parts, dn);
      if (n < 0) return n;
      const int r = op_dhat(c, u, out, t, 1, nullptr, dn);
      if (r < 0) return r;
    } else {
      n = op_dirac(c, in, t, 0, parts, dn);
      if (n < 0) return n;
      const int r = op_dirac(c, t, out, 1, nullptr, dn);
      if (r < 0) return r;
    }
    return n;
  }

  // r = bp - M x at the outer precision; |r|^2 into st->aux[0]
  int true_residual(const void* x) const {
    const int e = apply_normal(co, x, at(y.Ap), at(y.u), at(y.t), nullptr, nullptr);
    if (e < 0) return e;
    cudaMemcpyAsync(at(y.r), at(y.bp), y.vec64, cudaMemcpyDeviceToDevice, s);
    const int nb = axpby_launch(co.prec, -1.0, at(y.Ap), 1.0, at(y.r), y.vec64 / 16, partA, s);
    reduce_launch(partA, nb, &st->aux[0], s);
    return 0;
  }

  int read_state(CgState& h) const {
    cudaMemcpyAsync(&h, st, sizeof(CgState), cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return BSM_ECUDA;
    }
    return 0;
  }
  void write_state(const CgState& h) const { cudaMemcpyAsync(st, &h, sizeof(CgState), cudaMemcpyHostToDevice, s); }

  // `count` CG iterations; with a graph, the first call captures them on the
  // stream and later calls replay the instantiated graph
  cudaGraphExec_t graph_exec = nullptr;
  int iterate_batch(int count, bool use_graph, const OpCtx& c, void* x, void* r, void* p, void* Ap, void* u,
                    void* t, size_t vec) {
    if (graph_exec != nullptr) return cudaGraphLaunch(graph_exec, s) == cudaSuccess ? 0 : BSM_ECUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool can_capture = use_graph && s != nullptr && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
                             cs == cudaStreamCaptureStatusNone;
    if (can_capture && cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      int rc = 0;
      for (int k = 0; k < count && rc == 0; ++k) rc = iterate(c, x, r, p, Ap, u, t, vec);
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (rc != 0) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e == cudaSuccess && cudaGraphInstantiate(&graph_exec, graph, 0) == cudaSuccess) {
        cudaGraphDestroy(graph);
        return cudaGraphLaunch(graph_exec, s) == cudaSuccess ? 0 : BSM_ECUDA;
      }
      if (graph) cudaGraphDestroy(graph);
      graph_exec = nullptr;
      cudaGetLastError();  // capture unavailable: fall back to direct launches
    }
    for (int k = 0; k < count; ++k) {
      const int rc = iterate(c, x, r, p, Ap, u, t, vec);
      if (rc != 0) return rc;
    }
    return 0;
  }
  ~Solver() {
    if (graph_exec != nullptr) cudaGraphExecDestroy(graph_exec);
  }

  // one CG iteration at the precision of context c
  int iterate(const OpCtx& c, void* x, void* r, void* p, void* Ap, void* u, void* t, size_t vec) const {
    if (eo && vector_prec(c.prec) == BSM_F32) {
      // FP32 even-odd: the x and r updates ride in the epilogue of the last
      // hop of Dhat^+ Dhat p (Ap is never stored); alpha is known once
      // |Dhat p|^2 is reduced, before the Dhat^+ hops run
      cg_p_update_launch(BSM_F32, p, r, vec / 16, st, s);
      const int np = op_dhat(c, p, u, t, 0, partA, done);
      if (np < 0) return np;
      cg_alpha_launch(st, partA, np, s);
      const int nb = op_dhat_dag_cg(c, u, t, r, x, p, &st->alpha_f, partB, done);
      if (nb < 0) return nb;
      cg_beta_launch(st, partB, nb, s);
      return 0;
    }
    cg_p_update_launch(vector_prec(c.prec), p, r, vec / 16, st, s);
    const int np = apply_normal(c, p, Ap, u, t, partA, done);
    if (np < 0) return np;
    cg_alpha_launch(st, partA, np, s);
    const int nb = cg_xr_update_launch(vector_prec(c.prec), x, r, p, Ap, vec / 16, st, partB, s);
    cg_beta_launch(st, partB, nb, s);
    return 0;
  }
};

}  // namespace

size_t cg_workspace_bytes(const bsm_lattice& L, int prec_inner, int eo, int prec_outer) {
  return cg_layout(L, prec_inner, eo, prec_outer).total;
}

int cg_solve(const bsm_lattice& L, const void* U64, const void* U32, const void* b, void* x,
             const bsm_cg_opts& o, bsm_cg_stats* stats, void* ws, cudaStream_t s) {
  const int mixed = o.prec_inner == BSM_F32 || o.prec_inner == BSM_F32R12;
  const int eo = o.eo != 0;
  const int check = o.check_every > 0 ? o.check_every : 8;
  const double delta = o.delta > 0 ? o.delta : 0.1;
  const int po = o.prec_outer;
  Solver S(L, U64, U32, po, o.prec_inner, eo, ws, s);
  const OpCtx& co = S.co;
  const CgLayout& y = S.y;
  const size_t h64 = co.half_bytes;
  int rc;

  if (cudaStreamSynchronize(s) != cudaSuccess) return BSM_ECUDA;
  const auto t0 = std::chrono::steady_clock::now();

  // the outer-precision copies of b and x (DF64 keeps its own)
  const void* bo = b;
  void* xo = x;
  if (po == BSM_DF64) {
    f64_df64_launch(S.at(y.bdf), b, 2 * h64 / 16, true, s);
    if (o.use_x0) f64_df64_launch(S.at(y.xdf), x, 2 * h64 / 16, true, s);
    bo = S.at(y.bdf);
    xo = S.at(y.xdf);
  }
  const char* bc = reinterpret_cast<const char*>(bo);
  char* xc = reinterpret_cast<char*>(xo);

  // right-hand side bp of the normal equations, |bp|^2 -> aux[0], |b|^2 -> aux[1]
  int np;
  if (eo) {
    // bhat_e = b_e + 1/(2A) H_eo b_o  (into u), bp = Dhat^+ bhat_e
    rc = op_hop(co, 0, bc + h64, S.at(y.u), 0, bc, 1.0, 1.0 / (2.0 * co.A), nullptr, nullptr);
    if (rc < 0) return rc;
    np = op_dhat(co, S.at(y.u), S.at(y.bp), S.at(y.t), 1, S.partA, nullptr);
  } else {
    np = op_dirac(co, bo, S.at(y.bp), 1, S.partA, nullptr);
  }
  if (np < 0) return np;
  reduce_launch(S.partA, np, &S.st->aux[0], s);
  const int nbb = dot_launch(po, bo, bo, 2 * h64 / 16, S.partB, s);
  reduce_launch(S.partB, nbb, &S.st->aux[1], s);
  CgState h;
  memset(&h, 0, sizeof(h));
  if ((rc = S.read_state(h)) != 0) return rc;
  const double rhs2 = h.aux[0], b2 = h.aux[1];
  if (!isfinite(rhs2) || !isfinite(b2)) return BSM_ENAN;

  void* xs = xo;  // even half (eo) or the full solution vector
  int status = BSM_OK;
  int updates = 0;
  bool residual_fresh = false;  // st->aux[0] already holds |bp - M x|^2 for the final x
  CgState hs;
  memset(&hs, 0, sizeof(hs));
  hs.stop2 = o.tol * o.tol * rhs2;
  hs.max_iter = o.max_iter;
  hs.delta2 = delta * delta;

  if (rhs2 == 0.0) {
    cudaMemsetAsync(xo, 0, 2 * h64, s);
  } else {
    // initial residual
    double rr0 = rhs2;
    if (o.use_x0) {
      if ((rc = S.true_residual(xs)) != 0) return rc;
      if ((rc = S.read_state(h)) != 0) return rc;
      rr0 = h.aux[0];
    } else {
      cudaMemsetAsync(xs, 0, y.vec64, s);
      cudaMemcpyAsync(S.at(y.r), S.at(y.bp), y.vec64, cudaMemcpyDeviceToDevice, s);
    }
    hs.rr = hs.rr_max = rr0;
    hs.rr_prev = rr0;
    hs.beta = 0.0;
    hs.done = rr0 <= hs.stop2 ? kDoneConverged : kDoneRunning;
    const size_t n32 = S.ci.half_bytes / 16;  // float4 elements per FP32 half (mixed)
    const int halves = eo ? 1 : 2;
    if (mixed) {
      cudaMemsetAsync(S.at(y.x32), 0, y.vec32, s);
      cudaMemsetAsync(S.at(y.p32), 0, y.vec32, s);
      convert_to32_launch(po, S.at(y.r32), S.at(y.r), n32, halves, s);
    } else {
      cudaMemsetAsync(S.at(y.p), 0, y.vec64, s);
    }
    S.write_state(hs);

    int breakdowns = 0;
    while (hs.done != kDoneConverged || mixed) {
      if (hs.done == kDoneRunning) {
        rc = mixed ? S.iterate_batch(check, o.use_graph != 0, S.ci, S.at(y.x32), S.at(y.r32), S.at(y.p32),
                                     S.at(y.Ap32), S.at(y.u32), S.at(y.t32), y.vec32)
                   : S.iterate_batch(check, o.use_graph != 0, co, xs, S.at(y.r), S.at(y.p), S.at(y.Ap), S.at(y.u),
                                     S.at(y.t), y.vec64);
        if (rc < 0) return rc;
        if ((rc = S.read_state(hs)) != 0) return rc;
      }
      if (!mixed) {
        if (hs.done == kDoneConverged) break;
        if (hs.done == kDoneNaN) { status = BSM_ENAN; break; }
        if (hs.done == kDoneBreakdown) { status = BSM_EBREAKDOWN; break; }
        if (hs.done == kDoneMaxIter) { status = BSM_ENOCONV; break; }
        continue;
      }
      // mixed precision: reliable update when due
      if (hs.done == kDoneNaN) { status = BSM_ENAN; break; }
      if (hs.done == kDoneRunning && !hs.want_update) continue;
      accumulate32_launch(po, xs, S.at(y.x32), n32, halves, s);
      if ((rc = S.true_residual(xs)) != 0) return rc;
      if ((rc = S.read_state(h)) != 0) return rc;
      ++updates;
      const double rr_true = h.aux[0];
      if (!isfinite(rr_true)) { status = BSM_ENAN; break; }
      if (rr_true <= hs.stop2) {
        residual_fresh = true;
        break;
      }
      if (hs.done == kDoneMaxIter || hs.iter >= o.max_iter) { status = BSM_ENOCONV; break; }
      if (hs.done == kDoneBreakdown) {
        if (++breakdowns > 2) { status = BSM_EBREAKDOWN; break; }
      } else {
        breakdowns = 0;
      }
      // restart the FP32 iteration from the outer residual
      convert_to32_launch(po, S.at(y.r32), S.at(y.r), n32, halves, s);
      const int n1 = dot_launch(BSM_F32, S.at(y.r32), S.at(y.p32), y.vec32 / 16, S.partA, s);
      reduce_launch(S.partA, n1, &S.st->aux[1], s);
      const int n2 = dot_launch(BSM_F32, S.at(y.r32), S.at(y.r32), y.vec32 / 16, S.partB, s);
      reduce_launch(S.partB, n2, &S.st->aux[2], s);
      axpy_ratio32_launch(S.at(y.p32), S.at(y.r32), y.vec32 / 16, &S.st->aux[1], &S.st->aux[2], s);
      hs.beta = hs.done == kDoneBreakdown ? 0.0 : rr_true / hs.rr_prev;
      hs.rr = rr_true;
      hs.rr_max = rr_true;
      hs.done = kDoneRunning;
      hs.want_update = 0;
      S.write_state(hs);
    }
  }

  // true residual of the normal equations (unless the last reliable update
  // has just computed it for this x), odd-site reconstruction and the
  // full-system residual |D x - b| / |b|, all at the outer precision
  if (!residual_fresh && (rc = S.true_residual(xs)) != 0) return rc;
  if (eo) {
    rc = op_hop(co, 1, xs, xc + h64, 0, bc + h64, 1.0 / co.A, 1.0 / (2.0 * co.A), nullptr, nullptr);
    if (rc < 0) return rc;
  }
  void* full_tmp = eo ? S.at(y.u) : S.at(y.t);
  if ((rc = op_dirac(co, xo, full_tmp, 0, nullptr, nullptr)) < 0) return rc;
  const int nf = axpby_launch(po, -1.0, bo, 1.0, full_tmp, 2 * h64 / 16, S.partB, s);
  reduce_launch(S.partB, nf, &S.st->aux[1], s);
  if (po == BSM_DF64) f64_df64_launch(x, xo, 2 * h64 / 16, false, s);
  if ((rc = S.read_state(h)) != 0) return rc;
  const auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->iters = hs.iter;
    stats->reliable_updates = updates;
    stats->true_res_normal = rhs2 > 0 ? sqrt(h.aux[0] / rhs2) : 0.0;
    stats->true_res_full = b2 > 0 ? sqrt(h.aux[1] / b2) : 0.0;
    stats->seconds = std::chrono::duration<double>(t1 - t0).count();
  }
  if (status == BSM_OK && !(rhs2 == 0.0 || h.aux[0] <= o.tol * o.tol * rhs2)) status = BSM_ENOCONV;
  return status;
}

}  // namespace bsm
