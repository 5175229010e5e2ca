/*
 * bsm.h -- C ABI of the GB300 (sm_103a) library for the BSMBench hot path:
 * the even-odd preconditioned Wilson-Dirac operator and CG on its normal
 * equations (Bennett et al., "BSMBench", HPCS 2016, Sec. II-A field content,
 * Sec. II-B Dirac operator and CG, Sec. III benchmark tasks).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice (Sec. II-A): dims = {T, X, Y, Z}, mu = 0 is time, every extent even
 * and >= 2, V = T*X*Y*Z sites, V_h = V/2 sites per parity.  Canonical site
 * index s = ((t*X + x)*Y + y)*Z + z; parity(x) = (t+x+y+z) mod 2 (even = 0);
 * within a parity a site's index is s >> 1 (valid because Z is even).
 *
 * Fields (Sec. II-A): a link is an N x N complex matrix U_mu(x) (link from x
 * to x+mu).  The fermion at a site is 4 (spin) x d colour components in the
 * d-dimensional representation R of SU(N): fundamental (d = N), adjoint
 * (d = N^2-1, real), two-index symmetric (N(N+1)/2) or antisymmetric
 * (N(N-1)/2).
 *
 * Operator (Sec. II-B "Dphi"; the paper does not print the formula, the
 * standard Wilson form is used):
 *   (H psi)(x) = sum_mu [ (1 - g_mu) U^R_mu(x) psi(x+mu)
 *                       + (1 + g_mu) U^R_mu(x-mu)^+ psi(x-mu) ]
 *   D = A - H/2,  A = 4 + m0,
 * with U^R_mu(x) = R(U_mu(x)) times exp(i phi_mu) on the links that cross the
 * boundary (x_mu = L_mu - 1), and the chiral gamma basis g_0 = [[0,1],[1,0]],
 * g_k = [[0,-i s_k],[i s_k,0]], g_5 = diag(-1,-1,1,1).  The adjoint operator
 * is H^+ = g_5 H g_5 (the projectors exchanged).  Even-odd (Schur) operator on
 * the even sites: Dhat = A - 1/(4A) H_eo H_oe, Dhat^+ = A - 1/(4A) H^+_eo H^+_oe.
 * Representation bases: generalised Gell-Mann generators for the adjoint
 * (symmetric off-diagonal, antisymmetric off-diagonal, diagonal; Tr T^aT^b =
 * delta/2); e_(ii) = E_ii, e_(ij) = (E_ij +- E_ji)/sqrt2 (i<j, lexicographic)
 * for the two-index representations.
 *
 * Canonical host-order arrays (used only by pack/unpack and links_to_rep),
 * complex numbers as interleaved (re, im) FP64:
 *   fundamental links  [V][4][N][N]     spinors  [V][4][d]
 *
 * Device layouts (produced by this library; sizes from bsm_field_bytes):
 *   half spinor (one parity), FP64: 4d planes of V_h double2 (re, im),
 *       plane = spin*d + colour.
 *   half spinor, FP32: 2d planes of V_h float4, plane = s*d + colour for
 *       s = 0, 1, holding (psi[s][c], psi[s+2][c]) as (re, im, re, im).
 *   half spinor, DF64: as FP64 with each double2 replaced by a float4
 *       (re.hi, re.lo, im.hi, im.lo).
 *   half spinor, BF16: as FP32 with each float replaced by a bfloat16 (2d
 *       planes of 8-byte (re, im, re, im) quadruples).
 *   full spinor: the even half followed by the odd half.
 *   links, BSM_F32R12: per output parity 24 planes of float4, plane
 *       mu*6 + f*3 + q holding elements 2q and 2q+1 (row-major) of the first
 *       two rows of the forward (f = 0) / backward (f = 1) link, tiled as below.
 *   links: for each output parity p (p = 0 block first) the 8 links that a
 *       site x of parity p needs, forward U^R_mu(x) and backward
 *       U^R_mu(x-mu)^+, grouped in planes.  Complex representation, FP64:
 *       8 d^2 planes of double2, plane (2mu+f)*d^2 + c (f = 0 forward, 1
 *       backward, c = row*d + col); FP32: 4 d^2 planes of float4, plane
 *       mu*d^2 + c holding (forward[c], backward[c]).  Real (adjoint)
 *       representation: 4 d^2 planes of double2 (FP64) or float2 (FP32)
 *       holding (forward[c], backward[c]).  DF64 stores what FP64 stores
 *       with every double split into (hi, lo) floats: complex planes of
 *       float4 (re.hi, re.lo, im.hi, im.lo), real planes of float4
 *       (forward.hi, forward.lo, backward.hi, backward.lo).  BF16 stores what
 *       FP32 stores with every float replaced by a bfloat16.  The planes are tiled by 32 sites:
 *       element (plane, site i) sits at ((i/32)*planes + plane)*32 + i%32,
 *       with V_h rounded up to a multiple of 32, so the links of a warp's 32
 *       sites are one contiguous region.
 *   Every link is stored twice (as a forward link of its own site and as the
 *   backward link of its neighbour), so each hop reads its 8 links per site
 *   as aligned, coalesced 16-byte (8-byte for FP32 real) vectors.
 *
 * Ownership and execution: all pointers are device pointers unless stated;
 * the caller allocates and frees every buffer (workspace included) and the
 * library keeps no pointer past a call.  Buffers must be 16-byte aligned.
 * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * Every call is asynchronous on `stream` except bsm_cg_solve,
 * bsm_fgcr_solve and bsm_ptc_loss_grad, which synchronise `stream` before
 * they return.  Calls on different streams may
 * run concurrently if they share no output buffer.
 *
 * Errors: every call validates its arguments before it launches anything and
 * returns a bsm_status; nothing aborts or exits.  A CUDA launch or runtime
 * error returns BSM_ECUDA (bsm_last_cuda_error() gives its text).
 */
#ifndef BSM_GB300_H
#define BSM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BSM_OK = 0,
  BSM_EINVAL = -1,        /* bad argument: null/misaligned pointer, odd or zero extent, A == 0 */
  BSM_EUNSUPPORTED = -2,  /* (N, representation, precision, phase) not instantiated */
  BSM_ECUDA = -3,         /* CUDA launch or runtime error */
  BSM_EWORKSPACE = -4,    /* workspace smaller than bsm_workspace_bytes() */
  BSM_ENOCONV = -5,       /* a solver reached max_iter before the tolerance */
  BSM_EBREAKDOWN = -6,    /* CG breakdown: <p, M p> <= 0 */
  BSM_ENAN = -7,          /* NaN or Inf met in a solver reduction */
  BSM_ETIMEOUT = -8       /* a bounded device-side wait gave up */
} bsm_status;

typedef enum { BSM_FUND = 0, BSM_ADJ = 1, BSM_SYM = 2, BSM_ASYM = 3 } bsm_rep;
/* BSM_DF64: FP64-accurate "double-float" storage and arithmetic -- every real
 * is an unevaluated sum hi + lo of two FP32 numbers (about 48 significand
 * bits), computed with error-free transformations on the FP32 units; same
 * bytes as FP64, several times the speed on GB300, whose FP64 units are slow. */
/* BSM_BF16: bfloat16 storage of links and spinors with FP32 arithmetic
 * (Dslash only: error about 2^-9 relative per stored value). */
/* BSM_F32R12: FP32, with SU(3) fundamental links stored as their first two
 * rows (12 of 18 reals per link; the third row of an SU(3) matrix is the
 * complex conjugate of the cross product of the first two, and a link that
 * carries the boundary phase c needs the factor c^3 on it).  A quarter less
 * memory traffic per hop than BSM_F32 at FP32 accuracy.  Spinors are stored
 * exactly as BSM_F32.  N = 3 fundamental only (other lattices:
 * BSM_EUNSUPPORTED); accepted by bsm_field_bytes, bsm_workspace_bytes,
 * bsm_pack/unpack_spinor, bsm_links_to_rep, bsm_dslash, bsm_dirac_eo and as
 * bsm_cg_opts.prec_inner (U_rep32 then holds two-row links). */
typedef enum { BSM_F64 = 0, BSM_F32 = 1, BSM_DF64 = 2, BSM_BF16 = 3, BSM_F32R12 = 4 } bsm_prec;
typedef enum { BSM_EVEN = 0, BSM_ODD = 1, BSM_FULL = 2 } bsm_parity;
typedef enum { BSM_OP_DHAT = 0, BSM_OP_DHAT_DAG = 1, BSM_OP_DHAT_DAG_DHAT = 2 } bsm_eo_op;
typedef enum {
  BSM_FIELD_LINKS = 0,        /* representation links, device layout, both parities */
  BSM_FIELD_SPINOR = 1,       /* full-lattice spinor, device layout */
  BSM_FIELD_HALF_SPINOR = 2,  /* one parity, device layout */
  BSM_FIELD_FUND_CANON = 3,   /* canonical FP64 fundamental links [V][4][N][N] */
  BSM_FIELD_SPINOR_CANON = 4  /* canonical FP64 spinor [V][4][d] */
} bsm_field_kind;
typedef enum { BSM_CALL_DIRAC_EO = 0, BSM_CALL_CG = 1 } bsm_call;

typedef struct {
  int32_t dims[4];      /* {T, X, Y, Z}; all even and >= 2 */
  int32_t N;            /* gauge group SU(N) */
  int32_t rep;          /* bsm_rep */
  double m0;            /* Wilson bare mass; A = 4 + m0 must be nonzero */
  double bc_phase[4];   /* phi_mu in radians (pi = antiperiodic); a real
                           representation accepts only multiples of pi */
} bsm_lattice;

typedef struct {
  double tol;           /* stop when |rhs - M x_e| <= tol |rhs| (FP64, recomputed) */
  int32_t max_iter;     /* total CG iterations allowed */
  int32_t prec_inner;   /* equal to prec_outer: plain CG at that precision;
                           BSM_F32: mixed precision with reliable updates at
                           prec_outer (needs U_rep32) */
  double delta;         /* reliable-update trigger: |r| < delta * max|r| since the
                           last update (0 selects 0.1) */
  int32_t use_x0;       /* nonzero: x holds the initial guess on entry */
  int32_t eo;           /* nonzero: even-odd Schur system (default path);
                           zero: unpreconditioned D^+ D on the full lattice */
  int32_t check_every;  /* iterations between host convergence checks (0 = 8) */
  int32_t prec_outer;   /* precision of U_rep64, of the source preparation, the
                           reliable updates, the true residuals and (plain CG)
                           of the whole iteration: BSM_F64 or BSM_DF64.  b and
                           x are FP64 device-layout spinors either way. */
  int32_t use_graph;    /* nonzero: capture the check_every iterations between
                           host checks once as a CUDA graph and replay it
                           (fewer launch gaps on small lattices).  Ignored on
                           the legacy default stream and on a stream that is
                           already capturing. */
} bsm_cg_opts;

typedef struct {
  int32_t iters;            /* CG iterations performed */
  int32_t reliable_updates; /* FP64 residual recomputations (mixed precision) */
  double true_res_normal;   /* |rhs - M x| / |rhs| recomputed in FP64 */
  double true_res_full;     /* |D x - b| / |b| on the full lattice, FP64 */
  double seconds;           /* wall time of the solve (host clock, synchronised) */
} bsm_cg_stats;

/* d_R of (N, rep), or a negative bsm_status when unsupported.  Pure host. */
int bsm_rep_dim(int32_t N, int32_t rep);

/* Bytes of a field of `kind` at precision `prec` (canonical kinds ignore
 * prec).  0 when the lattice is invalid.  Pure host. */
size_t bsm_field_bytes(const bsm_lattice *lat, int32_t kind, int32_t prec);

/* Workspace bytes that bsm_dirac_eo (call = BSM_CALL_DIRAC_EO) or
 * bsm_cg_solve (BSM_CALL_CG, prec = the inner precision; enough for either
 * outer precision) needs.  Pure host. */
size_t bsm_workspace_bytes(const bsm_lattice *lat, int32_t call, int32_t prec);

/* Canonical FP64 spinor [V][4][d] (device) -> full device-layout spinor at
 * `prec`, and back (FP32 values are widened exactly on unpack). */
int bsm_pack_spinor(const bsm_lattice *lat, const double *canon, void *dev,
                    int32_t prec, void *stream);
int bsm_unpack_spinor(const bsm_lattice *lat, const void *dev, double *canon,
                      int32_t prec, void *stream);

/* Multi-RHS pack/unpack: canonical FP64 spinors [nrhs][V][4][d] (device) <->
 * the multi-RHS device layout at `prec` (BSM_F32 or BSM_BF16): the 2d
 * planes of the single-RHS layout, site-major with the RHS index innermost,
 * element (plane, site, rhs) at (site*2d + plane)*nrhs + rhs within each
 * parity, so that one site's spinors of all RHS are contiguous; nrhs times
 * bsm_field_bytes(lat, BSM_FIELD_SPINOR, prec) bytes.  V*nrhs <= 2^30. */
int bsm_pack_spinor_mrhs(const bsm_lattice *lat, const double *canon, void *dev,
                         int32_t nrhs, int32_t prec, void *stream);
int bsm_unpack_spinor_mrhs(const bsm_lattice *lat, const void *dev, double *canon,
                           int32_t nrhs, int32_t prec, void *stream);

/* Representation links (Sec. II-A: the fermion transforms under a
 * non-trivial representation of the gauge group).  U_fund: canonical FP64
 * fundamental links on the device.  U_rep: device-layout links at `prec`
 * (bsm_field_bytes(lat, BSM_FIELD_LINKS, prec) bytes), computed in FP64 and
 * rounded once, with the boundary phases folded in. */
int bsm_links_to_rep(const bsm_lattice *lat, const double *U_fund, void *U_rep,
                     int32_t prec, void *stream);

/* Dphi (Sec. II-B).  out_parity = BSM_EVEN / BSM_ODD: the hopping block
 * out_p = H_{p,1-p} in_{1-p} (raw hop, no 1/2, no mass), `in` and `out` half
 * spinors.  out_parity = BSM_FULL: out = D in on full spinors.  dagger != 0
 * applies the adjoint (H^+ = g_5 H g_5, D^+).  U_rep at the same `prec`. */
int bsm_dslash(const bsm_lattice *lat, const void *U_rep, const void *in,
               void *out, int32_t out_parity, int32_t dagger, int32_t prec,
               void *stream);

/* Dphi on nrhs right-hand sides at once (Sec. II-A: N_f fermion flavours in
 * one gauge field), the same operator as bsm_dslash applied to every RHS:
 * out_parity EVEN/ODD gives the hopping block on multi-RHS half spinors,
 * FULL gives D on full ones.  prec: BSM_F32 or BSM_BF16 (FP32 arithmetic).
 * Each link is read once per site and applied to all RHS; a thread owns a
 * site and a block of RHS whose size is tuned on the first call for each
 * (precision, d, nrhs, lattice) shape: that call times the candidates on
 * `stream` and synchronises it (set BSM_MRHS_TUNE=0 to take a fixed block
 * instead); later calls are asynchronous. */
int bsm_dslash_mrhs(const bsm_lattice *lat, const void *U_rep, const void *in, void *out,
                    int32_t nrhs, int32_t out_parity, int32_t dagger, int32_t prec,
                    void *stream);

/* The RHS block (RHS per thread) that bsm_dslash_mrhs uses for this
 * (lattice, nrhs, prec): 0 before the first call has tuned it, 1..4 for the
 * SIMT kernel, 102 and 104 for the SIMT kernel with 2 or 4 RHS per thread
 * held as lane pairs of packed FP32 instructions (one instruction serves two
 * RHS; 104 for d <= 3), 16 for the tensor-core kernel (BF16, complex d = 4,
 * 6, 8, nrhs = 4, 8, 12, 16: one warp per site, the link x spinor block
 * products as mma.sync m16n8k16 with FP32 accumulation); or a negative
 * bsm_status.  Pure host. */
int bsm_dslash_mrhs_block(const bsm_lattice *lat, int32_t nrhs, int32_t prec);

/* Pins the RHS block bsm_dslash_mrhs uses for (lattice, nrhs, prec) instead
 * of tuning it (block = 0 forgets the choice; the next call tunes again).
 * BSM_EUNSUPPORTED if that block does not exist for the shape.  Pure host;
 * the choice is process-wide. */
int bsm_dslash_mrhs_set_block(const bsm_lattice *lat, int32_t nrhs, int32_t prec, int32_t block);

/* Even-odd Schur operator on even half spinors: op = BSM_OP_DHAT (Dhat),
 * BSM_OP_DHAT_DAG (Dhat^+) or BSM_OP_DHAT_DAG_DHAT (Dhat^+ Dhat).  workspace:
 * at least bsm_workspace_bytes(lat, BSM_CALL_DIRAC_EO, prec) bytes. */
int bsm_dirac_eo(const bsm_lattice *lat, const void *U_rep, const void *in_e,
                 void *out_e, int32_t op, int32_t prec, void *workspace,
                 size_t workspace_bytes, void *stream);

/* Size of the library-owned scratch array of bsm_dirac_eo_noalloc: 64 MiB. */
#define BSM_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* bsm_dirac_eo without a caller workspace.  The paper has no counterpart:
 * this entry point serves callers that cannot allocate device memory
 * themselves -- a host that has handed all device memory to its own pool
 * allocator, a plugin or sandbox that exposes no allocation call, or a loop
 * that cannot afford the device-wide synchronisation that cudaMalloc and
 * cudaFree imply.  It takes the arguments of bsm_dirac_eo minus the
 * workspace, accepts the same lattices and precisions (BSM_F64, BSM_F32,
 * BSM_DF64, BSM_BF16, BSM_F32R12 for SU(3) fundamental) and computes the
 * same result with the same kernels.
 * Its two scratch half spinors live in one BSM_NOALLOC_SCRATCH_BYTES array
 * that the library declares as device memory.  The CUDA runtime reserves
 * that array on a device when it loads the library's module there: under
 * the default lazy module loading (CUDA_MODULE_LOADING=LAZY) that is the
 * first call of this entry point on the device, under
 * CUDA_MODULE_LOADING=EAGER it is the creation of every context that loads
 * the library, whether or not this entry point ever runs.  Either way the
 * device keeps the array until the process exits.  A caller whose pool
 * allocator takes all free device memory must therefore make its first call
 * before that pool is created (with less than the array free, the first
 * call returns BSM_ECUDA), and before any stream capture, because the first
 * call on a device also looks up the array's device address (with that
 * device current) and remembers it.  Calls after the first allocate nothing
 * (no cudaMalloc, cudaFree or allocating library routine).  A lattice whose
 * scratch, 2 * bsm_field_bytes(lat, BSM_FIELD_HALF_SPINOR, prec), exceeds
 * the array returns BSM_EWORKSPACE before any launch.  All calls on a
 * device share the one array and the scratch is fully rewritten by each
 * call, so nothing needs clearing between calls, but calls that overlap on
 * the GPU (e.g. on two streams) race on it: serialise them. */
int bsm_dirac_eo_noalloc(const bsm_lattice *lat, const void *U_rep, const void *in_e,
                         void *out_e, int32_t op, int32_t prec, void *stream);

/* A batch of lattices of uneven size in one persistent launch (several
 * gauge configurations or theories at once).  Each item is an SU(2) or SU(3)
 * fundamental lattice with FP32 links and its own nrhs multi-RHS FP32
 * spinors (bsm_pack_spinor_mrhs layout).  op BSM_BATCH_D: out = D in on full
 * spinors; BSM_BATCH_DHAT: out_e = Dhat in_e on even halves (two phases:
 * odd temporaries in the workspace, a grid barrier between them).  Blocks of a
 * cooperative grid take (lattice, parity, chunk) work items from a device
 * queue.  The barrier wait is bounded by timeout_s (0 selects 1 s): past it
 * the kernel raises an error flag and returns, and the call returns
 * BSM_ETIMEOUT.  barrier_extra > 0 adds arrivals that never come (a test of
 * that path).  items is a host array of 1..32 lattices; the call
 * synchronises `stream`. */
typedef enum { BSM_BATCH_D = 0, BSM_BATCH_DHAT = 1 } bsm_batch_op;
typedef struct {
  bsm_lattice lat;
  const void *U_rep;
  const void *in;
  void *out;
  int32_t nrhs;
} bsm_batch_item;
typedef struct {
  int32_t op;            /* bsm_batch_op */
  int32_t prec;          /* BSM_F32 */
  double timeout_s;      /* limit of the grid-barrier wait */
  int32_t barrier_extra; /* 0 in normal use */
} bsm_batch_opts;
size_t bsm_batch_workspace_bytes(const bsm_batch_item *items, int32_t count, const bsm_batch_opts *opts);
int bsm_dslash_batch(const bsm_batch_item *items, int32_t count, const bsm_batch_opts *opts,
                     void *workspace, size_t workspace_bytes, void *stream);
/* The same launch without the wait: it enqueues a memset of the workspace's
 * control block and the cooperative launch (the task table travels as a
 * launch parameter), nothing else, so a stream capture of this call gives a
 * CUDA graph that replays the whole batch.  bsm_dslash_batch_status waits
 * for `stream` and returns BSM_ETIMEOUT if the last batch run on this
 * workspace gave up a barrier wait, else BSM_OK. */
int bsm_dslash_batch_async(const bsm_batch_item *items, int32_t count, const bsm_batch_opts *opts,
                           void *workspace, size_t workspace_bytes, void *stream);
int bsm_dslash_batch_status(void *workspace, void *stream);

/* Solve D x = b (Sec. II-B: inverting the Dirac operator by CG) through CG on
 * the normal equations.  With opts->eo: Dhat^+ Dhat x_e = Dhat^+ bhat_e,
 * bhat_e = b_e + 1/(2A) H_eo b_o, then x_o = (b_o + H_oe x_e / 2) / A.
 * b, x: full FP64 device-layout spinors.  U_rep64: links at opts->prec_outer
 * (FP64 or DF64); U_rep32: FP32 links (required when opts->prec_inner ==
 * BSM_F32, else ignored).  stats is a
 * host pointer (may be NULL).  Synchronises `stream`.  Returns BSM_ENOCONV,
 * BSM_EBREAKDOWN or BSM_ENAN with x holding the last iterate. */
int bsm_cg_solve(const bsm_lattice *lat, const void *U_rep64, const void *U_rep32,
                 const void *b, void *x, const bsm_cg_opts *opts,
                 bsm_cg_stats *stats, void *workspace, size_t workspace_bytes,
                 void *stream);

/* ---------------------------------------------------------------------------
 * Learned preconditioner for the inversion of Sec. II-B (the paper itself
 * solves with plain CG; this is an extension).  A two-layer linear
 * parallel-transport convolution network M ~ D^{-1}, 1 -> C -> 1 channels:
 *
 *   layer(phi)_o(x)[s'] = sum_{k, i, s} (T_k phi_i)(x)[s] W[(k, i, s), (o, s')]
 *   T_0 = 1, T_{1+2mu} phi(x) = U_mu(x) phi(x+mu),
 *   T_{2+2mu} phi(x) = U_mu(x-mu)^+ phi(x-mu)
 *
 * with the representation links of the Dirac operator (boundary phases
 * included); the weights mix channels and spins only, so M commutes with
 * gauge transformations.  Supported: complex representations with d = 2, 3
 * (SU(2), SU(3) fundamental; SU(2) symmetric; SU(3) antisymmetric); others
 * give BSM_EUNSUPPORTED.  U_rep32: the FP32 links of bsm_links_to_rep.
 *
 * PTC field (device, complex FP32 = float2): rows (sample b, parity p, eo site
 * i, colour c) in that order, row index ((b*2 + p)*V_h + i)*d + c, each row
 * holding C channels x 4 spins, element [row][ch*4 + s].  A one-channel field
 * of nbatch samples is nbatch*V*d*4 float2.
 * Weights (device, complex FP32, row-major): W1 is 36 x 4C, W2 is 36C x 4,
 * row (k*C_in + i)*4 + s, column o*4 + s'.
 * --------------------------------------------------------------------------- */

/* FP64 full device-layout spinor (bsm_pack_spinor, prec BSM_F64) -> one-
 * channel PTC field of one sample (rounded to FP32), and back (widened). */
int bsm_ptc_pack(const bsm_lattice *lat, const void *psi, void *field, void *stream);
int bsm_ptc_unpack(const bsm_lattice *lat, const void *field, void *psi, void *stream);

/* Workspace bytes of bsm_ptc_apply (train = 0) or bsm_ptc_loss_grad
 * (train = 1) for `channels` hidden channels and nbatch samples; 0 for an
 * unsupported lattice or channels outside 1..64.  Pure host. */
size_t bsm_ptc_workspace_bytes(const bsm_lattice *lat, int32_t channels, int32_t nbatch, int32_t train);

/* out = M(in) for nbatch one-channel PTC fields.  prec BSM_F32: complex FP32
 * GEMMs; BSM_BF16: transported fields and weights rounded to BF16, products
 * accumulated in FP32 (inference).  Asynchronous on `stream`.  The BF16
 * path with 2, 4, 8 or 12 channels runs one tensor-core kernel whose waits
 * for MMA completion are bounded (2^20 polls; the environment variable
 * BSM_PTC_WAIT_POLLS lowers the bound, 0 making every first wait give up,
 * for tests of this path): a block whose wait gives up waits once more,
 * bounded, for its MMAs in flight, issues no further MMAs, stores NaN for
 * its remaining outputs and sets an error word in the workspace, which each
 * call clears first and bsm_ptc_status reads. */
int bsm_ptc_apply(const bsm_lattice *lat, const void *U_rep32, const void *W1, const void *W2,
                  int32_t channels, const void *in, void *out, int32_t nbatch, int32_t prec,
                  void *workspace, size_t workspace_bytes, void *stream);

/* Waits for `stream` and returns BSM_ETIMEOUT if the last bsm_ptc_apply on
 * this workspace had a bounded tensor-core wait give up, else BSM_OK
 * (BSM_EINVAL for a NULL or misaligned workspace). */
int bsm_ptc_status(void *workspace, void *stream);

/* Training loss and gradients, FP32:
 *   loss = sum_b |M(r_b) - e_b|^2 / |e_b|^2
 * G_W1, G_W2 (device, shaped like W1, W2) receive dloss/dRe W + i dloss/dIm W.
 * r, e: nbatch one-channel PTC fields.  *loss (host) is written.  Synchronises
 * `stream`. */
int bsm_ptc_loss_grad(const bsm_lattice *lat, const void *U_rep32, const void *W1, const void *W2,
                      int32_t channels, const void *r, const void *e, int32_t nbatch, void *G_W1,
                      void *G_W2, double *loss, void *workspace, size_t workspace_bytes, void *stream);

/* One Adam step (Kingma and Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8) on n
 * floats: W -= lr * mhat / (sqrt(vhat) + eps); m, v start at zero, step
 * counts from 1.  Asynchronous. */
int bsm_ptc_adam_step(void *W, const void *G, void *m, void *v, int64_t n, double lr, int32_t step,
                      void *stream);

/* Flexible GCR on the full operator, D x = b (FP64), with M = identity
 * (precond BSM_FGCR_NONE) or the network above (BSM_FGCR_PTC, in
 * ptc_prec BSM_F32 or BSM_BF16).  prec_inner BSM_F64: every vector and D in
 * FP64, restarted every `restart` directions.  BSM_F32: each restart cycle
 * solves D e = r in FP32 (FP32 links and vectors, FP64 reductions) from
 * e = 0 until |r32| <= inner_tol |r| or `restart` directions, then
 * x += e and r = b - D x are formed in FP64 (the stopping test always uses
 * this FP64 residual).  The solver stops when the residual of the system it
 * iterates on is <= tol |b|; with eo that residual is the full-system residual
 * of the reconstructed x (the odd sites' residual vanishes by construction).
 * The new direction of each step is orthogonalised against the cycle's
 * earlier ones by classical Gram-Schmidt in one pass (which, in the FP32
 * cycles, loses orthogonality faster than modified Gram-Schmidt would: more
 * steps, never a wrong residual, since the stopping test is the recomputed
 * FP64 residual). */
typedef enum { BSM_FGCR_NONE = 0, BSM_FGCR_PTC = 1 } bsm_fgcr_precond;
typedef struct {
  double tol;        /* stop when |r| <= tol |b| (iterated residual) */
  int32_t max_iter;
  int32_t restart;   /* directions kept, 1..64 */
  int32_t precond;   /* bsm_fgcr_precond */
  int32_t ptc_prec;  /* BSM_F32 or BSM_BF16 */
  int32_t channels;  /* hidden channels C of W1, W2 */
  int32_t prec_inner;/* BSM_F64 or BSM_F32 */
  double inner_tol;  /* BSM_F32 cycles: residual reduction per cycle (0 -> 0.1) */
  int32_t eo;        /* nonzero: solve the even-site Schur system Dhat x_e = bhat_e
                        (bhat_e = b_e + H_eo b_o / (2A)), preconditioned by the
                        even-even block of M, then x_o = (b_o + H_oe x_e / 2) / A */
  int32_t check_every;/* host convergence test every this many steps (0 -> 1);
                        up to check_every - 1 steps may run past convergence */
  int32_t prec_outer;/* arithmetic of the FP64-accurate operator (right-hand
                        side, the residual after each BSM_F32 cycle, the odd
                        sites, the final true residual): BSM_F64 (0), or
                        BSM_DF64 (double-float, about 48 significand bits), in
                        which case U_rep64 is a BSM_DF64 link field; the
                        vectors stay FP64 either way */
  int32_t fallback;  /* nonzero: when FGCR ends with BSM_ENOCONV, BSM_ENAN
                        or BSM_ETIMEOUT, solve the same system with CG on the
                        normal equations (bsm_cg_solve: mixed precision with
                        U_rep32 when it is given, else plain at prec_outer; eo
                        as above; from the FGCR iterate after BSM_ENOCONV,
                        from zero otherwise) to the normal-equation residual
                        tol, and return that solve's status */
  int32_t fallback_max_iter; /* CG iterations of the fallback (0 -> 20000) */
} bsm_fgcr_opts;
typedef struct {
  int32_t iters;     /* directions (preconditioner applications) in total */
  int32_t cycles;    /* restart cycles */
  double true_res;   /* |b - D x| / |b|, recomputed at the end (by the
                        fallback CG when it ran) */
  double seconds;    /* the whole call, the fallback included */
  int32_t fgcr_status;    /* status FGCR itself ended with */
  int32_t fallback_iters; /* CG iterations of the fallback, 0 if it did not run */
} bsm_fgcr_stats;
size_t bsm_fgcr_workspace_bytes(const bsm_lattice *lat, const bsm_fgcr_opts *opts);
/* b, x: full FP64 device-layout spinors (x is overwritten, start x = 0);
 * U_rep64: FP64 links (BSM_DF64 links with prec_outer BSM_DF64); U_rep32:
 * FP32 links, used with BSM_FGCR_PTC or
 * prec_inner BSM_F32 (may be NULL otherwise); W1, W2: used with BSM_FGCR_PTC
 * only.  Synchronises `stream` every check_every steps.  Returns
 * BSM_ENOCONV (max_iter reached), BSM_ENAN, or BSM_ETIMEOUT (a bounded
 * tensor-core wait of the BF16 network gave up, see bsm_ptc_apply; checked
 * after every restart cycle) with x holding the last iterate, unless
 * opts->fallback is set: then plain CG, the library's reference solver,
 * takes over and its status is returned (stats->fgcr_status keeps FGCR's).
 * The workspace is then sized for both solvers. */
int bsm_fgcr_solve(const bsm_lattice *lat, const void *U_rep64, const void *U_rep32,
                   const void *W1, const void *W2, const void *b, void *x,
                   const bsm_fgcr_opts *opts, bsm_fgcr_stats *stats, void *workspace,
                   size_t workspace_bytes, void *stream);

/* The launch configuration the last batch call on this thread used: RHS
 * per thread (1 or 2, or 102 / 104 for 2 / 4 RHS held as lane pairs of
 * packed FP32 instructions, as in bsm_dslash_mrhs_block; every lattice's
 * nrhs is a multiple of it) and chunks of 128 thread slots per work-queue grab
 * (1, 2, 4 or 8).  bsm_dslash_batch, bsm_dslash_batch_async and
 * bsm_cg_solve_batch pick it per batch shape (the lattices and their nrhs)
 * on their first call by timing every candidate on `stream` (which
 * synchronises it), unless the stream is capturing a graph or the
 * environment sets BSM_BATCH_TUNE=0; then the tuned choice if one exists,
 * else (1, 4).  BSM_BATCH_CONFIG="rb:grab" (e.g. "104:2") pins one
 * configuration for every batch whose nrhs are multiples of rb.  The
 * results do not depend on it.  Pure host. */
int bsm_batch_last_config(int32_t *rhs_per_thread, int32_t *chunks_per_grab);

/* A batch of systems solved together: mixed-precision CG (FP32 iterations,
 * reliable updates at opts->prec_outer) on the even-odd normal equations of
 * every right-hand side of several lattices of uneven size (Sec. II-B CG; the
 * N_f flavours of Sec. II-A as RHS sharing a gauge field).  Each iteration
 * runs Dhat^+ Dhat of the whole batch in one persistent launch (the
 * bsm_dslash_batch kernel, four phases) and the vector updates of all
 * systems in four more launches, with per-system scalars on the device; the
 * check_every iterations between host checks are captured once as a CUDA
 * graph (use_graph, not on the legacy default stream) and replayed.  At each
 * check every system whose residual fell by delta (or below the stop) gets a
 * reliable update; a system whose recomputed residual |bp - M x| <= tol |bp|
 * stops.  Items: SU(2) or SU(3) fundamental, up to 32 lattices.  opts:
 * prec_inner BSM_F32, prec_outer BSM_F64 or BSM_DF64, eo nonzero, use_x0 0;
 * tol, max_iter (iterations of the batch), delta, check_every, use_graph as
 * for bsm_cg_solve.  stats: one bsm_cg_stats per system, items in order and
 * RHS within an item (iters: the iteration at which that system stopped).
 * Synchronises `stream`.  A batch barrier that waits more than 1 s returns
 * BSM_ETIMEOUT. */
typedef struct {
  bsm_lattice lat;
  const void *U_rep64;  /* links at opts->prec_outer */
  const void *U_rep32;  /* FP32 links */
  const void *b;        /* nrhs FP64 full device-layout spinors, one after the other */
  void *x;              /* the solutions, same layout (overwritten) */
  int32_t nrhs;         /* 1, 2, 4, 8 or 16 */
} bsm_cg_batch_item;
size_t bsm_cg_batch_workspace_bytes(const bsm_cg_batch_item *items, int32_t count);
int bsm_cg_solve_batch(const bsm_cg_batch_item *items, int32_t count, const bsm_cg_opts *opts,
                       bsm_cg_stats *stats, void *workspace, size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------------
 * Domain decomposition in time (Sec. II-C: each process owns a block of the
 * lattice and exchanges boundary data with its neighbours for every Dphi).
 * A slab is the block of nt time slices [t0, t0 + nt) of `global`; t0 and nt
 * are even (so a site's parity is the same in the slab and in the global
 * lattice) and t0 + nt <= T.  A slab's spinors use the device layout of the
 * lattice `global` with dims[0] = nt (bsm_pack_spinor on that lattice).
 * Per hop each slab packs two faces of its input half spinor with
 * bsm_face_pack and hands them to its neighbours (BSM_FACE_LO, its first
 * slice, to the slab below; BSM_FACE_HI, its last slice, to the slab above;
 * the lattice is periodic, so the first slab's neighbour below is the last
 * slab) -- by NCCL send/receive or a copy into the receiver's memory -- and
 * then calls bsm_dslash_slab with the two faces it received.  A face holds
 * the spin projection that the receiver's time-direction term needs, 2 spin
 * x d colour complex per site: half of the boundary spinor.  Precisions
 * BSM_F64 and BSM_F32; errors as bsm_dslash.  Not in the paper's form: the
 * paper decomposes over MPI ranks with its own halo format. */
typedef struct {
  bsm_lattice global;  /* the whole lattice */
  int32_t t0, nt;      /* the slab's first time slice and number of slices */
} bsm_slab;
typedef enum { BSM_FACE_LO = 0, BSM_FACE_HI = 1 } bsm_face_side;

/* Bytes of one face (X Y Z / 2 sites x 2 x d complex at prec); 0 if invalid. */
size_t bsm_face_bytes(const bsm_slab *slab, int32_t prec);

/* face = the spin projection (1 -+ g_0) of one boundary slice of the slab's
 * half spinor in_slab (parity in_parity): side BSM_FACE_LO the first slice,
 * projected for the forward term of the slab below, BSM_FACE_HI the last
 * slice, for the backward term of the slab above.  dagger must match the
 * receiver's bsm_dslash_slab call. */
int bsm_face_pack(const bsm_slab *slab, const void *in_slab, void *face, int32_t side,
                  int32_t in_parity, int32_t dagger, int32_t prec, void *stream);

/* out_slab = the hop H_{p,1-p} (bsm_dslash with out_parity p) on the slab's
 * sites, from its half spinor in_slab of parity 1 - p and the faces received
 * from the slab below (face_lo, that slab's BSM_FACE_HI face) and above
 * (face_hi, that slab's BSM_FACE_LO face).  U_rep: the representation links of
 * the GLOBAL lattice (bsm_links_to_rep on `global`; the slab reads its own
 * sites' links, boundary phases included).  Equals the slab's part of
 * bsm_dslash on the global lattice up to the order of the sums. */
int bsm_dslash_slab(const bsm_slab *slab, const void *U_rep, const void *in_slab,
                    const void *face_lo, const void *face_hi, void *out_slab,
                    int32_t out_parity, int32_t dagger, int32_t prec, void *stream);

/* Static text for a bsm_status. */
const char *bsm_strerror(int status);

/* Text of the last CUDA error seen by this library on the calling thread
 * ("" if none). */
const char *bsm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
