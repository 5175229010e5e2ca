/*
 * oracle.h -- plain FP64 CPU oracle for the even-odd Wilson-Dirac hot path
 * of BSMBench (Bennett et al., "BSMBench: A Flexible and Scalable HPC
 * Benchmark from Beyond the Standard Model Physics", HPCS 2016).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no source with the CUDA path.
 *
 * Everything here is the plain definition, written as straightforward loops
 * in IEEE double precision (compiled as ISO C11, so no FMA contraction):
 *
 *   geometry      Sec. II-A: a periodic L^3 x T hypercubic lattice, 8 nearest
 *                 neighbours, 4 links per site.
 *   fields        Sec. II-A: an N x N complex link per link; the fermion is a
 *                 d_R-component complex vector per site, which transforms
 *                 under a non-trivial representation R of SU(N).  The paper's
 *                 per-site count omits the 4 Dirac spin components; they are
 *                 stored here ([site][spin 4][colour d]).
 *   operator      Sec. II-B: the nearest-neighbour Dirac operator "Dphi".
 *                 The paper does not write it out; the standard Wilson form
 *                 (mass form, hopping normalised by 1/2) is used:
 *                   (D psi)(x) = A psi(x) - 1/2 H psi(x),   A = 4 + m0,
 *                   (H psi)(x) = sum_mu [ (1 - g_mu) R(U_mu(x)) psi(x+mu)
 *                                       + (1 + g_mu) R(U_mu(x-mu))^+ psi(x-mu) ].
 *   solver        Sec. II-B: CG (Hestenes-Stiefel) on the normal equations.
 *
 * Conventions (not fixed by the paper):
 *   dims = {T, X, Y, Z}; mu = 0 is time; canonical site index
 *   s = ((t*X + x)*Y + y)*Z + z.  parity(x) = (t+x+y+z) mod 2, even = 0.
 *   Links U[s][mu][a][b] (U_mu(x): link from x to x+mu).
 *   Spinors psi[s][spin][colour].
 *   Chiral Euclidean gamma basis: g_0 = [[0,1],[1,0]],
 *   g_k = [[0,-i sigma_k],[i sigma_k,0]], g_5 = g_0 g_1 g_2 g_3.
 *   Boundary phases: a hop that crosses the boundary of direction mu in the
 *   forward sense picks up exp(+i phi_mu), in the backward sense exp(-i phi_mu)
 *   (phi = pi gives antiperiodic boundary conditions).
 *   Representation bases:
 *     FUND  R(U) = U.
 *     ADJ   R_ab = 2 Tr(T^a U T^b U^+), generalised Gell-Mann T^a with
 *           Tr(T^a T^b) = delta_ab / 2, ordered: symmetric off-diagonal
 *           (i<j lexicographic), antisymmetric off-diagonal, diagonal.
 *     SYM / ASYM  R_(ij),(kl) = Tr(e_(ij)^+ U e_(kl) U^T) with the orthonormal
 *           basis e_(ii) = E_ii, e_(ij) = (E_ij +- E_ji)/sqrt2 (i<j),
 *           lexicographic in (i,j), i<=j for SYM and i<j for ASYM.
 *
 * Complex numbers cross this interface as interleaved (re, im) doubles.
 */
#ifndef BSM_ORACLE_H
#define BSM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FUND = 0, ORC_ADJ = 1, ORC_SYM = 2, ORC_ASYM = 3 };
enum { ORC_EVEN = 0, ORC_ODD = 1, ORC_FULL = 2 };
enum { ORC_DHAT = 0, ORC_DHAT_DAG = 1, ORC_DHAT_DAG_DHAT = 2 };

typedef struct {
  int dims[4];      /* {T, X, Y, Z} */
  int N;            /* gauge group SU(N) */
  int rep;          /* ORC_FUND .. ORC_ASYM */
  double m0;        /* Wilson bare mass; A = 4 + m0 */
  double phase[4];  /* boundary phases phi_mu (radians) */
} orc_lattice;

/* Dimension d_R of representation `rep` of SU(N); -1 if N < 2 or the
 * representation is trivial (Sec. II-A requires a non-trivial one). */
int orc_rep_dim(int N, int rep);

/* g_mu for mu = 0..3 and g_5 for mu = 4, as a 4x4 row-major complex matrix. */
void orc_gamma(int mu, double *g);

/* R(U) for one N x N matrix U (Sec. II-A representation constraint). */
int orc_rep_matrix(int N, int rep, const double *U, double *R);

/* Representation links R[s][mu] = R(U_mu(s)) for the whole lattice.  No
 * boundary phase is folded in: the operator applies the phases itself. */
int orc_links_to_rep(const orc_lattice *L, const double *U, double *R);

/* Hopping term H (or its adjoint when dagger != 0) of Sec. II-B.  out is
 * written on the sites of parity out_parity (every site for ORC_FULL) and set
 * to zero elsewhere.  For a parity block only the neighbours, i.e. the sites
 * of the other parity, of `in` are read. */
void orc_hop(const orc_lattice *L, const double *R, const double *in,
             double *out, int out_parity, int dagger);

/* Full Wilson-Dirac operator D = A - H/2 (D^+ when dagger != 0). */
void orc_dirac(const orc_lattice *L, const double *R, const double *in,
               double *out, int dagger);

/* Even-odd Schur operator on the even sites:
 *   Dhat = A - 1/(4A) H_eo H_oe,  Dhat^+ = A - 1/(4A) H^+_eo H^+_oe.
 * in/out are full-lattice arrays; only even sites of `in` are read and the
 * odd sites of `out` are zeroed. */
void orc_dhat(const orc_lattice *L, const double *R, const double *in,
              double *out, int op);

/* CG on the normal equations (Sec. II-B).  eo = 0: D^+ D x = D^+ b on the
 * whole lattice.  eo = 1: the even-odd reduced system
 *   Dhat^+ Dhat x_e = Dhat^+ (b_e + 1/(2A) H_eo b_o),
 * followed by x_o = (b_o + H_oe x_e / 2) / A.  Stops when the iterated
 * residual satisfies |r| <= tol |rhs|.  x holds the initial guess on entry
 * when use_x0 != 0 (else zero) and the full-lattice solution on exit.
 * Returns the iteration count, or -1 if max_iter was reached.  *rel_res gets
 * the final iterated |r|/|rhs|. */
int orc_cg(const orc_lattice *L, const double *R, const double *b, double *x,
           int eo, double tol, int max_iter, int use_x0, double *rel_res);

/* Dense matrix of D, assembled entry by entry from the definition
 * (n = V*4*d rows, row index (s*4 + spin)*d + colour, row-major).  On a
 * lattice with L_mu = 2 both neighbours of a site coincide and both terms
 * add into the same block. */
void orc_dense_dirac(const orc_lattice *L, const double *R, double *M);

/* Gaussian elimination with partial pivoting: solves A x = b in place
 * (A is destroyed, b becomes x).  Returns 0, or -1 on a zero pivot. */
int orc_lu_solve(int n, double *A, double *b);

#ifdef __cplusplus
}
#endif
#endif
