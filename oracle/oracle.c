/*
 * oracle.c -- plain FP64 CPU oracle (test infrastructure only; see oracle.h
 * for the conventions).  Straight loops over sites, directions, spins and
 * colours, written from the definitions so that each line can be checked by
 * eye.  No blocking, no fusion, no reordering beyond the definitions.
 *
 * The only concession to speed is an OpenMP "parallel for" over output sites
 * in orc_hop: every output site is an independent sum, so the result does
 * not depend on the number of threads.  All inner products are sequential.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* geometry (Sec. II-A)                                                 */
/* ------------------------------------------------------------------ */

static long volume(const orc_lattice *L) {
  return (long)L->dims[0] * L->dims[1] * L->dims[2] * L->dims[3];
}

static void site_coords(const orc_lattice *L, long s, int c[4]) {
  c[3] = (int)(s % L->dims[3]); s /= L->dims[3];
  c[2] = (int)(s % L->dims[2]); s /= L->dims[2];
  c[1] = (int)(s % L->dims[1]); s /= L->dims[1];
  c[0] = (int)s;
}

static long site_index(const orc_lattice *L, const int c[4]) {
  return (((long)c[0] * L->dims[1] + c[1]) * L->dims[2] + c[2]) * L->dims[3] + c[3];
}

/* neighbour of s one step in direction mu, sense dir = +1 or -1 (periodic) */
static long neighbour(const orc_lattice *L, long s, int mu, int dir) {
  int c[4];
  site_coords(L, s, c);
  c[mu] = (c[mu] + dir + L->dims[mu]) % L->dims[mu];
  return site_index(L, c);
}

static int site_parity(const orc_lattice *L, long s) {
  int c[4];
  site_coords(L, s, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* ------------------------------------------------------------------ */
/* gamma matrices (chiral Euclidean basis)                             */
/* ------------------------------------------------------------------ */

static void matmul4(const cplx A[4][4], const cplx B[4][4], cplx C[4][4]) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cplx s = 0;
      for (int k = 0; k < 4; ++k) s += A[i][k] * B[k][j];
      C[i][j] = s;
    }
}

/* g[0..3] = gamma_mu, g[4] = gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 */
static void build_gammas(cplx g[5][4][4]) {
  /* Pauli matrices sigma_1..3 (index 0 unused) */
  const cplx sigma[4][2][2] = {
      {{1, 0}, {0, 1}},
      {{0, 1}, {1, 0}},
      {{0, -I}, {I, 0}},
      {{1, 0}, {0, -1}},
  };
  memset(g, 0, sizeof(cplx) * 5 * 16);
  for (int mu = 0; mu < 4; ++mu) {
    /* off-diagonal blocks: upper-right B, lower-left B^+ */
    cplx B[2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        B[a][b] = (mu == 0) ? (a == b ? 1.0 : 0.0) : -I * sigma[mu][a][b];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        g[mu][a][2 + b] = B[a][b];
        g[mu][2 + a][b] = conj(B[b][a]);
      }
  }
  cplx t1[4][4], t2[4][4];
  matmul4(g[0], g[1], t1);
  matmul4(t1, g[2], t2);
  matmul4(t2, g[3], g[4]);
}

void orc_gamma(int mu, double *out) {
  cplx g[5][4][4];
  build_gammas(g);
  memcpy(out, g[mu], sizeof(cplx) * 16);
}

/* ------------------------------------------------------------------ */
/* representations (Sec. II-A: the fermion transforms under a          */
/* non-trivial representation of SU(N))                                */
/* ------------------------------------------------------------------ */

int orc_rep_dim(int N, int rep) {
  if (N < 2) return -1;
  switch (rep) {
    case ORC_FUND: return N;
    case ORC_ADJ: return N * N - 1;
    case ORC_SYM: return N * (N + 1) / 2;
    case ORC_ASYM: return N * (N - 1) / 2 >= 2 ? N * (N - 1) / 2 : -1;
    default: return -1;
  }
}

/* generalised Gell-Mann generator number a of SU(N), N x N, row-major */
static void gellmann(int N, int a, cplx *T) {
  memset(T, 0, sizeof(cplx) * N * N);
  const int noff = N * (N - 1) / 2;
  if (a < 2 * noff) {
    int k = a < noff ? a : a - noff, i = 0, j = 1;
    for (int n = 0; n < k; ++n) {   /* k-th pair (i<j) in lexicographic order */
      if (++j == N) { ++i; j = i + 1; }
    }
    if (a < noff) {                 /* symmetric: (E_ij + E_ji)/2 */
      T[i * N + j] = 0.5;
      T[j * N + i] = 0.5;
    } else {                        /* antisymmetric: -i (E_ij - E_ji)/2 */
      T[i * N + j] = -0.5 * I;
      T[j * N + i] = 0.5 * I;
    }
  } else {                          /* diagonal: l = 1..N-1 */
    int l = a - 2 * noff + 1;
    double norm = 1.0 / sqrt(2.0 * l * (l + 1));
    for (int i = 0; i < l; ++i) T[i * N + i] = norm;
    T[l * N + l] = -l * norm;
  }
}

/* two-index basis matrix number k, N x N: sym -> (i<=j), asym -> (i<j) */
static void twoindex_basis(int N, int sym, int k, cplx *e) {
  memset(e, 0, sizeof(cplx) * N * N);
  int n = 0;
  for (int i = 0; i < N; ++i)
    for (int j = sym ? i : i + 1; j < N; ++j, ++n) {
      if (n != k) continue;
      if (i == j) {
        e[i * N + i] = 1.0;
      } else {
        e[i * N + j] = 1.0 / sqrt(2.0);
        e[j * N + i] = (sym ? 1.0 : -1.0) / sqrt(2.0);
      }
    }
}

static void matmul(int N, const cplx *A, const cplx *B, cplx *C) {
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      cplx s = 0;
      for (int k = 0; k < N; ++k) s += A[i * N + k] * B[k * N + j];
      C[i * N + j] = s;
    }
}

static cplx trace(int N, const cplx *A) {
  cplx s = 0;
  for (int i = 0; i < N; ++i) s += A[i * N + i];
  return s;
}

int orc_rep_matrix(int N, int rep, const double *Ud, double *Rd) {
  const int d = orc_rep_dim(N, rep);
  if (d < 0) return -1;
  const cplx *U = (const cplx *)Ud;
  cplx *R = (cplx *)Rd;
  if (rep == ORC_FUND) {
    memcpy(R, U, sizeof(cplx) * N * N);
    return 0;
  }
  cplx *Ea = malloc(sizeof(cplx) * N * N), *Eb = malloc(sizeof(cplx) * N * N);
  cplx *Ut = malloc(sizeof(cplx) * N * N), *t1 = malloc(sizeof(cplx) * N * N);
  cplx *t2 = malloc(sizeof(cplx) * N * N), *t3 = malloc(sizeof(cplx) * N * N);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      Ut[i * N + j] = (rep == ORC_ADJ) ? conj(U[j * N + i]) /* U^+ */
                                       : U[j * N + i];      /* U^T */
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      if (rep == ORC_ADJ) {
        gellmann(N, a, Ea);
        gellmann(N, b, Eb);
      } else {
        twoindex_basis(N, rep == ORC_SYM, a, Ea);
        twoindex_basis(N, rep == ORC_SYM, b, Eb);
        /* Ea <- Ea^+ (the basis is real, so a transpose) */
        for (int i = 0; i < N; ++i)
          for (int j = 0; j < i; ++j) {
            cplx tmp = Ea[i * N + j];
            Ea[i * N + j] = conj(Ea[j * N + i]);
            Ea[j * N + i] = conj(tmp);
          }
      }
      matmul(N, U, Eb, t1);    /* U E_b          */
      matmul(N, t1, Ut, t2);   /* U E_b U^+ / U^T */
      matmul(N, Ea, t2, t3);   /* E_a (...)       */
      R[a * d + b] = (rep == ORC_ADJ ? 2.0 : 1.0) * trace(N, t3);
    }
  free(Ea); free(Eb); free(Ut); free(t1); free(t2); free(t3);
  return 0;
}

int orc_links_to_rep(const orc_lattice *L, const double *U, double *R) {
  const int N = L->N, d = orc_rep_dim(N, L->rep);
  if (d < 0) return -1;
  const long nlinks = volume(L) * 4;
  for (long l = 0; l < nlinks; ++l)
    if (orc_rep_matrix(N, L->rep, U + 2 * l * N * N, R + 2 * l * d * d)) return -1;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Dirac operator (Sec. II-B)                                          */
/* ------------------------------------------------------------------ */

void orc_hop(const orc_lattice *L, const double *Rd, const double *ind,
             double *outd, int out_parity, int dagger) {
  const int d = orc_rep_dim(L->N, L->rep);
  const long V = volume(L);
  const cplx *R = (const cplx *)Rd, *in = (const cplx *)ind;
  cplx *out = (cplx *)outd;
  cplx g[5][4][4];
  build_gammas(g);
  /* H^+ has the projectors (1 -+ g_mu) exchanged: sgn = -1 */
  const double sgn = dagger ? -1.0 : 1.0;

#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    cplx *o = out + s * 4 * d;
    for (int k = 0; k < 4 * d; ++k) o[k] = 0;
    if (out_parity != ORC_FULL && site_parity(L, s) != out_parity) continue;
    int c[4];
    site_coords(L, s, c);
    for (int mu = 0; mu < 4; ++mu) {
      /* forward: (1 - sgn g_mu) R(U_mu(x)) psi(x + mu) */
      {
        const long sf = neighbour(L, s, mu, +1);
        const cplx ph = (c[mu] == L->dims[mu] - 1) ? cexp(I * L->phase[mu]) : 1.0;
        const cplx *Rl = R + (s * 4 + mu) * d * d;
        const cplx *p = in + sf * 4 * d;
        for (int al = 0; al < 4; ++al)
          for (int a = 0; a < d; ++a) {
            cplx acc = 0;
            for (int be = 0; be < 4; ++be) {
              const cplx P = (al == be ? 1.0 : 0.0) - sgn * g[mu][al][be];
              if (P == 0) continue;
              for (int b = 0; b < d; ++b) acc += P * Rl[a * d + b] * p[be * d + b];
            }
            o[al * d + a] += ph * acc;
          }
      }
      /* backward: (1 + sgn g_mu) R(U_mu(x - mu))^+ psi(x - mu) */
      {
        const long sb = neighbour(L, s, mu, -1);
        const cplx ph = (c[mu] == 0) ? cexp(-I * L->phase[mu]) : 1.0;
        const cplx *Rl = R + (sb * 4 + mu) * d * d;
        const cplx *p = in + sb * 4 * d;
        for (int al = 0; al < 4; ++al)
          for (int a = 0; a < d; ++a) {
            cplx acc = 0;
            for (int be = 0; be < 4; ++be) {
              const cplx P = (al == be ? 1.0 : 0.0) + sgn * g[mu][al][be];
              if (P == 0) continue;
              for (int b = 0; b < d; ++b) acc += P * conj(Rl[b * d + a]) * p[be * d + b];
            }
            o[al * d + a] += ph * acc;
          }
      }
    }
  }
}

void orc_dirac(const orc_lattice *L, const double *R, const double *ind,
               double *outd, int dagger) {
  const int d = orc_rep_dim(L->N, L->rep);
  const long n = volume(L) * 4 * d;
  const double A = 4.0 + L->m0;
  const cplx *in = (const cplx *)ind;
  cplx *out = (cplx *)outd;
  orc_hop(L, R, ind, outd, ORC_FULL, dagger);
  for (long k = 0; k < n; ++k) out[k] = A * in[k] - 0.5 * out[k];
}

static void dhat_once(const orc_lattice *L, const double *R, const cplx *in,
                      cplx *out, cplx *tmp, int dagger) {
  const int d = orc_rep_dim(L->N, L->rep);
  const long V = volume(L);
  const double A = 4.0 + L->m0;
  orc_hop(L, R, (const double *)in, (double *)tmp, ORC_ODD, dagger);   /* H_oe */
  orc_hop(L, R, (const double *)tmp, (double *)out, ORC_EVEN, dagger); /* H_eo */
  for (long s = 0; s < V; ++s) {
    if (site_parity(L, s) != ORC_EVEN) continue;  /* odd sites stay zero */
    for (int k = 0; k < 4 * d; ++k)
      out[s * 4 * d + k] = A * in[s * 4 * d + k] - out[s * 4 * d + k] / (4.0 * A);
  }
}

void orc_dhat(const orc_lattice *L, const double *R, const double *ind,
              double *outd, int op) {
  const int d = orc_rep_dim(L->N, L->rep);
  const long n = volume(L) * 4 * d;
  const cplx *in = (const cplx *)ind;
  cplx *out = (cplx *)outd;
  cplx *tmp = malloc(sizeof(cplx) * n);
  if (op == ORC_DHAT_DAG_DHAT) {
    cplx *mid = malloc(sizeof(cplx) * n);
    dhat_once(L, R, in, mid, tmp, 0);
    dhat_once(L, R, mid, out, tmp, 1);
    free(mid);
  } else {
    dhat_once(L, R, in, out, tmp, op == ORC_DHAT_DAG);
  }
  free(tmp);
}

/* ------------------------------------------------------------------ */
/* CG on the normal equations (Sec. II-B)                              */
/* ------------------------------------------------------------------ */

static double norm2(long n, const cplx *a) {
  double s = 0;
  for (long k = 0; k < n; ++k) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
  return s;
}

/* y = M x with M = D^+ D (eo = 0) or Dhat^+ Dhat (eo = 1) */
static void normal_op(const orc_lattice *L, const double *R, int eo,
                      const cplx *x, cplx *y, cplx *tmp) {
  if (eo) {
    orc_dhat(L, R, (const double *)x, (double *)y, ORC_DHAT_DAG_DHAT);
  } else {
    orc_dirac(L, R, (const double *)x, (double *)tmp, 0);
    orc_dirac(L, R, (const double *)tmp, (double *)y, 1);
  }
}

int orc_cg(const orc_lattice *L, const double *R, const double *bd, double *xd,
           int eo, double tol, int max_iter, int use_x0, double *rel_res) {
  const int d = orc_rep_dim(L->N, L->rep);
  const long V = volume(L), n = V * 4 * d;
  const double A = 4.0 + L->m0;
  const cplx *b = (const cplx *)bd;
  cplx *x = (cplx *)xd;
  cplx *rhs = calloc(n, sizeof(cplx)), *r = calloc(n, sizeof(cplx));
  cplx *p = calloc(n, sizeof(cplx)), *Mp = calloc(n, sizeof(cplx));
  cplx *t1 = calloc(n, sizeof(cplx)), *xs = calloc(n, sizeof(cplx));

  /* right-hand side of the normal equations */
  if (eo) {
    /* bhat_e = b_e + 1/(2A) H_eo b_o ; rhs = Dhat^+ bhat_e */
    orc_hop(L, R, bd, (double *)t1, ORC_EVEN, 0);
    for (long s = 0; s < V; ++s)
      for (int k = 0; k < 4 * d; ++k)
        t1[s * 4 * d + k] = site_parity(L, s) == ORC_EVEN
                                ? b[s * 4 * d + k] + t1[s * 4 * d + k] / (2.0 * A)
                                : 0.0;
    orc_dhat(L, R, (const double *)t1, (double *)rhs, ORC_DHAT_DAG);
  } else {
    orc_dirac(L, R, bd, (double *)rhs, 1);
  }

  /* initial guess (even sites only in the eo case) */
  for (long s = 0; s < V; ++s)
    for (int k = 0; k < 4 * d; ++k)
      xs[s * 4 * d + k] = (use_x0 && (!eo || site_parity(L, s) == ORC_EVEN))
                              ? x[s * 4 * d + k] : 0.0;

  /* r = rhs - M x, p = r */
  normal_op(L, R, eo, xs, Mp, t1);
  for (long k = 0; k < n; ++k) {
    r[k] = rhs[k] - Mp[k];
    p[k] = r[k];
  }
  const double rhs2 = norm2(n, rhs);
  double rr = norm2(n, r);
  int it = 0, converged = rr <= tol * tol * rhs2;
  while (!converged && it < max_iter) {
    normal_op(L, R, eo, p, Mp, t1);
    double pMp = 0;
    for (long k = 0; k < n; ++k) pMp += creal(conj(p[k]) * Mp[k]);
    const double alpha = rr / pMp;
    for (long k = 0; k < n; ++k) {
      xs[k] += alpha * p[k];
      r[k] -= alpha * Mp[k];
    }
    const double rr_new = norm2(n, r);
    ++it;
    if (rr_new <= tol * tol * rhs2) {
      converged = 1;
      rr = rr_new;
      break;
    }
    const double beta = rr_new / rr;
    for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
    rr = rr_new;
  }
  if (rel_res) *rel_res = sqrt(rr / rhs2);

  /* solution; in the eo case reconstruct the odd sites:
   * x_o = (b_o + H_oe x_e / 2) / A */
  if (eo) {
    orc_hop(L, R, (const double *)xs, (double *)t1, ORC_ODD, 0);
    for (long s = 0; s < V; ++s)
      for (int k = 0; k < 4 * d; ++k)
        x[s * 4 * d + k] = site_parity(L, s) == ORC_EVEN
                               ? xs[s * 4 * d + k]
                               : (b[s * 4 * d + k] + 0.5 * t1[s * 4 * d + k]) / A;
  } else {
    memcpy(x, xs, sizeof(cplx) * n);
  }
  free(rhs); free(r); free(p); free(Mp); free(t1); free(xs);
  return converged ? it : -1;
}

/* ------------------------------------------------------------------ */
/* dense assembly and LU (checks on tiny lattices)                     */
/* ------------------------------------------------------------------ */

void orc_dense_dirac(const orc_lattice *L, const double *Rd, double *Md) {
  const int d = orc_rep_dim(L->N, L->rep);
  const long V = volume(L), n = V * 4 * d;
  const double A = 4.0 + L->m0;
  const cplx *R = (const cplx *)Rd;
  cplx *M = (cplx *)Md;
  cplx g[5][4][4];
  build_gammas(g);
  memset(M, 0, sizeof(cplx) * n * n);
  for (long s = 0; s < V; ++s) {
    int c[4];
    site_coords(L, s, c);
    for (int al = 0; al < 4; ++al)
      for (int a = 0; a < d; ++a) {
        const long row = (s * 4 + al) * d + a;
        M[row * n + row] += A;
        for (int mu = 0; mu < 4; ++mu) {
          const long sf = neighbour(L, s, mu, +1), sb = neighbour(L, s, mu, -1);
          const cplx phf = (c[mu] == L->dims[mu] - 1) ? cexp(I * L->phase[mu]) : 1.0;
          const cplx phb = (c[mu] == 0) ? cexp(-I * L->phase[mu]) : 1.0;
          for (int be = 0; be < 4; ++be)
            for (int b = 0; b < d; ++b) {
              const cplx Pm = (al == be ? 1.0 : 0.0) - g[mu][al][be];
              const cplx Pp = (al == be ? 1.0 : 0.0) + g[mu][al][be];
              const cplx Uf = R[(s * 4 + mu) * d * d + a * d + b];
              const cplx Ub = conj(R[(sb * 4 + mu) * d * d + b * d + a]);
              M[row * n + (sf * 4 + be) * d + b] += -0.5 * phf * Pm * Uf;
              M[row * n + (sb * 4 + be) * d + b] += -0.5 * phb * Pp * Ub;
            }
        }
      }
  }
}

int orc_lu_solve(int n, double *Ad, double *bd) {
  cplx *A = (cplx *)Ad, *b = (cplx *)bd;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (cabs(A[(long)i * n + k]) > cabs(A[(long)piv * n + k])) piv = i;
    if (cabs(A[(long)piv * n + k]) == 0.0) return -1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        cplx t = A[(long)k * n + j];
        A[(long)k * n + j] = A[(long)piv * n + j];
        A[(long)piv * n + j] = t;
      }
      cplx t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      const cplx f = A[(long)i * n + k] / A[(long)k * n + k];
      for (int j = k; j < n; ++j) A[(long)i * n + j] -= f * A[(long)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    cplx s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[(long)i * n + j] * b[j];
    b[i] = s / A[(long)i * n + i];
  }
  return 0;
}
