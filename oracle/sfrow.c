/*
 * sfrow.c -- row-wise, sum-factorised FP64 formation of mass and Laplace-stiffness rows,
 * and of the weighted-quadrature load vector.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: only tests/, __graft_entry__.smoke()
 * and the CPU legs of bench.py load this library.  It shares no code with the CUDA library.
 *
 * It computes the oracle's method O2 (oracle/formation.py) row by row, with every 3D
 * quadrature sum evaluated one direction at a time -- the "row loop" + "sum factorization"
 * entry of the paper's cost table for weighted quadrature (Sec. 1, Table 2):
 *
 *   interior row i:  A_ij = sum_q w_i1(q1) w_i2(q2) w_i3(q3) c(x_q) B_j(x_q)      (mass)
 *                    stiffness: the sum over d of the same with the derivative rule w11
 *                    and B_j' in direction d;
 *   cut row i (Sec. 2.2, Eq. 1, support split into regular and cut parts): the DWQ box
 *                    (one-sided DWQ rule in the box direction, standard rules in the other
 *                    two), plus Gauss points of every inside support element outside the
 *                    box, plus the Gauss points of the octree pieces of every cut support
 *                    element (Sec. 3.1, sub-elements with Gauss rules).
 *
 * Variants (Sec. 3.1): DWQ (the method), Hybrid Gauss (no box: the whole regular part of a
 * cut row by element Gauss points) and Standard Gauss (every row, interior ones included,
 * by element Gauss points over its whole support; the rows of the element-loop matrix).
 *
 * The 1D rules (standard WQ and one-sided DWQ weights on the Gauss superset) and the
 * geometry (element states, octree pieces, function classes, boxes) are inputs, taken from
 * the numpy oracle.  B-spline values come from the Cox-de Boor recursion written out below;
 * the coefficient field is evaluated from its definition, sum_k c_k N_k1 N_k2 N_k3 over the
 * (p+1)^3 block of each point, with the three 1D sums nested.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OSF_MAXP 6
#define OSF_Q (OSF_MAXP + 1)
#define OSF_NB (2 * OSF_MAXP + 1)
#define OSF_NPT 64 /* points per direction of one rule (a rule has at most (p+1)^2 = 49) */

typedef struct {
  int32_t p, variant, coef_kind, src_kind;
  int32_t n_el[3], n[3], nsup[3];
  const double* U[3];      /* open knot vectors, n_el + 2p + 1 */
  const double* t_sup[3];  /* Gauss superset points, n_el (p+1) */
  const double* w_sup[3];  /* Gauss superset weights */
  const double* std00[3];  /* standard WQ rules, dense over the superset: [n][nsup] */
  const double* std11[3];
  const int32_t* dwq_id[3]; /* [n][p][2]: index of the one-sided DWQ rule (i, b, side) or -1 */
  const double* dwq00[3];  /* [rules][nsup] */
  const double* dwq11[3];
  const int8_t* elem_state; /* n_el1 n_el2 n_el3: 0 out, 1 in, 2 cut with pieces, 3 cut without */
  const int8_t* fclass;     /* n1 n2 n3: 0 exterior, 1 interior, 2 cut */
  const int32_t* box;       /* n1 n2 n3: -1 or d | side << 2 | b << 3 */
  const int64_t* piece_ptr; /* pieces of element e: [piece_ptr[e], piece_ptr[e + 1]) */
  const double* piece_box;  /* [pieces][3][2]: (lo, hi) per direction */
  const double* xg;         /* (p+1)-point Gauss-Legendre nodes on [-1, 1] */
  const double* wg;
  double c0;                /* constant coefficient */
  const double* ck;         /* B-spline coefficients, index k1 + n1 (k2 + n2 k3) */
  const int64_t* rowptr;
  const int32_t* colind;
} osf_mesh;

enum { COEF_CONST = 0, COEF_ANALYTIC = 1, COEF_BSPLINE = 2 };
enum { VAR_DWQ = 0, VAR_HYBRID = 1, VAR_GAUSS = 2 };
enum { E_OUT = 0, E_IN = 1, E_CUT = 2 };
enum { F_EXT = 0, F_INT = 1, F_CUT = 2 };
/* load-vector source f: the coefficient field itself, or the paper's sin(2xz) cos(3yz) */
enum { SRC_COEF = 0, SRC_PAPER = 1 };

/* ---------------------------------------------------------------------------------------
 * B-spline values by the Cox-de Boor recursion (de Boor 1978):
 *   N_{j,0} = 1 on [U_j, U_{j+1}),
 *   N_{j,k} = (x - U_j) / (U_{j+k} - U_j) N_{j,k-1} + (U_{j+k+1} - x) / (U_{j+k+1} - U_{j+1}) N_{j+1,k-1}
 * (a term with a zero denominator is dropped), and the derivative
 *   N'_{j,p} = p / (U_{j+p} - U_j) N_{j,p-1} - p / (U_{j+p+1} - U_{j+1}) N_{j+1,p-1}.
 * With span s (U_s <= x < U_{s+1}) the nonzero functions are j = s - p .. s; N[r] and dN[r]
 * receive function s - p + r. */
static void basis(const double* U, int p, int s, double x, double* N, double* dN) {
  double T[OSF_Q][OSF_Q]; /* T[k][r] = N_{s-k+r, k}(x), r = 0..k */
  T[0][0] = 1.0;
  for (int k = 1; k <= p; ++k) {
    for (int r = 0; r <= k; ++r) {
      const int j = s - k + r;
      double v = 0.0;
      if (r >= 1) {
        const double den = U[j + k] - U[j];
        if (den != 0.0) v += (x - U[j]) / den * T[k - 1][r - 1];
      }
      if (r <= k - 1) {
        const double den = U[j + k + 1] - U[j + 1];
        if (den != 0.0) v += (U[j + k + 1] - x) / den * T[k - 1][r];
      }
      T[k][r] = v;
    }
  }
  for (int r = 0; r <= p; ++r) {
    const int j = s - p + r;
    double d = 0.0;
    if (r >= 1) {
      const double den = U[j + p] - U[j];
      if (den != 0.0) d += p / den * T[p - 1][r - 1];
    }
    if (r <= p - 1) {
      const double den = U[j + p + 1] - U[j + 1];
      if (den != 0.0) d -= p / den * T[p - 1][r];
    }
    N[r] = T[p][r];
    dN[r] = d;
  }
}

/* Element containing x: the e with U[e+p] <= x < U[e+p+1], clipped to [0, n_el - 1]. */
static int element_of(const double* U, int p, int n_el, double x) {
  int lo = 0, hi = n_el - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (U[mid + p] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

/* ---------------------------------------------------------------------------------------
 * Per-thread scratch. */
typedef struct {
  double c[OSF_NPT * OSF_NPT * OSF_NPT];         /* coefficient (or source) on a point grid */
  double s1[OSF_NPT * OSF_NB * OSF_NB];          /* coefficient sums, stage 1 */
  double s2[OSF_NPT * OSF_NPT * OSF_NB];         /* stage 2 */
  double F[OSF_NPT * OSF_NPT * OSF_NPT];         /* weighted integrand */
  double t1[OSF_NB * OSF_NPT * OSF_NPT];         /* contraction stages */
  double t2[OSF_NB * OSF_NB * OSF_NPT];
  double V[OSF_NB * OSF_NB * OSF_NB];            /* the row's dense band, [j3][j2][j1] */
} scratch_t;

/* Points of one direction of a tensor grid with their element and basis values. */
typedef struct {
  int np;
  double t[OSF_NPT], w[OSF_NPT];
  int e[OSF_NPT];
  double N[OSF_NPT][OSF_Q], dN[OSF_NPT][OSF_Q];
} dirpts_t;

static void dir_basis(const osf_mesh* m, int d, dirpts_t* P) {
  for (int k = 0; k < P->np; ++k) {
    P->e[k] = element_of(m->U[d], m->p, m->n_el[d], P->t[k]);
    basis(m->U[d], m->p, P->e[k] + m->p, P->t[k], P->N[k], P->dN[k]);
  }
}

/* B^(kind)_j(t_k) for function j (0 outside the p+1 nonzero functions at t_k). */
static double bval(const dirpts_t* P, int p, int k, int j, int kind) {
  const int r = j - P->e[k];
  if (r < 0 || r > p) return 0.0;
  return kind ? P->dN[k][r] : P->N[k][r];
}

/* Coefficient c(x) at every point of the grid P0 x P1 x P2 (index k0 + n0 (k1 + n1 k2)). */
static void coef_grid(const osf_mesh* m, const dirpts_t* P, scratch_t* S, int which) {
  const int n0 = P[0].np, n1 = P[1].np, n2 = P[2].np, p = m->p;
  double* c = S->c;
  if (which == 1) { /* the paper's load-vector source f = sin(2 x z) cos(3 y z) */
    for (int k2 = 0; k2 < n2; ++k2)
      for (int k1 = 0; k1 < n1; ++k1)
        for (int k0 = 0; k0 < n0; ++k0) {
          const double x = P[0].t[k0], y = P[1].t[k1], z = P[2].t[k2];
          c[k0 + n0 * (k1 + n1 * k2)] = sin(2.0 * x * z) * cos(3.0 * y * z);
        }
    return;
  }
  if (m->coef_kind == COEF_CONST) {
    for (int k = 0; k < n0 * n1 * n2; ++k) c[k] = m->c0;
    return;
  }
  if (m->coef_kind == COEF_ANALYTIC) {
    const double twopi = 2.0 * 3.14159265358979323846;
    for (int k2 = 0; k2 < n2; ++k2)
      for (int k1 = 0; k1 < n1; ++k1)
        for (int k0 = 0; k0 < n0; ++k0)
          c[k0 + n0 * (k1 + n1 * k2)] =
              1.0 + 0.5 * sin(twopi * P[0].t[k0]) * cos(twopi * P[1].t[k1]) * P[2].t[k2];
    return;
  }
  /* B-spline field: c(x) = sum_{a} ck[e1+a1, e2+a2, e3+a3] N_a1(x1) N_a2(x2) N_a3(x3), the
   * sums over a1, a2, a3 nested (coefficient rows b of directions 1 and 2 that the grid's
   * points touch: [lo_d, lo_d + nb_d)). */
  int lo[3], nb[3];
  for (int d = 0; d < 3; ++d) {
    int a = P[d].e[0], b = P[d].e[0];
    for (int k = 1; k < P[d].np; ++k) {
      if (P[d].e[k] < a) a = P[d].e[k];
      if (P[d].e[k] > b) b = P[d].e[k];
    }
    lo[d] = a;
    nb[d] = b + p - a + 1;
  }
  const int cn0 = m->n[0], cn1 = m->n[1];
  /* s1[k0][b1][b2] = sum_a0 N0(k0, a0) ck[e0(k0) + a0, b1, b2] */
  for (int k0 = 0; k0 < n0; ++k0)
    for (int b2 = 0; b2 < nb[2]; ++b2)
      for (int b1 = 0; b1 < nb[1]; ++b1) {
        double s = 0.0;
        for (int a0 = 0; a0 <= p; ++a0)
          s += P[0].N[k0][a0] * m->ck[(P[0].e[k0] + a0) + (int64_t)cn0 * ((lo[1] + b1) + (int64_t)cn1 * (lo[2] + b2))];
        S->s1[(k0 * nb[1] + b1) * nb[2] + b2] = s;
      }
  /* s2[k0][k1][b2] = sum_a1 N1(k1, a1) s1[k0][e1(k1) + a1 - lo1][b2] */
  for (int k0 = 0; k0 < n0; ++k0)
    for (int k1 = 0; k1 < n1; ++k1)
      for (int b2 = 0; b2 < nb[2]; ++b2) {
        double s = 0.0;
        for (int a1 = 0; a1 <= p; ++a1)
          s += P[1].N[k1][a1] * S->s1[(k0 * nb[1] + (P[1].e[k1] + a1 - lo[1])) * nb[2] + b2];
        S->s2[(k0 * n1 + k1) * nb[2] + b2] = s;
      }
  /* c[k0, k1, k2] = sum_a2 N2(k2, a2) s2[k0][k1][e2(k2) + a2 - lo2] */
  for (int k2 = 0; k2 < n2; ++k2)
    for (int k1 = 0; k1 < n1; ++k1)
      for (int k0 = 0; k0 < n0; ++k0) {
        double s = 0.0;
        for (int a2 = 0; a2 <= p; ++a2) s += P[2].N[k2][a2] * S->s2[(k0 * n1 + k1) * nb[2] + (P[2].e[k2] + a2 - lo[2])];
        c[k0 + n0 * (k1 + n1 * k2)] = s;
      }
}

/* V[j] += sum_g F(g) Phi_j1(g0) Phi_j2(g1) Phi_j3(g2) over a tensor grid, for the band
 * columns j_d in [blo_d, blo_d + bw_d): three contractions, direction 1 first.
 * Phi[d][k][jj] is the trial factor of direction d at point k for column blo_d + jj. */
static void contract_band(const int* np, const int* bw, const double* F, double (*Phi[3])[OSF_NB], scratch_t* S,
                          double* V) {
  const int n0 = np[0], n1 = np[1], n2 = np[2];
  /* t1[j0][k1][k2] = sum_k0 Phi0[k0][j0] F[k0, k1, k2] */
  for (int j0 = 0; j0 < bw[0]; ++j0)
    for (int k2 = 0; k2 < n2; ++k2)
      for (int k1 = 0; k1 < n1; ++k1) {
        double s = 0.0;
        for (int k0 = 0; k0 < n0; ++k0) s += Phi[0][k0][j0] * F[k0 + n0 * (k1 + n1 * k2)];
        S->t1[(j0 * n1 + k1) * n2 + k2] = s;
      }
  /* t2[j0][j1][k2] = sum_k1 Phi1[k1][j1] t1[j0][k1][k2] */
  for (int j0 = 0; j0 < bw[0]; ++j0)
    for (int j1 = 0; j1 < bw[1]; ++j1)
      for (int k2 = 0; k2 < n2; ++k2) {
        double s = 0.0;
        for (int k1 = 0; k1 < n1; ++k1) s += Phi[1][k1][j1] * S->t1[(j0 * n1 + k1) * n2 + k2];
        S->t2[(j0 * bw[1] + j1) * n2 + k2] = s;
      }
  /* V[j2][j1][j0] += sum_k2 Phi2[k2][j2] t2[j0][j1][k2] */
  for (int j2 = 0; j2 < bw[2]; ++j2)
    for (int j1 = 0; j1 < bw[1]; ++j1)
      for (int j0 = 0; j0 < bw[0]; ++j0) {
        double s = 0.0;
        for (int k2 = 0; k2 < n2; ++k2) s += Phi[2][k2][j2] * S->t2[(j0 * bw[1] + j1) * n2 + k2];
        V[(j2 * bw[1] + j1) * bw[0] + j0] += s;
      }
}

/* Kinds of the terms: mass one term (0,0,0); stiffness the three placements of the
 * derivative (kind 1 = derivative rule w11 and B' in that direction). */
static int op_terms(int op, int kinds[3][3]) {
  if (op == 0) {
    kinds[0][0] = kinds[0][1] = kinds[0][2] = 0;
    return 1;
  }
  for (int t = 0; t < 3; ++t)
    for (int d = 0; d < 3; ++d) kinds[t][d] = (t == d);
  return 3;
}

/* The weighted-quadrature part of row i: the tensor grid of each direction's rule (standard,
 * or the one-sided DWQ rule in the box direction), with the test function folded into the
 * weights.  mode 0: matrix band into V; mode 1: load value sum_q W(q) f(x_q) into *load. */
static int wq_part(const osf_mesh* m, const int* idx, int box, int op, const int* blo, const int* bw, scratch_t* S,
                   double* V, int mode, double* load) {
  const int p = m->p;
  int kinds[3][3];
  const int nt = mode ? 1 : op_terms(op, kinds);
  if (mode) kinds[0][0] = kinds[0][1] = kinds[0][2] = 0;
  const int bd = box >= 0 ? (box & 3) : -1, bside = (box >> 2) & 1, bb = box >> 3;
  for (int t = 0; t < nt; ++t) {
    dirpts_t P[3];
    for (int d = 0; d < 3; ++d) {
      const double* w;
      const int id = idx[d], ns = m->nsup[d];
      if (d == bd) {
        const int elo = id - p > 0 ? id - p : 0;
        const int slot = bb - elo - 1;
        if (slot < 0 || slot >= p) return -2;
        const int r = m->dwq_id[d][(id * p + slot) * 2 + bside];
        if (r < 0) return -3; /* rule not supplied */
        w = (kinds[t][d] ? m->dwq11[d] : m->dwq00[d]) + (int64_t)r * ns;
      } else {
        w = (kinds[t][d] ? m->std11[d] : m->std00[d]) + (int64_t)id * ns;
      }
      /* points of the rule: the superset points with a nonzero weight (a zero weight adds an
       * exact zero to every sum it appears in) */
      int np = 0;
      for (int s = 0; s < ns; ++s)
        if (w[s] != 0.0) {
          if (np >= OSF_NPT) return -4;
          P[d].t[np] = m->t_sup[d][s];
          P[d].w[np] = w[s];
          ++np;
        }
      P[d].np = np;
      if (np == 0) goto next_term;
      dir_basis(m, d, &P[d]);
    }
    {
      coef_grid(m, P, S, mode ? m->src_kind : 0);
      const int np3[3] = {P[0].np, P[1].np, P[2].np};
      for (int k2 = 0; k2 < np3[2]; ++k2)
        for (int k1 = 0; k1 < np3[1]; ++k1)
          for (int k0 = 0; k0 < np3[0]; ++k0) {
            const int k = k0 + np3[0] * (k1 + np3[1] * k2);
            S->F[k] = P[0].w[k0] * P[1].w[k1] * P[2].w[k2] * S->c[k];
          }
      if (mode) {
        double s = 0.0;
        for (int k = 0; k < np3[0] * np3[1] * np3[2]; ++k) s += S->F[k];
        *load += s;
        continue;
      }
      static __thread double phi[3][OSF_NPT][OSF_NB];
      for (int d = 0; d < 3; ++d)
        for (int k = 0; k < P[d].np; ++k)
          for (int jj = 0; jj < bw[d]; ++jj) phi[d][k][jj] = bval(&P[d], p, k, blo[d] + jj, kinds[t][d]);
      double(*Phi[3])[OSF_NB] = {phi[0], phi[1], phi[2]};
      contract_band(np3, bw, S->F, Phi, S, V);
    }
  next_term:;
  }
  return 0;
}

/* Gauss points of one tensor-product cell (an inside element, or an octree piece of a cut
 * element) inside element (e0, e1, e2): adds sum_g w_g c(x_g) Phi_i(x_g) Phi_j(x_g) to the
 * band for the p+1 local functions j_d = e_d .. e_d + p (mode 0), or sum_g w_g f(x_g) Phi_i
 * to *load (mode 1). */
static void gauss_cell(const osf_mesh* m, const int* idx, const int* e, const dirpts_t* Pin, int op, const int* blo,
                       const int* bw, scratch_t* S, double* V, int mode, double* load) {
  const int p = m->p, Q = p + 1;
  dirpts_t P[3];
  for (int d = 0; d < 3; ++d) {
    P[d] = Pin[d];
    for (int k = 0; k < Q; ++k) {
      P[d].e[k] = e[d];
      basis(m->U[d], p, e[d] + p, P[d].t[k], P[d].N[k], P[d].dN[k]);
    }
  }
  coef_grid(m, P, S, mode ? m->src_kind : 0);
  int kinds[3][3];
  const int nt = mode ? 1 : op_terms(op, kinds);
  if (mode) kinds[0][0] = kinds[0][1] = kinds[0][2] = 0;
  const int np3[3] = {Q, Q, Q};
  for (int t = 0; t < nt; ++t) {
    for (int g2 = 0; g2 < Q; ++g2)
      for (int g1 = 0; g1 < Q; ++g1)
        for (int g0 = 0; g0 < Q; ++g0) {
          const int g = g0 + Q * (g1 + Q * g2);
          const double fi = bval(&P[0], p, g0, idx[0], kinds[t][0]) * bval(&P[1], p, g1, idx[1], kinds[t][1]) *
                            bval(&P[2], p, g2, idx[2], kinds[t][2]);
          S->F[g] = P[0].w[g0] * P[1].w[g1] * P[2].w[g2] * S->c[g] * fi;
        }
    if (mode) {
      double s = 0.0;
      for (int g = 0; g < Q * Q * Q; ++g) s += S->F[g];
      *load += s;
      continue;
    }
    /* the p+1 local functions j_d = e_d + b of each direction (all inside the row's band),
     * then added into the band */
    static __thread double phi[3][OSF_NPT][OSF_NB];
    static __thread double loc[OSF_Q * OSF_Q * OSF_Q];
    for (int d = 0; d < 3; ++d)
      for (int k = 0; k < Q; ++k)
        for (int b = 0; b < Q; ++b) phi[d][k][b] = bval(&P[d], p, k, e[d] + b, kinds[t][d]);
    double(*Phi[3])[OSF_NB] = {phi[0], phi[1], phi[2]};
    memset(loc, 0, sizeof(double) * Q * Q * Q);
    contract_band(np3, np3, S->F, Phi, S, loc);
    for (int b2 = 0; b2 < Q; ++b2)
      for (int b1 = 0; b1 < Q; ++b1)
        for (int b0 = 0; b0 < Q; ++b0)
          V[((e[2] + b2 - blo[2]) * bw[1] + (e[1] + b1 - blo[1])) * bw[0] + (e[0] + b0 - blo[0])] +=
              loc[(b2 * Q + b1) * Q + b0];
  }
}

/* The Gauss part of row i: every inside support element outside the box (all of them with
 * no box), with its own (p+1)^3 Gauss points, and every cut support element with the Gauss
 * points of its octree pieces. */
static void gauss_part(const osf_mesh* m, const int* idx, int box, int op, const int* blo, const int* bw, scratch_t* S,
                       double* V, int mode, double* load) {
  const int p = m->p, Q = p + 1;
  int elo[3], ehi[3];
  for (int d = 0; d < 3; ++d) {
    elo[d] = idx[d] - p > 0 ? idx[d] - p : 0;
    ehi[d] = idx[d] < m->n_el[d] - 1 ? idx[d] : m->n_el[d] - 1;
  }
  const int bd = box >= 0 ? (box & 3) : -1, bside = (box >> 2) & 1, bb = box >> 3;
  for (int e2 = elo[2]; e2 <= ehi[2]; ++e2)
    for (int e1 = elo[1]; e1 <= ehi[1]; ++e1)
      for (int e0 = elo[0]; e0 <= ehi[0]; ++e0) {
        const int64_t e = e0 + (int64_t)m->n_el[0] * (e1 + (int64_t)m->n_el[1] * e2);
        const int st = m->elem_state[e];
        const int ee[3] = {e0, e1, e2};
        dirpts_t P[3];
        if (st == E_IN) {
          if (bd >= 0) {
            const int ed = ee[bd];
            if ((bside == 0 && ed < bb) || (bside == 1 && ed >= bb)) continue; /* in the DWQ box */
          }
          for (int d = 0; d < 3; ++d) {
            P[d].np = Q;
            for (int g = 0; g < Q; ++g) {
              P[d].t[g] = m->t_sup[d][ee[d] * Q + g];
              P[d].w[g] = m->w_sup[d][ee[d] * Q + g];
            }
          }
          gauss_cell(m, idx, ee, P, op, blo, bw, S, V, mode, load);
        } else if (st == E_CUT) {
          for (int64_t pc = m->piece_ptr[e]; pc < m->piece_ptr[e + 1]; ++pc) {
            const double* bx = m->piece_box + pc * 6;
            for (int d = 0; d < 3; ++d) {
              const double a = bx[2 * d], b = bx[2 * d + 1];
              const double mid = 0.5 * (a + b), half = 0.5 * (b - a);
              P[d].np = Q;
              for (int g = 0; g < Q; ++g) {
                P[d].t[g] = mid + half * m->xg[g];
                P[d].w[g] = half * m->wg[g];
              }
            }
            gauss_cell(m, idx, ee, P, op, blo, bw, S, V, mode, load);
          }
        }
      }
}

/* One row: its dense band (order j3, j2, j1) written onto its pattern columns. */
static int form_row(const osf_mesh* m, int op, int64_t i, scratch_t* S, double* out) {
  const int p = m->p, n0 = m->n[0], n1 = m->n[1];
  const int idx[3] = {(int)(i % n0), (int)((i / n0) % n1), (int)(i / ((int64_t)n0 * n1))};
  int blo[3], bw[3];
  for (int d = 0; d < 3; ++d) {
    blo[d] = idx[d] - p > 0 ? idx[d] - p : 0;
    const int bhi = idx[d] + p < m->n[d] - 1 ? idx[d] + p : m->n[d] - 1;
    bw[d] = bhi - blo[d] + 1;
  }
  memset(S->V, 0, sizeof(double) * bw[0] * bw[1] * bw[2]);
  const int cls = m->fclass[i];
  if (cls == F_EXT) return 0;
  const int box = (cls == F_CUT && m->variant == VAR_DWQ) ? m->box[i] : -1;
  if (m->variant == VAR_GAUSS) {
    gauss_part(m, idx, -1, op, blo, bw, S, S->V, 0, NULL);
  } else {
    if (cls == F_INT || box >= 0) {
      const int r = wq_part(m, idx, box, op, blo, bw, S, S->V, 0, NULL);
      if (r) return r;
    }
    if (cls == F_CUT) gauss_part(m, idx, box, op, blo, bw, S, S->V, 0, NULL);
  }
  for (int64_t k = m->rowptr[i]; k < m->rowptr[i + 1]; ++k) {
    const int64_t j = m->colind[k];
    const int j0 = (int)(j % n0), j1 = (int)((j / n0) % n1), j2 = (int)(j / ((int64_t)n0 * n1));
    out[k - m->rowptr[i]] = S->V[((j2 - blo[2]) * bw[1] + (j1 - blo[1])) * bw[0] + (j0 - blo[0])];
  }
  return 0;
}

/* Load value b_i = "int f B_i" of row i by the same rules (Sec. 3.1 target function). */
static int load_row(const osf_mesh* m, int64_t i, scratch_t* S, double* out) {
  const int p = m->p, n0 = m->n[0], n1 = m->n[1];
  const int idx[3] = {(int)(i % n0), (int)((i / n0) % n1), (int)(i / ((int64_t)n0 * n1))};
  int blo[3], bw[3];
  for (int d = 0; d < 3; ++d) {
    blo[d] = idx[d] - p > 0 ? idx[d] - p : 0;
    bw[d] = 1;
  }
  double b = 0.0;
  const int cls = m->fclass[i];
  if (cls != F_EXT) {
    const int box = (cls == F_CUT && m->variant == VAR_DWQ) ? m->box[i] : -1;
    if (m->variant == VAR_GAUSS) {
      gauss_part(m, idx, -1, 0, blo, bw, S, NULL, 1, &b);
    } else {
      if (cls == F_INT || box >= 0) {
        const int r = wq_part(m, idx, box, 0, blo, bw, S, NULL, 1, &b);
        if (r) return r;
      }
      if (cls == F_CUT) gauss_part(m, idx, box, 0, blo, bw, S, NULL, 1, &b);
    }
  }
  *out = b;
  return 0;
}

typedef struct {
  const osf_mesh* m;
  int op, load;
  const int64_t* rows;
  int64_t nrows;
  const int64_t* out_off;
  double* out;
  int64_t next;
  int err;
} job_t;

static void* worker(void* arg) {
  job_t* J = (job_t*)arg;
  scratch_t* S = (scratch_t*)malloc(sizeof(scratch_t));
  if (!S) {
    __atomic_store_n(&J->err, -1, __ATOMIC_RELAXED);
    return NULL;
  }
  for (;;) {
    const int64_t k = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
    if (k >= J->nrows) break;
    const int r = J->load ? load_row(J->m, J->rows[k], S, J->out + k)
                          : form_row(J->m, J->op, J->rows[k], S, J->out + J->out_off[k]);
    if (r) __atomic_store_n(&J->err, r, __ATOMIC_RELAXED);
  }
  free(S);
  return NULL;
}

static int run(job_t* J, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 1; t < nthreads; ++t)
    if (pthread_create(&th[started], NULL, worker, J) == 0) ++started;
  worker(J);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  return J->err;
}

/* Rows rows[0..nrows) of operator op (0 mass, 1 stiffness); row k's values (its pattern
 * columns, ascending) go to out + out_off[k].  Returns 0, or a negative code if a DWQ rule
 * a box needs was not supplied. */
int osf_form_rows(const osf_mesh* m, int op, const int64_t* rows, int64_t nrows, const int64_t* out_off, double* out,
                  int nthreads) {
  if (!m || m->p < 1 || m->p > OSF_MAXP) return -1;
  job_t J = {m, op, 0, rows, nrows, out_off, out, 0, 0};
  return run(&J, nthreads);
}

/* Load values b_i for rows rows[0..nrows) into out[k]. */
int osf_load_rows(const osf_mesh* m, const int64_t* rows, int64_t nrows, double* out, int nthreads) {
  if (!m || m->p < 1 || m->p > OSF_MAXP) return -1;
  job_t J = {m, 0, 1, rows, nrows, NULL, out, 0, 0};
  return run(&J, nthreads);
}

/* B-spline values and derivatives of the p+1 functions nonzero at x (for the pins). */
int osf_basis(const double* U, int p, int n_el, double x, double* N, double* dN, int* first) {
  if (p < 1 || p > OSF_MAXP) return -1;
  const int e = element_of(U, p, n_el, x);
  basis(U, p, e + p, x, N, dN);
  *first = e;
  return 0;
}
