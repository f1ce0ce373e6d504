/*
 * cgks_oracle3.c -- serial FP64 CPU oracle of the p-multigrid compact
 * gas-kinetic scheme (Ji, Shyy & Xu, arXiv:2109.09965), 3-D.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA library (nor with the 2-D oracle,
 * whose results the 3-D tests compare against): it re-derives the polyhedral
 * geometry, the face list, the face quadrature, the reconstruction, the
 * kinetic moments, the fluxes, the time stepping, the low-order smoother and
 * the sweep order from the paper.  Plain loops over array-of-structs data in
 * double precision; kinetic moments by a generic polynomial integrator in
 * (u, v, w, xi^2); small dense solves by Gaussian elimination and
 * Householder QR.
 *
 * Paper passages followed (section / equation of arXiv:2109.09965):
 *   3-D BGK model, psi, K = (5-3 gamma)/(gamma-1) .... Section 2, Eq. (bgk)
 *   polyhedral cells, N_f faces, face quadrature:
 *     3 Gauss points per triangle, 4 per quadrilateral . Section 2.1
 *   Maxwellian, micro-slopes a_{x_i}, A .............. Section 2.2
 *   smooth GKS flux .................................. Section 2.2, Eq. (2nd-smooth-flux)
 *   interface state, Gauss-Green gradients ........... Section 2.3
 *   S1O2 ............................................. Section 2.4
 *   V-cycle, backward Euler, L-F split, local dt,
 *     point relaxation ............................... Section 3, Algorithm 1
 *   density residual Res ............................. Section 4
 *
 * Readings (in addition to those of the 2-D oracle, which carry over):
 *   cells tet / prism / pyramid / hex with "positive" node order (first face
 *   counter-clockwise seen from the rest of the cell); triangle faces with
 *   the symmetric 3-point rule of degree 2; quadrilateral faces as bilinear
 *   patches with the 2 x 2 Gauss rule, one normal and area from the exact
 *   area vector of the patch and Gauss weights |J_k| / sum |J|; cell volume,
 *   centroid and second moments by tets from the mean of the cell's nodes to
 *   the face triangles (a quad face cut into 4 triangles at its centre);
 *   h_i = |Omega_i|^(1/3); quadratic reconstruction (9 monomials) when the
 *   centroids of the cell's stencil (face neighbours plus wall mirror cells)
 *   spread in all three directions -- T = sum_j d_j d_j^T of the scaled
 *   offsets with det(T) / (tr(T)/3)^3 >= 1e-3 -- linear otherwise (a stencil
 *   in one plane leaves the curvature across it undetermined); explicit dt
 *   with h_i = 3|Omega_i| / sum_p S_p.  Full flux (Eq. (2nd-flux)) and
 *   compact WENO on conservative variables as in the 2-D oracle, with the
 *   9-monomial quadratic and the three local slope directions; their tau_n
 *   constants and weight form are readings, parity unpinned against the
 *   cited papers.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NV 5          /* rho, rho u, rho v, rho w, rho E */
#define ND 3
#define NM 9          /* xi eta zeta xi^2 xi*eta xi*zeta eta^2 eta*zeta zeta^2 */
#define MAXBC 16
#define MAXMOM 12
#define MAXFC 6       /* faces per cell */
#define MAXGP 4       /* Gauss points per face */
#define MAXROWS (4 * MAXFC + 3)

enum { O3_BC_SLIP = 0, O3_BC_NOSLIP = 1, O3_BC_FARFIELD = 2 };

typedef struct {
  int kind;
  int pad_;
  double uw[3];               /* wall velocity of a no-slip wall */
  double rho, u[3], p;        /* free stream of a far-field boundary */
} o3_bc;

typedef struct {
  double gamma, mu, alpha, cfl_hi, cfl_lo;
  int n_implicit, n_sweeps, time_scheme, n_bc;
  int flux_lo;                /* low-level flux: 0 = KFVS, 1 = Lax-Friedrichs */
  int flux_hi;                /* high-level flux: 0 = smooth, 1 = full, Eq. (2nd-flux) */
  double tau_c1, tau_c2;      /* tau_n = tau + C1 dt + C2 dt |p_l - p_r| / (p_l + p_r) */
  double weno_eps;            /* > 0: nonlinear compact WENO weights; <= 0: linear weights */
  double weno_g0;             /* linear weight of the quadratic candidate */
  o3_bc bc[MAXBC];
  int lo_viscous;             /* 1: the low-order residual carries a first-order viscous flux */
  int pad2_;
} o3_params;

typedef struct {
  long c0, c1;                /* c1 < 0 on a boundary face */
  int tag;
  int nv;
  long node[4];
  double n[3], S;             /* unit normal out of c0, area */
  double xf[3];               /* face centre */
  int ng;
  double xg[MAXGP][3], wg[MAXGP];
  double delta;
} o3_face;

typedef struct {
  int type, nv;
  long node[8];
  double vol, xc[3], h;
  double M2[6];               /* central second moments / vol: xx xy xz yy yz zz */
  int nf;
  long face[MAXFC];
  int sgn[MAXFC];
  int nb;
  long nbr[MAXFC];
} o3_cell;

typedef struct {
  long nn, nc, nf;
  double *x;
  o3_cell *cell;
  o3_face *face;
  long *rcm;
  int *colour;
  int ncolour;
} o3_mesh;

/* faces of each cell type, outward, counter-clockwise seen from outside */
static const int TET_F[4][4] = { { 0, 2, 1, -1 }, { 0, 1, 3, -1 }, { 1, 2, 3, -1 }, { 2, 0, 3, -1 } };
static const int PRI_F[5][4] = { { 0, 2, 1, -1 }, { 3, 4, 5, -1 }, { 0, 1, 4, 3 }, { 1, 2, 5, 4 }, { 2, 0, 3, 5 } };
static const int PYR_F[5][4] = { { 0, 3, 2, 1 }, { 0, 1, 4, -1 }, { 1, 2, 4, -1 }, { 2, 3, 4, -1 }, { 3, 0, 4, -1 } };
static const int HEX_F[6][4] = { { 0, 3, 2, 1 }, { 4, 5, 6, 7 }, { 0, 1, 5, 4 }, { 1, 2, 6, 5 }, { 2, 3, 7, 6 }, { 3, 0, 4, 7 } };

static int cell_faces(int type, const int (**tab)[4]) {
  switch (type) {
    case 2: *tab = TET_F; return 4;
    case 3: *tab = PRI_F; return 5;
    case 4: *tab = PYR_F; return 5;
    case 5: *tab = HEX_F; return 6;
  }
  return 0;
}
static int type_nodes(int type) { return type == 2 ? 4 : type == 3 ? 6 : type == 4 ? 5 : type == 5 ? 8 : 0; }

static double o3_K(double gamma) { return (5.0 - 3.0 * gamma) / (gamma - 1.0); }

static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ */
/* dense solves                                                        */
/* ------------------------------------------------------------------ */
static int gauss_solve(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int r = k + 1; r < n; ++r)
      if (fabs(A[r * n + k]) > fabs(A[piv * n + k])) piv = r;
    if (A[piv * n + k] == 0.0) return -1;
    if (piv != k) {
      for (int c = 0; c < n; ++c) { double t = A[k * n + c]; A[k * n + c] = A[piv * n + c]; A[piv * n + c] = t; }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int r = k + 1; r < n; ++r) {
      double f = A[r * n + k] / A[k * n + k];
      for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
      b[r] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * b[c];
    b[k] = s / A[k * n + k];
  }
  return 0;
}

/* min ||A x - B|| by Householder QR; A m x n (row major), B m x nr, X n x nr */
static int householder_ls(int m, int n, double *A, int nr, double *B, double *X) {
  for (int k = 0; k < n; ++k) {
    double norm = 0.0;
    for (int i = k; i < m; ++i) norm += A[i * n + k] * A[i * n + k];
    norm = sqrt(norm);
    if (!(norm > 1e-13)) return -1;   /* rank-deficient (columns are O(1) in scaled coordinates) */
    double alpha = A[k * n + k] > 0 ? -norm : norm;
    double v[MAXROWS + 8];
    for (int i = 0; i < m; ++i) v[i] = 0.0;
    for (int i = k; i < m; ++i) v[i] = A[i * n + k];
    v[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int c = k; c < n; ++c) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += v[i] * A[i * n + c];
      s = 2.0 * s / vv;
      for (int i = k; i < m; ++i) A[i * n + c] -= s * v[i];
    }
    for (int c = 0; c < nr; ++c) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += v[i] * B[i * nr + c];
      s = 2.0 * s / vv;
      for (int i = k; i < m; ++i) B[i * nr + c] -= s * v[i];
    }
  }
  for (int c = 0; c < nr; ++c)
    for (int k = n - 1; k >= 0; --k) {
      double s = B[k * nr + c];
      for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * X[j * nr + c];
      if (fabs(A[k * n + k]) < 1e-13 * (fabs(A[0]) + 1e-300)) return -1;
      X[k * nr + c] = s / A[k * n + k];
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Kinetic moments: polynomials in (u, v, w, xi^2) against a Maxwellian */
/* ------------------------------------------------------------------ */
typedef struct { double c; int a, b, d, k; } o3_term;   /* c u^a v^b w^d (xi^2)^k */
typedef struct { int n; o3_term t[512]; } o3_poly;
typedef struct { double mu[MAXMOM], mv[MAXMOM], mw[MAXMOM], mx[4]; } o3_mom;
typedef struct { double rho, U, V, Wv, lam; } o3_maxw;

static void poly_zero(o3_poly *p) { p->n = 0; }
static void poly_add(o3_poly *p, double c, int a, int b, int d, int k) {
  if (p->n >= 512) { fprintf(stderr, "oracle3: polynomial overflow\n"); abort(); }
  o3_term *t = &p->t[p->n++];
  t->c = c; t->a = a; t->b = b; t->d = d; t->k = k;
}
/* psi: 1, u, v, w, (u^2 + v^2 + w^2 + xi^2) / 2 */
static void poly_psi(int r, o3_poly *p) {
  poly_zero(p);
  if (r == 0) poly_add(p, 1.0, 0, 0, 0, 0);
  else if (r == 1) poly_add(p, 1.0, 1, 0, 0, 0);
  else if (r == 2) poly_add(p, 1.0, 0, 1, 0, 0);
  else if (r == 3) poly_add(p, 1.0, 0, 0, 1, 0);
  else {
    poly_add(p, 0.5, 2, 0, 0, 0); poly_add(p, 0.5, 0, 2, 0, 0);
    poly_add(p, 0.5, 0, 0, 2, 0); poly_add(p, 0.5, 0, 0, 0, 1);
  }
}
static void poly_slope(const double s[NV], o3_poly *p) {
  poly_zero(p);
  for (int r = 0; r < NV; ++r) {
    o3_poly q; poly_psi(r, &q);
    for (int i = 0; i < q.n; ++i) poly_add(p, s[r] * q.t[i].c, q.t[i].a, q.t[i].b, q.t[i].d, q.t[i].k);
  }
}
static void poly_mul(const o3_poly *x, const o3_poly *y, o3_poly *out) {
  poly_zero(out);
  for (int i = 0; i < x->n; ++i)
    for (int j = 0; j < y->n; ++j)
      poly_add(out, x->t[i].c * y->t[j].c, x->t[i].a + y->t[j].a, x->t[i].b + y->t[j].b,
               x->t[i].d + y->t[j].d, x->t[i].k + y->t[j].k);
}
static void poly_mono(double c, int a, int b, int d, o3_poly *p) { poly_zero(p); poly_add(p, c, a, b, d, 0); }
static double poly_int(const o3_poly *p, const o3_mom *m) {
  double s = 0.0;
  for (int i = 0; i < p->n; ++i) {
    const o3_term *t = &p->t[i];
    if (t->a >= MAXMOM || t->b >= MAXMOM || t->d >= MAXMOM || t->k > 3) { fprintf(stderr, "oracle3: moment order\n"); abort(); }
    s += t->c * m->mu[t->a] * m->mv[t->b] * m->mw[t->d] * m->mx[t->k];
  }
  return s;
}

static o3_maxw maxw_from_W(const double W[NV], double K) {
  o3_maxw g;
  g.rho = W[0]; g.U = W[1] / W[0]; g.V = W[2] / W[0]; g.Wv = W[3] / W[0];
  double ke = 0.5 * g.rho * (g.U * g.U + g.V * g.V + g.Wv * g.Wv);
  g.lam = (K + 3.0) * g.rho / (4.0 * (W[4] - ke));
  return g;
}

static void full_range(double mean, double l, double *m) {
  m[0] = 1.0; m[1] = mean;
  for (int a = 2; a < MAXMOM; ++a) m[a] = mean * m[a - 1] + (a - 1) / (2.0 * l) * m[a - 2];
}
/* range: 0 full, +1 u > 0, -1 u < 0 (normal velocity only) */
static void moments(const o3_maxw *g, double K, int range, o3_mom *m) {
  double l = g->lam;
  if (range == 0) full_range(g->U, l, m->mu);
  else {
    double e = exp(-l * g->U * g->U) / sqrt(M_PI * l);
    if (range > 0) { m->mu[0] = 0.5 * erfc(-sqrt(l) * g->U); m->mu[1] = g->U * m->mu[0] + 0.5 * e; }
    else           { m->mu[0] = 0.5 * erfc(sqrt(l) * g->U);  m->mu[1] = g->U * m->mu[0] - 0.5 * e; }
    for (int a = 2; a < MAXMOM; ++a) m->mu[a] = g->U * m->mu[a - 1] + (a - 1) / (2.0 * l) * m->mu[a - 2];
  }
  full_range(g->V, l, m->mv);
  full_range(g->Wv, l, m->mw);
  m->mx[0] = 1.0;
  m->mx[1] = K / (2.0 * l);
  m->mx[2] = K * (K + 2.0) / (4.0 * l * l);
  m->mx[3] = K * (K + 2.0) * (K + 4.0) / (8.0 * l * l * l);
}

/* <psi_r c u^a v^b w^d> */
static double mom_psi(int r, double c, int a, int b, int d, const o3_mom *m) {
  o3_poly ps, mono, pr; poly_psi(r, &ps); poly_mono(c, a, b, d, &mono); poly_mul(&ps, &mono, &pr);
  return poly_int(&pr, m);
}
/* <psi_r u^a v^b w^d slope> */
static double mom_psi_slope(int r, int a, int b, int d, const double s[NV], const o3_mom *m) {
  o3_poly ps, mono, sl, t1, t2;
  poly_psi(r, &ps); poly_mono(1.0, a, b, d, &mono); poly_slope(s, &sl);
  poly_mul(&ps, &mono, &t1); poly_mul(&t1, &sl, &t2);
  return poly_int(&t2, m);
}

/* <a psi> = dW / rho, M_rs = <psi_r psi_s> (Section 2.2) */
static int micro_slope(const o3_mom *m, double rho, const double dW[NV], double s[NV]) {
  double M[NV * NV], b[NV];
  for (int r = 0; r < NV; ++r) {
    b[r] = dW[r] / rho;
    for (int c = 0; c < NV; ++c) {
      o3_poly pr, pc, pp; poly_psi(r, &pr); poly_psi(c, &pc); poly_mul(&pr, &pc, &pp);
      M[r * NV + c] = poly_int(&pp, m);
    }
  }
  int rc = gauss_solve(NV, M, b);
  for (int r = 0; r < NV; ++r) s[r] = b[r];
  return rc;
}

/* ------------------------------------------------------------------ */
/* frames: e1 = n, e2 = t1, e3 = t2 (right-handed)                     */
/* ------------------------------------------------------------------ */
static void frame(const double n[3], double E[3][3]) {
  double a[3] = { 0, 0, 0 };
  int k = 0;
  for (int d = 1; d < 3; ++d) if (fabs(n[d]) < fabs(n[k])) k = d;
  a[k] = 1.0;
  double t1[3], t2[3];
  cross3(a, n, t1);
  double l = sqrt(dot3(t1, t1));
  for (int d = 0; d < 3; ++d) t1[d] /= l;
  cross3(n, t1, t2);
  for (int d = 0; d < 3; ++d) { E[0][d] = n[d]; E[1][d] = t1[d]; E[2][d] = t2[d]; }
}
static void to_local(double E[3][3], const double Wg[NV], double Wl[NV]) {
  Wl[0] = Wg[0]; Wl[4] = Wg[4];
  for (int a = 0; a < 3; ++a) Wl[1 + a] = E[a][0] * Wg[1] + E[a][1] * Wg[2] + E[a][2] * Wg[3];
}
static void to_global(double E[3][3], const double Wl[NV], double Wg[NV]) {
  Wg[0] = Wl[0]; Wg[4] = Wl[4];
  for (int d = 0; d < 3; ++d) Wg[1 + d] = E[0][d] * Wl[1] + E[1][d] * Wl[2] + E[2][d] * Wl[3];
}

/* ------------------------------------------------------------------ */
/* Smooth GKS flux at one Gauss point (Eq. (2nd-smooth-flux)), 3-D.     */
/*   grad[d * NV + v] = dW_v / dx_d (global); n from l to r             */
/* ------------------------------------------------------------------ */
void o3_gks_flux_point(const o3_params *P, const double Wl_g[NV], const double Wr_g[NV],
                       const double gl[ND * NV], const double gr[ND * NV], const double n[3], double delta,
                       double F0[NV], double F1[NV], double Wc_out[NV], double Wt_out[NV]) {
  double K = o3_K(P->gamma);
  double E[3][3];
  frame(n, E);
  double Wl[NV], Wr[NV];
  to_local(E, Wl_g, Wl);
  to_local(E, Wr_g, Wr);
  /* derivative along each local axis, as a local-frame vector */
  double dl[3][NV], dr[3][NV];
  for (int a = 0; a < 3; ++a) {
    double tl[NV], tr[NV];
    for (int v = 0; v < NV; ++v) {
      tl[v] = E[a][0] * gl[v] + E[a][1] * gl[NV + v] + E[a][2] * gl[2 * NV + v];
      tr[v] = E[a][0] * gr[v] + E[a][1] * gr[NV + v] + E[a][2] * gr[2 * NV + v];
    }
    to_local(E, tl, dl[a]);
    to_local(E, tr, dr[a]);
  }
  o3_maxw gL = maxw_from_W(Wl, K), gR = maxw_from_W(Wr, K);
  o3_mom ml, mr;
  moments(&gL, K, +1, &ml);
  moments(&gR, K, -1, &mr);
  double Wc[NV];
  for (int r = 0; r < NV; ++r) Wc[r] = gL.rho * mom_psi(r, 1.0, 0, 0, 0, &ml) + gR.rho * mom_psi(r, 1.0, 0, 0, 0, &mr);
  double dW[3][NV];
  for (int v = 0; v < NV; ++v) {
    for (int a = 0; a < 3; ++a) dW[a][v] = 0.5 * (dl[a][v] + dr[a][v]);
    if (delta > 0.0) dW[0][v] += P->alpha * (Wr[v] - Wl[v]) / delta;
  }
  o3_maxw gc = maxw_from_W(Wc, K);
  o3_mom mc;
  moments(&gc, K, 0, &mc);
  double a[3][NV], A[NV], bA[NV];
  for (int k = 0; k < 3; ++k) micro_slope(&mc, gc.rho, dW[k], a[k]);
  for (int r = 0; r < NV; ++r)
    bA[r] = -(mom_psi_slope(r, 1, 0, 0, a[0], &mc) + mom_psi_slope(r, 0, 1, 0, a[1], &mc) +
              mom_psi_slope(r, 0, 0, 1, a[2], &mc)) * gc.rho;
  micro_slope(&mc, gc.rho, bA, A);
  double pc = gc.rho / (2.0 * gc.lam);
  double tau = P->mu / pc;
  double F0l[NV], F1l[NV], Wtl[NV];
  for (int r = 0; r < NV; ++r) {
    double feq = mom_psi(r, 1.0, 1, 0, 0, &mc);
    double visc = mom_psi_slope(r, 2, 0, 0, a[0], &mc) + mom_psi_slope(r, 1, 1, 0, a[1], &mc) +
                  mom_psi_slope(r, 1, 0, 1, a[2], &mc) + mom_psi_slope(r, 1, 0, 0, A, &mc);
    F0l[r] = gc.rho * (feq - tau * visc);
    F1l[r] = gc.rho * mom_psi_slope(r, 1, 0, 0, A, &mc);
    Wtl[r] = gc.rho * mom_psi_slope(r, 0, 0, 0, A, &mc);
  }
  to_global(E, F0l, F0);
  to_global(E, F1l, F1);
  to_global(E, Wc, Wc_out);
  to_global(E, Wtl, Wt_out);
}

/* ------------------------------------------------------------------ */
/* Full GKS flux at one Gauss point, Eq. (2nd-flux), 3-D:              */
/*   f = (1 - e) g^c + [(t + tau) e - tau] a^c.u g^c                    */
/*       + (t - tau + tau e) A^c g^c                                    */
/*       + e g^l [1 - (tau + t) a^l.u - tau A^l] H(u_n)                 */
/*       + e g^r [1 - (tau + t) a^r.u - tau A^r] (1 - H(u_n)),          */
/* e = exp(-t / tau_n), tau = mu / p^c, tau_n = tau + C1 dt             */
/* + C2 dt |p_l - p_r| / (p_l + p_r) (reading).  As in 2-D, the time    */
/* dependence is brought to F0 + t F1 through the integrals over        */
/* [0, dt] and [0, dt/2], and the interface state to the line through   */
/* its values at dt/2 and dt.                                           */
/* ------------------------------------------------------------------ */
typedef struct { double c1, c2, c3, e, te; } o3_tcoef;

static o3_tcoef tcoef_at(double t, double tau, double taun) {
  o3_tcoef c;
  double e = taun > 0.0 ? exp(-t / taun) : 0.0;
  c.c1 = 1.0 - e; c.c2 = (t + tau) * e - tau; c.c3 = t - tau + tau * e; c.e = e; c.te = t * e;
  return c;
}
static o3_tcoef tcoef_int(double T, double tau, double taun) {
  o3_tcoef c;
  double E = taun > 0.0 ? exp(-T / taun) : 0.0;
  double om = taun > 0.0 ? -expm1(-T / taun) : 1.0;
  c.e = taun * om;
  c.te = taun * taun * om - taun * T * E;
  c.c1 = T - c.e;
  c.c2 = c.te + tau * c.e - tau * T;
  c.c3 = 0.5 * T * T - tau * T + tau * c.e;
  return c;
}

/* slopes a_1..a_3 (local axes) and A of a Maxwellian from its derivatives */
static void maxw_slopes3(const o3_mom *m, double rho, double dW[3][NV], double a[3][NV], double A[NV]) {
  double bA[NV];
  for (int k = 0; k < 3; ++k) micro_slope(m, rho, dW[k], a[k]);
  for (int r = 0; r < NV; ++r)
    bA[r] = -(mom_psi_slope(r, 1, 0, 0, a[0], m) + mom_psi_slope(r, 0, 1, 0, a[1], m) +
              mom_psi_slope(r, 0, 0, 1, a[2], m)) * rho;
  micro_slope(m, rho, bA, A);
}

/* Q = rho (<u psi>, <u (a.u) psi>, <u A psi>), Pm = rho (<psi>, <(a.u) psi>, <A psi>) */
static void piece3(double rho, const o3_mom *m, double a[3][NV], const double A[NV], double Q[3][NV],
                   double Pm[3][NV]) {
  for (int r = 0; r < NV; ++r) {
    Q[0][r] = rho * mom_psi(r, 1.0, 1, 0, 0, m);
    Q[1][r] = rho * (mom_psi_slope(r, 2, 0, 0, a[0], m) + mom_psi_slope(r, 1, 1, 0, a[1], m) +
                     mom_psi_slope(r, 1, 0, 1, a[2], m));
    Q[2][r] = rho * mom_psi_slope(r, 1, 0, 0, A, m);
    Pm[0][r] = rho * mom_psi(r, 1.0, 0, 0, 0, m);
    Pm[1][r] = rho * (mom_psi_slope(r, 1, 0, 0, a[0], m) + mom_psi_slope(r, 0, 1, 0, a[1], m) +
                      mom_psi_slope(r, 0, 0, 1, a[2], m));
    Pm[2][r] = rho * mom_psi_slope(r, 0, 0, 0, A, m);
  }
}

static void full_combine3(const o3_tcoef *c, double tau, double X[3][3][NV], double out[NV]) {
  for (int r = 0; r < NV; ++r)
    out[r] = c->c1 * X[0][0][r] + c->c2 * X[0][1][r] + c->c3 * X[0][2][r]
           + c->e * (X[1][0][r] - tau * X[1][1][r] - tau * X[1][2][r]
                     + X[2][0][r] - tau * X[2][1][r] - tau * X[2][2][r])
           - c->te * (X[1][1][r] + X[2][1][r]);
}

void o3_gks_full_flux_point(const o3_params *P, const double Wl_g[NV], const double Wr_g[NV],
                            const double gl[ND * NV], const double gr[ND * NV], const double n[3], double delta,
                            double dt, double F0[NV], double F1[NV], double Wc_out[NV], double Wt_out[NV]) {
  double K = o3_K(P->gamma);
  double E[3][3];
  frame(n, E);
  double Wl[NV], Wr[NV];
  to_local(E, Wl_g, Wl);
  to_local(E, Wr_g, Wr);
  double dl[3][NV], dr[3][NV];
  for (int a = 0; a < 3; ++a) {
    double tl[NV], tr[NV];
    for (int v = 0; v < NV; ++v) {
      tl[v] = E[a][0] * gl[v] + E[a][1] * gl[NV + v] + E[a][2] * gl[2 * NV + v];
      tr[v] = E[a][0] * gr[v] + E[a][1] * gr[NV + v] + E[a][2] * gr[2 * NV + v];
    }
    to_local(E, tl, dl[a]);
    to_local(E, tr, dr[a]);
  }
  o3_maxw gL = maxw_from_W(Wl, K), gR = maxw_from_W(Wr, K);
  o3_mom mlh, mrh, mlf, mrf;
  moments(&gL, K, +1, &mlh);
  moments(&gR, K, -1, &mrh);
  moments(&gL, K, 0, &mlf);
  moments(&gR, K, 0, &mrf);
  double al[3][NV], Al[NV], ar[3][NV], Ar[NV];
  maxw_slopes3(&mlf, gL.rho, dl, al, Al);
  maxw_slopes3(&mrf, gR.rho, dr, ar, Ar);
  double Wc[NV];
  for (int r = 0; r < NV; ++r) Wc[r] = gL.rho * mom_psi(r, 1.0, 0, 0, 0, &mlh) + gR.rho * mom_psi(r, 1.0, 0, 0, 0, &mrh);
  double dW[3][NV];
  for (int v = 0; v < NV; ++v) {
    for (int a = 0; a < 3; ++a) dW[a][v] = 0.5 * (dl[a][v] + dr[a][v]);
    if (delta > 0.0) dW[0][v] += P->alpha * (Wr[v] - Wl[v]) / delta;
  }
  o3_maxw gc = maxw_from_W(Wc, K);
  o3_mom mc;
  moments(&gc, K, 0, &mc);
  double ac[3][NV], Ac[NV];
  maxw_slopes3(&mc, gc.rho, dW, ac, Ac);
  double pc = gc.rho / (2.0 * gc.lam), pl = gL.rho / (2.0 * gL.lam), pr = gR.rho / (2.0 * gR.lam);
  double tau = P->mu / pc;
  double taun = tau + P->tau_c1 * dt + P->tau_c2 * dt * fabs(pl - pr) / (pl + pr);
  double Q[3][3][NV], Pm[3][3][NV];
  piece3(gc.rho, &mc, ac, Ac, Q[0], Pm[0]);
  piece3(gL.rho, &mlh, al, Al, Q[1], Pm[1]);
  piece3(gR.rho, &mrh, ar, Ar, Q[2], Pm[2]);
  o3_tcoef I1 = tcoef_int(dt, tau, taun), Ih = tcoef_int(0.5 * dt, tau, taun);
  o3_tcoef C1 = tcoef_at(dt, tau, taun), Ch = tcoef_at(0.5 * dt, tau, taun);
  double Fd[NV], Fh[NV], Wd[NV], Wh[NV];
  full_combine3(&I1, tau, Q, Fd);
  full_combine3(&Ih, tau, Q, Fh);
  full_combine3(&C1, tau, Pm, Wd);
  full_combine3(&Ch, tau, Pm, Wh);
  double F0l[NV], F1l[NV], Wcl[NV], Wtl[NV];
  for (int r = 0; r < NV; ++r) {
    F0l[r] = (4.0 * Fh[r] - Fd[r]) / dt;
    F1l[r] = 4.0 * (Fd[r] - 2.0 * Fh[r]) / (dt * dt);
    Wcl[r] = 2.0 * Wh[r] - Wd[r];
    Wtl[r] = 2.0 * (Wd[r] - Wh[r]) / dt;
  }
  to_global(E, F0l, F0);
  to_global(E, F1l, F1);
  to_global(E, Wcl, Wc_out);
  to_global(E, Wtl, Wt_out);
}

/* first-order KFVS flux of two cell-average states (Section 3) */
void o3_kfvs(const o3_params *P, const double Wl_g[NV], const double Wr_g[NV], const double n[3], double F[NV]) {
  double K = o3_K(P->gamma);
  double E[3][3];
  frame(n, E);
  double Wl[NV], Wr[NV], Fl[NV];
  to_local(E, Wl_g, Wl);
  to_local(E, Wr_g, Wr);
  o3_maxw gL = maxw_from_W(Wl, K), gR = maxw_from_W(Wr, K);
  o3_mom ml, mr;
  moments(&gL, K, +1, &ml);
  moments(&gR, K, -1, &mr);
  for (int r = 0; r < NV; ++r) Fl[r] = gL.rho * mom_psi(r, 1.0, 1, 0, 0, &ml) + gR.rho * mom_psi(r, 1.0, 1, 0, 0, &mr);
  to_global(E, Fl, F);
}

void o3_euler_flux(double gamma, const double W[NV], const double n[3], double F[NV]) {
  double rho = W[0], u[3] = { W[1] / rho, W[2] / rho, W[3] / rho };
  double p = (gamma - 1.0) * (W[4] - 0.5 * rho * dot3(u, u));
  double un = dot3(u, n);
  F[0] = rho * un;
  for (int d = 0; d < 3; ++d) F[1 + d] = W[1 + d] * un + p * n[d];
  F[4] = (W[4] + p) * un;
}

/* ------------------------------------------------------------------ */
/* boundary ghost states                                                */
/* ------------------------------------------------------------------ */
static void prim3(double g, const double W[NV], double *rho, double u[3], double *p) {
  *rho = W[0];
  for (int d = 0; d < 3; ++d) u[d] = W[1 + d] / W[0];
  *p = (g - 1.0) * (W[4] - 0.5 * W[0] * dot3(u, u));
}
static void cons3(double g, double rho, const double u[3], double p, double W[NV]) {
  W[0] = rho;
  for (int d = 0; d < 3; ++d) W[1 + d] = rho * u[d];
  W[4] = p / (g - 1.0) + 0.5 * rho * dot3(u, u);
}

static void farfield_state(const o3_params *P, const o3_bc *bc, const double W[NV], const double n[3], double Wg[NV]) {
  double g = P->gamma, ri, ui[3], pi;
  prim3(g, W, &ri, ui, &pi);
  double ci = sqrt(g * pi / ri), uni = dot3(ui, n);
  double re = bc->rho, pe = bc->p, ue[3] = { bc->u[0], bc->u[1], bc->u[2] };
  double ce = sqrt(g * pe / re), une = dot3(ue, n);
  if (uni <= -ci) { cons3(g, re, ue, pe, Wg); return; }
  if (uni >= ci) { memcpy(Wg, W, sizeof(double) * NV); return; }
  double Rp = uni + 2.0 * ci / (g - 1.0), Rm = une - 2.0 * ce / (g - 1.0);
  double unb = 0.5 * (Rp + Rm), cb = 0.25 * (g - 1.0) * (Rp - Rm);
  double s, ut[3];
  if (unb >= 0.0) { s = pi / pow(ri, g); for (int d = 0; d < 3; ++d) ut[d] = ui[d] - uni * n[d]; }
  else            { s = pe / pow(re, g); for (int d = 0; d < 3; ++d) ut[d] = ue[d] - une * n[d]; }
  double rb = pow(cb * cb / (g * s), 1.0 / (g - 1.0)), pb = rb * cb * cb / g;
  double ub[3];
  for (int d = 0; d < 3; ++d) ub[d] = ut[d] + unb * n[d];
  cons3(g, rb, ub, pb, Wg);
}

/* Ghost value and gradient across a boundary face with outward normal n;
 * grad[d * NV + v].  Mirror M = I - 2 n n^T. */
void o3_ghost(const o3_params *P, int tag, const double W[NV], const double grad[ND * NV], const double n[3],
              double Wg[NV], double gradg[ND * NV]) {
  const o3_bc *bc = &P->bc[tag];
  double g = P->gamma, M[3][3];
  for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) M[a][b] = (a == b) - 2.0 * n[a] * n[b];
  if (bc->kind == O3_BC_SLIP) {
    Wg[0] = W[0]; Wg[4] = W[4];
    for (int a = 0; a < 3; ++a) Wg[1 + a] = M[a][0] * W[1] + M[a][1] * W[2] + M[a][2] * W[3];
    for (int d = 0; d < 3; ++d) {
      gradg[d * NV + 0] = M[d][0] * grad[0] + M[d][1] * grad[NV] + M[d][2] * grad[2 * NV];
      gradg[d * NV + 4] = M[d][0] * grad[4] + M[d][1] * grad[NV + 4] + M[d][2] * grad[2 * NV + 4];
    }
    double J[3][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) J[a][b] = grad[b * NV + 1 + a];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int c = 0; c < 3; ++c) for (int e = 0; e < 3; ++e) s += M[a][c] * J[c][e] * M[e][b];
      gradg[b * NV + 1 + a] = s;
    }
  } else if (bc->kind == O3_BC_NOSLIP) {
    double rho, u[3], p;
    prim3(g, W, &rho, u, &p);
    double drho[3], du[3][3], dp[3];
    for (int b = 0; b < 3; ++b) {
      drho[b] = grad[b * NV];
      for (int a = 0; a < 3; ++a) du[a][b] = (grad[b * NV + 1 + a] - u[a] * drho[b]) / rho;
      double ke = u[0] * du[0][b] + u[1] * du[1][b] + u[2] * du[2][b];
      dp[b] = (g - 1.0) * (grad[b * NV + 4] - 0.5 * dot3(u, u) * drho[b] - rho * ke);
    }
    double ug[3], drg[3], dpg[3], dug[3][3];
    for (int a = 0; a < 3; ++a) ug[a] = 2.0 * bc->uw[a] - u[a];
    for (int d = 0; d < 3; ++d) {
      drg[d] = M[d][0] * drho[0] + M[d][1] * drho[1] + M[d][2] * drho[2];
      dpg[d] = M[d][0] * dp[0] + M[d][1] * dp[1] + M[d][2] * dp[2];
    }
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
      dug[a][b] = -(du[a][0] * M[0][b] + du[a][1] * M[1][b] + du[a][2] * M[2][b]);
    cons3(g, rho, ug, p, Wg);
    for (int b = 0; b < 3; ++b) {
      gradg[b * NV] = drg[b];
      for (int a = 0; a < 3; ++a) gradg[b * NV + 1 + a] = ug[a] * drg[b] + rho * dug[a][b];
      double ke = ug[0] * dug[0][b] + ug[1] * dug[1][b] + ug[2] * dug[2][b];
      gradg[b * NV + 4] = dpg[b] / (g - 1.0) + 0.5 * dot3(ug, ug) * drg[b] + rho * ke;
    }
  } else {
    farfield_state(P, bc, W, n, Wg);
    for (int k = 0; k < ND * NV; ++k) gradg[k] = 0.0;
  }
}

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */
/* accumulate a tet (p, a, b, c): signed volume, first and second raw moments */
static void tet_moments(const double p[3], const double a[3], const double b[3], const double c[3], double *V,
                        double S1[3], double S2[6]) {
  double u[3], v[3], w[3], x[3];
  for (int d = 0; d < 3; ++d) { u[d] = a[d] - p[d]; v[d] = b[d] - p[d]; w[d] = c[d] - p[d]; }
  cross3(u, v, x);
  double vol = dot3(x, w) / 6.0;
  const double *P4[4] = { p, a, b, c };
  double s[3] = { 0, 0, 0 };
  for (int k = 0; k < 4; ++k) for (int d = 0; d < 3; ++d) s[d] += P4[k][d];
  *V += vol;
  for (int d = 0; d < 3; ++d) S1[d] += vol * s[d] / 4.0;
  /* int x_i x_j over a tet = V/20 (sum_k x_i^k x_j^k + s_i s_j) */
  int q = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j, ++q) {
      double t = s[i] * s[j];
      for (int k = 0; k < 4; ++k) t += P4[k][i] * P4[k][j];
      S2[q] += vol / 20.0 * t;
    }
}

/* volume, centroid and central second moments of a cell with nodes X0;
 * the moments are taken about the mean of the nodes (no cancellation for
 * small cells far from the origin) */
static void polyhedron(int type, const double X0[8][3], double *vol, double xc[3], double M2[6]) {
  const int (*tab)[4];
  int nf = cell_faces(type, &tab);
  int nv = type_nodes(type);
  double o[3] = { 0, 0, 0 }, X[8][3];
  for (int k = 0; k < nv; ++k) for (int d = 0; d < 3; ++d) o[d] += X0[k][d] / nv;
  for (int k = 0; k < nv; ++k) for (int d = 0; d < 3; ++d) X[k][d] = X0[k][d] - o[d];
  double p[3] = { 0, 0, 0 };
  double V = 0.0, S1[3] = { 0, 0, 0 }, S2[6] = { 0, 0, 0, 0, 0, 0 };
  for (int f = 0; f < nf; ++f) {
    int m = tab[f][3] < 0 ? 3 : 4;
    if (m == 3) tet_moments(p, X[tab[f][0]], X[tab[f][1]], X[tab[f][2]], &V, S1, S2);
    else {
      double fc[3];
      for (int d = 0; d < 3; ++d) fc[d] = 0.25 * (X[tab[f][0]][d] + X[tab[f][1]][d] + X[tab[f][2]][d] + X[tab[f][3]][d]);
      for (int e = 0; e < 4; ++e) tet_moments(p, X[tab[f][e]], X[tab[f][(e + 1) % 4]], fc, &V, S1, S2);
    }
  }
  *vol = V;
  double c[3];
  for (int d = 0; d < 3; ++d) c[d] = S1[d] / V;
  int q = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j, ++q) M2[q] = S2[q] / V - c[i] * c[j];
  for (int d = 0; d < 3; ++d) xc[d] = o[d] + c[d];
}

/* face of nodes X[0..m-1] (counter-clockwise seen from outside) */
static void face_geometry(int m, const double X[4][3], o3_face *F) {
  double A[3] = { 0, 0, 0 };
  F->ng = m == 3 ? 3 : 4;
  if (m == 3) {
    double u[3], v[3];
    for (int d = 0; d < 3; ++d) { u[d] = X[1][d] - X[0][d]; v[d] = X[2][d] - X[0][d]; }
    cross3(u, v, A);
    for (int d = 0; d < 3; ++d) A[d] *= 0.5;
    static const double bary[3][3] = { { 2.0 / 3, 1.0 / 6, 1.0 / 6 }, { 1.0 / 6, 2.0 / 3, 1.0 / 6 }, { 1.0 / 6, 1.0 / 6, 2.0 / 3 } };
    for (int k = 0; k < 3; ++k) {
      for (int d = 0; d < 3; ++d) F->xg[k][d] = bary[k][0] * X[0][d] + bary[k][1] * X[1][d] + bary[k][2] * X[2][d];
      F->wg[k] = 1.0 / 3.0;
    }
    for (int d = 0; d < 3; ++d) F->xf[d] = (X[0][d] + X[1][d] + X[2][d]) / 3.0;
  } else {
    /* bilinear patch x(s, t) on [-1, 1]^2, nodes at (-1,-1) (1,-1) (1,1) (-1,1) */
    double g = 1.0 / sqrt(3.0), J[4];
    static const double sg[4][2] = { { -1, -1 }, { 1, -1 }, { 1, 1 }, { -1, 1 } };
    double Jsum = 0.0;
    for (int k = 0; k < 4; ++k) {
      double s = sg[k][0] * g, t = sg[k][1] * g;
      double N[4] = { 0.25 * (1 - s) * (1 - t), 0.25 * (1 + s) * (1 - t), 0.25 * (1 + s) * (1 + t), 0.25 * (1 - s) * (1 + t) };
      double Ns[4] = { -0.25 * (1 - t), 0.25 * (1 - t), 0.25 * (1 + t), -0.25 * (1 + t) };
      double Nt[4] = { -0.25 * (1 - s), -0.25 * (1 + s), 0.25 * (1 + s), 0.25 * (1 - s) };
      double xs[3] = { 0, 0, 0 }, xt[3] = { 0, 0, 0 }, c[3];
      for (int d = 0; d < 3; ++d) {
        F->xg[k][d] = 0.0;
        for (int a = 0; a < 4; ++a) { F->xg[k][d] += N[a] * X[a][d]; xs[d] += Ns[a] * X[a][d]; xt[d] += Nt[a] * X[a][d]; }
      }
      cross3(xs, xt, c);
      for (int d = 0; d < 3; ++d) A[d] += c[d];
      J[k] = sqrt(dot3(c, c));
      Jsum += J[k];
    }
    for (int k = 0; k < 4; ++k) F->wg[k] = J[k] / Jsum;
    for (int d = 0; d < 3; ++d) F->xf[d] = 0.25 * (X[0][d] + X[1][d] + X[2][d] + X[3][d]);
  }
  F->S = sqrt(dot3(A, A));
  for (int d = 0; d < 3; ++d) F->n[d] = A[d] / F->S;
}

typedef struct { long key[4]; long cell; int k; } o3_fkey;

static int fkey_cmp(const void *x, const void *y) {
  const o3_fkey *p = (const o3_fkey *)x, *q = (const o3_fkey *)y;
  for (int i = 0; i < 4; ++i)
    if (p->key[i] != q->key[i]) return p->key[i] < q->key[i] ? -1 : 1;
  if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
  return 0;
}
static void sort_key(int m, const long *nodes, long key[4]) {
  long t[4] = { -1, -1, -1, -1 };
  for (int i = 0; i < m; ++i) t[i] = nodes[i];
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j)
      if (t[j] < t[i]) { long s = t[i]; t[i] = t[j]; t[j] = s; }
  for (int i = 0; i < 4; ++i) key[i] = i < m ? t[i] : -1;
}

static void mesh_free(o3_mesh *m) {
  if (!m) return;
  free(m->x); free(m->cell); free(m->face); free(m->rcm); free(m->colour); free(m);
}
void o3_mesh_destroy(o3_mesh *m) { mesh_free(m); }

static void mesh_ordering(o3_mesh *m);

/* err: 1 bad input, 2 non-manifold face, 3 boundary face without tag,
 * 4 non-positive volume */
o3_mesh *o3_mesh_create(long nn, const double *xyz, long nc, const uint8_t *ctype, const int64_t *cptr,
                        const int64_t *cnodes, long nbf, const int64_t *bptr, const int64_t *bnodes,
                        const int32_t *btag, int *err) {
  *err = 0;
  o3_mesh *m = (o3_mesh *)calloc(1, sizeof(o3_mesh));
  m->nn = nn; m->nc = nc;
  m->x = (double *)malloc(sizeof(double) * 3 * nn);
  memcpy(m->x, xyz, sizeof(double) * 3 * nn);
  m->cell = (o3_cell *)calloc(nc, sizeof(o3_cell));
  long nfk = 0;
  for (long c = 0; c < nc; ++c) {
    o3_cell *C = &m->cell[c];
    C->type = ctype[c];
    C->nv = type_nodes(C->type);
    if (C->nv == 0 || cptr[c + 1] - cptr[c] != C->nv) { *err = 1; mesh_free(m); return NULL; }
    double X[8][3];
    for (int k = 0; k < C->nv; ++k) {
      C->node[k] = cnodes[cptr[c] + k];
      for (int d = 0; d < 3; ++d) X[k][d] = m->x[3 * C->node[k] + d];
    }
    polyhedron(C->type, X, &C->vol, C->xc, C->M2);
    if (!(C->vol > 0.0)) { *err = 4; mesh_free(m); return NULL; }
    C->h = cbrt(C->vol);
    const int (*tab)[4];
    nfk += cell_faces(C->type, &tab);
  }
  o3_fkey *E = (o3_fkey *)malloc(sizeof(o3_fkey) * nfk);
  long q = 0;
  for (long c = 0; c < nc; ++c) {
    const int (*tab)[4];
    int nf = cell_faces(m->cell[c].type, &tab);
    for (int f = 0; f < nf; ++f) {
      int mm = tab[f][3] < 0 ? 3 : 4;
      long nodes[4];
      for (int i = 0; i < mm; ++i) nodes[i] = m->cell[c].node[tab[f][i]];
      sort_key(mm, nodes, E[q].key);
      E[q].cell = c; E[q].k = f; ++q;
    }
  }
  qsort(E, nfk, sizeof(o3_fkey), fkey_cmp);
  o3_fkey *B = (o3_fkey *)malloc(sizeof(o3_fkey) * (nbf > 0 ? nbf : 1));
  for (long f = 0; f < nbf; ++f) {
    int mm = (int)(bptr[f + 1] - bptr[f]);
    if (mm != 3 && mm != 4) { *err = 1; free(E); free(B); mesh_free(m); return NULL; }
    long nodes[4];
    for (int i = 0; i < mm; ++i) nodes[i] = bnodes[bptr[f] + i];
    sort_key(mm, nodes, B[f].key);
    B[f].cell = btag[f]; B[f].k = 0;
  }
  qsort(B, nbf, sizeof(o3_fkey), fkey_cmp);
  m->face = (o3_face *)calloc(nfk, sizeof(o3_face));
  long nf = 0;
  for (long i = 0; i < nfk;) {
    long j = i + 1;
    while (j < nfk && memcmp(E[j].key, E[i].key, sizeof E[i].key) == 0) ++j;
    if (j - i > 2) { *err = 2; break; }
    o3_face *F = &m->face[nf];
    long c0 = E[i].cell;
    const o3_cell *C = &m->cell[c0];
    const int (*tab)[4];
    cell_faces(C->type, &tab);
    int mm = tab[E[i].k][3] < 0 ? 3 : 4;
    double X[4][3];
    F->nv = mm;
    for (int a = 0; a < mm; ++a) {
      F->node[a] = C->node[tab[E[i].k][a]];
      for (int d = 0; d < 3; ++d) X[a][d] = m->x[3 * F->node[a] + d];
    }
    face_geometry(mm, X, F);
    F->c0 = c0;
    if (j - i == 2) { F->c1 = E[i + 1].cell; F->tag = -1; }
    else {
      F->c1 = -1;
      long lo = 0, hi = nbf - 1, found = -1;
      while (lo <= hi) {
        long mid = (lo + hi) / 2;
        int cmp = memcmp(B[mid].key, E[i].key, sizeof E[i].key);
        int less = 0;
        for (int t = 0; t < 4; ++t) if (B[mid].key[t] != E[i].key[t]) { less = B[mid].key[t] < E[i].key[t]; break; }
        if (cmp != 0 && less) lo = mid + 1;
        else { if (cmp == 0) found = mid; hi = mid - 1; }
      }
      if (found < 0) { *err = 3; break; }
      F->tag = (int)B[found].cell;
    }
    ++nf;
    i = j;
  }
  free(E); free(B);
  if (*err) { mesh_free(m); return NULL; }
  m->nf = nf;
  for (long f = 0; f < nf; ++f) {
    o3_face *F = &m->face[f];
    const double *x0 = m->cell[F->c0].xc;
    double d[3];
    if (F->c1 >= 0) {
      const double *x1 = m->cell[F->c1].xc;
      for (int k = 0; k < 3; ++k) d[k] = x1[k] - x0[k];
      F->delta = fabs(dot3(d, F->n));
    } else {
      for (int k = 0; k < 3; ++k) d[k] = F->xf[k] - x0[k];
      F->delta = 2.0 * fabs(dot3(d, F->n));
    }
    o3_cell *C0 = &m->cell[F->c0];
    C0->face[C0->nf] = f; C0->sgn[C0->nf] = +1; C0->nf++;
    if (F->c1 >= 0) {
      o3_cell *C1 = &m->cell[F->c1];
      C1->face[C1->nf] = f; C1->sgn[C1->nf] = -1; C1->nf++;
      C0->nbr[C0->nb++] = F->c1;
      C1->nbr[C1->nb++] = F->c0;
    }
  }
  mesh_ordering(m);
  return m;
}

long o3_mesh_nfaces(const o3_mesh *m) { return m->nf; }
int o3_mesh_ncolours(const o3_mesh *m) { return m->ncolour; }
void o3_mesh_geometry(const o3_mesh *m, double *vol, double *xc, double *M2) {
  for (long c = 0; c < m->nc; ++c) {
    vol[c] = m->cell[c].vol;
    for (int d = 0; d < 3; ++d) xc[3 * c + d] = m->cell[c].xc[d];
    for (int q = 0; q < 6; ++q) M2[6 * c + q] = m->cell[c].M2[q];
  }
}
/* per face: c0, c1, tag, n[3], S, number of Gauss points, xg[4][3], wg[4] */
void o3_mesh_faces(const o3_mesh *m, int64_t *c0, int64_t *c1, int32_t *tag, double *n, double *S, int32_t *ng,
                   double *xg, double *wg) {
  for (long f = 0; f < m->nf; ++f) {
    const o3_face *F = &m->face[f];
    c0[f] = F->c0; c1[f] = F->c1; tag[f] = F->tag; S[f] = F->S; ng[f] = F->ng;
    for (int d = 0; d < 3; ++d) n[3 * f + d] = F->n[d];
    for (int k = 0; k < MAXGP; ++k) {
      for (int d = 0; d < 3; ++d) xg[12 * f + 3 * k + d] = k < F->ng ? F->xg[k][d] : 0.0;
      wg[4 * f + k] = k < F->ng ? F->wg[k] : 0.0;
    }
  }
}

/* reverse Cuthill-McKee from the lowest-index cell of minimum degree,
 * neighbours by (degree, index); greedy smallest-free colouring in RCM order */
static const o3_mesh *g_mesh;
static int nbr_cmp(const void *x, const void *y) {
  long a = *(const long *)x, b = *(const long *)y;
  int da = g_mesh->cell[a].nb, db = g_mesh->cell[b].nb;
  if (da != db) return da < db ? -1 : 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}
static void mesh_ordering(o3_mesh *m) {
  long nc = m->nc;
  long *cm = (long *)malloc(sizeof(long) * nc);
  char *seen = (char *)calloc(nc, 1);
  long head = 0, tail = 0;
  g_mesh = m;
  /* minimum-degree start: one pass to find it, then rescan from there */
  long scan = 0;
  while (tail < nc) {
    long start = -1;
    int mind = 1 << 30;
    for (long c = 0; c < nc; ++c)
      if (!seen[c] && m->cell[c].nb < mind) { mind = m->cell[c].nb; start = c; }
    (void)scan;
    seen[start] = 1; cm[tail++] = start;
    while (head < tail) {
      long v = cm[head++], nb[MAXFC];
      int k = 0;
      for (int i = 0; i < m->cell[v].nb; ++i) if (!seen[m->cell[v].nbr[i]]) nb[k++] = m->cell[v].nbr[i];
      qsort(nb, k, sizeof(long), nbr_cmp);
      for (int i = 0; i < k; ++i) { seen[nb[i]] = 1; cm[tail++] = nb[i]; }
    }
  }
  m->rcm = (long *)malloc(sizeof(long) * nc);
  for (long i = 0; i < nc; ++i) m->rcm[i] = cm[nc - 1 - i];
  m->colour = (int *)malloc(sizeof(int) * nc);
  for (long c = 0; c < nc; ++c) m->colour[c] = -1;
  m->ncolour = 0;
  for (long i = 0; i < nc; ++i) {
    long v = m->rcm[i];
    int used[16] = { 0 };
    for (int k = 0; k < m->cell[v].nb; ++k) {
      int cc = m->colour[m->cell[v].nbr[k]];
      if (cc >= 0) used[cc] = 1;
    }
    int col = 0;
    while (used[col]) ++col;
    m->colour[v] = col;
    if (col + 1 > m->ncolour) m->ncolour = col + 1;
  }
  free(cm); free(seen);
}
void o3_mesh_ordering(const o3_mesh *m, int64_t *rcm, int32_t *colour) {
  for (long i = 0; i < m->nc; ++i) { rcm[i] = m->rcm[i]; colour[i] = m->colour[i]; }
}

/* ------------------------------------------------------------------ */
/* solver                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
  const o3_mesh *m;
  o3_params P;
  double *W, *Wx;             /* [nc][NV], [nc][3][NV] */
  double *coef;               /* [nc][NM][NV] */
  double *mom_self;           /* [nc][NM] */
  double *F0, *F1, *Wc, *Wt;  /* [nf][NV] */
  double *Rp0;
  double res, dt_last;
  int status;
} o3_solver;

/* means over a cell (volume V, centroid xj, central moments M2j) of the
 * monomials in the scaled coordinates of cell i */
static void monomial_means(const double xi[3], double h, const double xj[3], const double M2j[6], double out[NM]) {
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = (xj[k] - xi[k]) / h;
  double h2 = h * h;
  out[0] = d[0]; out[1] = d[1]; out[2] = d[2];
  out[3] = M2j[0] / h2 + d[0] * d[0];
  out[4] = M2j[1] / h2 + d[0] * d[1];
  out[5] = M2j[2] / h2 + d[0] * d[2];
  out[6] = M2j[3] / h2 + d[1] * d[1];
  out[7] = M2j[4] / h2 + d[1] * d[2];
  out[8] = M2j[5] / h2 + d[2] * d[2];
}

o3_solver *o3_solver_create(const o3_mesh *m, const o3_params *P) {
  o3_solver *s = (o3_solver *)calloc(1, sizeof(o3_solver));
  s->m = m; s->P = *P;
  long nc = m->nc, nf = m->nf;
  s->W = (double *)calloc(nc * NV, sizeof(double));
  s->Wx = (double *)calloc(nc * ND * NV, sizeof(double));
  s->coef = (double *)calloc(nc * NM * NV, sizeof(double));
  s->mom_self = (double *)calloc(nc * NM, sizeof(double));
  s->F0 = (double *)calloc(nf * NV, sizeof(double));
  s->F1 = (double *)calloc(nf * NV, sizeof(double));
  s->Wc = (double *)calloc(nf * NV, sizeof(double));
  s->Wt = (double *)calloc(nf * NV, sizeof(double));
  s->Rp0 = (double *)calloc(nc * NV, sizeof(double));
  for (long c = 0; c < nc; ++c)
    monomial_means(m->cell[c].xc, m->cell[c].h, m->cell[c].xc, m->cell[c].M2, &s->mom_self[c * NM]);
  return s;
}
void o3_solver_destroy(o3_solver *s) {
  if (!s) return;
  free(s->W); free(s->Wx); free(s->coef); free(s->mom_self);
  free(s->F0); free(s->F1); free(s->Wc); free(s->Wt); free(s->Rp0); free(s);
}
void o3_set_state(o3_solver *s, const double *W, const double *Wx) {
  memcpy(s->W, W, sizeof(double) * s->m->nc * NV);
  if (Wx) memcpy(s->Wx, Wx, sizeof(double) * s->m->nc * ND * NV);
  else memset(s->Wx, 0, sizeof(double) * s->m->nc * ND * NV);
}
void o3_get_state(const o3_solver *s, double *W, double *Wx) {
  if (W) memcpy(W, s->W, sizeof(double) * s->m->nc * NV);
  if (Wx) memcpy(Wx, s->Wx, sizeof(double) * s->m->nc * ND * NV);
}
double o3_last_residual(const o3_solver *s) { return s->res; }
int o3_status(const o3_solver *s) { return s->status; }

static int is_wall(const o3_solver *s, const o3_face *F) {
  return F->c1 < 0 && s->P.bc[F->tag].kind != O3_BC_FARFIELD;
}

/* the mirror image of cell i across the plane of face F: its nodes
 * reflected, then the same tet decomposition (orientation reversed) */
static void mirror_means(const o3_mesh *m, long i, const o3_face *F, double out[NM]) {
  const o3_cell *C = &m->cell[i];
  double X[8][3];
  for (int a = 0; a < C->nv; ++a) {
    const double *x = &m->x[3 * C->node[a]];
    double d = (x[0] - F->xf[0]) * F->n[0] + (x[1] - F->xf[1]) * F->n[1] + (x[2] - F->xf[2]) * F->n[2];
    for (int k = 0; k < 3; ++k) X[a][k] = x[k] - 2.0 * d * F->n[k];
  }
  double V, xc[3], M2[6];
  polyhedron(C->type, X, &V, xc, M2);   /* V < 0 (reflected), ratios still exact */
  monomial_means(C->xc, C->h, xc, M2, out);
}

/* derivatives of the monomials averaged over a cell with monomial means mj:
 * rows d/dx, d/dy, d/dz (times h) */
static void grad_rows(const double mj[NM], double gx[NM], double gy[NM], double gz[NM]) {
  double a = mj[0], b = mj[1], c = mj[2];
  double X[NM] = { 1, 0, 0, 2 * a, b, c, 0, 0, 0 };
  double Y[NM] = { 0, 1, 0, 0, a, 0, 2 * b, c, 0 };
  double Z[NM] = { 0, 0, 1, 0, 0, a, 0, b, 2 * c };
  memcpy(gx, X, sizeof X); memcpy(gy, Y, sizeof Y); memcpy(gz, Z, sizeof Z);
}

/* Smoothness indicator of a candidate with scaled coefficients c (stride
 * between monomials): the cell mean of the squared first derivatives in
 * the scaled coordinates (linear functions, so the mean is the square of
 * the centroid value plus the quadratic form of the central second
 * moments M2 / h^2) plus the squared second derivatives, each multi-index
 * once. */
static double weno_beta3(const o3_cell *C, const double *c, int stride) {
  double q[NM];
  for (int k = 0; k < NM; ++k) q[k] = c[k * stride];
  /* gradient of P = g0 + G (xi, eta, zeta) */
  double g0[3] = { q[0], q[1], q[2] };
  double G[3][3] = { { 2 * q[3], q[4], q[5] }, { q[4], 2 * q[6], q[7] }, { q[5], q[7], 2 * q[8] } };
  double h2 = C->h * C->h;
  double M[3][3] = { { C->M2[0] / h2, C->M2[1] / h2, C->M2[2] / h2 },
                     { C->M2[1] / h2, C->M2[3] / h2, C->M2[4] / h2 },
                     { C->M2[2] / h2, C->M2[4] / h2, C->M2[5] / h2 } };
  double b = 0.0;
  for (int d = 0; d < 3; ++d) {
    b += g0[d] * g0[d];
    for (int a = 0; a < 3; ++a)
      for (int e = 0; e < 3; ++e) b += G[d][a] * M[a][e] * G[d][e];
  }
  return b + 4 * q[3] * q[3] + q[4] * q[4] + q[5] * q[5] + 4 * q[6] * q[6] + q[7] * q[7] + 4 * q[8] * q[8];
}

/* Compact WENO (conservative variables), as in 2-D: candidates P2 (X) and
 * the linear polynomials of the mean gradients of the cell and its face
 * neighbours; gamma_0 = g0, the rest (1 - g0)/m; w ~ gamma/(beta + eps)^2;
 * P = (w_0/gamma_0)(P2 - sum gamma_k P1_k) + sum w_k P1_k.  In place. */
static void weno_combine3(const o3_solver *s, const double *Wx, long i, double *X) {
  const o3_cell *C = &s->m->cell[i];
  double g0 = s->P.weno_g0, eps = s->P.weno_eps;
  long cand[MAXFC + 1];
  int m = 0;
  cand[m++] = i;
  for (int k = 0; k < C->nb; ++k) cand[m++] = C->nbr[k];
  double gk = (1.0 - g0) / m;
  for (int v = 0; v < NV; ++v) {
    double G[MAXFC + 1][3], wt[MAXFC + 2], wsum = 0.0;
    double b0 = weno_beta3(C, &X[v], NV);
    wt[0] = g0 / ((b0 + eps) * (b0 + eps));
    for (int k = 0; k < m; ++k) {
      double cl[NM] = { 0 };
      for (int d = 0; d < 3; ++d) cl[d] = G[k][d] = C->h * Wx[(cand[k] * ND + d) * NV + v];
      double b = weno_beta3(C, cl, 1);
      wt[k + 1] = gk / ((b + eps) * (b + eps));
    }
    for (int k = 0; k <= m; ++k) wsum += wt[k];
    for (int k = 0; k <= m; ++k) wt[k] /= wsum;
    for (int q = 0; q < NM; ++q) {
      double lin = 0.0, sel = 0.0;
      if (q < 3)
        for (int k = 0; k < m; ++k) { lin += gk * G[k][q]; sel += wt[k + 1] * G[k][q]; }
      X[q * NV + v] = wt[0] / g0 * (X[q * NV + v] - lin) + sel;
    }
  }
}

static void reconstruct_cell(o3_solver *s, const double *W, const double *Wx, long i) {
  const o3_mesh *m = s->m;
  const o3_cell *C = &m->cell[i];
  double *c = &s->coef[i * NM * NV];
  const double *mi = &s->mom_self[i * NM];
  /* quadratic only when the stencil cells' centroids spread in all three
   * directions: the normalised determinant of T = sum_j d_j d_j^T, d_j the
   * scaled centroid offsets of the neighbours and wall mirror cells */
  double T[3][3] = { { 0 } };
  int nst = 0;
  for (int k = 0; k < C->nf; ++k) {
    const o3_face *F = &m->face[C->face[k]];
    double d[3];
    if (F->c1 >= 0) {
      long j = C->sgn[k] > 0 ? F->c1 : F->c0;
      for (int a = 0; a < 3; ++a) d[a] = (m->cell[j].xc[a] - C->xc[a]) / C->h;
    } else if (is_wall(s, F)) {
      double t = dot3(F->n, F->xf) - dot3(F->n, C->xc);
      for (int a = 0; a < 3; ++a) d[a] = 2.0 * t * F->n[a] / C->h;
    } else continue;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) T[a][b] += d[a] * d[b];
    ++nst;
  }
  double tr = T[0][0] + T[1][1] + T[2][2];
  double det = T[0][0] * (T[1][1] * T[2][2] - T[1][2] * T[2][1]) - T[0][1] * (T[1][0] * T[2][2] - T[1][2] * T[2][0]) +
               T[0][2] * (T[1][0] * T[2][1] - T[1][1] * T[2][0]);
  int quadratic = nst >= 3 && tr > 0.0 && det / (tr * tr * tr / 27.0) >= 1e-3;
  if (!quadratic) {
    for (int q = 0; q < NM * NV; ++q) c[q] = 0.0;
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < NV; ++v) c[d * NV + v] = C->h * Wx[(i * ND + d) * NV + v];
    return;
  }
  double A[MAXROWS * NM], B[MAXROWS * NV], X[NM * NV];
  int row = 0;
  for (int k = 0; k < C->nb; ++k) {
    long j = C->nbr[k];
    double mj[NM], g[3][NM];
    monomial_means(C->xc, C->h, m->cell[j].xc, m->cell[j].M2, mj);
    for (int q = 0; q < NM; ++q) A[row * NM + q] = mj[q] - mi[q];
    for (int v = 0; v < NV; ++v) B[row * NV + v] = W[j * NV + v] - W[i * NV + v];
    ++row;
    grad_rows(mj, g[0], g[1], g[2]);
    for (int d = 0; d < 3; ++d, ++row) {
      for (int q = 0; q < NM; ++q) A[row * NM + q] = g[d][q];
      for (int v = 0; v < NV; ++v) B[row * NV + v] = C->h * Wx[(j * ND + d) * NV + v];
    }
  }
  for (int k = 0; k < C->nf; ++k) {
    const o3_face *F = &m->face[C->face[k]];
    if (!is_wall(s, F)) continue;
    double mg[NM], Wg[NV], Gg[ND * NV], g[3][NM];
    mirror_means(m, i, F, mg);
    o3_ghost(&s->P, F->tag, &W[i * NV], &Wx[i * ND * NV], F->n, Wg, Gg);
    for (int q = 0; q < NM; ++q) A[row * NM + q] = mg[q] - mi[q];
    for (int v = 0; v < NV; ++v) B[row * NV + v] = Wg[v] - W[i * NV + v];
    ++row;
    grad_rows(mg, g[0], g[1], g[2]);
    for (int d = 0; d < 3; ++d, ++row) {
      for (int q = 0; q < NM; ++q) A[row * NM + q] = g[d][q];
      for (int v = 0; v < NV; ++v) B[row * NV + v] = C->h * Gg[d * NV + v];
    }
  }
  {
    double g[3][NM];
    grad_rows(mi, g[0], g[1], g[2]);
    for (int d = 0; d < 3; ++d, ++row) {
      for (int q = 0; q < NM; ++q) A[row * NM + q] = g[d][q];
      for (int v = 0; v < NV; ++v) B[row * NV + v] = C->h * Wx[(i * ND + d) * NV + v];
    }
  }
  if (householder_ls(row, NM, A, NV, B, X) != 0) {
    /* rank-deficient stencil: the same linear reconstruction as above */
    for (int q = 0; q < NM * NV; ++q) c[q] = 0.0;
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < NV; ++v) c[d * NV + v] = C->h * Wx[(i * ND + d) * NV + v];
    return;
  }
  if (s->P.weno_eps > 0.0) weno_combine3(s, Wx, i, X);
  for (int q = 0; q < NM * NV; ++q) c[q] = X[q];
}

static void reconstruct_all(o3_solver *s, const double *W, const double *Wx) {
  for (long i = 0; i < s->m->nc; ++i) reconstruct_cell(s, W, Wx, i);
}

static void recon_eval(const o3_solver *s, const double *W, long i, const double x[3], double val[NV],
                       double grad[ND * NV]) {
  const o3_cell *C = &s->m->cell[i];
  const double *c = &s->coef[i * NM * NV];
  const double *mi = &s->mom_self[i * NM];
  double a = (x[0] - C->xc[0]) / C->h, b = (x[1] - C->xc[1]) / C->h, e = (x[2] - C->xc[2]) / C->h;
  double phi[NM] = { a, b, e, a * a, a * b, a * e, b * b, b * e, e * e };
  double dx[NM] = { 1, 0, 0, 2 * a, b, e, 0, 0, 0 };
  double dy[NM] = { 0, 1, 0, 0, a, 0, 2 * b, e, 0 };
  double dz[NM] = { 0, 0, 1, 0, 0, a, 0, b, 2 * e };
  for (int v = 0; v < NV; ++v) {
    double p = W[i * NV + v], gx = 0, gy = 0, gz = 0;
    for (int q = 0; q < NM; ++q) {
      p += c[q * NV + v] * (phi[q] - mi[q]);
      gx += c[q * NV + v] * dx[q]; gy += c[q * NV + v] * dy[q]; gz += c[q * NV + v] * dz[q];
    }
    val[v] = p; grad[v] = gx / C->h; grad[NV + v] = gy / C->h; grad[2 * NV + v] = gz / C->h;
  }
}

void o3_reconstruct(o3_solver *s) { reconstruct_all(s, s->W, s->Wx); }
void o3_recon_eval(const o3_solver *s, long cell, const double x[3], double val[NV], double grad[ND * NV]) {
  recon_eval(s, s->W, cell, x, val, grad);
}

/* reconstruction + face fluxes; per face the weighted Gauss sums */
static void hi_eval(o3_solver *s, const double *W, const double *Wx, double dt) {
  const o3_mesh *m = s->m;
  reconstruct_all(s, W, Wx);
  for (long f = 0; f < m->nf; ++f) {
    const o3_face *F = &m->face[f];
    double sF0[NV] = { 0 }, sF1[NV] = { 0 }, sWc[NV] = { 0 }, sWt[NV] = { 0 };
    for (int k = 0; k < F->ng; ++k) {
      double Wl[NV], gl[ND * NV], Wr[NV], gr[ND * NV];
      recon_eval(s, W, F->c0, F->xg[k], Wl, gl);
      if (F->c1 >= 0) recon_eval(s, W, F->c1, F->xg[k], Wr, gr);
      else if (is_wall(s, F)) o3_ghost(&s->P, F->tag, Wl, gl, F->n, Wr, gr);
      else {
        double zero[ND * NV] = { 0 };
        o3_ghost(&s->P, F->tag, &W[F->c0 * NV], zero, F->n, Wr, gr);
      }
      double f0[NV], f1[NV], wc[NV], wt[NV];
      if (s->P.flux_hi) o3_gks_full_flux_point(&s->P, Wl, Wr, gl, gr, F->n, F->delta, dt, f0, f1, wc, wt);
      else o3_gks_flux_point(&s->P, Wl, Wr, gl, gr, F->n, F->delta, f0, f1, wc, wt);
      for (int v = 0; v < NV; ++v) {
        sF0[v] += F->wg[k] * f0[v]; sF1[v] += F->wg[k] * f1[v];
        sWc[v] += F->wg[k] * wc[v]; sWt[v] += F->wg[k] * wt[v];
      }
    }
    for (int v = 0; v < NV; ++v) {
      s->F0[f * NV + v] = sF0[v]; s->F1[f * NV + v] = sF1[v];
      s->Wc[f * NV + v] = sWc[v]; s->Wt[f * NV + v] = sWt[v];
    }
  }
}

/* Wall loads (Section 4's sphere drag and surface quantities): for every
 * boundary face carrying tag, in the oracle's face order, the face centre
 * (vertex mean), the unit normal out of the fluid, the area, and the
 * momentum part of the face's high-order flux F0 at the current state
 * (the weighted Gauss-point sum; with the full flux, of its fit over a
 * step dt; global frame): on a wall the traction the fluid exerts.
 * Arrays hold max_faces entries; returns the number of faces with the tag. */
long o3_wall_loads(o3_solver *s, int tag, double dt, long max_faces, double *x, double *n, double *S,
                   double *traction) {
  const o3_mesh *m = s->m;
  hi_eval(s, s->W, s->Wx, dt);
  long k = 0;
  for (long f = 0; f < m->nf; ++f) {
    const o3_face *F = &m->face[f];
    if (F->c1 >= 0 || F->tag != tag) continue;
    if (k < max_faces) {
      for (int d = 0; d < 3; ++d) {
        x[3 * k + d] = F->xf[d];
        n[3 * k + d] = F->n[d];
        traction[3 * k + d] = s->F0[f * NV + 1 + d];
      }
      S[k] = F->S;
    }
    ++k;
  }
  return k;
}

static void net_flux(const o3_solver *s, const double *F0, const double *F1, double a, double b, double *out) {
  const o3_mesh *m = s->m;
  memset(out, 0, sizeof(double) * m->nc * NV);
  for (long f = 0; f < m->nf; ++f) {
    const o3_face *F = &m->face[f];
    for (int v = 0; v < NV; ++v) {
      double fl = F->S * (a * F0[f * NV + v] + b * F1[f * NV + v]);
      out[F->c0 * NV + v] -= fl;
      if (F->c1 >= 0) out[F->c1 * NV + v] += fl;
    }
  }
}

static void gauss_green(const o3_solver *s, const double *Wc, const double *Wt, double t, double *Wx) {
  const o3_mesh *m = s->m;
  memset(Wx, 0, sizeof(double) * m->nc * ND * NV);
  for (long f = 0; f < m->nf; ++f) {
    const o3_face *F = &m->face[f];
    for (int v = 0; v < NV; ++v) {
      double wp = Wc[f * NV + v] + t * Wt[f * NV + v];
      for (int d = 0; d < 3; ++d) {
        double g = F->S * F->n[d] * wp;
        Wx[(F->c0 * ND + d) * NV + v] += g;
        if (F->c1 >= 0) Wx[(F->c1 * ND + d) * NV + v] -= g;
      }
    }
  }
  for (long c = 0; c < m->nc; ++c)
    for (int q = 0; q < ND * NV; ++q) Wx[c * ND * NV + q] /= m->cell[c].vol;
}

/* dt = CFL_hi min_i h_i / (|U_i| + c_i + 2 nu_i / h_i), h_i = 3|Omega_i| / sum_p S_p */
double o3_explicit_dt(const o3_solver *s) {
  const o3_mesh *m = s->m;
  double dt = INFINITY;
  for (long c = 0; c < m->nc; ++c) {
    const o3_cell *C = &m->cell[c];
    double area = 0.0;
    for (int k = 0; k < C->nf; ++k) area += m->face[C->face[k]].S;
    double h = 3.0 * C->vol / area, rho, u[3], p;
    prim3(s->P.gamma, &s->W[c * NV], &rho, u, &p);
    double speed = sqrt(dot3(u, u)) + sqrt(s->P.gamma * p / rho) + 2.0 * (s->P.mu / rho) / h;
    double d = h / speed;
    if (d < dt) dt = d;
  }
  return s->P.cfl_hi * dt;
}

static int check_state(o3_solver *s, const double *W) {
  for (long c = 0; c < s->m->nc; ++c) {
    double rho, u[3], p;
    prim3(s->P.gamma, &W[c * NV], &rho, u, &p);
    if (!(rho > 0.0) || !(p > 0.0) || !isfinite(rho) || !isfinite(p)) { s->status = 1; return 1; }
  }
  return 0;
}

static void hi_step(o3_solver *s, const double *W, const double *Wx, double dt, double *Wn, double *Wxn,
                    double *Rlag) {
  const o3_mesh *m = s->m;
  long nc = m->nc, nf = m->nf;
  hi_eval(s, W, Wx, dt);
  if (s->P.time_scheme == 0) {
    net_flux(s, s->F0, s->F1, 1.0, 0.5 * dt, Rlag);
    for (long c = 0; c < nc; ++c)
      for (int v = 0; v < NV; ++v) Wn[c * NV + v] = W[c * NV + v] + dt / m->cell[c].vol * Rlag[c * NV + v];
    gauss_green(s, s->Wc, s->Wt, dt, Wxn);
  } else {
    double *F0n = (double *)malloc(sizeof(double) * nf * NV), *F1n = (double *)malloc(sizeof(double) * nf * NV);
    double *Wcn = (double *)malloc(sizeof(double) * nf * NV);
    double *Ws = (double *)malloc(sizeof(double) * nc * NV), *Wxs = (double *)malloc(sizeof(double) * nc * ND * NV);
    double *R = (double *)malloc(sizeof(double) * nc * NV), *F1c = (double *)malloc(sizeof(double) * nf * NV);
    memcpy(F0n, s->F0, sizeof(double) * nf * NV);
    memcpy(F1n, s->F1, sizeof(double) * nf * NV);
    memcpy(Wcn, s->Wc, sizeof(double) * nf * NV);
    net_flux(s, F0n, F1n, 0.5, 0.125 * dt, R);
    for (long c = 0; c < nc; ++c)
      for (int v = 0; v < NV; ++v) Ws[c * NV + v] = W[c * NV + v] + dt / m->cell[c].vol * R[c * NV + v];
    gauss_green(s, Wcn, s->Wt, 0.5 * dt, Wxs);
    hi_eval(s, Ws, Wxs, dt);
    for (long q = 0; q < nf * NV; ++q) F1c[q] = F1n[q] + 2.0 * s->F1[q];
    net_flux(s, F0n, F1c, 1.0, dt / 6.0, Rlag);
    for (long c = 0; c < nc; ++c)
      for (int v = 0; v < NV; ++v) Wn[c * NV + v] = W[c * NV + v] + dt / m->cell[c].vol * Rlag[c * NV + v];
    gauss_green(s, Wcn, s->Wt, dt, Wxn);
    free(F0n); free(F1n); free(Wcn); free(Ws); free(Wxs); free(R); free(F1c);
  }
}

static double density_residual(const o3_mesh *m, const double *Wold, const double *Wnew) {
  double num = 0.0, den = 0.0;
  for (long c = 0; c < m->nc; ++c) { num += fabs(Wnew[c * NV] - Wold[c * NV]); den += Wold[c * NV]; }
  return num / den;
}

double o3_highorder_step(o3_solver *s, double dt) {
  long nc = s->m->nc;
  if (dt <= 0.0) dt = o3_explicit_dt(s);
  double *Wn = (double *)malloc(sizeof(double) * nc * NV), *Wxn = (double *)malloc(sizeof(double) * nc * ND * NV);
  hi_step(s, s->W, s->Wx, dt, Wn, Wxn, s->Rp0);
  s->res = density_residual(s->m, s->W, Wn);
  memcpy(s->W, Wn, sizeof(double) * nc * NV);
  memcpy(s->Wx, Wxn, sizeof(double) * nc * ND * NV);
  free(Wn); free(Wxn);
  s->dt_last = dt;
  check_state(s, s->W);
  return dt;
}

void o3_hi_residual(o3_solver *s, double dt, double *R) {
  hi_eval(s, s->W, s->Wx, dt);
  net_flux(s, s->F0, s->F1, 1.0, 0.5 * dt, R);
}

/* ---- low-order level ---- */
static void lo_ghost(const o3_solver *s, int tag, const double U[NV], const double n[3], double Ug[NV]) {
  double g0[ND * NV] = { 0 }, gg[ND * NV];
  o3_ghost(&s->P, tag, U, g0, n, Ug, gg);
}
static double lo_lambda_side(const o3_solver *s, const double U[NV], const double n[3], double S, double vol) {
  double rho, u[3], p;
  prim3(s->P.gamma, U, &rho, u, &p);
  return fabs(dot3(u, n)) + sqrt(s->P.gamma * p / rho) + 2.0 * (s->P.mu / rho) * S / vol;
}
/* R_lo,i(U) = -sum_p S_p F_lo(U_i, U_ip; n_p): KFVS, or the Lax-Friedrichs
 * alternative of Section 3 with the implicit operator's lambda_p,
 * (F_n(U_l) + F_n(U_r)) / 2 - lambda_p (U_r - U_l) / 2 */
/* First-order viscous flux of the low-order level, as in 2-D: normal
 * gradients from the two cell states over the centre distance delta along
 * n (boundary faces: twice the centre-to-face distance, ghost state),
 *   tau.n = mu / delta (du + (n.du) n / 3),  q.n = -kappa (T_r - T_l) / delta,
 * F -= (0, tau.n, tau.n . (u_l + u_r)/2 - q.n). */
static void lo_viscous_flux(const o3_solver *s, const double Ul[NV], const double Ur[NV], const double n[3],
                            double delta, double F[NV]) {
  double rl, ul[3], pl, rr, ur[3], pr;
  prim3(s->P.gamma, Ul, &rl, ul, &pl);
  prim3(s->P.gamma, Ur, &rr, ur, &pr);
  const double mu = s->P.mu, kappa = mu * s->P.gamma / (s->P.gamma - 1.0);
  const double du[3] = { ur[0] - ul[0], ur[1] - ul[1], ur[2] - ul[2] };
  const double dn = dot3(du, n);
  double tau[3], work = 0.0;
  for (int d = 0; d < 3; ++d) {
    tau[d] = mu / delta * (du[d] + dn * n[d] / 3.0);
    work += tau[d] * 0.5 * (ul[d] + ur[d]);
  }
  const double qn = -kappa * (pr / rr - pl / rl) / delta;
  F[1] -= tau[0];
  F[2] -= tau[1];
  F[3] -= tau[2];
  F[4] -= work - qn;
}

static void lo_residual(const o3_solver *s, const double *U, double *R) {
  const o3_mesh *m = s->m;
  memset(R, 0, sizeof(double) * m->nc * NV);
  for (long f = 0; f < m->nf; ++f) {
    const o3_face *F = &m->face[f];
    double Ur[NV], Fl[NV];
    if (F->c1 >= 0) memcpy(Ur, &U[F->c1 * NV], sizeof Ur);
    else lo_ghost(s, F->tag, &U[F->c0 * NV], F->n, Ur);
    if (s->P.flux_lo == 1) {
      const double v0 = m->cell[F->c0].vol, v1 = F->c1 >= 0 ? m->cell[F->c1].vol : v0;
      const double l0 = lo_lambda_side(s, &U[F->c0 * NV], F->n, F->S, v0);
      const double l1 = lo_lambda_side(s, Ur, F->n, F->S, v1);
      const double lam = l0 > l1 ? l0 : l1;
      double Fa[NV], Fb[NV];
      o3_euler_flux(s->P.gamma, &U[F->c0 * NV], F->n, Fa);
      o3_euler_flux(s->P.gamma, Ur, F->n, Fb);
      for (int v = 0; v < NV; ++v) Fl[v] = 0.5 * (Fa[v] + Fb[v]) - 0.5 * lam * (Ur[v] - U[F->c0 * NV + v]);
    } else {
      o3_kfvs(&s->P, &U[F->c0 * NV], Ur, F->n, Fl);
    }
    if (s->P.lo_viscous && s->P.mu > 0.0) lo_viscous_flux(s, &U[F->c0 * NV], Ur, F->n, F->delta, Fl);
    for (int v = 0; v < NV; ++v) {
      R[F->c0 * NV + v] -= F->S * Fl[v];
      if (F->c1 >= 0) R[F->c1 * NV + v] += F->S * Fl[v];
    }
  }
}
static void lo_lambda(const o3_solver *s, const double *U, double *lam) {
  const o3_mesh *m = s->m;
  for (long f = 0; f < m->nf; ++f) {
    const o3_face *F = &m->face[f];
    double l0 = lo_lambda_side(s, &U[F->c0 * NV], F->n, F->S, m->cell[F->c0].vol), l1;
    if (F->c1 >= 0) l1 = lo_lambda_side(s, &U[F->c1 * NV], F->n, F->S, m->cell[F->c1].vol);
    else { double Ug[NV]; lo_ghost(s, F->tag, &U[F->c0 * NV], F->n, Ug); l1 = lo_lambda_side(s, Ug, F->n, F->S, m->cell[F->c0].vol); }
    lam[f] = l0 > l1 ? l0 : l1;
  }
}
static void fminus(const o3_solver *s, const double U[NV], const double n[3], double lam, double out[NV]) {
  double F[NV];
  o3_euler_flux(s->P.gamma, U, n, F);
  for (int v = 0; v < NV; ++v) out[v] = 0.5 * (F[v] - lam * U[v]);
}
static void relax_cell(const o3_solver *s, long i, const double *U, const double *R, const double *lam,
                       const double *D, double *dU) {
  const o3_mesh *m = s->m;
  const o3_cell *C = &m->cell[i];
  double acc[NV];
  for (int v = 0; v < NV; ++v) acc[v] = R[i * NV + v];
  for (int k = 0; k < C->nf; ++k) {
    const o3_face *F = &m->face[C->face[k]];
    if (F->c1 < 0) continue;
    long j = C->sgn[k] > 0 ? F->c1 : F->c0;
    double n[3] = { C->sgn[k] * F->n[0], C->sgn[k] * F->n[1], C->sgn[k] * F->n[2] };
    double Up[NV], fa[NV], fb[NV];
    for (int v = 0; v < NV; ++v) Up[v] = U[j * NV + v] + dU[j * NV + v];
    fminus(s, Up, n, lam[C->face[k]], fa);
    fminus(s, &U[j * NV], n, lam[C->face[k]], fb);
    for (int v = 0; v < NV; ++v) acc[v] -= F->S * (fa[v] - fb[v]);
  }
  for (int v = 0; v < NV; ++v) dU[i * NV + v] = acc[v] / D[i];
}
static void lo_diag(const o3_solver *s, const double *lam, double *D) {
  const o3_mesh *m = s->m;
  for (long i = 0; i < m->nc; ++i) {
    const o3_cell *C = &m->cell[i];
    double sum = 0.0;
    for (int k = 0; k < C->nf; ++k) sum += lam[C->face[k]] * m->face[C->face[k]].S;
    double dti = s->P.cfl_lo * C->vol / sum;
    D[i] = C->vol / dti + 0.5 * sum;
  }
}
static void point_relaxation(const o3_solver *s, const double *U, const double *R, const double *lam,
                             const double *D, int n_sweeps, double *dU) {
  const o3_mesh *m = s->m;
  memset(dU, 0, sizeof(double) * m->nc * NV);
  for (int sw = 0; sw < n_sweeps; ++sw) {
    for (int col = 0; col < m->ncolour; ++col)
      for (long i = 0; i < m->nc; ++i) if (m->colour[i] == col) relax_cell(s, i, U, R, lam, D, dU);
    for (int col = m->ncolour - 1; col >= 0; --col)
      for (long i = 0; i < m->nc; ++i) if (m->colour[i] == col) relax_cell(s, i, U, R, lam, D, dU);
  }
}
static void lo_solve(o3_solver *s, const double *Wp0, const double *Rp0, double *U) {
  const o3_mesh *m = s->m;
  long nc = m->nc, nf = m->nf;
  double *Src = (double *)malloc(sizeof(double) * nc * NV), *R = (double *)malloc(sizeof(double) * nc * NV);
  double *lam = (double *)malloc(sizeof(double) * nf), *D = (double *)malloc(sizeof(double) * nc);
  double *dU = (double *)malloc(sizeof(double) * nc * NV);
  lo_residual(s, Wp0, R);
  for (long q = 0; q < nc * NV; ++q) Src[q] = Rp0[q] - R[q];
  memcpy(U, Wp0, sizeof(double) * nc * NV);
  for (int k = 0; k < s->P.n_implicit; ++k) {
    lo_residual(s, U, R);
    for (long q = 0; q < nc * NV; ++q) R[q] += Src[q];
    lo_lambda(s, U, lam);
    lo_diag(s, lam, D);
    point_relaxation(s, U, R, lam, D, s->P.n_sweeps, dU);
    for (long q = 0; q < nc * NV; ++q) U[q] += dU[q];
  }
  free(Src); free(R); free(lam); free(D); free(dU);
}
static void pmg_cycle(o3_solver *s) {
  const o3_mesh *m = s->m;
  long nc = m->nc;
  double dt = o3_explicit_dt(s);
  double *Wn = (double *)malloc(sizeof(double) * nc * NV), *Wxn = (double *)malloc(sizeof(double) * nc * ND * NV);
  double *Rlag = (double *)malloc(sizeof(double) * nc * NV), *U = (double *)malloc(sizeof(double) * nc * NV);
  hi_step(s, s->W, s->Wx, dt, Wn, Wxn, Rlag);
  hi_eval(s, Wn, Wxn, dt);
  net_flux(s, s->F0, s->F1, 1.0, 0.5 * dt, s->Rp0);
  lo_solve(s, Wn, s->Rp0, U);
  for (long q = 0; q < nc * NV; ++q) Wn[q] += U[q] - Wn[q];
  s->res = density_residual(m, s->W, Wn);
  memcpy(s->W, Wn, sizeof(double) * nc * NV);
  memcpy(s->Wx, Wxn, sizeof(double) * nc * ND * NV);
  s->dt_last = dt;
  free(Wn); free(Wxn); free(Rlag); free(U);
  check_state(s, s->W);
}
int o3_pmg_cycle(o3_solver *s, int n, double *res_hist) {
  for (int k = 0; k < n; ++k) {
    pmg_cycle(s);
    if (res_hist) res_hist[k] = s->res;
    if (s->status) return s->status;
  }
  return s->status;
}
int o3_explicit_steps(o3_solver *s, int n, double *res_hist) {
  for (int k = 0; k < n; ++k) {
    o3_highorder_step(s, -1.0);
    if (res_hist) res_hist[k] = s->res;
    if (s->status) return s->status;
  }
  return s->status;
}
void o3_loworder_smooth(o3_solver *s) {
  long nc = s->m->nc;
  double *U = (double *)malloc(sizeof(double) * nc * NV), *Wp0 = (double *)malloc(sizeof(double) * nc * NV);
  memcpy(Wp0, s->W, sizeof(double) * nc * NV);
  lo_solve(s, Wp0, s->Rp0, U);
  s->res = density_residual(s->m, s->W, U);
  memcpy(s->W, U, sizeof(double) * nc * NV);
  free(U); free(Wp0);
}
void o3_lo_residual(const o3_solver *s, const double *U, double *R) { lo_residual(s, U, R); }
void o3_lo_lambda(const o3_solver *s, const double *U, double *lam) { lo_lambda(s, U, lam); }
void o3_lo_diag(const o3_solver *s, const double *U, double *D) {
  double *lam = (double *)malloc(sizeof(double) * s->m->nf);
  lo_lambda(s, U, lam); lo_diag(s, lam, D); free(lam);
}
void o3_lo_relax(const o3_solver *s, const double *U, const double *R, int n_sweeps, double *dU) {
  const o3_mesh *m = s->m;
  double *lam = (double *)malloc(sizeof(double) * m->nf), *D = (double *)malloc(sizeof(double) * m->nc);
  lo_lambda(s, U, lam); lo_diag(s, lam, D);
  if (n_sweeps >= 0) point_relaxation(s, U, R, lam, D, n_sweeps, dU);
  else {
    memset(dU, 0, sizeof(double) * m->nc * NV);
    for (int col = 0; col < m->ncolour; ++col)
      for (long i = 0; i < m->nc; ++i) if (m->colour[i] == col) relax_cell(s, i, U, R, lam, D, dU);
  }
  free(lam); free(D);
}
void o3_set_rp0(o3_solver *s, const double *R) { memcpy(s->Rp0, R, sizeof(double) * s->m->nc * NV); }
void o3_get_rp0(const o3_solver *s, double *R) { memcpy(R, s->Rp0, sizeof(double) * s->m->nc * NV); }
int o3_micro_slope(double gamma, const double W[NV], const double dW[NV], double s[NV]) {
  double K = o3_K(gamma);
  o3_maxw g = maxw_from_W(W, K);
  o3_mom m;
  moments(&g, K, 0, &m);
  return micro_slope(&m, g.rho, dW, s);
}
