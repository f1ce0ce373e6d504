/*
 * cgks_oracle.c -- serial FP64 CPU oracle of the p-multigrid compact
 * gas-kinetic scheme (Ji, Shyy & Xu, "A p-multigrid compact gas-kinetic
 * scheme for steady-state acceleration", arXiv:2109.09965), 2-D.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA library: it re-derives the mesh
 * geometry, the face list, the reconstruction, the kinetic moments, the
 * fluxes, the time stepping, the low-order smoother and the sweep order
 * from the paper on its own.  Everything is plain loops over
 * array-of-structs data in double precision; the kinetic moments are
 * evaluated by a generic polynomial integrator, the small dense solves by
 * Gaussian elimination / Householder QR, so each step can be checked
 * against the paper by eye.
 *
 * Paper passages followed (section / equation of arXiv:2109.09965):
 *   BGK model, compatibility, psi, K ......... Section 2, Eq. (bgk)
 *   FV semi-discretisation, Gauss points ..... Section 2.1, Eq. (semidiscrete)
 *   Maxwellian, micro-slopes a, A ............ Section 2.2
 *   smooth GKS flux .......................... Section 2.2, Eq. (2nd-smooth-flux)
 *   full GKS flux, tau_n ..................... Section 2.2, Eq. (2nd-flux)
 *   compact WENO (eps), characteristic vars .. Section 4 (transonic / supersonic
 *                                              cases, shock reflection)
 *   Dirichlet, supersonic outflow ............ Section 4 (shock reflection)
 *   interface state W_{p,k}(t) ............... Section 2.3
 *   Gauss-Green gradient update .............. Section 2.3 (gauss-formula)
 *   S1O2 ..................................... Section 2.4, Eqs. (s1o2), (flux-operator)
 *   two-level V-cycle, steps 1-5 ............. Section 3 (enumerated algorithm)
 *   backward Euler + L-F split ............... Section 3, Eqs. (implicit), (implicit-dis)
 *   local time step .......................... Section 3, Eq. (implicit-local)
 *   point relaxation ......................... Section 3, Algorithm 1
 *   density residual Res ..................... Section 4 (Res definition)
 *
 * Readings where the paper is silent:
 *   K in 2-D = (4-2*gamma)/(gamma-1); 2-point Gauss-Legendre per edge;
 *   compact least-squares quadratic (cell means + cell-mean gradients of the
 *   face neighbours, own cell-mean gradient); W^c from half-range moments
 *   of g^l, g^r; W^c_x = mean of the two side gradients; tau = mu/p^c with
 *   constant mu; S2O4 after Li & Du (2016) with gradient stages at t/2 and
 *   midpoint; global dt from CFL_hi; residual re-evaluated at W^{n+1};
 *   first-order inviscid KFVS on the low level (or, as the alternative the
 *   paper names, Lax-Friedrichs with the implicit operator's lambda_p as
 *   its dissipation coefficient); lambda with nu = mu/rho;
 *   dt_i = CFL_lo |Omega_i| / sum(lambda S); coloured sweep order (colours
 *   ascending = forward, descending = backward); ghost-state boundaries:
 *   walls mirror the reconstructed point state (and enter the wall cell's
 *   reconstruction as mirror-image ghost cells), the far field takes
 *   Riemann invariants of the cell mean and the free stream; the
 *   equilibrium normal slope adds alpha * jump / delta (Nishikawa 2010);
 *   full flux: tau_n = tau + C1 dt + C2 dt |p_l - p_r| / (p_l + p_r) in the
 *   exponentials, time dependence through the integrals over [0, dt] and
 *   [0, dt/2]; WENO: candidates P2 and the linear polynomials of the own
 *   and neighbours' mean gradients, Jiang-Shu weights gamma/(beta + eps)^2
 *   with gamma_0 = 0.95; characteristic fields of the Euler Jacobian along
 *   the face normal at the mean of the two cell averages.  The tau_n
 *   constants and the WENO weight form are readings of cited schemes:
 *   parity unpinned against those papers (the tests pin the structure,
 *   the limits and the exactness of what is implemented).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NV 4          /* conserved variables in 2-D: rho, rho u, rho v, rho E */
#define NM 5          /* quadratic monomials: xi, eta, xi^2, xi*eta, eta^2 */
#define MAXBC 16
#define MAXMOM 12

/* ------------------------------------------------------------------ */
/* parameters (layout mirrored by the Python ctypes wrapper)           */
/* ------------------------------------------------------------------ */
enum { OR_BC_SLIP = 0, OR_BC_NOSLIP = 1, OR_BC_FARFIELD = 2, OR_BC_DIRICHLET = 3, OR_BC_OUTFLOW = 4 };

typedef struct {
  int kind;
  int pad_;
  double uw[2];               /* wall velocity of a no-slip wall */
  double rho, u[2], p;        /* free stream of a far-field boundary, state of a Dirichlet one */
} or_bc;

typedef struct {
  double gamma, mu;
  double alpha;               /* jump coefficient of the equilibrium normal slope */
  double cfl_hi, cfl_lo;
  int n_implicit, n_sweeps;
  int time_scheme;            /* 0 = S1O2, 1 = S2O4 */
  int restrict_mode;          /* reserved, must be 0: R_p0 is re-evaluated at W^{n+1} */
  int n_bc;
  int flux_lo;                /* low-level flux: 0 = KFVS, 1 = Lax-Friedrichs */
  int sweep_order;            /* 0 = colour classes, 1 = element index (serial),
                                 2 = index partitions with lagged exchange,
                                 3 = RCM partitions, colour classes inside,
                                     lagged exchange per sweep */
  int n_parts;                /* partitions of sweep_order 2 and 3 */
  int flux_hi;                /* high-level flux: 0 = smooth, Eq. (2nd-smooth-flux);
                                 1 = full, Eq. (2nd-flux) */
  int pad_;
  double tau_c1, tau_c2;      /* numerical collision time of the full flux:
                                 tau_n = tau + C1 dt + C2 dt |p_l - p_r| / (p_l + p_r) */
  double weno_eps;            /* > 0: nonlinear compact WENO weights with this epsilon;
                                 <= 0: linear weights */
  double weno_g0;             /* linear weight of the quadratic candidate */
  int weno_char;              /* 1: WENO weights on characteristic variables, per face side */
  int pad2_;
  or_bc bc[MAXBC];
  int lo_viscous;             /* 1: the low-order residual carries a first-order viscous flux */
  int pad3_;
} or_params;

/* ------------------------------------------------------------------ */
/* mesh                                                                */
/* ------------------------------------------------------------------ */
typedef struct {
  long c0, c1;                /* c1 < 0 on a boundary face */
  int tag;                    /* boundary tag, -1 inside */
  double n[2];                /* unit normal pointing out of c0 */
  double S;                   /* edge length */
  double xg[2][2];            /* Gauss points */
  double wg[2];               /* Gauss weights (sum to 1) */
  double delta;               /* distance of the two cell centres along n */
} or_face;

typedef struct {
  int nv;
  long node[4];
  double vol, xc[2], h;       /* area, centroid, length scale sqrt(area) */
  int nf;
  long face[4];
  int sgn[4];                 /* +1 if this cell is c0 of the face */
  int nb;
  long nbr[4];                /* cells across interior faces */
} or_cell;

typedef struct {
  long nn, nc, nf;
  double *x;                  /* [nn][2] */
  or_cell *cell;
  or_face *face;
  long *rcm;                  /* reverse Cuthill-McKee order of the cells */
  int *colour;                /* greedy colour of each cell */
  int ncolour;
} or_mesh;

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */
static double or_K(double gamma) { return (4.0 - 2.0 * gamma) / (gamma - 1.0); }

/* Gaussian elimination with partial pivoting, n <= 8, in place. */
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

/* Least squares min ||A x - B|| by Householder QR.  A is m x n (row major,
 * destroyed), B is m x nr (destroyed), X is n x nr. */
static int householder_ls(int m, int n, double *A, int nr, double *B, double *X) {
  for (int k = 0; k < n; ++k) {
    double norm = 0.0;
    for (int i = k; i < m; ++i) norm += A[i * n + k] * A[i * n + k];
    norm = sqrt(norm);
    if (!(norm > 1e-13)) return -1;   /* rank-deficient (columns are O(1) in scaled coordinates) */
    double alpha = A[k * n + k] > 0 ? -norm : norm;
    double v[64];
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
  for (int c = 0; c < nr; ++c) {
    for (int k = n - 1; k >= 0; --k) {
      double s = B[k * nr + c];
      for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * X[j * nr + c];
      if (A[k * n + k] == 0.0) return -1;
      X[k * nr + c] = s / A[k * n + k];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Kinetic moments (Section 2.2): polynomials in (u, v, xi^2) integrated */
/* against a Maxwellian, normalised by rho.                           */
/* ------------------------------------------------------------------ */
typedef struct { double c; int a, b, k; } or_term;     /* c u^a v^b (xi^2)^k */
typedef struct { int n; or_term t[256]; } or_poly;

typedef struct {
  double mu[MAXMOM];          /* <u^a> over the chosen u range */
  double mv[MAXMOM];          /* <v^b> full range */
  double mx[4];               /* <(xi^2)^k> */
} or_mom;

static void poly_zero(or_poly *p) { p->n = 0; }
static void poly_add_term(or_poly *p, double c, int a, int b, int k) {
  if (p->n >= 256) { fprintf(stderr, "oracle: polynomial overflow\n"); abort(); }
  p->t[p->n].c = c; p->t[p->n].a = a; p->t[p->n].b = b; p->t[p->n].k = k; p->n++;
}
/* psi_r: 1, u, v, (u^2 + v^2 + xi^2)/2 */
static void poly_psi(int r, or_poly *p) {
  poly_zero(p);
  if (r == 0) poly_add_term(p, 1.0, 0, 0, 0);
  else if (r == 1) poly_add_term(p, 1.0, 1, 0, 0);
  else if (r == 2) poly_add_term(p, 1.0, 0, 1, 0);
  else { poly_add_term(p, 0.5, 2, 0, 0); poly_add_term(p, 0.5, 0, 2, 0); poly_add_term(p, 0.5, 0, 0, 1); }
}
/* micro-slope a = sum_r s_r psi_r */
static void poly_slope(const double s[NV], or_poly *p) {
  poly_zero(p);
  for (int r = 0; r < NV; ++r) {
    or_poly q; poly_psi(r, &q);
    for (int i = 0; i < q.n; ++i) poly_add_term(p, s[r] * q.t[i].c, q.t[i].a, q.t[i].b, q.t[i].k);
  }
}
static void poly_mul(const or_poly *x, const or_poly *y, or_poly *out) {
  poly_zero(out);
  for (int i = 0; i < x->n; ++i)
    for (int j = 0; j < y->n; ++j)
      poly_add_term(out, x->t[i].c * y->t[j].c, x->t[i].a + y->t[j].a,
                    x->t[i].b + y->t[j].b, x->t[i].k + y->t[j].k);
}
static void poly_monomial(double c, int a, int b, or_poly *p) { poly_zero(p); poly_add_term(p, c, a, b, 0); }
static double poly_integrate(const or_poly *p, const or_mom *m) {
  double s = 0.0;
  for (int i = 0; i < p->n; ++i) {
    const or_term *t = &p->t[i];
    if (t->a >= MAXMOM || t->b >= MAXMOM || t->k > 3) { fprintf(stderr, "oracle: moment order\n"); abort(); }
    s += t->c * m->mu[t->a] * m->mv[t->b] * m->mx[t->k];
  }
  return s;
}

typedef struct { double rho, U, V, lam; } or_maxw;

/* Maxwellian parameters from local-frame conservative variables. */
static or_maxw maxw_from_W(const double W[NV], double K) {
  or_maxw g;
  g.rho = W[0]; g.U = W[1] / W[0]; g.V = W[2] / W[0];
  g.lam = (K + 2.0) * g.rho / (4.0 * (W[3] - 0.5 * g.rho * (g.U * g.U + g.V * g.V)));
  return g;
}

/* range: 0 = full, +1 = u > 0 half, -1 = u < 0 half */
static void moments(const or_maxw *g, double K, int range, or_mom *m) {
  double l = g->lam;
  if (range == 0) {
    m->mu[0] = 1.0; m->mu[1] = g->U;
  } else {
    double e = exp(-l * g->U * g->U) / sqrt(M_PI * l);
    if (range > 0) { m->mu[0] = 0.5 * erfc(-sqrt(l) * g->U); m->mu[1] = g->U * m->mu[0] + 0.5 * e; }
    else           { m->mu[0] = 0.5 * erfc(sqrt(l) * g->U);  m->mu[1] = g->U * m->mu[0] - 0.5 * e; }
  }
  for (int a = 2; a < MAXMOM; ++a) m->mu[a] = g->U * m->mu[a - 1] + (a - 1) / (2.0 * l) * m->mu[a - 2];
  m->mv[0] = 1.0; m->mv[1] = g->V;
  for (int b = 2; b < MAXMOM; ++b) m->mv[b] = g->V * m->mv[b - 1] + (b - 1) / (2.0 * l) * m->mv[b - 2];
  m->mx[0] = 1.0;
  m->mx[1] = K / (2.0 * l);
  m->mx[2] = K * (K + 2.0) / (4.0 * l * l);
  m->mx[3] = K * (K + 2.0) * (K + 4.0) / (8.0 * l * l * l);
}

/* <psi_r * extra>, extra = c u^a v^b */
static double mom_psi_uv(int r, double c, int a, int b, const or_mom *m) {
  or_poly ps, mono, pr; poly_psi(r, &ps); poly_monomial(c, a, b, &mono); poly_mul(&ps, &mono, &pr);
  return poly_integrate(&pr, m);
}
/* <psi_r * u^a v^b * slope> */
static double mom_psi_uv_slope(int r, int a, int b, const double s[NV], const or_mom *m) {
  or_poly ps, mono, sl, t1, t2;
  poly_psi(r, &ps); poly_monomial(1.0, a, b, &mono); poly_slope(s, &sl);
  poly_mul(&ps, &mono, &t1); poly_mul(&t1, &sl, &t2);
  return poly_integrate(&t2, m);
}

/* Micro-slope from the compatibility condition <a> = dW (Section 2.2):
 * solve M s = dW / rho with M_rs = <psi_r psi_s>. */
static int micro_slope(const or_mom *m, double rho, const double dW[NV], double s[NV]) {
  double M[NV * NV], b[NV];
  for (int r = 0; r < NV; ++r) {
    b[r] = dW[r] / rho;
    for (int c = 0; c < NV; ++c) {
      or_poly pr, pc, pp; poly_psi(r, &pr); poly_psi(c, &pc); poly_mul(&pr, &pc, &pp);
      M[r * NV + c] = poly_integrate(&pp, m);
    }
  }
  int rc = gauss_solve(NV, M, b);
  for (int r = 0; r < NV; ++r) s[r] = b[r];
  return rc;
}

/* ------------------------------------------------------------------ */
/* frames                                                              */
/* ------------------------------------------------------------------ */
/* global -> local (normal n, tangent t = (-ny, nx)) for one state vector */
static void to_local(const double n[2], const double Wg[NV], double Wl[NV]) {
  Wl[0] = Wg[0];
  Wl[1] = Wg[1] * n[0] + Wg[2] * n[1];
  Wl[2] = -Wg[1] * n[1] + Wg[2] * n[0];
  Wl[3] = Wg[3];
}
static void to_global(const double n[2], const double Wl[NV], double Wg[NV]) {
  Wg[0] = Wl[0];
  Wg[1] = Wl[1] * n[0] - Wl[2] * n[1];
  Wg[2] = Wl[1] * n[1] + Wl[2] * n[0];
  Wg[3] = Wl[3];
}

/* ------------------------------------------------------------------ */
/* Gas-kinetic smooth flux at one Gauss point (Section 2.2, Eq.        */
/* (2nd-smooth-flux); interface state of Section 2.3).                  */
/*   in : W^l, W^r (global), grad[d][v] = dW_v/dx_d of each side,       */
/*        unit normal n pointing from l to r                            */
/*   out: F0, F1 with F(t) = F0 + t F1 (global frame, per unit length), */
/*        W^c and W_t = <A psi> (global frame)                          */
/* ------------------------------------------------------------------ */
void or_gks_flux_point(const or_params *P, const double Wl_g[NV], const double Wr_g[NV],
                       const double gl[2 * NV], const double gr[2 * NV], const double n[2], double delta,
                       double F0[NV], double F1[NV], double Wc_out[NV], double Wt_out[NV]) {
  double K = or_K(P->gamma);
  double t[2] = { -n[1], n[0] };
  double Wl[NV], Wr[NV];
  to_local(n, Wl_g, Wl);
  to_local(n, Wr_g, Wr);
  /* directional derivatives along n and t, then rotated to the local frame */
  double dn_l[NV], dt_l[NV], dn_r[NV], dt_r[NV], tmp_n[NV], tmp_t[NV];
  for (int v = 0; v < NV; ++v) {
    tmp_n[v] = n[0] * gl[v] + n[1] * gl[NV + v];
    tmp_t[v] = t[0] * gl[v] + t[1] * gl[NV + v];
  }
  to_local(n, tmp_n, dn_l); to_local(n, tmp_t, dt_l);
  for (int v = 0; v < NV; ++v) {
    tmp_n[v] = n[0] * gr[v] + n[1] * gr[NV + v];
    tmp_t[v] = t[0] * gr[v] + t[1] * gr[NV + v];
  }
  to_local(n, tmp_n, dn_r); to_local(n, tmp_t, dt_r);

  /* equilibrium state W^c from the particles of g^l moving right and of
   * g^r moving left (kinetic collision of the two initial states) */
  or_maxw gl_ = maxw_from_W(Wl, K), gr_ = maxw_from_W(Wr, K);
  or_mom ml, mr;
  moments(&gl_, K, +1, &ml);
  moments(&gr_, K, -1, &mr);
  double Wc[NV];
  for (int r = 0; r < NV; ++r)
    Wc[r] = gl_.rho * mom_psi_uv(r, 1.0, 0, 0, &ml) + gr_.rho * mom_psi_uv(r, 1.0, 0, 0, &mr);

  /* slopes of the equilibrium: mean of the two side gradients, plus in the
   * normal direction the jump of the two side values over the distance
   * delta between the cell centres along n (alpha-damping interface
   * gradient, Nishikawa 2010); the jump is O(h^3) for smooth data */
  double dWn[NV], dWt[NV];
  for (int v = 0; v < NV; ++v) {
    dWn[v] = 0.5 * (dn_l[v] + dn_r[v]);
    if (delta > 0.0) dWn[v] += P->alpha * (Wr[v] - Wl[v]) / delta;
    dWt[v] = 0.5 * (dt_l[v] + dt_r[v]);
  }

  or_maxw gc = maxw_from_W(Wc, K);
  or_mom mc;
  moments(&gc, K, 0, &mc);
  double an[NV], at[NV], A[NV];
  micro_slope(&mc, gc.rho, dWn, an);
  micro_slope(&mc, gc.rho, dWt, at);
  /* temporal slope from <A + a_n u + a_t v> = 0 */
  double bA[NV];
  for (int r = 0; r < NV; ++r)
    bA[r] = -(mom_psi_uv_slope(r, 1, 0, an, &mc) + mom_psi_uv_slope(r, 0, 1, at, &mc)) * gc.rho;
  micro_slope(&mc, gc.rho, bA, A);

  double pc = gc.rho / (2.0 * gc.lam);
  double tau = P->mu / pc;

  double F0l[NV], F1l[NV], Wtl[NV];
  for (int r = 0; r < NV; ++r) {
    double flux_eq = mom_psi_uv(r, 1.0, 1, 0, &mc);
    double visc = mom_psi_uv_slope(r, 2, 0, an, &mc) + mom_psi_uv_slope(r, 1, 1, at, &mc)
                + mom_psi_uv_slope(r, 1, 0, A, &mc);
    F0l[r] = gc.rho * (flux_eq - tau * visc);
    F1l[r] = gc.rho * mom_psi_uv_slope(r, 1, 0, A, &mc);
    Wtl[r] = gc.rho * mom_psi_uv_slope(r, 0, 0, A, &mc);
  }
  to_global(n, F0l, F0);
  to_global(n, F1l, F1);
  to_global(n, Wc, Wc_out);
  to_global(n, Wtl, Wt_out);
}

/* ------------------------------------------------------------------ */
/* Full gas-kinetic flux at one Gauss point, Eq. (2nd-flux), for flows  */
/* with discontinuities (Section 4: transonic and supersonic cases):    */
/*   f = (1 - e) g^c + [(t + tau) e - tau] a^c.u g^c                    */
/*       + (t - tau + tau e) A^c g^c                                    */
/*       + e g^l [1 - (tau + t) a^l.u - tau A^l] H(u)                   */
/*       + e g^r [1 - (tau + t) a^r.u - tau A^r] (1 - H(u)),            */
/* e = exp(-t / tau_n), tau = mu / p^c (Section 2.3).  tau_n (the paper */
/* adopts the one of its compact-GKS reference without printing it) is  */
/* read as tau + C1 dt + C2 dt |p_l - p_r| / (p_l + p_r).  The time     */
/* dependence is brought to the form F0 + t F1 used by the time         */
/* schemes through the integrals over [0, dt] and [0, dt/2]            */
/* (two-stage GKS): F0 dt + F1 dt^2/2 = Fhat(dt),                       */
/* F0 dt/2 + F1 dt^2/8 = Fhat(dt/2); likewise the interface state       */
/* W_p(t) = <psi f(t)> is represented by the line through its values at */
/* dt/2 and dt.  Same arguments as or_gks_flux_point plus dt.           */
/* ------------------------------------------------------------------ */
typedef struct { double c1, c2, c3, e, te; } or_tcoef;

/* the five coefficient functions of Eq. (2nd-flux) at time t */
static or_tcoef tcoef_at(double t, double tau, double taun) {
  or_tcoef c;
  double e = taun > 0.0 ? exp(-t / taun) : 0.0;
  c.c1 = 1.0 - e;
  c.c2 = (t + tau) * e - tau;
  c.c3 = t - tau + tau * e;
  c.e = e;
  c.te = t * e;
  return c;
}
/* their integrals over [0, T] */
static or_tcoef tcoef_int(double T, double tau, double taun) {
  or_tcoef c;
  double E = taun > 0.0 ? exp(-T / taun) : 0.0;
  double om = taun > 0.0 ? -expm1(-T / taun) : 1.0;      /* 1 - E */
  c.e = taun * om;                                       /* int e */
  c.te = taun * taun * om - taun * T * E;                /* int t e */
  c.c1 = T - c.e;
  c.c2 = c.te + tau * c.e - tau * T;
  c.c3 = 0.5 * T * T - tau * T + tau * c.e;
  return c;
}

/* Moments of one Maxwellian piece (full or half range table m) with its
 * slopes an, at, A: Q* the normal fluxes, P* the states, each times rho:
 *   Q0 = <u psi>, Q1 = <u (an u + at v) psi>, Q2 = <u A psi>,
 *   P0 = <psi>,   P1 = <(an u + at v) psi>,   P2 = <A psi>. */
static void piece_moments(double rho, const or_mom *m, const double an[NV], const double at[NV],
                          const double A[NV], double Q[3][NV], double Pm[3][NV]) {
  for (int r = 0; r < NV; ++r) {
    Q[0][r] = rho * mom_psi_uv(r, 1.0, 1, 0, m);
    Q[1][r] = rho * (mom_psi_uv_slope(r, 2, 0, an, m) + mom_psi_uv_slope(r, 1, 1, at, m));
    Q[2][r] = rho * mom_psi_uv_slope(r, 1, 0, A, m);
    Pm[0][r] = rho * mom_psi_uv(r, 1.0, 0, 0, m);
    Pm[1][r] = rho * (mom_psi_uv_slope(r, 1, 0, an, m) + mom_psi_uv_slope(r, 0, 1, at, m));
    Pm[2][r] = rho * mom_psi_uv_slope(r, 0, 0, A, m);
  }
}

/* spatial slopes of a Maxwellian from its normal / tangential derivatives,
 * and the temporal slope from <A + a_n u + a_t v> = 0 */
static void maxw_slopes(const or_mom *m, double rho, const double dn[NV], const double dt[NV], double an[NV],
                        double at[NV], double A[NV]) {
  micro_slope(m, rho, dn, an);
  micro_slope(m, rho, dt, at);
  double bA[NV];
  for (int r = 0; r < NV; ++r)
    bA[r] = -(mom_psi_uv_slope(r, 1, 0, an, m) + mom_psi_uv_slope(r, 0, 1, at, m)) * rho;
  micro_slope(m, rho, bA, A);
}

/* the combination of Eq. (2nd-flux) with coefficients c of the pieces
 * X[piece][moment][r] (piece 0 = equilibrium, 1 = left, 2 = right) */
static void full_combine(const or_tcoef *c, double tau, double X[3][3][NV], double out[NV]) {
  for (int r = 0; r < NV; ++r)
    out[r] = c->c1 * X[0][0][r] + c->c2 * X[0][1][r] + c->c3 * X[0][2][r]
           + c->e * (X[1][0][r] - tau * X[1][1][r] - tau * X[1][2][r]
                     + X[2][0][r] - tau * X[2][1][r] - tau * X[2][2][r])
           - c->te * (X[1][1][r] + X[2][1][r]);
}

void or_gks_full_flux_point(const or_params *P, const double Wl_g[NV], const double Wr_g[NV],
                            const double gl[2 * NV], const double gr[2 * NV], const double n[2], double delta,
                            double dt, double F0[NV], double F1[NV], double Wc_out[NV], double Wt_out[NV]) {
  double K = or_K(P->gamma);
  double t[2] = { -n[1], n[0] };
  double Wl[NV], Wr[NV];
  to_local(n, Wl_g, Wl);
  to_local(n, Wr_g, Wr);
  double dn_l[NV], dt_l[NV], dn_r[NV], dt_r[NV], tmp_n[NV], tmp_t[NV];
  for (int v = 0; v < NV; ++v) {
    tmp_n[v] = n[0] * gl[v] + n[1] * gl[NV + v];
    tmp_t[v] = t[0] * gl[v] + t[1] * gl[NV + v];
  }
  to_local(n, tmp_n, dn_l); to_local(n, tmp_t, dt_l);
  for (int v = 0; v < NV; ++v) {
    tmp_n[v] = n[0] * gr[v] + n[1] * gr[NV + v];
    tmp_t[v] = t[0] * gr[v] + t[1] * gr[NV + v];
  }
  to_local(n, tmp_n, dn_r); to_local(n, tmp_t, dt_r);

  /* the two initial Maxwellians: half-range tables for the free-transport
   * terms, full-range tables for their slopes */
  or_maxw gl_ = maxw_from_W(Wl, K), gr_ = maxw_from_W(Wr, K);
  or_mom mlh, mrh, mlf, mrf;
  moments(&gl_, K, +1, &mlh);
  moments(&gr_, K, -1, &mrh);
  moments(&gl_, K, 0, &mlf);
  moments(&gr_, K, 0, &mrf);
  double an_l[NV], at_l[NV], A_l[NV], an_r[NV], at_r[NV], A_r[NV];
  maxw_slopes(&mlf, gl_.rho, dn_l, dt_l, an_l, at_l, A_l);
  maxw_slopes(&mrf, gr_.rho, dn_r, dt_r, an_r, at_r, A_r);

  /* equilibrium W^c and its slopes, as for the smooth flux */
  double Wc[NV];
  for (int r = 0; r < NV; ++r)
    Wc[r] = gl_.rho * mom_psi_uv(r, 1.0, 0, 0, &mlh) + gr_.rho * mom_psi_uv(r, 1.0, 0, 0, &mrh);
  double dWn[NV], dWt[NV];
  for (int v = 0; v < NV; ++v) {
    dWn[v] = 0.5 * (dn_l[v] + dn_r[v]);
    if (delta > 0.0) dWn[v] += P->alpha * (Wr[v] - Wl[v]) / delta;
    dWt[v] = 0.5 * (dt_l[v] + dt_r[v]);
  }
  or_maxw gc = maxw_from_W(Wc, K);
  or_mom mc;
  moments(&gc, K, 0, &mc);
  double an[NV], at[NV], A[NV];
  maxw_slopes(&mc, gc.rho, dWn, dWt, an, at, A);

  /* collision times */
  double pc = gc.rho / (2.0 * gc.lam);
  double pl = gl_.rho / (2.0 * gl_.lam), pr = gr_.rho / (2.0 * gr_.lam);
  double tau = P->mu / pc;
  double taun = tau + P->tau_c1 * dt + P->tau_c2 * dt * fabs(pl - pr) / (pl + pr);

  double Q[3][3][NV], Pm[3][3][NV];
  piece_moments(gc.rho, &mc, an, at, A, Q[0], Pm[0]);
  piece_moments(gl_.rho, &mlh, an_l, at_l, A_l, Q[1], Pm[1]);
  piece_moments(gr_.rho, &mrh, an_r, at_r, A_r, Q[2], Pm[2]);

  or_tcoef I1 = tcoef_int(dt, tau, taun), Ih = tcoef_int(0.5 * dt, tau, taun);
  or_tcoef C1 = tcoef_at(dt, tau, taun), Ch = tcoef_at(0.5 * dt, tau, taun);
  double Fd[NV], Fh[NV], Wd[NV], Wh[NV];
  full_combine(&I1, tau, Q, Fd);
  full_combine(&Ih, tau, Q, Fh);
  full_combine(&C1, tau, Pm, Wd);
  full_combine(&Ch, tau, Pm, Wh);
  double F0l[NV], F1l[NV], Wcl[NV], Wtl[NV];
  for (int r = 0; r < NV; ++r) {
    F0l[r] = (4.0 * Fh[r] - Fd[r]) / dt;
    F1l[r] = 4.0 * (Fd[r] - 2.0 * Fh[r]) / (dt * dt);
    Wcl[r] = 2.0 * Wh[r] - Wd[r];
    Wtl[r] = 2.0 * (Wd[r] - Wh[r]) / dt;
  }
  to_global(n, F0l, F0);
  to_global(n, F1l, F1);
  to_global(n, Wcl, Wc_out);
  to_global(n, Wtl, Wt_out);
}

/* First-order kinetic flux vector splitting (Section 3, step 3): the
 * half-range fluxes of the two cell-average Maxwellians. */
void or_kfvs(const or_params *P, const double Wl_g[NV], const double Wr_g[NV], const double n[2],
             double F[NV]) {
  double K = or_K(P->gamma);
  double Wl[NV], Wr[NV], Fl[NV];
  to_local(n, Wl_g, Wl);
  to_local(n, Wr_g, Wr);
  or_maxw gl_ = maxw_from_W(Wl, K), gr_ = maxw_from_W(Wr, K);
  or_mom ml, mr;
  moments(&gl_, K, +1, &ml);
  moments(&gr_, K, -1, &mr);
  for (int r = 0; r < NV; ++r)
    Fl[r] = gl_.rho * mom_psi_uv(r, 1.0, 1, 0, &ml) + gr_.rho * mom_psi_uv(r, 1.0, 1, 0, &mr);
  to_global(n, Fl, F);
}

/* Euler normal flux F(U).n */
void or_euler_flux(double gamma, const double W[NV], const double n[2], double F[NV]) {
  double rho = W[0], u = W[1] / rho, v = W[2] / rho;
  double p = (gamma - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v));
  double un = u * n[0] + v * n[1];
  F[0] = rho * un;
  F[1] = W[1] * un + p * n[0];
  F[2] = W[2] * un + p * n[1];
  F[3] = (W[3] + p) * un;
}

/* ------------------------------------------------------------------ */
/* Boundary ghost states (readings of the boundary conditions named in  */
/* Section 4: reflective wall, non-slip adiabatic wall, Riemann far     */
/* field).                                                             */
/* ------------------------------------------------------------------ */
static void prim(double gamma, const double W[NV], double *rho, double u[2], double *p) {
  *rho = W[0]; u[0] = W[1] / W[0]; u[1] = W[2] / W[0];
  *p = (gamma - 1.0) * (W[3] - 0.5 * W[0] * (u[0] * u[0] + u[1] * u[1]));
}
static void cons(double gamma, double rho, const double u[2], double p, double W[NV]) {
  W[0] = rho; W[1] = rho * u[0]; W[2] = rho * u[1];
  W[3] = p / (gamma - 1.0) + 0.5 * rho * (u[0] * u[0] + u[1] * u[1]);
}

/* 1-D Riemann invariants normal to the face, from the interior state and
 * the free stream */
static void farfield_state(const or_params *P, const or_bc *bc, const double W[NV], const double n[2],
                           double Wg[NV]) {
  double g = P->gamma;
  double ri, ui[2], pi;
  prim(g, W, &ri, ui, &pi);
  double ci = sqrt(g * pi / ri);
  double uni = ui[0] * n[0] + ui[1] * n[1];
  double re = bc->rho, pe = bc->p;
  double ue[2] = { bc->u[0], bc->u[1] };
  double ce = sqrt(g * pe / re);
  double une = ue[0] * n[0] + ue[1] * n[1];
  if (uni <= -ci) { cons(g, re, ue, pe, Wg); return; }        /* supersonic inflow */
  if (uni >= ci) { for (int v = 0; v < NV; ++v) Wg[v] = W[v]; return; } /* supersonic outflow */
  double Rp = uni + 2.0 * ci / (g - 1.0);
  double Rm = une - 2.0 * ce / (g - 1.0);
  double unb = 0.5 * (Rp + Rm);
  double cb = 0.25 * (g - 1.0) * (Rp - Rm);
  double s, ut[2];
  if (unb >= 0.0) {
    s = pi / pow(ri, g);
    ut[0] = ui[0] - uni * n[0]; ut[1] = ui[1] - uni * n[1];
  } else {
    s = pe / pow(re, g);
    ut[0] = ue[0] - une * n[0]; ut[1] = ue[1] - une * n[1];
  }
  double rb = pow(cb * cb / (g * s), 1.0 / (g - 1.0));
  double pb = rb * cb * cb / g;
  double ub[2] = { ut[0] + unb * n[0], ut[1] + unb * n[1] };
  cons(g, rb, ub, pb, Wg);
}

/* Ghost value and gradient across a boundary face with outward normal n.
 * grad[d][v] layout: grad[d * NV + v].  Mirror M = I - 2 n n^T. */
void or_ghost(const or_params *P, int tag, const double W[NV], const double grad[2 * NV],
              const double n[2], double Wg[NV], double gradg[2 * NV]) {
  const or_bc *bc = &P->bc[tag];
  double g = P->gamma;
  double M[2][2] = { { 1.0 - 2.0 * n[0] * n[0], -2.0 * n[0] * n[1] },
                     { -2.0 * n[1] * n[0], 1.0 - 2.0 * n[1] * n[1] } };
  if (bc->kind == OR_BC_SLIP) {
    /* rho, E even; momentum reflected: m_g(x) = M m(Mx) */
    Wg[0] = W[0]; Wg[3] = W[3];
    Wg[1] = M[0][0] * W[1] + M[0][1] * W[2];
    Wg[2] = M[1][0] * W[1] + M[1][1] * W[2];
    for (int v = 0; v < NV; ++v)
      for (int d = 0; d < 2; ++d) gradg[d * NV + v] = 0.0;
    /* scalars: grad_g = M grad */
    for (int d = 0; d < 2; ++d) {
      gradg[d * NV + 0] = M[d][0] * grad[0 * NV + 0] + M[d][1] * grad[1 * NV + 0];
      gradg[d * NV + 3] = M[d][0] * grad[0 * NV + 3] + M[d][1] * grad[1 * NV + 3];
    }
    /* momentum Jacobian J[a][b] = d m_a / d x_b ; J_g = M J M */
    double J[2][2], Jg[2][2];
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b) J[a][b] = grad[b * NV + 1 + a];
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b) {
      double s = 0.0;
      for (int c = 0; c < 2; ++c) for (int e = 0; e < 2; ++e) s += M[a][c] * J[c][e] * M[e][b];
      Jg[a][b] = s;
    }
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b) gradg[b * NV + 1 + a] = Jg[a][b];
  } else if (bc->kind == OR_BC_NOSLIP) {
    /* rho(Mx), p(Mx) even; u_g(x) = 2 u_w - u(Mx) */
    double rho, u[2], p;
    prim(g, W, &rho, u, &p);
    double drho[2], du[2][2], dp[2];       /* du[a][b] = d u_a / d x_b */
    for (int b = 0; b < 2; ++b) {
      drho[b] = grad[b * NV + 0];
      for (int a = 0; a < 2; ++a) du[a][b] = (grad[b * NV + 1 + a] - u[a] * drho[b]) / rho;
      double ke_b = u[0] * du[0][b] + u[1] * du[1][b];
      dp[b] = (g - 1.0) * (grad[b * NV + 3] - 0.5 * (u[0] * u[0] + u[1] * u[1]) * drho[b] - rho * ke_b);
    }
    double ug[2] = { 2.0 * bc->uw[0] - u[0], 2.0 * bc->uw[1] - u[1] };
    double drg[2], dpg[2], dug[2][2];
    for (int d = 0; d < 2; ++d) {
      drg[d] = M[d][0] * drho[0] + M[d][1] * drho[1];
      dpg[d] = M[d][0] * dp[0] + M[d][1] * dp[1];
    }
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b)
      dug[a][b] = -(du[a][0] * M[0][b] + du[a][1] * M[1][b]);
    cons(g, rho, ug, p, Wg);
    for (int b = 0; b < 2; ++b) {
      gradg[b * NV + 0] = drg[b];
      for (int a = 0; a < 2; ++a) gradg[b * NV + 1 + a] = ug[a] * drg[b] + rho * dug[a][b];
      double ke_b = ug[0] * dug[0][b] + ug[1] * dug[1][b];
      gradg[b * NV + 3] = dpg[b] / (g - 1.0) + 0.5 * (ug[0] * ug[0] + ug[1] * ug[1]) * drg[b] + rho * ke_b;
    }
  } else if (bc->kind == OR_BC_DIRICHLET) {
    /* prescribed state, uniform outside (Section 4, shock reflection) */
    cons(g, bc->rho, bc->u, bc->p, Wg);
    for (int k = 0; k < 2 * NV; ++k) gradg[k] = 0.0;
  } else if (bc->kind == OR_BC_OUTFLOW) {
    /* supersonic outflow: every characteristic leaves the domain, the
     * outside continues the inside (state and gradient copied) */
    for (int v = 0; v < NV; ++v) Wg[v] = W[v];
    for (int k = 0; k < 2 * NV; ++k) gradg[k] = grad[k];
  } else {
    farfield_state(P, bc, W, n, Wg);
    for (int k = 0; k < 2 * NV; ++k) gradg[k] = 0.0;
  }
}

/* ------------------------------------------------------------------ */
/* Mesh: faces, geometry, Gauss points (Section 2.1)                   */
/* ------------------------------------------------------------------ */
typedef struct { long a, b, cell; int k; } or_edge;

static int edge_cmp(const void *x, const void *y) {
  const or_edge *p = (const or_edge *)x, *q = (const or_edge *)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
  return 0;
}

/* triangle fan of cell c: triangles (v0, v_k, v_{k+1}) */
static void cell_geometry(const or_mesh *m, or_cell *c) {
  double A = 0.0, cx = 0.0, cy = 0.0;
  const double *x0 = &m->x[2 * c->node[0]];
  for (int k = 1; k + 1 < c->nv; ++k) {
    const double *x1 = &m->x[2 * c->node[k]], *x2 = &m->x[2 * c->node[k + 1]];
    double a = 0.5 * ((x1[0] - x0[0]) * (x2[1] - x0[1]) - (x2[0] - x0[0]) * (x1[1] - x0[1]));
    A += a;
    cx += a * (x0[0] + x1[0] + x2[0]) / 3.0;
    cy += a * (x0[1] + x1[1] + x2[1]) / 3.0;
  }
  c->vol = A; c->xc[0] = cx / A; c->xc[1] = cy / A;
  c->h = sqrt(A);
}

/* Means over cell j of the monomials phi_m((x - xc_i)/h_i), exact for
 * degree 2: triangle fan, edge-midpoint rule on each triangle. */
static void cell_mean_monomials(const or_mesh *m, long j, const double xc[2], double h, double out[NM]) {
  const or_cell *c = &m->cell[j];
  for (int q = 0; q < NM; ++q) out[q] = 0.0;
  double A = 0.0;
  const double *x0 = &m->x[2 * c->node[0]];
  for (int k = 1; k + 1 < c->nv; ++k) {
    const double *x1 = &m->x[2 * c->node[k]], *x2 = &m->x[2 * c->node[k + 1]];
    double a = 0.5 * ((x1[0] - x0[0]) * (x2[1] - x0[1]) - (x2[0] - x0[0]) * (x1[1] - x0[1]));
    const double *P[3] = { x0, x1, x2 };
    for (int e = 0; e < 3; ++e) {
      double mx = 0.5 * (P[e][0] + P[(e + 1) % 3][0]), my = 0.5 * (P[e][1] + P[(e + 1) % 3][1]);
      double xi = (mx - xc[0]) / h, eta = (my - xc[1]) / h;
      out[0] += a / 3.0 * xi;
      out[1] += a / 3.0 * eta;
      out[2] += a / 3.0 * xi * xi;
      out[3] += a / 3.0 * xi * eta;
      out[4] += a / 3.0 * eta * eta;
    }
    A += a;
  }
  for (int q = 0; q < NM; ++q) out[q] /= A;
}

static void mesh_free(or_mesh *m) {
  if (!m) return;
  free(m->x); free(m->cell); free(m->face); free(m->rcm); free(m->colour); free(m);
}
void or_mesh_destroy(or_mesh *m) { mesh_free(m); }

static void mesh_ordering(or_mesh *m);

/* Build the mesh.  err: 0 ok, 1 bad input, 2 non-manifold edge, 3 boundary
 * edge without tag, 4 non-positive area. */
or_mesh *or_mesh_create(long nn, const double *xy, long nc, const uint8_t *ctype,
                        const int64_t *cptr, const int64_t *cnodes, long nbf,
                        const int64_t *bptr, const int64_t *bnodes, const int32_t *btag, int *err) {
  *err = 0;
  or_mesh *m = (or_mesh *)calloc(1, sizeof(or_mesh));
  m->nn = nn; m->nc = nc;
  m->x = (double *)malloc(sizeof(double) * 2 * nn);
  memcpy(m->x, xy, sizeof(double) * 2 * nn);
  m->cell = (or_cell *)calloc(nc, sizeof(or_cell));
  long ne = 0;
  for (long c = 0; c < nc; ++c) {
    int nv = (int)(cptr[c + 1] - cptr[c]);
    if ((ctype[c] == 0 && nv != 3) || (ctype[c] == 1 && nv != 4) || ctype[c] > 1) { *err = 1; mesh_free(m); return NULL; }
    m->cell[c].nv = nv;
    for (int k = 0; k < nv; ++k) m->cell[c].node[k] = cnodes[cptr[c] + k];
    cell_geometry(m, &m->cell[c]);
    if (!(m->cell[c].vol > 0.0)) { *err = 4; mesh_free(m); return NULL; }
    ne += nv;
  }
  or_edge *E = (or_edge *)malloc(sizeof(or_edge) * ne);
  long q = 0;
  for (long c = 0; c < nc; ++c)
    for (int k = 0; k < m->cell[c].nv; ++k) {
      long a = m->cell[c].node[k], b = m->cell[c].node[(k + 1) % m->cell[c].nv];
      E[q].a = a < b ? a : b; E[q].b = a < b ? b : a; E[q].cell = c; E[q].k = k; ++q;
    }
  qsort(E, ne, sizeof(or_edge), edge_cmp);
  or_edge *B = (or_edge *)malloc(sizeof(or_edge) * (nbf > 0 ? nbf : 1));
  for (long f = 0; f < nbf; ++f) {
    if (bptr[f + 1] - bptr[f] != 2) { *err = 1; free(E); free(B); mesh_free(m); return NULL; }
    long a = bnodes[bptr[f]], b = bnodes[bptr[f] + 1];
    B[f].a = a < b ? a : b; B[f].b = a < b ? b : a; B[f].cell = btag[f]; B[f].k = 0;
  }
  qsort(B, nbf, sizeof(or_edge), edge_cmp);
  m->face = (or_face *)calloc(ne, sizeof(or_face));
  long nf = 0;
  for (long i = 0; i < ne;) {
    long j = i + 1;
    while (j < ne && E[j].a == E[i].a && E[j].b == E[i].b) ++j;
    if (j - i > 2) { *err = 2; break; }
    or_face *F = &m->face[nf];
    long c0 = E[i].cell;
    int k = E[i].k;
    const or_cell *C = &m->cell[c0];
    const double *xa = &m->x[2 * C->node[k]], *xb = &m->x[2 * C->node[(k + 1) % C->nv]];
    double dx = xb[0] - xa[0], dy = xb[1] - xa[1];
    F->S = sqrt(dx * dx + dy * dy);
    F->n[0] = dy / F->S; F->n[1] = -dx / F->S;          /* outward for a counter-clockwise cell */
    double s3 = 1.0 / (2.0 * sqrt(3.0));
    F->xg[0][0] = xa[0] + (0.5 - s3) * dx; F->xg[0][1] = xa[1] + (0.5 - s3) * dy;
    F->xg[1][0] = xa[0] + (0.5 + s3) * dx; F->xg[1][1] = xa[1] + (0.5 + s3) * dy;
    F->wg[0] = F->wg[1] = 0.5;
    F->c0 = c0;
    if (j - i == 2) {
      F->c1 = E[i + 1].cell; F->tag = -1;
    } else {
      F->c1 = -1;
      or_edge key = { E[i].a, E[i].b, -1, 0 };
      long lo = 0, hi = nbf - 1, found = -1;
      while (lo <= hi) {                      /* first boundary record with this node pair */
        long mid = (lo + hi) / 2;
        if (B[mid].a < key.a || (B[mid].a == key.a && B[mid].b < key.b)) lo = mid + 1;
        else { if (B[mid].a == key.a && B[mid].b == key.b) found = mid; hi = mid - 1; }
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
    or_face *F = &m->face[f];
    const double *x0 = m->cell[F->c0].xc;
    if (F->c1 >= 0) {
      const double *x1 = m->cell[F->c1].xc;
      F->delta = fabs((x1[0] - x0[0]) * F->n[0] + (x1[1] - x0[1]) * F->n[1]);
    } else {  /* mirror image of the cell centre across the boundary edge */
      F->delta = 2.0 * fabs((F->xg[0][0] - x0[0]) * F->n[0] + (F->xg[0][1] - x0[1]) * F->n[1]);
    }
    or_cell *C0 = &m->cell[F->c0];
    C0->face[C0->nf] = f; C0->sgn[C0->nf] = +1; C0->nf++;
    if (F->c1 >= 0) {
      or_cell *C1 = &m->cell[F->c1];
      C1->face[C1->nf] = f; C1->sgn[C1->nf] = -1; C1->nf++;
      C0->nbr[C0->nb++] = F->c1;
      C1->nbr[C1->nb++] = F->c0;
    }
  }
  mesh_ordering(m);
  return m;
}

long or_mesh_nfaces(const or_mesh *m) { return m->nf; }
int or_mesh_ncolours(const or_mesh *m) { return m->ncolour; }

void or_mesh_geometry(const or_mesh *m, double *vol, double *xc) {
  for (long c = 0; c < m->nc; ++c) {
    vol[c] = m->cell[c].vol; xc[2 * c] = m->cell[c].xc[0]; xc[2 * c + 1] = m->cell[c].xc[1];
  }
}
void or_mesh_faces(const or_mesh *m, int64_t *c0, int64_t *c1, int32_t *tag, double *n, double *S, double *xg) {
  for (long f = 0; f < m->nf; ++f) {
    const or_face *F = &m->face[f];
    c0[f] = F->c0; c1[f] = F->c1; tag[f] = F->tag;
    n[2 * f] = F->n[0]; n[2 * f + 1] = F->n[1]; S[f] = F->S;
    for (int k = 0; k < 2; ++k) { xg[4 * f + 2 * k] = F->xg[k][0]; xg[4 * f + 2 * k + 1] = F->xg[k][1]; }
  }
}

/* ------------------------------------------------------------------ */
/* Sweep order: reverse Cuthill-McKee from the lowest-index cell of     */
/* minimum degree, neighbours visited by (degree, index), then greedy   */
/* smallest-free colouring in RCM order (replaces the index order of    */
/* Algorithm 1 so cells of one colour can relax together).              */
/* ------------------------------------------------------------------ */
static const or_mesh *g_sort_mesh;
static int nbr_cmp(const void *x, const void *y) {
  long a = *(const long *)x, b = *(const long *)y;
  int da = g_sort_mesh->cell[a].nb, db = g_sort_mesh->cell[b].nb;
  if (da != db) return da < db ? -1 : 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}

static void mesh_ordering(or_mesh *m) {
  long nc = m->nc;
  long *cm = (long *)malloc(sizeof(long) * nc);
  char *seen = (char *)calloc(nc, 1);
  long head = 0, tail = 0;
  g_sort_mesh = m;
  while (tail < nc) {
    long start = -1;
    for (long c = 0; c < nc; ++c)
      if (!seen[c] && (start < 0 || m->cell[c].nb < m->cell[start].nb)) start = c;
    seen[start] = 1; cm[tail++] = start;
    while (head < tail) {
      long v = cm[head++];
      long nb[4]; int k = 0;
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
    int used[8] = { 0 };
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

void or_mesh_ordering(const or_mesh *m, int64_t *rcm, int32_t *colour) {
  for (long i = 0; i < m->nc; ++i) { rcm[i] = m->rcm[i]; colour[i] = m->colour[i]; }
}

/* ------------------------------------------------------------------ */
/* Solver state                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
  const or_mesh *m;
  or_params P;
  double *W;                  /* [nc][NV]   cell averages */
  double *Wx;                 /* [nc][2][NV] cell-averaged gradients */
  double *coef;               /* [nc][NM][NV] reconstruction coefficients */
  double *mom_self;           /* [nc][NM] own monomial means */
  unsigned char *quad;        /* [nc] 1: least-squares quadratic, 0: linear fallback */
  /* per-face quadrature sums of one high-order evaluation */
  double *F0, *F1, *Wc, *Wt;  /* [nf][NV] */
  double *Rp0;                /* [nc][NV] transferred residual */
  double res;                 /* Res of the last update */
  double dt_last;
  int status;
} or_solver;

or_solver *or_solver_create(const or_mesh *m, const or_params *P) {
  or_solver *s = (or_solver *)calloc(1, sizeof(or_solver));
  s->m = m; s->P = *P;
  long nc = m->nc, nf = m->nf;
  s->W = (double *)calloc(nc * NV, sizeof(double));
  s->Wx = (double *)calloc(nc * 2 * NV, sizeof(double));
  s->coef = (double *)calloc(nc * NM * NV, sizeof(double));
  s->quad = (unsigned char *)calloc(nc, 1);
  s->mom_self = (double *)calloc(nc * NM, sizeof(double));
  s->F0 = (double *)calloc(nf * NV, sizeof(double));
  s->F1 = (double *)calloc(nf * NV, sizeof(double));
  s->Wc = (double *)calloc(nf * NV, sizeof(double));
  s->Wt = (double *)calloc(nf * NV, sizeof(double));
  s->Rp0 = (double *)calloc(nc * NV, sizeof(double));
  for (long c = 0; c < nc; ++c)
    cell_mean_monomials(m, c, m->cell[c].xc, m->cell[c].h, &s->mom_self[c * NM]);
  return s;
}

void or_solver_destroy(or_solver *s) {
  if (!s) return;
  free(s->W); free(s->Wx); free(s->coef); free(s->mom_self); free(s->quad);
  free(s->F0); free(s->F1); free(s->Wc); free(s->Wt); free(s->Rp0); free(s);
}

void or_set_state(or_solver *s, const double *W, const double *Wx) {
  memcpy(s->W, W, sizeof(double) * s->m->nc * NV);
  if (Wx) memcpy(s->Wx, Wx, sizeof(double) * s->m->nc * 2 * NV);
  else memset(s->Wx, 0, sizeof(double) * s->m->nc * 2 * NV);
}
void or_get_state(const or_solver *s, double *W, double *Wx) {
  if (W) memcpy(W, s->W, sizeof(double) * s->m->nc * NV);
  if (Wx) memcpy(Wx, s->Wx, sizeof(double) * s->m->nc * 2 * NV);
}
double or_last_residual(const or_solver *s) { return s->res; }
int or_status(const or_solver *s) { return s->status; }

/* ------------------------------------------------------------------ */
/* Compact reconstruction (linear weights; scheme cited at Section 2.2) */
/* per cell: P_i(x) = W_i + sum_m c_m (phi_m(x) - mean_i phi_m), fitted in */
/* least squares to the face neighbours' cell means and cell-mean       */
/* gradients and to the own cell-mean gradient.                        */
/* ------------------------------------------------------------------ */
/* Means over the mirror image of cell i across the line of face f of the
 * monomials phi_m((x - xc_i)/h_i); same quadrature as cell_mean_monomials. */
static void mirror_mean_monomials(const or_mesh *m, long i, const or_face *F, double out[NM]) {
  const or_cell *C = &m->cell[i];
  double xm[4][2];
  for (int a = 0; a < C->nv; ++a) {
    const double *x = &m->x[2 * C->node[a]];
    double d = (x[0] - F->xg[0][0]) * F->n[0] + (x[1] - F->xg[0][1]) * F->n[1];
    xm[a][0] = x[0] - 2.0 * d * F->n[0];
    xm[a][1] = x[1] - 2.0 * d * F->n[1];
  }
  for (int q = 0; q < NM; ++q) out[q] = 0.0;
  double A = 0.0;
  for (int k = 1; k + 1 < C->nv; ++k) {
    const double *P[3] = { xm[0], xm[k], xm[k + 1] };
    double a = 0.5 * fabs((P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]));
    for (int e = 0; e < 3; ++e) {
      double mx = 0.5 * (P[e][0] + P[(e + 1) % 3][0]), my = 0.5 * (P[e][1] + P[(e + 1) % 3][1]);
      double xi = (mx - C->xc[0]) / C->h, eta = (my - C->xc[1]) / C->h;
      out[0] += a / 3.0 * xi;
      out[1] += a / 3.0 * eta;
      out[2] += a / 3.0 * xi * xi;
      out[3] += a / 3.0 * xi * eta;
      out[4] += a / 3.0 * eta * eta;
    }
    A += a;
  }
  for (int q = 0; q < NM; ++q) out[q] /= A;
}

static int is_wall(const or_solver *s, const or_face *F) {
  if (F->c1 >= 0) return 0;
  int k = s->P.bc[F->tag].kind;
  return k == OR_BC_SLIP || k == OR_BC_NOSLIP;
}

/* Smoothness indicator of a candidate polynomial with scaled coefficients
 * c (monomials of (x - xc)/h, h^2 = |Omega|): the sum over the
 * derivative multi-indices alpha with 1 <= |alpha| <= 2 of the cell mean of
 * (h^|alpha| D^alpha P)^2.  The cell mean of the squared first derivatives
 * is taken by the edge-midpoint rule on a fan of triangles (exact for the
 * quadratic integrand). */
static double weno_beta(const or_mesh *m, long i, const double *c, int stride) {
  const or_cell *C = &m->cell[i];
  double c0 = c[0], c1 = c[stride], c2 = c[2 * stride], c3 = c[3 * stride], c4 = c[4 * stride];
  double sum = 0.0, A = 0.0;
  const double *x0 = &m->x[2 * C->node[0]];
  for (int k = 1; k + 1 < C->nv; ++k) {
    const double *x1 = &m->x[2 * C->node[k]], *x2 = &m->x[2 * C->node[k + 1]];
    double a = 0.5 * ((x1[0] - x0[0]) * (x2[1] - x0[1]) - (x2[0] - x0[0]) * (x1[1] - x0[1]));
    const double *P[3] = { x0, x1, x2 };
    for (int e = 0; e < 3; ++e) {
      double xi = (0.5 * (P[e][0] + P[(e + 1) % 3][0]) - C->xc[0]) / C->h;
      double eta = (0.5 * (P[e][1] + P[(e + 1) % 3][1]) - C->xc[1]) / C->h;
      double px = c0 + 2.0 * c2 * xi + c3 * eta, py = c1 + c3 * xi + 2.0 * c4 * eta;
      sum += a / 3.0 * (px * px + py * py);
    }
    A += a;
  }
  return sum / A + 4.0 * c2 * c2 + c3 * c3 + 4.0 * c4 * c4;
}

/* Compact WENO with nonlinear weights (Section 4 names it for the
 * transonic and supersonic cases and gives its epsilon; the scheme itself
 * is the cited one, read here as follows).  Candidates of cell i: the
 * compact quadratic P2 (coefficients X) and the linear polynomials
 * W_i + h g.(xi, eta) with g the cell-mean gradient of the cell itself and
 * of each face neighbour.  Linear weights gamma_0 = g0 for P2 and
 * (1 - g0)/m for each of the m linear ones; nonlinear weights
 * w_k ~ gamma_k / (beta_k + eps)^2, normalised; the result
 *   P = (w_0 / gamma_0) (P2 - sum_k gamma_k P1_k) + sum_k w_k P1_k
 * equals P2 when w = gamma and keeps the cell mean.  Per component.
 * weno_mix does it for the NV components of X (in place, [q][v] layout)
 * with the m scaled candidate gradients G[k][d][v]. */
static void weno_mix(const or_solver *s, long i, double *X, int m, double G[5][2][NV]) {
  double g0 = s->P.weno_g0, eps = s->P.weno_eps;
  double gk = (1.0 - g0) / m;
  for (int v = 0; v < NV; ++v) {
    double wt[6], wsum = 0.0;
    double b0 = weno_beta(s->m, i, &X[v], NV);
    wt[0] = g0 / ((b0 + eps) * (b0 + eps));
    for (int k = 0; k < m; ++k) {
      double cl[NM] = { G[k][0][v], G[k][1][v], 0.0, 0.0, 0.0 };
      double b = weno_beta(s->m, i, cl, 1);
      wt[k + 1] = gk / ((b + eps) * (b + eps));
    }
    for (int k = 0; k <= m; ++k) wsum += wt[k];
    for (int k = 0; k <= m; ++k) wt[k] /= wsum;
    for (int q = 0; q < NM; ++q) {
      double lin = 0.0, sel = 0.0;
      if (q < 2)
        for (int k = 0; k < m; ++k) { lin += gk * G[k][q][v]; sel += wt[k + 1] * G[k][q][v]; }
      X[q * NV + v] = wt[0] / g0 * (X[q * NV + v] - lin) + sel;
    }
  }
}

/* the scaled linear candidates h_i * (mean gradient) of cell i and its
 * face neighbours; returns their number */
static int weno_candidates(const or_solver *s, const double *Wx, long i, double G[5][2][NV]) {
  const or_cell *C = &s->m->cell[i];
  long cand[5];
  int m = 0;
  cand[m++] = i;
  for (int k = 0; k < C->nb; ++k) cand[m++] = C->nbr[k];
  for (int k = 0; k < m; ++k)
    for (int d = 0; d < 2; ++d)
      for (int v = 0; v < NV; ++v) G[k][d][v] = C->h * Wx[(cand[k] * 2 + d) * NV + v];
  return m;
}

static void weno_combine(const or_solver *s, const double *Wx, long i, double *X) {
  double G[5][2][NV];
  int m = weno_candidates(s, Wx, i, G);
  weno_mix(s, i, X, m, G);
}

/* Right eigenvectors (columns) of the Euler flux Jacobian along the unit
 * normal n at the conservative state W: the waves u_n - c, u_n (entropy),
 * u_n (shear) and u_n + c. */
static void euler_right_eigvecs(double gamma, const double W[NV], const double n[2], double R[NV][NV]) {
  double rho, u[2], p;
  prim(gamma, W, &rho, u, &p);
  double c = sqrt(gamma * p / rho), H = (W[3] + p) / rho;
  double un = u[0] * n[0] + u[1] * n[1], ut = -u[0] * n[1] + u[1] * n[0];
  double col[NV][NV] = { { 1.0, u[0] - c * n[0], u[1] - c * n[1], H - c * un },
                         { 1.0, u[0], u[1], 0.5 * (u[0] * u[0] + u[1] * u[1]) },
                         { 0.0, -n[1], n[0], ut },
                         { 1.0, u[0] + c * n[0], u[1] + c * n[1], H + c * un } };
  for (int r = 0; r < NV; ++r)
    for (int k = 0; k < NV; ++k) R[r][k] = col[k][r];
}

/* exposed for the eigenvector pin */
void or_euler_right_eigvecs(double gamma, const double W[NV], const double n[2], double *R) {
  double Rm[NV][NV];
  euler_right_eigvecs(gamma, W, n, Rm);
  for (int r = 0; r < NV; ++r) for (int k = 0; k < NV; ++k) R[r * NV + k] = Rm[r][k];
}

/* Compact WENO on characteristic variables (Section 4, shock reflection):
 * the candidates of cell i are projected on the left eigenvectors L = R^-1
 * of the Euler flux Jacobian along the face normal, taken at the mean of
 * the cell averages on the two sides of the face (the cell's own average
 * on a boundary face); the nonlinear weights are formed per
 * characteristic field, and the combination is projected back with R.
 * X: the linear-weight quadratic of cell i; out: the face-side polynomial. */
static void weno_char_side(const or_solver *s, const double *Wx, long i, const double Wref[NV], const double n[2],
                           const double *X, double *out) {
  double R[NV][NV], L[NV][NV];
  euler_right_eigvecs(s->P.gamma, Wref, n, R);
  for (int k = 0; k < NV; ++k) {
    double A[NV * NV], e[NV] = { 0 };
    for (int r = 0; r < NV; ++r) for (int c = 0; c < NV; ++c) A[r * NV + c] = R[r][c];
    e[k] = 1.0;
    gauss_solve(NV, A, e);                 /* column k of R^-1 */
    for (int r = 0; r < NV; ++r) L[r][k] = e[r];
  }
  double G[5][2][NV], GQ[5][2][NV], XQ[NM * NV];
  int m = weno_candidates(s, Wx, i, G);
  for (int q = 0; q < NM; ++q)
    for (int a = 0; a < NV; ++a) {
      double acc = 0.0;
      for (int v = 0; v < NV; ++v) acc += L[a][v] * X[q * NV + v];
      XQ[q * NV + a] = acc;
    }
  for (int k = 0; k < m; ++k)
    for (int d = 0; d < 2; ++d)
      for (int a = 0; a < NV; ++a) {
        double acc = 0.0;
        for (int v = 0; v < NV; ++v) acc += L[a][v] * G[k][d][v];
        GQ[k][d][a] = acc;
      }
  weno_mix(s, i, XQ, m, GQ);
  for (int q = 0; q < NM; ++q)
    for (int v = 0; v < NV; ++v) {
      double acc = 0.0;
      for (int a = 0; a < NV; ++a) acc += R[v][a] * XQ[q * NV + a];
      out[q * NV + v] = acc;
    }
}

static void reconstruct_cell(or_solver *s, const double *W, const double *Wx, long i) {
  const or_mesh *m = s->m;
  const or_cell *C = &m->cell[i];
  double *c = &s->coef[i * NM * NV];
  const double *mi = &s->mom_self[i * NM];
  int nwall = 0;
  for (int k = 0; k < C->nf; ++k) nwall += is_wall(s, &m->face[C->face[k]]);
  s->quad[i] = 0;
  if (C->nb + nwall < 2) {
    /* too few neighbours for a quadratic: linear from the own gradient */
    for (int q = 0; q < NM * NV; ++q) c[q] = 0.0;
    for (int v = 0; v < NV; ++v) {
      c[0 * NV + v] = C->h * Wx[(i * 2 + 0) * NV + v];
      c[1 * NV + v] = C->h * Wx[(i * 2 + 1) * NV + v];
    }
    return;
  }
  int neq = 3 * (C->nb + nwall) + 2;
  double A[64 * NM], B[64 * NV], X[NM * NV];
  int row = 0;
  for (int k = 0; k < C->nb; ++k) {
    long j = C->nbr[k];
    double mj[NM];
    cell_mean_monomials(m, j, C->xc, C->h, mj);
    /* mean over Omega_j of P_i equals W_j */
    for (int q = 0; q < NM; ++q) A[row * NM + q] = mj[q] - mi[q];
    for (int v = 0; v < NV; ++v) B[row * NV + v] = W[j * NV + v] - W[i * NV + v];
    ++row;
    /* h_i * mean over Omega_j of grad P_i equals h_i * gradient mean of j */
    double gx[NM] = { 1.0, 0.0, 2.0 * mj[0], mj[1], 0.0 };
    double gy[NM] = { 0.0, 1.0, 0.0, mj[0], 2.0 * mj[1] };
    for (int q = 0; q < NM; ++q) { A[row * NM + q] = gx[q]; A[(row + 1) * NM + q] = gy[q]; }
    for (int v = 0; v < NV; ++v) {
      B[row * NV + v] = C->h * Wx[(j * 2 + 0) * NV + v];
      B[(row + 1) * NV + v] = C->h * Wx[(j * 2 + 1) * NV + v];
    }
    row += 2;
  }
  /* wall faces: the mirror-image ghost cell enters like a face neighbour,
   * its mean and mean gradient given by the wall condition applied to the
   * own cell mean and mean gradient */
  for (int k = 0; k < C->nf; ++k) {
    const or_face *F = &m->face[C->face[k]];
    if (!is_wall(s, F)) continue;
    double mg[NM], Wg[NV], Gg[2 * NV];
    mirror_mean_monomials(m, i, F, mg);
    or_ghost(&s->P, F->tag, &W[i * NV], &Wx[i * 2 * NV], F->n, Wg, Gg);
    for (int q = 0; q < NM; ++q) A[row * NM + q] = mg[q] - mi[q];
    for (int v = 0; v < NV; ++v) B[row * NV + v] = Wg[v] - W[i * NV + v];
    ++row;
    double gx[NM] = { 1.0, 0.0, 2.0 * mg[0], mg[1], 0.0 };
    double gy[NM] = { 0.0, 1.0, 0.0, mg[0], 2.0 * mg[1] };
    for (int q = 0; q < NM; ++q) { A[row * NM + q] = gx[q]; A[(row + 1) * NM + q] = gy[q]; }
    for (int v = 0; v < NV; ++v) {
      B[row * NV + v] = C->h * Gg[v];
      B[(row + 1) * NV + v] = C->h * Gg[NV + v];
    }
    row += 2;
  }
  {
    double gx[NM] = { 1.0, 0.0, 2.0 * mi[0], mi[1], 0.0 };
    double gy[NM] = { 0.0, 1.0, 0.0, mi[0], 2.0 * mi[1] };
    for (int q = 0; q < NM; ++q) { A[row * NM + q] = gx[q]; A[(row + 1) * NM + q] = gy[q]; }
    for (int v = 0; v < NV; ++v) {
      B[row * NV + v] = C->h * Wx[(i * 2 + 0) * NV + v];
      B[(row + 1) * NV + v] = C->h * Wx[(i * 2 + 1) * NV + v];
    }
    row += 2;
  }
  if (householder_ls(neq, NM, A, NV, B, X) != 0) {
    /* rank-deficient stencil (e.g. a lone cell between two parallel walls):
     * the same linear reconstruction as for too few neighbours */
    for (int q = 0; q < NM * NV; ++q) c[q] = 0.0;
    for (int v = 0; v < NV; ++v) {
      c[0 * NV + v] = C->h * Wx[(i * 2 + 0) * NV + v];
      c[1 * NV + v] = C->h * Wx[(i * 2 + 1) * NV + v];
    }
    return;
  }
  if (s->P.weno_eps > 0.0 && !s->P.weno_char) weno_combine(s, Wx, i, X);
  for (int q = 0; q < NM * NV; ++q) c[q] = X[q];
  s->quad[i] = 1;
}

static void reconstruct_all(or_solver *s, const double *W, const double *Wx) {
  for (long i = 0; i < s->m->nc; ++i) reconstruct_cell(s, W, Wx, i);
}

/* value and gradient at point x of the polynomial of cell i with
 * coefficients c ([q][v]) */
static void poly_eval(const or_solver *s, const double *W, long i, const double *c, const double x[2],
                      double val[NV], double grad[2 * NV]);

/* value and gradient of P_i at point x */
static void recon_eval(const or_solver *s, const double *W, long i, const double x[2],
                       double val[NV], double grad[2 * NV]) {
  poly_eval(s, W, i, &s->coef[i * NM * NV], x, val, grad);
}

static void poly_eval(const or_solver *s, const double *W, long i, const double *c, const double x[2],
                      double val[NV], double grad[2 * NV]) {
  const or_cell *C = &s->m->cell[i];
  const double *mi = &s->mom_self[i * NM];
  double xi = (x[0] - C->xc[0]) / C->h, eta = (x[1] - C->xc[1]) / C->h;
  double phi[NM] = { xi, eta, xi * xi, xi * eta, eta * eta };
  double dphix[NM] = { 1.0, 0.0, 2.0 * xi, eta, 0.0 };
  double dphiy[NM] = { 0.0, 1.0, 0.0, xi, 2.0 * eta };
  for (int v = 0; v < NV; ++v) {
    double p = W[i * NV + v], gx = 0.0, gy = 0.0;
    for (int q = 0; q < NM; ++q) {
      p += c[q * NV + v] * (phi[q] - mi[q]);
      gx += c[q * NV + v] * dphix[q];
      gy += c[q * NV + v] * dphiy[q];
    }
    val[v] = p; grad[v] = gx / C->h; grad[NV + v] = gy / C->h;
  }
}

/* test hooks: reconstruct and evaluate */
void or_reconstruct(or_solver *s) { reconstruct_all(s, s->W, s->Wx); }
void or_recon_eval(const or_solver *s, long cell, const double x[2], double val[NV], double grad[2 * NV]) {
  recon_eval(s, s->W, cell, x, val, grad);
}

/* test hook: value and gradient at x of the polynomial the face flux uses
 * on one side of face f (side 0: c0, 1: c1) after or_reconstruct: the
 * cell's own, or with characteristic WENO the one limited for this face */
void or_face_side_eval(or_solver *s, long f, int side, const double x[2], double val[NV], double grad[2 * NV]) {
  const or_face *F = &s->m->face[f];
  long c = side == 0 ? F->c0 : F->c1;
  const double *p = &s->coef[c * NM * NV];
  double q[NM * NV];
  if (s->P.weno_eps > 0.0 && s->P.weno_char && s->quad[c]) {
    double Wref[NV];
    for (int v = 0; v < NV; ++v)
      Wref[v] = F->c1 >= 0 ? 0.5 * (s->W[F->c0 * NV + v] + s->W[F->c1 * NV + v]) : s->W[F->c0 * NV + v];
    weno_char_side(s, s->Wx, c, Wref, F->n, p, q);
    p = q;
  }
  poly_eval(s, s->W, c, p, x, val, grad);
}

/* ------------------------------------------------------------------ */
/* High-order evaluation: reconstruction + face fluxes (Sections 2.1-2.3) */
/* Stores per face the weighted Gauss sums of F0, F1, W^c and W_t.      */
/* ------------------------------------------------------------------ */
static void hi_eval(or_solver *s, const double *W, const double *Wx, double dt) {
  const or_mesh *m = s->m;
  reconstruct_all(s, W, Wx);
  for (long f = 0; f < m->nf; ++f) {
    const or_face *F = &m->face[f];
    double sF0[NV] = { 0 }, sF1[NV] = { 0 }, sWc[NV] = { 0 }, sWt[NV] = { 0 };
    /* the polynomials of the two sides: the cell's own, or with
     * characteristic WENO one limited for this face */
    const double *p0 = &s->coef[F->c0 * NM * NV], *p1 = F->c1 >= 0 ? &s->coef[F->c1 * NM * NV] : NULL;
    double q0[NM * NV], q1[NM * NV];
    if (s->P.weno_eps > 0.0 && s->P.weno_char) {
      double Wref[NV];
      for (int v = 0; v < NV; ++v)
        Wref[v] = F->c1 >= 0 ? 0.5 * (W[F->c0 * NV + v] + W[F->c1 * NV + v]) : W[F->c0 * NV + v];
      if (s->quad[F->c0]) { weno_char_side(s, Wx, F->c0, Wref, F->n, p0, q0); p0 = q0; }
      if (F->c1 >= 0 && s->quad[F->c1]) { weno_char_side(s, Wx, F->c1, Wref, F->n, p1, q1); p1 = q1; }
    }
    for (int k = 0; k < 2; ++k) {
      double Wl[NV], gl[2 * NV], Wr[NV], gr[2 * NV];
      poly_eval(s, W, F->c0, p0, F->xg[k], Wl, gl);
      if (F->c1 >= 0) poly_eval(s, W, F->c1, p1, F->xg[k], Wr, gr);
      else if (is_wall(s, F) || s->P.bc[F->tag].kind == OR_BC_OUTFLOW)
        or_ghost(&s->P, F->tag, Wl, gl, F->n, Wr, gr);
      else {
        /* far field: Riemann-invariant state from the cell mean and the free
         * stream, uniform (zero gradient) outside; Dirichlet: the given
         * state, uniform outside */
        double zero[2 * NV] = { 0 };
        or_ghost(&s->P, F->tag, &W[F->c0 * NV], zero, F->n, Wr, gr);
      }
      double f0[NV], f1[NV], wc[NV], wt[NV];
      if (s->P.flux_hi) or_gks_full_flux_point(&s->P, Wl, Wr, gl, gr, F->n, F->delta, dt, f0, f1, wc, wt);
      else or_gks_flux_point(&s->P, Wl, Wr, gl, gr, F->n, F->delta, f0, f1, wc, wt);
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

/* Net integrated flux sum_p S_p n-flux of the linear combination
 * a*F0 + b*F1 into each cell: out_i = -sum_p sgn S_p (a F0 + b F1). */
static void net_flux(const or_solver *s, const double *F0, const double *F1, double a, double b, double *out) {
  const or_mesh *m = s->m;
  memset(out, 0, sizeof(double) * m->nc * NV);
  for (long f = 0; f < m->nf; ++f) {
    const or_face *F = &m->face[f];
    for (int v = 0; v < NV; ++v) {
      double fl = F->S * (a * F0[f * NV + v] + b * F1[f * NV + v]);
      out[F->c0 * NV + v] -= fl;
      if (F->c1 >= 0) out[F->c1 * NV + v] += fl;
    }
  }
}

/* Gauss-Green (Section 2.3): |Omega| grad W = sum_p S_p n_p sum_k w_k W_{p,k}
 * with the interface states W_{p,k} = W^c + t W_t. */
static void gauss_green(const or_solver *s, const double *Wc, const double *Wt, double t, double *Wx) {
  const or_mesh *m = s->m;
  memset(Wx, 0, sizeof(double) * m->nc * 2 * NV);
  for (long f = 0; f < m->nf; ++f) {
    const or_face *F = &m->face[f];
    for (int v = 0; v < NV; ++v) {
      double wp = Wc[f * NV + v] + t * Wt[f * NV + v];
      for (int d = 0; d < 2; ++d) {
        double g = F->S * F->n[d] * wp;
        Wx[(F->c0 * 2 + d) * NV + v] += g;
        if (F->c1 >= 0) Wx[(F->c1 * 2 + d) * NV + v] -= g;
      }
    }
  }
  for (long c = 0; c < m->nc; ++c)
    for (int q = 0; q < 2 * NV; ++q) Wx[c * 2 * NV + q] /= m->cell[c].vol;
}

/* Explicit global time step (reading of CFL_hi, Section 4):
 * dt = CFL_hi * min_i h_i / (|U_i| + c_i + 2 nu_i / h_i), h_i = 2|Omega_i| / sum_p S_p */
double or_explicit_dt(const or_solver *s) {
  const or_mesh *m = s->m;
  double dt = INFINITY;
  for (long c = 0; c < m->nc; ++c) {
    const or_cell *C = &m->cell[c];
    double per = 0.0;
    for (int k = 0; k < C->nf; ++k) per += m->face[C->face[k]].S;
    double h = 2.0 * C->vol / per;
    double rho, u[2], p;
    prim(s->P.gamma, &s->W[c * NV], &rho, u, &p);
    double a = sqrt(s->P.gamma * p / rho);
    double speed = sqrt(u[0] * u[0] + u[1] * u[1]) + a + 2.0 * (s->P.mu / rho) / h;
    double d = h / speed;
    if (d < dt) dt = d;
  }
  return s->P.cfl_hi * dt;
}

static int check_state(or_solver *s, const double *W) {
  for (long c = 0; c < s->m->nc; ++c) {
    double rho, u[2], p;
    prim(s->P.gamma, &W[c * NV], &rho, u, &p);
    if (!(rho > 0.0) || !(p > 0.0) || !isfinite(rho) || !isfinite(p)) { s->status = 1; return 1; }
  }
  return 0;
}

/* One explicit high-order step from (W, Wx) with time step dt.  Writes the
 * new state to (Wn, Wxn) and the time-averaged net flux of the step to Rlag
 * (so that Wn = W + dt/|Omega| Rlag). */
static void hi_step(or_solver *s, const double *W, const double *Wx, double dt,
                    double *Wn, double *Wxn, double *Rlag) {
  const or_mesh *m = s->m;
  long nc = m->nc, nf = m->nf;
  hi_eval(s, W, Wx, dt);
  if (s->P.time_scheme == 0) {
    /* S1O2 (Section 2.4): W^{n+1} = W^n + dt L + dt^2/2 dL/dt; the
     * interface state at t^{n+1} feeds the Gauss-Green update */
    net_flux(s, s->F0, s->F1, 1.0, 0.5 * dt, Rlag);
    for (long c = 0; c < nc; ++c)
      for (int v = 0; v < NV; ++v) Wn[c * NV + v] = W[c * NV + v] + dt / m->cell[c].vol * Rlag[c * NV + v];
    gauss_green(s, s->Wc, s->Wt, dt, Wxn);
  } else {
    /* S2O4 (two-stage fourth order, Li & Du 2016, named in Section 1):
     *   W*      = W^n + dt/2 L^n + dt^2/8 dL^n
     *   W^{n+1} = W^n + dt L^n + dt^2/6 (dL^n + 2 dL*) */
    double *F0n = (double *)malloc(sizeof(double) * nf * NV), *F1n = (double *)malloc(sizeof(double) * nf * NV);
    double *Wcn = (double *)malloc(sizeof(double) * nf * NV);
    double *Ws = (double *)malloc(sizeof(double) * nc * NV), *Wxs = (double *)malloc(sizeof(double) * nc * 2 * NV);
    double *R = (double *)malloc(sizeof(double) * nc * NV);
    memcpy(F0n, s->F0, sizeof(double) * nf * NV);
    memcpy(F1n, s->F1, sizeof(double) * nf * NV);
    memcpy(Wcn, s->Wc, sizeof(double) * nf * NV);
    net_flux(s, F0n, F1n, 0.5, 0.125 * dt, R);
    for (long c = 0; c < nc; ++c)
      for (int v = 0; v < NV; ++v) Ws[c * NV + v] = W[c * NV + v] + dt / m->cell[c].vol * R[c * NV + v];
    gauss_green(s, Wcn, s->Wt, 0.5 * dt, Wxs);
    hi_eval(s, Ws, Wxs, dt);
    /* Rlag = -sum S (F0^n + dt/6 (F1^n + 2 F1*)) */
    double *F1c = (double *)malloc(sizeof(double) * nf * NV);
    for (long q = 0; q < nf * NV; ++q) F1c[q] = F1n[q] + 2.0 * s->F1[q];
    net_flux(s, F0n, F1c, 1.0, dt / 6.0, Rlag);
    for (long c = 0; c < nc; ++c)
      for (int v = 0; v < NV; ++v) Wn[c * NV + v] = W[c * NV + v] + dt / m->cell[c].vol * Rlag[c * NV + v];
    /* gradients at t^{n+1}: W^{c,n} + dt * W_t^{c,*} (midpoint reading) */
    gauss_green(s, Wcn, s->Wt, dt, Wxn);
    free(F0n); free(F1n); free(Wcn); free(Ws); free(Wxs); free(R); free(F1c);
  }
}

static double density_residual(const or_mesh *m, const double *Wold, const double *Wnew) {
  double num = 0.0, den = 0.0;
  for (long c = 0; c < m->nc; ++c) { num += fabs(Wnew[c * NV] - Wold[c * NV]); den += Wold[c * NV]; }
  return num / den;
}

/* Public explicit step.  dt <= 0: from CFL_hi.  Returns dt used. */
double or_highorder_step(or_solver *s, double dt) {
  const or_mesh *m = s->m;
  long nc = m->nc;
  if (dt <= 0.0) dt = or_explicit_dt(s);
  double *Wn = (double *)malloc(sizeof(double) * nc * NV), *Wxn = (double *)malloc(sizeof(double) * nc * 2 * NV);
  hi_step(s, s->W, s->Wx, dt, Wn, Wxn, s->Rp0);
  s->res = density_residual(m, s->W, Wn);
  memcpy(s->W, Wn, sizeof(double) * nc * NV);
  memcpy(s->Wx, Wxn, sizeof(double) * nc * 2 * NV);
  free(Wn); free(Wxn);
  s->dt_last = dt;
  check_state(s, s->W);
  return dt;
}

/* High-order residual R_i = -sum_p S_p (F0 + dt/2 F1).n at the current
 * state: the time-averaged net flux over [t, t+dt] (Section 3, step 2). */
void or_hi_residual(or_solver *s, double dt, double *R) {
  hi_eval(s, s->W, s->Wx, dt);
  net_flux(s, s->F0, s->F1, 1.0, 0.5 * dt, R);
}

/* Wall loads (the surface quantities of Section 4's cylinder tables and
 * sphere drag): for every boundary face carrying tag, in the oracle's face
 * order, the face centre (mean of its two Gauss points), the unit normal
 * out of the fluid, the length, and the momentum part of the face's
 * high-order flux F0 at the current state (the weighted Gauss-point sum of
 * Eq. (2nd-smooth-flux), or of Eq. (2nd-flux) over a step dt; global
 * frame), which on a wall is the traction the fluid exerts.  Arrays hold
 * max_faces entries; returns the number of faces with the tag. */
long or_wall_loads(or_solver *s, int tag, double dt, long max_faces, double *x, double *n, double *S,
                   double *traction) {
  const or_mesh *m = s->m;
  hi_eval(s, s->W, s->Wx, dt);
  long k = 0;
  for (long f = 0; f < m->nf; ++f) {
    const or_face *F = &m->face[f];
    if (F->c1 >= 0 || F->tag != tag) continue;
    if (k < max_faces) {
      for (int d = 0; d < 2; ++d) {
        x[2 * k + d] = 0.5 * (F->xg[0][d] + F->xg[1][d]);
        n[2 * k + d] = F->n[d];
        traction[2 * k + d] = s->F0[f * NV + 1 + d];
      }
      S[k] = F->S;
    }
    ++k;
  }
  return k;
}

/* ------------------------------------------------------------------ */
/* Low-order level (Section 3): first-order KFVS residual, L-F split,  */
/* local time step, point relaxation.                                   */
/* ------------------------------------------------------------------ */
static void lo_ghost(const or_solver *s, int tag, const double U[NV], const double n[2], double Ug[NV]) {
  double g0[2 * NV] = { 0 }, gg[2 * NV];
  or_ghost(&s->P, tag, U, g0, n, Ug, gg);
}

/* modified spectral radius |U_n| + c + 2 nu S / |Omega| of one side */
static double lo_lambda_side(const or_solver *s, const double U[NV], const double n[2], double S, double vol) {
  double rho, u[2], p;
  prim(s->P.gamma, U, &rho, u, &p);
  double c = sqrt(s->P.gamma * p / rho);
  return fabs(u[0] * n[0] + u[1] * n[1]) + c + 2.0 * (s->P.mu / rho) * S / vol;
}

/* The Lax-Friedrichs alternative of the low-level flux (Section 3 names the
 * solver; its dissipation coefficient is read as the implicit operator's
 * lambda_p = max of the two sides):
 *   F = (F_n(U_l) + F_n(U_r)) / 2 - lambda_p (U_r - U_l) / 2. */
static void lo_lf(const or_solver *s, const double Ul[NV], const double Ur[NV], const double n[2], double lam,
                  double F[NV]) {
  double Fl[NV], Fr[NV];
  or_euler_flux(s->P.gamma, Ul, n, Fl);
  or_euler_flux(s->P.gamma, Ur, n, Fr);
  for (int v = 0; v < NV; ++v) F[v] = 0.5 * (Fl[v] + Fr[v]) - 0.5 * lam * (Ur[v] - Ul[v]);
}

/* R_lo,i(U) = -sum_p S_p F_lo(U_i, U_ip; n_p), F_lo = KFVS or L-F */
/* First-order viscous flux of the low-order level (reading: Section 3's
 * "first-order finite volume scheme" for the Navier-Stokes equations; its
 * implicit operator already carries the viscous spectral radius in lambda).
 * Gradients along the face normal from the two cell states over the
 * distance delta of the cell centres along n (a boundary face: twice the
 * centre-to-face distance, against the ghost state): with du = u_r - u_l,
 *   tau.n = mu / delta (du + (n.du) n / 3)          (Stokes' hypothesis),
 *   q.n   = -kappa (T_r - T_l) / delta,  T = p / rho, kappa = mu c_p (Pr = 1),
 * subtracted from the inviscid flux: F -= (0, tau.n, tau.n . (u_l + u_r)/2 - q.n). */
static void lo_viscous_flux(const or_solver *s, const double Ul[NV], const double Ur[NV], const double n[2],
                            double delta, double F[NV]) {
  double rl, ul[2], pl, rr, ur[2], pr;
  prim(s->P.gamma, Ul, &rl, ul, &pl);
  prim(s->P.gamma, Ur, &rr, ur, &pr);
  const double mu = s->P.mu, kappa = mu * s->P.gamma / (s->P.gamma - 1.0);
  const double du[2] = { ur[0] - ul[0], ur[1] - ul[1] };
  const double dn = du[0] * n[0] + du[1] * n[1];
  double tau[2];
  for (int d = 0; d < 2; ++d) tau[d] = mu / delta * (du[d] + dn * n[d] / 3.0);
  const double qn = -kappa * (pr / rr - pl / rl) / delta;
  F[1] -= tau[0];
  F[2] -= tau[1];
  F[3] -= tau[0] * 0.5 * (ul[0] + ur[0]) + tau[1] * 0.5 * (ul[1] + ur[1]) - qn;
}

static void lo_residual(const or_solver *s, const double *U, double *R) {
  const or_mesh *m = s->m;
  memset(R, 0, sizeof(double) * m->nc * NV);
  for (long f = 0; f < m->nf; ++f) {
    const or_face *F = &m->face[f];
    double Ur[NV], Fl[NV];
    if (F->c1 >= 0) memcpy(Ur, &U[F->c1 * NV], sizeof Ur);
    else lo_ghost(s, F->tag, &U[F->c0 * NV], F->n, Ur);
    if (s->P.flux_lo == 1) {
      const double v0 = m->cell[F->c0].vol, v1 = F->c1 >= 0 ? m->cell[F->c1].vol : v0;
      const double l0 = lo_lambda_side(s, &U[F->c0 * NV], F->n, F->S, v0);
      const double l1 = lo_lambda_side(s, Ur, F->n, F->S, v1);
      lo_lf(s, &U[F->c0 * NV], Ur, F->n, l0 > l1 ? l0 : l1, Fl);
    } else {
      or_kfvs(&s->P, &U[F->c0 * NV], Ur, F->n, Fl);
    }
    if (s->P.lo_viscous && s->P.mu > 0.0) lo_viscous_flux(s, &U[F->c0 * NV], Ur, F->n, F->delta, Fl);
    for (int v = 0; v < NV; ++v) {
      R[F->c0 * NV + v] -= F->S * Fl[v];
      if (F->c1 >= 0) R[F->c1 * NV + v] += F->S * Fl[v];
    }
  }
}

/* lambda_p = max(lambda_i, lambda_ip) per face */
static void lo_lambda(const or_solver *s, const double *U, double *lam) {
  const or_mesh *m = s->m;
  for (long f = 0; f < m->nf; ++f) {
    const or_face *F = &m->face[f];
    double l0 = lo_lambda_side(s, &U[F->c0 * NV], F->n, F->S, m->cell[F->c0].vol);
    double l1;
    if (F->c1 >= 0) l1 = lo_lambda_side(s, &U[F->c1 * NV], F->n, F->S, m->cell[F->c1].vol);
    else { double Ug[NV]; lo_ghost(s, F->tag, &U[F->c0 * NV], F->n, Ug); l1 = lo_lambda_side(s, Ug, F->n, F->S, m->cell[F->c0].vol); }
    lam[f] = l0 > l1 ? l0 : l1;
  }
}

/* F^-(U; n) = (F_n(U) - lambda U) / 2 */
static void fminus(const or_solver *s, const double U[NV], const double n[2], double lam, double out[NV]) {
  double F[NV];
  or_euler_flux(s->P.gamma, U, n, F);
  for (int v = 0; v < NV; ++v) out[v] = 0.5 * (F[v] - lam * U[v]);
}

/* Point-relaxation update of one cell, Eq. (implicit-local):
 * dU_i = (R_i - sum_p S_p [F^-(U_ip + dU_ip) - F^-(U_ip)]) / D_i,
 * D_i = |Omega_i| / dt_i + 1/2 sum_p lambda_p S_p, ghost increments zero.
 * Neighbour increments come from dU, or, with a partition map, from dU_old
 * for neighbours in another partition (the lagged exchange of the paper's
 * threaded sweep). */
static void relax_cell(const or_solver *s, long i, const double *U, const double *R, const double *lam,
                       const double *D, double *dU, const double *dU_old, const int *part) {
  const or_mesh *m = s->m;
  const or_cell *C = &m->cell[i];
  double acc[NV];
  for (int v = 0; v < NV; ++v) acc[v] = R[i * NV + v];
  for (int k = 0; k < C->nf; ++k) {
    const or_face *F = &m->face[C->face[k]];
    if (F->c1 < 0) continue;
    long j = C->sgn[k] > 0 ? F->c1 : F->c0;
    const double *dj = (part && part[j] != part[i]) ? &dU_old[j * NV] : &dU[j * NV];
    double n[2] = { C->sgn[k] * F->n[0], C->sgn[k] * F->n[1] };
    double Up[NV], fa[NV], fb[NV];
    for (int v = 0; v < NV; ++v) Up[v] = U[j * NV + v] + dj[v];
    fminus(s, Up, n, lam[C->face[k]], fa);
    fminus(s, &U[j * NV], n, lam[C->face[k]], fb);
    for (int v = 0; v < NV; ++v) acc[v] -= F->S * (fa[v] - fb[v]);
  }
  for (int v = 0; v < NV; ++v) dU[i * NV + v] = acc[v] / D[i];
}

static void lo_diag(const or_solver *s, const double *lam, double *D) {
  const or_mesh *m = s->m;
  for (long i = 0; i < m->nc; ++i) {
    const or_cell *C = &m->cell[i];
    double sum = 0.0;
    for (int k = 0; k < C->nf; ++k) sum += lam[C->face[k]] * m->face[C->face[k]].S;
    double dti = s->P.cfl_lo * C->vol / sum;      /* local time step */
    D[i] = C->vol / dti + 0.5 * sum;
  }
}

/* Algorithm 1, n_sweeps x (forward pass, backward pass), in one of four
 * orders.  0: colour classes (colours ascending, then descending); the
 * default and the GPU's.  1: element index 1..N, then N..1 (Algorithm 1 as
 * printed, serial).  2: the paper's threaded sweep made deterministic: the
 * index range cut into n_parts partitions, each swept in index order, with
 * neighbours in other partitions read as they were at the start of the
 * pass (Section 4, parallel strategy).  3: the same idea with colour
 * classes inside each partition: the reverse Cuthill-McKee order cut into
 * n_parts partitions (the cell at RCM position k is in partition
 * floor(k n_parts / N)); each sweep relaxes colours ascending then
 * descending within every partition, and a neighbour in another partition
 * is read as it was at the start of the sweep (the forward and backward
 * pass together). */
static void point_relaxation(const or_solver *s, const double *U, const double *R, const double *lam,
                             const double *D, int n_sweeps, double *dU) {
  const or_mesh *m = s->m;
  const long nc = m->nc;
  memset(dU, 0, sizeof(double) * nc * NV);
  if (s->P.sweep_order == 0) {
    for (int sw = 0; sw < n_sweeps; ++sw) {
      for (int col = 0; col < m->ncolour; ++col)
        for (long i = 0; i < nc; ++i) if (m->colour[i] == col) relax_cell(s, i, U, R, lam, D, dU, NULL, NULL);
      for (int col = m->ncolour - 1; col >= 0; --col)
        for (long i = 0; i < nc; ++i) if (m->colour[i] == col) relax_cell(s, i, U, R, lam, D, dU, NULL, NULL);
    }
    return;
  }
  if (s->P.sweep_order == 3) {
    const long np = s->P.n_parts > 0 ? s->P.n_parts : 1;
    int *part = (int *)malloc(sizeof(int) * nc);
    double *old = (double *)malloc(sizeof(double) * nc * NV);
    for (long k = 0; k < nc; ++k) part[m->rcm[k]] = (int)((k * np) / nc);
    for (int sw = 0; sw < n_sweeps; ++sw) {
      memcpy(old, dU, sizeof(double) * nc * NV);
      for (int col = 0; col < m->ncolour; ++col)
        for (long i = 0; i < nc; ++i) if (m->colour[i] == col) relax_cell(s, i, U, R, lam, D, dU, old, part);
      for (int col = m->ncolour - 1; col >= 0; --col)
        for (long i = 0; i < nc; ++i) if (m->colour[i] == col) relax_cell(s, i, U, R, lam, D, dU, old, part);
    }
    free(part);
    free(old);
    return;
  }
  int *part = NULL;
  double *old = NULL;
  if (s->P.sweep_order == 2) {
    const int np = s->P.n_parts > 0 ? s->P.n_parts : 1;
    part = (int *)malloc(sizeof(int) * nc);
    old = (double *)malloc(sizeof(double) * nc * NV);
    for (long i = 0; i < nc; ++i) part[i] = (int)((i * np) / nc);
  }
  for (int sw = 0; sw < n_sweeps; ++sw) {
    if (old) memcpy(old, dU, sizeof(double) * nc * NV);
    for (long i = 0; i < nc; ++i) relax_cell(s, i, U, R, lam, D, dU, old, part);
    if (old) memcpy(old, dU, sizeof(double) * nc * NV);
    for (long i = nc - 1; i >= 0; --i) relax_cell(s, i, U, R, lam, D, dU, old, part);
  }
  free(part);
  free(old);
}

/* Low-order solve of R(W~) + S = 0 from U = W_p0 (Section 3, step 4):
 * n_implicit backward-Euler steps, each solved by point relaxation. */
static void lo_solve(or_solver *s, const double *Wp0, const double *Rp0, double *U) {
  const or_mesh *m = s->m;
  long nc = m->nc, nf = m->nf;
  double *Src = (double *)malloc(sizeof(double) * nc * NV), *R = (double *)malloc(sizeof(double) * nc * NV);
  double *lam = (double *)malloc(sizeof(double) * nf), *D = (double *)malloc(sizeof(double) * nc);
  double *dU = (double *)malloc(sizeof(double) * nc * NV);
  /* forcing S = R_p0 - R(W_p0) (step 3) */
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

/* One two-level V-cycle (Section 3, steps 1-5). */
static void pmg_cycle(or_solver *s) {
  const or_mesh *m = s->m;
  long nc = m->nc;
  double dt = or_explicit_dt(s);
  double *Wn = (double *)malloc(sizeof(double) * nc * NV), *Wxn = (double *)malloc(sizeof(double) * nc * 2 * NV);
  double *Rlag = (double *)malloc(sizeof(double) * nc * NV), *U = (double *)malloc(sizeof(double) * nc * NV);
  /* 1: high-order step */
  hi_step(s, s->W, s->Wx, dt, Wn, Wxn, Rlag);
  /* 2: restriction W_p0 = W^{n+1}, residual R_p0 = R(W^{n+1}): the
   * time-averaged net flux over [t^{n+1}, t^{n+1} + dt] */
  hi_eval(s, Wn, Wxn, dt);
  net_flux(s, s->F0, s->F1, 1.0, 0.5 * dt, s->Rp0);
  /* 3-4: forcing and low-order implicit solve */
  lo_solve(s, Wn, s->Rp0, U);
  /* 5: prolongation of the correction C = W~ - W_p0; gradients unchanged */
  for (long q = 0; q < nc * NV; ++q) Wn[q] += U[q] - Wn[q];
  s->res = density_residual(m, s->W, Wn);
  memcpy(s->W, Wn, sizeof(double) * nc * NV);
  memcpy(s->Wx, Wxn, sizeof(double) * nc * 2 * NV);
  s->dt_last = dt;
  free(Wn); free(Wxn); free(Rlag); free(U);
  check_state(s, s->W);
}

int or_pmg_cycle(or_solver *s, int n, double *res_hist) {
  for (int k = 0; k < n; ++k) {
    pmg_cycle(s);
    if (res_hist) res_hist[k] = s->res;
    if (s->status) return s->status;
  }
  return s->status;
}

int or_explicit_steps(or_solver *s, int n, double *res_hist) {
  for (int k = 0; k < n; ++k) {
    or_highorder_step(s, -1.0);
    if (res_hist) res_hist[k] = s->res;
    if (s->status) return s->status;
  }
  return s->status;
}

/* low-order smoothing alone, using R_p0 of the last high-order evaluation
 * held in the solver (step 3-5 of Section 3 on the current state) */
void or_loworder_smooth(or_solver *s) {
  long nc = s->m->nc;
  double *U = (double *)malloc(sizeof(double) * nc * NV), *Wp0 = (double *)malloc(sizeof(double) * nc * NV);
  memcpy(Wp0, s->W, sizeof(double) * nc * NV);
  lo_solve(s, Wp0, s->Rp0, U);
  s->res = density_residual(s->m, s->W, U);
  memcpy(s->W, U, sizeof(double) * nc * NV);
  free(U); free(Wp0);
}

/* ---- test hooks for the low level ---- */
void or_lo_residual(const or_solver *s, const double *U, double *R) { lo_residual(s, U, R); }
void or_lo_lambda(const or_solver *s, const double *U, double *lam) { lo_lambda(s, U, lam); }
void or_lo_diag(const or_solver *s, const double *U, double *D) {
  double *lam = (double *)malloc(sizeof(double) * s->m->nf);
  lo_lambda(s, U, lam); lo_diag(s, lam, D); free(lam);
}
/* relax with a given right-hand side: dU from n_sweeps (forward+backward) passes;
 * n_sweeps < 0 means a single forward pass */
void or_lo_relax(const or_solver *s, const double *U, const double *R, int n_sweeps, double *dU) {
  const or_mesh *m = s->m;
  double *lam = (double *)malloc(sizeof(double) * m->nf), *D = (double *)malloc(sizeof(double) * m->nc);
  lo_lambda(s, U, lam); lo_diag(s, lam, D);
  if (n_sweeps >= 0) point_relaxation(s, U, R, lam, D, n_sweeps, dU);
  else {
    memset(dU, 0, sizeof(double) * m->nc * NV);
    for (int col = 0; col < m->ncolour; ++col)
      for (long i = 0; i < m->nc; ++i) if (m->colour[i] == col) relax_cell(s, i, U, R, lam, D, dU, NULL, NULL);
  }
  free(lam); free(D);
}
void or_set_rp0(or_solver *s, const double *R) { memcpy(s->Rp0, R, sizeof(double) * s->m->nc * NV); }
void or_get_rp0(const or_solver *s, double *R) { memcpy(R, s->Rp0, sizeof(double) * s->m->nc * NV); }

/* micro-slope solve exposed for the compatibility pin */
int or_micro_slope(double gamma, const double W[NV], const double dW[NV], double s[NV]) {
  double K = or_K(gamma);
  or_maxw g = maxw_from_W(W, K);
  or_mom m;
  moments(&g, K, 0, &m);
  return micro_slope(&m, g.rho, dW, s);
}
