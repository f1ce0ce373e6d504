// Device-side gas-kinetic physics of the compact GKS, 2-D (Sections 2.2-2.3
// and 3 of Ji, Shyy & Xu, arXiv:2109.09965).
//
// All routines work in the local face frame (normal n, tangent t = (-ny, nx))
// on conservative variables (rho, rho*u_n, rho*u_t, rho*E) and their
// derivatives along n and t.  Moments of the Maxwellian are normalised by
// rho: <u^a> by the standard recurrence, <xi^2> = K/(2 lambda),
// <xi^4> = K(K+2)/(4 lambda^2).  The micro-slope solve <a psi> = b uses its
// closed form.  Templated on the arithmetic type so the same code serves
// the FP64 path and the FP32 flux of the mixed path.
#pragma once

#include <cuda_runtime.h>

namespace cgks {
namespace dev {

constexpr int NV = 4;

template <typename T> __device__ __forceinline__ T d_erfc(T x);
template <> __device__ __forceinline__ double d_erfc<double>(double x) { return erfc(x); }
template <> __device__ __forceinline__ float d_erfc<float>(float x) { return erfcf(x); }
template <typename T> __device__ __forceinline__ T d_exp(T x);
template <> __device__ __forceinline__ double d_exp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float d_exp<float>(float x) { return expf(x); }
template <typename T> __device__ __forceinline__ T d_expm1(T x);
template <> __device__ __forceinline__ double d_expm1<double>(double x) { return expm1(x); }
template <> __device__ __forceinline__ float d_expm1<float>(float x) { return expm1f(x); }
template <typename T> __device__ __forceinline__ T d_sqrt(T x);
template <> __device__ __forceinline__ double d_sqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float d_sqrt<float>(float x) { return sqrtf(x); }
template <typename T> __device__ __forceinline__ T d_pi();
template <> __device__ __forceinline__ double d_pi<double>() { return 3.141592653589793238462643; }
template <> __device__ __forceinline__ float d_pi<float>() { return 3.14159265358979f; }

// Rotate a conservative vector between global and face frames.
template <typename T>
__device__ __forceinline__ void rot_in(T nx, T ny, const T g[NV], T l[NV]) {
  l[0] = g[0];
  l[1] = g[1] * nx + g[2] * ny;
  l[2] = -g[1] * ny + g[2] * nx;
  l[3] = g[3];
}
template <typename T>
__device__ __forceinline__ void rot_out(T nx, T ny, const T l[NV], T g[NV]) {
  g[0] = l[0];
  g[1] = l[1] * nx - l[2] * ny;
  g[2] = l[1] * ny + l[2] * nx;
  g[3] = l[3];
}

// Constants of the kinetic model with K internal degrees of freedom,
// computed once on the host: c2K = 2/(K+2), c4K = 4/(K+2).
template <typename T>
struct KC {
  T K, c2K, c4K;
};
constexpr double kInvSqrtPi = 0.56418958354775628694807945156;

// Maxwellian of local-frame conservative W: rho, 1/rho, U, V, lambda and
// 1/(2 lambda).  Two divisions; everything downstream multiplies.
template <typename T>
struct Maxw {
  T rho, ir, U, V, lam, i2l;
};
template <typename T>
__device__ __forceinline__ Maxw<T> maxw(const T W[NV], T c2K) {
  // lambda = (K+2) rho / (4 (rho E - rho |U|^2 / 2)),  c2K = 2 / (K+2)
  Maxw<T> g;
  g.rho = W[0];
  g.ir = T(1) / W[0];
  g.U = W[1] * g.ir;
  g.V = W[2] * g.ir;
  T eps = W[3] - T(0.5) * g.rho * (g.U * g.U + g.V * g.V);
  g.i2l = c2K * eps * g.ir;
  g.lam = T(0.5) / g.i2l;
  return g;
}

template <typename T> __device__ __forceinline__ T d_rsqrt(T x);
template <> __device__ __forceinline__ double d_rsqrt<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float d_rsqrt<float>(float x) { return rsqrtf(x); }

// Half-range moments <u^k>, k = 0..KMAX, over u > 0 (sgn = +1) or u < 0
// (-1), of the Maxwellian with mean U, 1/(2 lambda) = i2l, sqrt(lambda) = sl
// and 1/sqrt(pi lambda) = isp.
template <typename T, int KMAX>
__device__ __forceinline__ void half_moments(T U, T i2l, T sl, T isp, int sgn, T mu[KMAX + 1]) {
  T z = sl * U;
  T e = d_exp(-z * z) * isp;
  if (sgn > 0) {
    mu[0] = T(0.5) * d_erfc(-z);
    mu[1] = U * mu[0] + T(0.5) * e;
  } else {
    mu[0] = T(0.5) * d_erfc(z);
    mu[1] = U * mu[0] - T(0.5) * e;
  }
#pragma unroll
  for (int k = 2; k <= KMAX; ++k) mu[k] = U * mu[k - 1] + T(k - 1) * i2l * mu[k - 2];
}

// Full-range moment tables of the equilibrium used by the flux.
template <typename T>
struct Mom {
  T mu[7], mv[7], x2, x4;   // <u^k>, <v^k>, <xi^2>, <xi^4>
};
template <typename T>
__device__ __forceinline__ void full_moments(const Maxw<T> &g, T K, Mom<T> &m) {
  const T i2l = g.i2l;
  m.mu[0] = T(1); m.mu[1] = g.U;
  m.mv[0] = T(1); m.mv[1] = g.V;
#pragma unroll
  for (int k = 2; k < 7; ++k) {
    m.mu[k] = g.U * m.mu[k - 1] + T(k - 1) * i2l * m.mu[k - 2];
    m.mv[k] = g.V * m.mv[k - 1] + T(k - 1) * i2l * m.mv[k - 2];
  }
  m.x2 = K * i2l;
  m.x4 = K * (K + T(2)) * i2l * i2l;
}

// <u^a v^b xi^(2d) * s>, slope s = s0 + s1 u + s2 v + s3 (u^2+v^2+xi^2)/2
template <typename T>
__device__ __forceinline__ T mslope(const Mom<T> &m, int a, int b, int d, const T s[NV]) {
  const T xd = d == 0 ? T(1) : (d == 1 ? m.x2 : m.x4);
  const T xd1 = d == 0 ? m.x2 : m.x4;
  T r = s[0] * m.mu[a] * m.mv[b] * xd + s[1] * m.mu[a + 1] * m.mv[b] * xd + s[2] * m.mu[a] * m.mv[b + 1] * xd;
  r += T(0.5) * s[3] * (m.mu[a + 2] * m.mv[b] * xd + m.mu[a] * m.mv[b + 2] * xd + m.mu[a] * m.mv[b] * xd1);
  return r;
}
// vector <u^a v^b s psi>
template <typename T>
__device__ __forceinline__ void gpsi(const Mom<T> &m, int a, int b, const T s[NV], T out[NV]) {
  out[0] = mslope(m, a, b, 0, s);
  out[1] = mslope(m, a + 1, b, 0, s);
  out[2] = mslope(m, a, b + 1, 0, s);
  out[3] = T(0.5) * (mslope(m, a + 2, b, 0, s) + mslope(m, a, b + 2, 0, s) + mslope(m, a, b, 1, s));
}

// Closed-form solution of <s psi> = b (b already divided by rho), 2-D,
// K internal degrees of freedom.  q = U^2 + V^2 + (K+2)/(2 lambda),
// tl = 2 lambda, l2 = 4 lambda^2 / (K+2): shared by the three solves.
template <typename T>
struct SlopeSolver {
  T U, V, q, tl, l2;
};
template <typename T>
__device__ __forceinline__ SlopeSolver<T> slope_solver(const Maxw<T> &g, const KC<T> &kc) {
  SlopeSolver<T> S;
  S.U = g.U; S.V = g.V;
  S.q = g.U * g.U + g.V * g.V + (kc.K + T(2)) * g.i2l;
  S.tl = T(2) * g.lam;
  S.l2 = kc.c4K * g.lam * g.lam;
  return S;
}
template <typename T>
__device__ __forceinline__ void micro_slope(const SlopeSolver<T> &S, const T b[NV], T s[NV]) {
  T R4 = T(2) * b[3] - S.q * b[0];
  T R3 = b[2] - S.V * b[0];
  T R2 = b[1] - S.U * b[0];
  s[3] = S.l2 * (R4 - T(2) * S.U * R2 - T(2) * S.V * R3);
  s[2] = S.tl * R3 - S.V * s[3];
  s[1] = S.tl * R2 - S.U * s[3];
  s[0] = b[0] - S.U * s[1] - S.V * s[2] - T(0.5) * s[3] * S.q;
}

// Smooth gas-kinetic flux at one Gauss point, Eq. (2nd-smooth-flux):
//   f = g^c - tau (a_n u + a_t v + A) g^c + A g^c t,   tau = mu / p^c
// with W^c from the half-range moments of g^l (u>0) and g^r (u<0), the
// equilibrium slopes from the mean of the side derivatives plus, along n,
// ajump * (W^r - W^l) with ajump = alpha / delta.  Inputs and outputs in
// the local frame: F0 + t F1 = flux, Wc + t Wt = interface state.
template <typename T>
__device__ __forceinline__ void gks_point_local(const KC<T> &kc, T mu_visc, T ajump,
                                                const T Wl[NV], const T Wr[NV],
                                                const T dnl[NV], const T dtl[NV],
                                                const T dnr[NV], const T dtr[NV],
                                                T F0[NV], T F1[NV], T Wc[NV], T Wt[NV]) {
  const T K = kc.K, c2K = kc.c2K;
  Maxw<T> gl = maxw(Wl, c2K), gr = maxw(Wr, c2K);
  T ml[3], mr[3];
  half_moments<T, 2>(gl.U, gl.i2l, d_sqrt(gl.lam), d_rsqrt(gl.lam) * T(kInvSqrtPi), +1, ml);
  half_moments<T, 2>(gr.U, gr.i2l, d_sqrt(gr.lam), d_rsqrt(gr.lam) * T(kInvSqrtPi), -1, mr);
  T el = gl.V * gl.V + (K + T(1)) * gl.i2l;
  T er = gr.V * gr.V + (K + T(1)) * gr.i2l;
  Wc[0] = gl.rho * ml[0] + gr.rho * mr[0];
  Wc[1] = gl.rho * ml[1] + gr.rho * mr[1];
  Wc[2] = gl.rho * ml[0] * gl.V + gr.rho * mr[0] * gr.V;
  Wc[3] = gl.rho * T(0.5) * (ml[2] + ml[0] * el) + gr.rho * T(0.5) * (mr[2] + mr[0] * er);
  Maxw<T> gc = maxw(Wc, c2K);
  Mom<T> m;
  full_moments(gc, K, m);
  SlopeSolver<T> SS = slope_solver(gc, kc);
  T bn[NV], bt[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T dn = T(0.5) * (dnl[v] + dnr[v]) + ajump * (Wr[v] - Wl[v]);
    bn[v] = dn * gc.ir;
    bt[v] = T(0.5) * (dtl[v] + dtr[v]) * gc.ir;
  }
  T an[NV], at[NV], A[NV], bA[NV], g1[NV], g2[NV];
  micro_slope(SS, bn, an);
  micro_slope(SS, bt, at);
  gpsi(m, 1, 0, an, g1);
  gpsi(m, 0, 1, at, g2);
#pragma unroll
  for (int v = 0; v < NV; ++v) bA[v] = -(g1[v] + g2[v]);
  micro_slope(SS, bA, A);
  T tau = mu_visc * SS.tl * gc.ir;          // mu / p^c, p^c = rho / (2 lambda)
  T gAu[NV], gA[NV], gn2[NV], gtuv[NV];
  gpsi(m, 1, 0, A, gAu);
  gpsi(m, 0, 0, A, gA);
  gpsi(m, 2, 0, an, gn2);
  gpsi(m, 1, 1, at, gtuv);
  T feq[NV] = { m.mu[1], m.mu[2], m.mu[1] * gc.V,
                T(0.5) * (m.mu[3] + m.mu[1] * m.mv[2] + m.mu[1] * m.x2) };
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    F0[v] = gc.rho * (feq[v] - tau * (gn2[v] + gtuv[v] + gAu[v]));
    F1[v] = gc.rho * gAu[v];
    Wt[v] = gc.rho * gA[v];
  }
}

// ---------------- full flux, Eq. (2nd-flux) ----------------
// Moment table of one Maxwellian whose u-moments are taken over a half
// range (sgn = +1: u > 0, -1: u < 0); v and xi moments full.
template <typename T>
__device__ __forceinline__ void half_table(const Maxw<T> &g, T K, int sgn, Mom<T> &m) {
  half_moments<T, 6>(g.U, g.i2l, d_sqrt(g.lam), d_rsqrt(g.lam) * T(kInvSqrtPi), sgn, m.mu);
  m.mv[0] = T(1); m.mv[1] = g.V;
#pragma unroll
  for (int k = 2; k < 7; ++k) m.mv[k] = g.V * m.mv[k - 1] + T(k - 1) * g.i2l * m.mv[k - 2];
  m.x2 = K * g.i2l;
  m.x4 = K * (K + T(2)) * g.i2l * g.i2l;
}

// Spatial micro-slopes of a Maxwellian from its normal / tangential
// derivatives (dn, dt), and the temporal one from <A + a_n u + a_t v> = 0.
template <typename T>
__device__ __forceinline__ void maxw_slopes(const Maxw<T> &g, const Mom<T> &mf, const KC<T> &kc, const T dn[NV],
                                            const T dt[NV], T an[NV], T at[NV], T A[NV]) {
  SlopeSolver<T> SS = slope_solver(g, kc);
  T b[NV], g1[NV], g2[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) b[v] = dn[v] * g.ir;
  micro_slope(SS, b, an);
#pragma unroll
  for (int v = 0; v < NV; ++v) b[v] = dt[v] * g.ir;
  micro_slope(SS, b, at);
  gpsi(mf, 1, 0, an, g1);
  gpsi(mf, 0, 1, at, g2);
#pragma unroll
  for (int v = 0; v < NV; ++v) b[v] = -(g1[v] + g2[v]);
  micro_slope(SS, b, A);
}

// rho-weighted moments of one piece of the distribution: flux moments
// Q = (<u psi>, <u (a_n u + a_t v) psi>, <u A psi>) and state moments
// P = (<psi>, <(a_n u + a_t v) psi>, <A psi>).
template <typename T>
__device__ __forceinline__ void piece(T rho, const Mom<T> &m, const T an[NV], const T at[NV], const T A[NV],
                                      T Q[3][NV], T P[3][NV]) {
  const T one[NV] = { T(1), T(0), T(0), T(0) };
  T a[NV], b[NV];
  gpsi(m, 1, 0, one, a);
#pragma unroll
  for (int v = 0; v < NV; ++v) Q[0][v] = rho * a[v];
  gpsi(m, 2, 0, an, a);
  gpsi(m, 1, 1, at, b);
#pragma unroll
  for (int v = 0; v < NV; ++v) Q[1][v] = rho * (a[v] + b[v]);
  gpsi(m, 1, 0, A, a);
#pragma unroll
  for (int v = 0; v < NV; ++v) Q[2][v] = rho * a[v];
  gpsi(m, 0, 0, one, a);
#pragma unroll
  for (int v = 0; v < NV; ++v) P[0][v] = rho * a[v];
  gpsi(m, 1, 0, an, a);
  gpsi(m, 0, 1, at, b);
#pragma unroll
  for (int v = 0; v < NV; ++v) P[1][v] = rho * (a[v] + b[v]);
  gpsi(m, 0, 0, A, a);
#pragma unroll
  for (int v = 0; v < NV; ++v) P[2][v] = rho * a[v];
}

// Eq. (2nd-flux) with time coefficients (c1, c2, c3, e, te) applied to the
// equilibrium (X0), left (XL) and right (XR) pieces.
template <typename T>
__device__ __forceinline__ void full_sum(T c1, T c2, T c3, T e, T te, T tau, const T X0[3][NV], const T XL[3][NV],
                                         const T XR[3][NV], T out[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v)
    out[v] = c1 * X0[0][v] + c2 * X0[1][v] + c3 * X0[2][v] +
             e * ((XL[0][v] + XR[0][v]) - tau * (XL[1][v] + XR[1][v]) - tau * (XL[2][v] + XR[2][v])) -
             te * (XL[1][v] + XR[1][v]);
}

// Full gas-kinetic flux at one Gauss point, Eq. (2nd-flux):
//   f = (1 - e) g^c + [(t + tau) e - tau] a^c.u g^c + (t - tau + tau e) A^c g^c
//     + e g^l [1 - (tau + t) a^l.u - tau A^l] H(u) + e g^r [...] (1 - H(u)),
// e = exp(-t / tau_n), tau = mu / p^c,
// tau_n = tau + c1 dt + c2 dt |p_l - p_r| / (p_l + p_r).
// Brought to the linear-in-time form of the time schemes through the time
// integrals over [0, dt] and [0, dt/2]: F0 dt + F1 dt^2/2 = Fhat(dt),
// F0 dt/2 + F1 dt^2/8 = Fhat(dt/2); the interface state W_p(t) = <psi f(t)>
// by the line Wc + t Wt through its values at dt/2 and dt.  Same frame and
// arguments as gks_point_local, plus dt and the two tau_n constants.
template <typename T>
__device__ void gks_full_point_local(const KC<T> &kc, T mu_visc, T ajump, T dt, T tc1, T tc2, const T Wl[NV],
                                     const T Wr[NV], const T dnl[NV], const T dtl[NV], const T dnr[NV],
                                     const T dtr[NV], T F0[NV], T F1[NV], T Wc[NV], T Wt[NV]) {
  const T K = kc.K, c2K = kc.c2K;
  Maxw<T> gl = maxw(Wl, c2K), gr = maxw(Wr, c2K);
  T Q0[3][NV], P0[3][NV], QL[3][NV], PL[3][NV], QR[3][NV], PR[3][NV];
  T anl[NV], atl[NV], Al[NV], anr[NV], atr[NV], Ar[NV];
  {
    Mom<T> mf;
    full_moments(gl, K, mf);
    maxw_slopes(gl, mf, kc, dnl, dtl, anl, atl, Al);
    full_moments(gr, K, mf);
    maxw_slopes(gr, mf, kc, dnr, dtr, anr, atr, Ar);
  }
  T W0[NV];
  {
    Mom<T> mh;
    half_table(gl, K, +1, mh);
    piece(gl.rho, mh, anl, atl, Al, QL, PL);
    half_table(gr, K, -1, mh);
    piece(gr.rho, mh, anr, atr, Ar, QR, PR);
  }
  // W^c: the collision of the particles of g^l moving right and g^r moving left
#pragma unroll
  for (int v = 0; v < NV; ++v) W0[v] = PL[0][v] + PR[0][v];
  Maxw<T> gc = maxw(W0, c2K);
  T an[NV], at[NV], A[NV];
  {
    Mom<T> m;
    full_moments(gc, K, m);
    T dn[NV], dtg[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      dn[v] = T(0.5) * (dnl[v] + dnr[v]) + ajump * (Wr[v] - Wl[v]);
      dtg[v] = T(0.5) * (dtl[v] + dtr[v]);
    }
    maxw_slopes(gc, m, kc, dn, dtg, an, at, A);
    piece(gc.rho, m, an, at, A, Q0, P0);
  }
  const T tau = mu_visc * T(2) * gc.lam * gc.ir;          // mu / p^c
  const T pl = gl.rho * gl.i2l, pr = gr.rho * gr.i2l;
  const T taun = tau + tc1 * dt + tc2 * dt * fabs(pl - pr) / (pl + pr);
  T Fd[NV], Fh[NV], Wd[NV], Wh[NV];
#pragma unroll 1
  for (int k = 0; k < 2; ++k) {
    const T t = k == 0 ? dt : T(0.5) * dt;
    // coefficient functions at t and their integrals over [0, t]
    const T e = taun > T(0) ? d_exp(-t / taun) : T(0);
    const T om = taun > T(0) ? -d_expm1(-t / taun) : T(1);
    const T ie = taun * om, ite = taun * taun * om - taun * t * e;
    full_sum(t - ie, ite + tau * ie - tau * t, T(0.5) * t * t - tau * t + tau * ie, ie, ite, tau, Q0, QL, QR,
             k == 0 ? Fd : Fh);
    full_sum(T(1) - e, (t + tau) * e - tau, t - tau + tau * e, e, t * e, tau, P0, PL, PR, k == 0 ? Wd : Wh);
  }
  const T idt = T(1) / dt;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    F0[v] = (T(4) * Fh[v] - Fd[v]) * idt;
    F1[v] = T(4) * (Fd[v] - T(2) * Fh[v]) * idt * idt;
    Wc[v] = T(2) * Wh[v] - Wd[v];
    Wt[v] = T(2) * (Wd[v] - Wh[v]) * idt;
  }
}

// Cell-average primitives used by the low level (one set per cell and
// implicit step): rho, u, v, p, 1/(2 lambda), sqrt(lambda), 1/sqrt(pi
// lambda), sound speed c, 1/rho.
constexpr int NPRIM = 9;
template <typename T>
struct Prim {
  T rho, u, v, p, i2l, sl, isp, c, ir;
};
template <typename T>
__device__ __forceinline__ Prim<T> prim_of(const T W[NV], T gamma, const KC<T> &kc) {
  Prim<T> q;
  q.rho = W[0];
  q.ir = T(1) / W[0];
  q.u = W[1] * q.ir;
  q.v = W[2] * q.ir;
  T eps = W[3] - T(0.5) * q.rho * (q.u * q.u + q.v * q.v);
  q.p = (gamma - T(1)) * eps;
  q.i2l = kc.c2K * eps * q.ir;
  T lam = T(0.5) / q.i2l;
  q.sl = d_sqrt(lam);
  q.isp = d_rsqrt(lam) * T(kInvSqrtPi);
  q.c = d_sqrt(gamma * q.p * q.ir);
  return q;
}

// First-order KFVS flux of two cell-average states, local frame, from
// their primitives (normal / tangential velocities already rotated).
template <typename T>
__device__ __forceinline__ void kfvs_prims(T K, T rl, T unl, T utl, T i2ll, T sll, T ispl,
                                           T rr, T unr, T utr, T i2lr, T slr, T ispr, T F[NV]) {
  T ml[4], mr[4];
  half_moments<T, 3>(unl, i2ll, sll, ispl, +1, ml);
  half_moments<T, 3>(unr, i2lr, slr, ispr, -1, mr);
  T el = utl * utl + (K + T(1)) * i2ll;
  T er = utr * utr + (K + T(1)) * i2lr;
  F[0] = rl * ml[1] + rr * mr[1];
  F[1] = rl * ml[2] + rr * mr[2];
  F[2] = rl * ml[1] * utl + rr * mr[1] * utr;
  F[3] = rl * T(0.5) * (ml[3] + ml[1] * el) + rr * T(0.5) * (mr[3] + mr[1] * er);
}

// Euler normal flux F(U).n, global frame.
template <typename T>
__device__ __forceinline__ void euler_flux(T gamma, const T W[NV], T nx, T ny, T F[NV]) {
  T ir = T(1) / W[0];
  T u = W[1] * ir, v = W[2] * ir;
  T p = (gamma - T(1)) * (W[3] - T(0.5) * W[0] * (u * u + v * v));
  T un = u * nx + v * ny;
  F[0] = W[0] * un;
  F[1] = W[1] * un + p * nx;
  F[2] = W[2] * un + p * ny;
  F[3] = (W[3] + p) * un;
}

// F_n(U + dU) - F_n(U) of the Euler normal flux, written so that every
// term is proportional to the increment (no cancellation between two
// nearly equal fluxes): exact algebra, accurate to the working precision
// relative to the difference itself.  Base state: conservative W, velocity
// (u, v), pressure p; dW the increment; (nx, ny) the normal.
template <typename T>
__device__ __forceinline__ void euler_flux_delta(T gamma, const T W[NV], T u, T v, T p, const T dW[NV],
                                                 T nx, T ny, T dF[NV]) {
  const T rho = W[0], r1 = W[0] + dW[0];
  const T inv = T(1) / (rho * r1);
  const T mn = W[1] * nx + W[2] * ny, dmn = dW[1] * nx + dW[2] * ny;
  const T un = u * nx + v * ny;
  const T dun = (rho * dmn - mn * dW[0]) * inv;                       // (un)' - un
  const T un1 = un + dun;
  const T m2 = W[1] * W[1] + W[2] * W[2];
  const T dm2 = T(2) * (W[1] * dW[1] + W[2] * dW[2]) + dW[1] * dW[1] + dW[2] * dW[2];
  const T dke = T(0.5) * (rho * dm2 - m2 * dW[0]) * inv;              // d(|m|^2 / (2 rho))
  const T dp = (gamma - T(1)) * (dW[3] - dke);
  dF[0] = dmn;
  dF[1] = dW[1] * un1 + W[1] * dun + dp * nx;
  dF[2] = dW[2] * un1 + W[2] * dun + dp * ny;
  dF[3] = (dW[3] + dp) * un1 + (W[3] + p) * dun;
}

// ---------------- boundary ghost states (local frame) ----------------
// Wall velocity (wn, wt) and free stream (rho, un, ut, p) are given in the
// face frame of the boundary face.
template <typename T>
__device__ __forceinline__ void ghost_slip(const T W[NV], const T dn[NV], const T dt[NV],
                                           T Wg[NV], T dng[NV], T dtg[NV]) {
  // rho, rho u_t, rho E even across the wall, rho u_n odd
  Wg[0] = W[0]; Wg[1] = -W[1]; Wg[2] = W[2]; Wg[3] = W[3];
  dng[0] = -dn[0]; dng[1] = dn[1]; dng[2] = -dn[2]; dng[3] = -dn[3];
  dtg[0] = dt[0]; dtg[1] = -dt[1]; dtg[2] = dt[2]; dtg[3] = dt[3];
}

template <typename T>
__device__ __forceinline__ void ghost_noslip(T gamma, T wn, T wt, const T W[NV], const T dn[NV],
                                             const T dt[NV], T Wg[NV], T dng[NV], T dtg[NV]) {
  // rho, p even; u_g = 2 u_w - u  (derivatives: along n kept, along t flipped)
  T rho = W[0], ir = T(1) / rho;
  T u = W[1] * ir, v = W[2] * ir;
  T ke = T(0.5) * (u * u + v * v);
  T p = (gamma - T(1)) * (W[3] - rho * ke);
  T ug = T(2) * wn - u, vg = T(2) * wt - v;
  T keg = T(0.5) * (ug * ug + vg * vg);
  Wg[0] = rho; Wg[1] = rho * ug; Wg[2] = rho * vg; Wg[3] = p / (gamma - T(1)) + rho * keg;
  const T *D[2] = { dn, dt };
  T *G[2] = { dng, dtg };
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    T dr = D[b][0];
    T du = (D[b][1] - u * dr) * ir, dv = (D[b][2] - v * dr) * ir;
    T dp = (gamma - T(1)) * (D[b][3] - ke * dr - rho * (u * du + v * dv));
    T s = b == 0 ? T(-1) : T(1);   // scalars: normal derivative flips
    T drg = s * dr, dpg = s * dp;
    T dug = -s * du, dvg = -s * dv;  // velocity: tangential derivative flips
    G[b][0] = drg;
    G[b][1] = ug * drg + rho * dug;
    G[b][2] = vg * drg + rho * dvg;
    G[b][3] = dpg / (gamma - T(1)) + keg * drg + rho * (ug * dug + vg * dvg);
  }
}

// 1-D Riemann invariants normal to the face between the interior state W
// and the free stream (rho_e, une, ute, pe); local frame.
template <typename T>
__device__ __forceinline__ void ghost_farfield(T gamma, T re, T une, T ute, T pe, const T W[NV], T Wg[NV]) {
  T ri = W[0], ir = T(1) / ri;
  T uni = W[1] * ir, uti = W[2] * ir;
  T pi = (gamma - T(1)) * (W[3] - T(0.5) * ri * (uni * uni + uti * uti));
  T ci = d_sqrt(gamma * pi / ri), ce = d_sqrt(gamma * pe / re);
  T rb, unb, utb, pb;
  if (uni <= -ci) {
    rb = re; unb = une; utb = ute; pb = pe;
  } else if (uni >= ci) {
    rb = ri; unb = uni; utb = uti; pb = pi;
  } else {
    T Rp = uni + T(2) * ci / (gamma - T(1));
    T Rm = une - T(2) * ce / (gamma - T(1));
    unb = T(0.5) * (Rp + Rm);
    T cb = T(0.25) * (gamma - T(1)) * (Rp - Rm);
    T s;
    if (unb >= T(0)) { s = pi / pow(ri, gamma); utb = uti; }
    else { s = pe / pow(re, gamma); utb = ute; }
    rb = pow(cb * cb / (gamma * s), T(1) / (gamma - T(1)));
    pb = rb * cb * cb / gamma;
  }
  Wg[0] = rb; Wg[1] = rb * unb; Wg[2] = rb * utb;
  Wg[3] = pb / (gamma - T(1)) + T(0.5) * rb * (unb * unb + utb * utb);
}

}  // namespace dev
}  // namespace cgks
