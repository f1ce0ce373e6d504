// Device-side gas-kinetic physics of the compact GKS in 3-D (Sections 2.2-2.3
// and 3 of Ji, Shyy & Xu, arXiv:2109.09965).
//
// Local face frame: e1 = n, e2 = t1, e3 = t2 (right-handed, precomputed per
// face).  Conservative variables (rho, rho u_n, rho u_t1, rho u_t2, rho E).
// Moments normalised by rho; K = (5 - 3 gamma)/(gamma - 1) internal degrees
// of freedom, so <xi^2> = K/(2 lambda), <xi^4> = K(K+2)/(4 lambda^2).
// kc holds K, c2K = 2/(K+3), c4K = 4/(K+3).  The micro-slope solve
// <a psi> = b uses its closed form.
#pragma once

#include "cgks_physics.cuh"

namespace cgks {
namespace dev3 {

using dev::KC;
using dev::d_sqrt;
using dev::d_rsqrt;
using dev::half_moments;
constexpr int NV = 5;

// the face frame: n, t1, t2 as three rows
template <typename T>
struct Frame {
  T e[3][3];
};

template <typename T>
__device__ __forceinline__ void rot_in(const Frame<T> &F, const T g[NV], T l[NV]) {
  l[0] = g[0];
  l[4] = g[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) l[1 + a] = F.e[a][0] * g[1] + F.e[a][1] * g[2] + F.e[a][2] * g[3];
}
template <typename T>
__device__ __forceinline__ void rot_out(const Frame<T> &F, const T l[NV], T g[NV]) {
  g[0] = l[0];
  g[4] = l[4];
#pragma unroll
  for (int d = 0; d < 3; ++d) g[1 + d] = F.e[0][d] * l[1] + F.e[1][d] * l[2] + F.e[2][d] * l[3];
}

template <typename T>
struct Maxw {
  T rho, ir, U, V, W, lam, i2l;
};
template <typename T>
__device__ __forceinline__ Maxw<T> maxw(const T Wc[NV], T c2K) {
  // lambda = (K+3) rho / (4 (rho E - rho |U|^2 / 2)), c2K = 2 / (K+3)
  Maxw<T> g;
  g.rho = Wc[0];
  g.ir = T(1) / Wc[0];
  g.U = Wc[1] * g.ir;
  g.V = Wc[2] * g.ir;
  g.W = Wc[3] * g.ir;
  T eps = Wc[4] - T(0.5) * g.rho * (g.U * g.U + g.V * g.V + g.W * g.W);
  g.i2l = c2K * eps * g.ir;
  g.lam = T(0.5) / g.i2l;
  return g;
}

template <typename T>
struct Mom {
  T mu[7], mv[6], mw[6], x2, x4;
};
template <typename T>
__device__ __forceinline__ void full_moments(const Maxw<T> &g, T K, Mom<T> &m) {
  const T i2l = g.i2l;
  m.mu[0] = T(1); m.mu[1] = g.U;
  m.mv[0] = T(1); m.mv[1] = g.V;
  m.mw[0] = T(1); m.mw[1] = g.W;
#pragma unroll
  for (int k = 2; k < 7; ++k) m.mu[k] = g.U * m.mu[k - 1] + T(k - 1) * i2l * m.mu[k - 2];
#pragma unroll
  for (int k = 2; k < 6; ++k) {
    m.mv[k] = g.V * m.mv[k - 1] + T(k - 1) * i2l * m.mv[k - 2];
    m.mw[k] = g.W * m.mw[k - 1] + T(k - 1) * i2l * m.mw[k - 2];
  }
  m.x2 = K * i2l;
  m.x4 = K * (K + T(2)) * i2l * i2l;
}

// <u^a v^b w^c xi^(2d) s>, s = s0 + s1 u + s2 v + s3 w + s4 (u^2+v^2+w^2+xi^2)/2
template <typename T>
__device__ __forceinline__ T mslope(const Mom<T> &m, int a, int b, int c, int d, const T s[NV]) {
  const T xd = d == 0 ? T(1) : (d == 1 ? m.x2 : m.x4);
  const T xd1 = d == 0 ? m.x2 : m.x4;
  const T base = m.mu[a] * m.mv[b] * m.mw[c];
  T r = (s[0] * base + s[1] * m.mu[a + 1] * m.mv[b] * m.mw[c] + s[2] * m.mu[a] * m.mv[b + 1] * m.mw[c] +
         s[3] * m.mu[a] * m.mv[b] * m.mw[c + 1]) * xd;
  r += T(0.5) * s[4] *
       ((m.mu[a + 2] * m.mv[b] * m.mw[c] + m.mu[a] * m.mv[b + 2] * m.mw[c] + m.mu[a] * m.mv[b] * m.mw[c + 2]) * xd +
        base * xd1);
  return r;
}
// vector <u^a v^b w^c s psi>
template <typename T>
__device__ __forceinline__ void gpsi(const Mom<T> &m, int a, int b, int c, const T s[NV], T out[NV]) {
  out[0] = mslope(m, a, b, c, 0, s);
  out[1] = mslope(m, a + 1, b, c, 0, s);
  out[2] = mslope(m, a, b + 1, c, 0, s);
  out[3] = mslope(m, a, b, c + 1, 0, s);
  out[4] = T(0.5) * (mslope(m, a + 2, b, c, 0, s) + mslope(m, a, b + 2, c, 0, s) + mslope(m, a, b, c + 2, 0, s) +
                     mslope(m, a, b, c, 1, s));
}

// Closed-form <s psi> = b (b divided by rho): q = |U|^2 + (K+3)/(2 lambda),
// tl = 2 lambda, l2 = 4 lambda^2 / (K+3).
template <typename T>
struct SlopeSolver {
  T U, V, W, q, tl, l2;
};
template <typename T>
__device__ __forceinline__ SlopeSolver<T> slope_solver(const Maxw<T> &g, const KC<T> &kc) {
  SlopeSolver<T> S;
  S.U = g.U; S.V = g.V; S.W = g.W;
  S.q = g.U * g.U + g.V * g.V + g.W * g.W + (kc.K + T(3)) * g.i2l;
  S.tl = T(2) * g.lam;
  S.l2 = kc.c4K * g.lam * g.lam;
  return S;
}
template <typename T>
__device__ __forceinline__ void micro_slope(const SlopeSolver<T> &S, const T b[NV], T s[NV]) {
  const T R5 = T(2) * b[4] - S.q * b[0];
  const T R2 = b[1] - S.U * b[0], R3 = b[2] - S.V * b[0], R4 = b[3] - S.W * b[0];
  s[4] = S.l2 * (R5 - T(2) * (S.U * R2 + S.V * R3 + S.W * R4));
  s[3] = S.tl * R4 - S.W * s[4];
  s[2] = S.tl * R3 - S.V * s[4];
  s[1] = S.tl * R2 - S.U * s[4];
  s[0] = b[0] - S.U * s[1] - S.V * s[2] - S.W * s[3] - T(0.5) * s[4] * S.q;
}

// Smooth GKS flux at one Gauss point, Eq. (2nd-smooth-flux), local frame:
//   f = g^c - tau (a_n u + a_t1 v + a_t2 w + A) g^c + A g^c t,  tau = mu / p^c
// W^c from the half-range moments of g^l (u > 0) and g^r (u < 0); the
// equilibrium slopes from the mean of the side derivatives (dl[k], dr[k]:
// derivatives along e_k as local-frame vectors) plus, along n,
// ajump * (W^r - W^l).
template <typename T>
__device__ __forceinline__ void gks_point_local(const KC<T> &kc, T mu_visc, T ajump, const T Wl[NV],
                                                const T Wr[NV], const T dl[3][NV], const T dr[3][NV], T F0[NV],
                                                T F1[NV], T Wc[NV], T Wt[NV]) {
  const T K = kc.K, c2K = kc.c2K;
  Maxw<T> gl = maxw(Wl, c2K), gr = maxw(Wr, c2K);
  T ml[3], mr[3];
  half_moments<T, 2>(gl.U, gl.i2l, d_sqrt(gl.lam), d_rsqrt(gl.lam) * T(dev::kInvSqrtPi), +1, ml);
  half_moments<T, 2>(gr.U, gr.i2l, d_sqrt(gr.lam), d_rsqrt(gr.lam) * T(dev::kInvSqrtPi), -1, mr);
  const T el = gl.V * gl.V + gl.W * gl.W + (K + T(2)) * gl.i2l;
  const T er = gr.V * gr.V + gr.W * gr.W + (K + T(2)) * gr.i2l;
  Wc[0] = gl.rho * ml[0] + gr.rho * mr[0];
  Wc[1] = gl.rho * ml[1] + gr.rho * mr[1];
  Wc[2] = gl.rho * ml[0] * gl.V + gr.rho * mr[0] * gr.V;
  Wc[3] = gl.rho * ml[0] * gl.W + gr.rho * mr[0] * gr.W;
  Wc[4] = gl.rho * T(0.5) * (ml[2] + ml[0] * el) + gr.rho * T(0.5) * (mr[2] + mr[0] * er);
  Maxw<T> gc = maxw(Wc, c2K);
  Mom<T> m;
  full_moments(gc, K, m);
  SlopeSolver<T> SS = slope_solver(gc, kc);
  T b[3][NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    b[0][v] = (T(0.5) * (dl[0][v] + dr[0][v]) + ajump * (Wr[v] - Wl[v])) * gc.ir;
    b[1][v] = T(0.5) * (dl[1][v] + dr[1][v]) * gc.ir;
    b[2][v] = T(0.5) * (dl[2][v] + dr[2][v]) * gc.ir;
  }
  T an[NV], a1[NV], a2[NV], A[NV], bA[NV], g0[NV], g1[NV], g2[NV];
  micro_slope(SS, b[0], an);
  micro_slope(SS, b[1], a1);
  micro_slope(SS, b[2], a2);
  gpsi(m, 1, 0, 0, an, g0);
  gpsi(m, 0, 1, 0, a1, g1);
  gpsi(m, 0, 0, 1, a2, g2);
#pragma unroll
  for (int v = 0; v < NV; ++v) bA[v] = -(g0[v] + g1[v] + g2[v]);
  micro_slope(SS, bA, A);
  const T tau = mu_visc * SS.tl * gc.ir;   // mu / p^c, p^c = rho / (2 lambda)
  T gAu[NV], gA[NV], gn2[NV], g1u[NV], g2u[NV];
  gpsi(m, 1, 0, 0, A, gAu);
  gpsi(m, 0, 0, 0, A, gA);
  gpsi(m, 2, 0, 0, an, gn2);
  gpsi(m, 1, 1, 0, a1, g1u);
  gpsi(m, 1, 0, 1, a2, g2u);
  const T feq[NV] = { m.mu[1], m.mu[2], m.mu[1] * gc.V, m.mu[1] * gc.W,
                      T(0.5) * (m.mu[3] + m.mu[1] * (m.mv[2] + m.mw[2] + m.x2)) };
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    F0[v] = gc.rho * (feq[v] - tau * (gn2[v] + g1u[v] + g2u[v] + gAu[v]));
    F1[v] = gc.rho * gAu[v];
    Wt[v] = gc.rho * gA[v];
  }
}

// ---------------- full flux, Eq. (2nd-flux), 3-D ----------------
// u-moments over a half range (sgn +1: u > 0, -1: u < 0), v, w, xi full
template <typename T>
__device__ __forceinline__ void half_table(const Maxw<T> &g, T K, int sgn, Mom<T> &m) {
  half_moments<T, 6>(g.U, g.i2l, d_sqrt(g.lam), d_rsqrt(g.lam) * T(dev::kInvSqrtPi), sgn, m.mu);
  m.mv[0] = T(1); m.mv[1] = g.V;
  m.mw[0] = T(1); m.mw[1] = g.W;
#pragma unroll
  for (int k = 2; k < 6; ++k) {
    m.mv[k] = g.V * m.mv[k - 1] + T(k - 1) * g.i2l * m.mv[k - 2];
    m.mw[k] = g.W * m.mw[k - 1] + T(k - 1) * g.i2l * m.mw[k - 2];
  }
  m.x2 = K * g.i2l;
  m.x4 = K * (K + T(2)) * g.i2l * g.i2l;
}

// slopes along the three local axes from the derivatives d[k] (local
// vectors), and A from <A + a.u> = 0; mf the full-range table of g
template <typename T>
__device__ __forceinline__ void maxw_slopes(const Maxw<T> &g, const Mom<T> &mf, const KC<T> &kc, const T d[3][NV],
                                            T a[3][NV], T A[NV]) {
  SlopeSolver<T> SS = slope_solver(g, kc);
  T b[NV], g0[NV], g1[NV], g2[NV];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int v = 0; v < NV; ++v) b[v] = d[k][v] * g.ir;
    micro_slope(SS, b, a[k]);
  }
  gpsi(mf, 1, 0, 0, a[0], g0);
  gpsi(mf, 0, 1, 0, a[1], g1);
  gpsi(mf, 0, 0, 1, a[2], g2);
#pragma unroll
  for (int v = 0; v < NV; ++v) b[v] = -(g0[v] + g1[v] + g2[v]);
  micro_slope(SS, b, A);
}

// rho-weighted flux moments Q = (<u psi>, <u a.u psi>, <u A psi>) and state
// moments P = (<psi>, <a.u psi>, <A psi>) of one piece
template <typename T>
__device__ __forceinline__ void piece(T rho, const Mom<T> &m, const T a[3][NV], const T A[NV], T Q[3][NV],
                                      T P[3][NV]) {
  const T one[NV] = { T(1), T(0), T(0), T(0), T(0) };
  T x[NV], y[NV], z[NV];
  gpsi(m, 1, 0, 0, one, x);
#pragma unroll
  for (int v = 0; v < NV; ++v) Q[0][v] = rho * x[v];
  gpsi(m, 2, 0, 0, a[0], x);
  gpsi(m, 1, 1, 0, a[1], y);
  gpsi(m, 1, 0, 1, a[2], z);
#pragma unroll
  for (int v = 0; v < NV; ++v) Q[1][v] = rho * (x[v] + y[v] + z[v]);
  gpsi(m, 1, 0, 0, A, x);
#pragma unroll
  for (int v = 0; v < NV; ++v) Q[2][v] = rho * x[v];
  gpsi(m, 0, 0, 0, one, x);
#pragma unroll
  for (int v = 0; v < NV; ++v) P[0][v] = rho * x[v];
  gpsi(m, 1, 0, 0, a[0], x);
  gpsi(m, 0, 1, 0, a[1], y);
  gpsi(m, 0, 0, 1, a[2], z);
#pragma unroll
  for (int v = 0; v < NV; ++v) P[1][v] = rho * (x[v] + y[v] + z[v]);
  gpsi(m, 0, 0, 0, A, x);
#pragma unroll
  for (int v = 0; v < NV; ++v) P[2][v] = rho * x[v];
}

template <typename T>
__device__ __forceinline__ void full_sum(T c1, T c2, T c3, T e, T te, T tau, const T X0[3][NV], const T XL[3][NV],
                                         const T XR[3][NV], T out[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v)
    out[v] = c1 * X0[0][v] + c2 * X0[1][v] + c3 * X0[2][v] +
             e * ((XL[0][v] + XR[0][v]) - tau * (XL[1][v] + XR[1][v]) - tau * (XL[2][v] + XR[2][v])) -
             te * (XL[1][v] + XR[1][v]);
}

// Full gas-kinetic flux at one Gauss point, Eq. (2nd-flux), 3-D, local
// frame; same construction as the 2-D dev::gks_full_point_local (tau_n in
// the exponentials, time integrals over [0, dt] and [0, dt/2] fitted to
// F0 + t F1, the interface state by the line through t = dt/2 and dt).
template <typename T>
__device__ void gks_full_point_local(const KC<T> &kc, T mu_visc, T ajump, T dt, T tc1, T tc2, const T Wl[NV],
                                     const T Wr[NV], const T dl[3][NV], const T dr[3][NV], T F0[NV], T F1[NV],
                                     T Wc[NV], T Wt[NV]) {
  const T K = kc.K, c2K = kc.c2K;
  Maxw<T> gl = maxw(Wl, c2K), gr = maxw(Wr, c2K);
  T Q0[3][NV], P0[3][NV], QL[3][NV], PL[3][NV], QR[3][NV], PR[3][NV];
  {
    T al[3][NV], Al[NV];
    Mom<T> m;
    full_moments(gl, K, m);
    maxw_slopes(gl, m, kc, dl, al, Al);
    half_table(gl, K, +1, m);
    piece(gl.rho, m, al, Al, QL, PL);
  }
  {
    T ar[3][NV], Ar[NV];
    Mom<T> m;
    full_moments(gr, K, m);
    maxw_slopes(gr, m, kc, dr, ar, Ar);
    half_table(gr, K, -1, m);
    piece(gr.rho, m, ar, Ar, QR, PR);
  }
  T W0[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) W0[v] = PL[0][v] + PR[0][v];
  Maxw<T> gc = maxw(W0, c2K);
  {
    T d[3][NV], ac[3][NV], Ac[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      d[0][v] = T(0.5) * (dl[0][v] + dr[0][v]) + ajump * (Wr[v] - Wl[v]);
      d[1][v] = T(0.5) * (dl[1][v] + dr[1][v]);
      d[2][v] = T(0.5) * (dl[2][v] + dr[2][v]);
    }
    Mom<T> m;
    full_moments(gc, K, m);
    maxw_slopes(gc, m, kc, d, ac, Ac);
    piece(gc.rho, m, ac, Ac, Q0, P0);
  }
  const T tau = mu_visc * T(2) * gc.lam * gc.ir;
  const T pl = gl.rho * gl.i2l, pr = gr.rho * gr.i2l;
  const T taun = tau + tc1 * dt + tc2 * dt * fabs(pl - pr) / (pl + pr);
  T Fd[NV], Fh[NV], Wd[NV], Wh[NV];
#pragma unroll 1
  for (int k = 0; k < 2; ++k) {
    const T t = k == 0 ? dt : T(0.5) * dt;
    const T e = taun > T(0) ? dev::d_exp(-t / taun) : T(0);
    const T om = taun > T(0) ? -dev::d_expm1(-t / taun) : T(1);
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

// cell primitives of the low level: rho, u, v, w, p, 1/(2 lambda),
// sqrt(lambda), 1/sqrt(pi lambda), c, 1/rho
constexpr int NPRIM = 10;
template <typename T>
struct Prim {
  T rho, u, v, w, p, i2l, sl, isp, c, ir;
};
template <typename T>
__device__ __forceinline__ Prim<T> prim_of(const T W[NV], T gamma, const KC<T> &kc) {
  Prim<T> q;
  q.rho = W[0];
  q.ir = T(1) / W[0];
  q.u = W[1] * q.ir;
  q.v = W[2] * q.ir;
  q.w = W[3] * q.ir;
  const T eps = W[4] - T(0.5) * q.rho * (q.u * q.u + q.v * q.v + q.w * q.w);
  q.p = (gamma - T(1)) * eps;
  q.i2l = kc.c2K * eps * q.ir;
  const T lam = T(0.5) / q.i2l;
  q.sl = d_sqrt(lam);
  q.isp = d_rsqrt(lam) * T(dev::kInvSqrtPi);
  q.c = d_sqrt(gamma * q.p * q.ir);
  return q;
}

// first-order KFVS flux of two cell states (local velocities), local frame
template <typename T>
__device__ __forceinline__ void kfvs(T K, T rl, T unl, T v1l, T v2l, T i2ll, T sll, T ispl, T rr, T unr, T v1r,
                                     T v2r, T i2lr, T slr, T ispr, T F[NV]) {
  T ml[4], mr[4];
  half_moments<T, 3>(unl, i2ll, sll, ispl, +1, ml);
  half_moments<T, 3>(unr, i2lr, slr, ispr, -1, mr);
  const T el = v1l * v1l + v2l * v2l + (K + T(2)) * i2ll;
  const T er = v1r * v1r + v2r * v2r + (K + T(2)) * i2lr;
  F[0] = rl * ml[1] + rr * mr[1];
  F[1] = rl * ml[2] + rr * mr[2];
  F[2] = rl * ml[1] * v1l + rr * mr[1] * v1r;
  F[3] = rl * ml[1] * v2l + rr * mr[1] * v2r;
  F[4] = rl * T(0.5) * (ml[3] + ml[1] * el) + rr * T(0.5) * (mr[3] + mr[1] * er);
}

template <typename T>
__device__ __forceinline__ void euler_flux(T gamma, const T W[NV], const T n[3], T F[NV]) {
  const T ir = T(1) / W[0];
  const T u = W[1] * ir, v = W[2] * ir, w = W[3] * ir;
  const T p = (gamma - T(1)) * (W[4] - T(0.5) * W[0] * (u * u + v * v + w * w));
  const T un = u * n[0] + v * n[1] + w * n[2];
  F[0] = W[0] * un;
  F[1] = W[1] * un + p * n[0];
  F[2] = W[2] * un + p * n[1];
  F[3] = W[3] * un + p * n[2];
  F[4] = (W[4] + p) * un;
}

// F_n(W + dW) - F_n(W), every term proportional to the increment
// (see the 2-D version): base velocity (u, v, w) and pressure p.
template <typename T>
__device__ __forceinline__ void euler_flux_delta(T gamma, const T W[NV], T u, T v, T w, T p, const T dW[NV],
                                                 const T n[3], T dF[NV]) {
  const T rho = W[0], r1 = W[0] + dW[0];
  const T inv = T(1) / (rho * r1);
  const T mn = W[1] * n[0] + W[2] * n[1] + W[3] * n[2], dmn = dW[1] * n[0] + dW[2] * n[1] + dW[3] * n[2];
  const T un = u * n[0] + v * n[1] + w * n[2];
  const T dun = (rho * dmn - mn * dW[0]) * inv;
  const T un1 = un + dun;
  const T m2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  const T dm2 = T(2) * (W[1] * dW[1] + W[2] * dW[2] + W[3] * dW[3]) + dW[1] * dW[1] + dW[2] * dW[2] + dW[3] * dW[3];
  const T dke = T(0.5) * (rho * dm2 - m2 * dW[0]) * inv;
  const T dp = (gamma - T(1)) * (dW[4] - dke);
  dF[0] = dmn;
  dF[1] = dW[1] * un1 + W[1] * dun + dp * n[0];
  dF[2] = dW[2] * un1 + W[2] * dun + dp * n[1];
  dF[3] = dW[3] * un1 + W[3] * dun + dp * n[2];
  dF[4] = (dW[4] + dp) * un1 + (W[4] + p) * dun;
}

// ---- boundary ghosts, local frame.  d[k]: derivative along e_k (local
// vector).  Mirror across the wall: normal coordinate flips.
template <typename T>
__device__ __forceinline__ void ghost_slip(const T W[NV], const T d[3][NV], T Wg[NV], T dg[3][NV]) {
  // rho, rho u_t1, rho u_t2, rho E even; rho u_n odd
  Wg[0] = W[0]; Wg[1] = -W[1]; Wg[2] = W[2]; Wg[3] = W[3]; Wg[4] = W[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T s = k == 0 ? T(-1) : T(1);   // derivative along n flips
#pragma unroll
    for (int v = 0; v < NV; ++v) dg[k][v] = (v == 1 ? -s : s) * d[k][v];
  }
}

template <typename T>
__device__ __forceinline__ void ghost_noslip(T gamma, const T uw[3], const T W[NV], const T d[3][NV], T Wg[NV],
                                             T dg[3][NV]) {
  // rho, p even; u_g = 2 u_w - u (local components)
  const T rho = W[0], ir = T(1) / rho;
  const T u[3] = { W[1] * ir, W[2] * ir, W[3] * ir };
  const T ke = T(0.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const T p = (gamma - T(1)) * (W[4] - rho * ke);
  T ug[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) ug[a] = T(2) * uw[a] - u[a];
  const T keg = T(0.5) * (ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2]);
  Wg[0] = rho; Wg[1] = rho * ug[0]; Wg[2] = rho * ug[1]; Wg[3] = rho * ug[2];
  Wg[4] = p / (gamma - T(1)) + rho * keg;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T dr = d[k][0];
    T du[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) du[a] = (d[k][1 + a] - u[a] * dr) * ir;
    const T dp = (gamma - T(1)) * (d[k][4] - ke * dr - rho * (u[0] * du[0] + u[1] * du[1] + u[2] * du[2]));
    const T s = k == 0 ? T(-1) : T(1);   // scalars: normal derivative flips
    const T drg = s * dr, dpg = s * dp;
    T dug[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) dug[a] = -s * du[a];   // velocity: tangential derivatives flip
    dg[k][0] = drg;
#pragma unroll
    for (int a = 0; a < 3; ++a) dg[k][1 + a] = ug[a] * drg + rho * dug[a];
    dg[k][4] = dpg / (gamma - T(1)) + keg * drg + rho * (ug[0] * dug[0] + ug[1] * dug[1] + ug[2] * dug[2]);
  }
}

// Riemann invariants normal to the face: interior W and free stream
// (re, une, ut1e, ut2e, pe), local frame
template <typename T>
__device__ __forceinline__ void ghost_farfield(T gamma, T re, const T ue[3], T pe, const T W[NV], T Wg[NV]) {
  const T ri = W[0], ir = T(1) / ri;
  const T ui[3] = { W[1] * ir, W[2] * ir, W[3] * ir };
  const T pi = (gamma - T(1)) * (W[4] - T(0.5) * ri * (ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]));
  const T ci = d_sqrt(gamma * pi / ri), ce = d_sqrt(gamma * pe / re);
  T rb, ub[3], pb;
  if (ui[0] <= -ci) {
    rb = re; ub[0] = ue[0]; ub[1] = ue[1]; ub[2] = ue[2]; pb = pe;
  } else if (ui[0] >= ci) {
    rb = ri; ub[0] = ui[0]; ub[1] = ui[1]; ub[2] = ui[2]; pb = pi;
  } else {
    const T Rp = ui[0] + T(2) * ci / (gamma - T(1));
    const T Rm = ue[0] - T(2) * ce / (gamma - T(1));
    ub[0] = T(0.5) * (Rp + Rm);
    const T cb = T(0.25) * (gamma - T(1)) * (Rp - Rm);
    T s;
    if (ub[0] >= T(0)) { s = pi / pow(ri, gamma); ub[1] = ui[1]; ub[2] = ui[2]; }
    else { s = pe / pow(re, gamma); ub[1] = ue[1]; ub[2] = ue[2]; }
    rb = pow(cb * cb / (gamma * s), T(1) / (gamma - T(1)));
    pb = rb * cb * cb / gamma;
  }
  Wg[0] = rb; Wg[1] = rb * ub[0]; Wg[2] = rb * ub[1]; Wg[3] = rb * ub[2];
  Wg[4] = pb / (gamma - T(1)) + T(0.5) * rb * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
}

}  // namespace dev3
}  // namespace cgks
