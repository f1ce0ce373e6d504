// Kernels of the 3-D hot path (included by cgks_device3.cu only).
//
// One solve; cells colour-major with reverse Cuthill-McKee order inside a
// colour, faces sorted by their lower cell; structure-of-arrays
// [component][n].  Flux kernels are templated on the flux type TF (double,
// or float in the mixed path, where W, W_x, U and every accumulation into
// them stay double).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "cgks_internal.h"
#include "cgks_physics3.cuh"
#include "cgks_pdl.cuh"
#include "cgks_shapes.h"
#include "cgks_vec.cuh"

namespace cgks {
namespace kern3 {

namespace D3 = cgks::dev3;
constexpr int NV = 5;
constexpr int kCellBlock = 256;
constexpr int kSweepLanes = 8;                     // lanes per cell (6 face slots)
constexpr int kFO = 4 * NV;                        // face outputs of the high level: F0, F1, Wc, Wt
constexpr int kLo = 8;                             // low-level face run: flux (NV), lambda_p, 2 pad
constexpr int kEu = 6;                             // Euler flux cache run of one face side: NV, 1 pad
constexpr int kBadState = 1;

template <typename T>
__host__ __device__ constexpr bool is_f32() { return std::is_same<T, float>::value; }

template <typename T>
struct ParamsT {
  T gamma, K, cfl_hi, cfl_lo, mu;
  D3::KC<T> kc;
  const int *bc_kind;          // [16]
  const T *bc_uw;              // [16][3] wall velocity (global)
  const T *bc_rho, *bc_u, *bc_p;  // [16], [16][3], [16] free stream (global)
  int flux_lo;                    // low-level flux: CGKS_FLUX_KFVS or CGKS_FLUX_LF
  T tau_c1, tau_c2;               // numerical collision time constants of the full flux
  T weno_eps, weno_g0;            // compact WENO epsilon (0: linear weights), linear weight of P2
  int lo_viscous;                 // 1: the low-order residual carries a first-order viscous flux
};

template <typename T>
struct MeshT {
  int nc, nf;
  const T *vol, *ivol, *ih, *hdt, *m2, *op;       // m2 [6][nc], op [27*9][nc]
  const T *fe, *fS, *fjump, *fw, *fxi;            // fe [9][nf] (n, t1, t2), fw [4][nf], fxi [24][nf]
  const T *fidl;                                  // 1/delta: centre distance along n (boundary: twice to the face)
  const T *sn, *shs;                              // [6*3][nc] outward normal per slot, [6][nc] S/2
  const int *fng, *cface, *cnbr, *fc0, *fc1;
};

struct Ctl {
  double dt_fixed;
  int res_ctr, pad_;
};

__device__ __forceinline__ double dt_of(const Ctl *ctl, const unsigned long long *dt_bits, double cfl) {
  if (ctl->dt_fixed > 0.0) return ctl->dt_fixed;
  return cfl * __longlong_as_double(static_cast<long long>(*dt_bits));
}
__device__ __forceinline__ bool state_ok(double gamma, const double w[NV]) {
  const double p = (gamma - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0]);
  return w[0] > 0.0 && p > 0.0 && isfinite(w[0]) && isfinite(p) && isfinite(w[1]) && isfinite(w[2]) &&
         isfinite(w[3]);
}

__device__ __forceinline__ void block_sum2(double a, double b, double *out2) {
  __shared__ double sa[32], sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { out2[0] = a; out2[1] = b; }
  }
}

template <typename T>
__device__ __forceinline__ D3::Frame<T> frame_of(const MeshT<T> &m, int f) {
  D3::Frame<T> F;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int d = 0; d < 3; ++d) F.e[a][d] = m.fe[(3 * a + d) * m.nf + f];
  return F;
}

// ------------------------------------------------------------------
__global__ void k_reset_dt(Ctl *ctl, unsigned long long *dt_bits, double dt_fixed) {
  pdl_enter();
  if (threadIdx.x == 0) { *dt_bits = 0x7ff0000000000000ull; ctl->dt_fixed = dt_fixed; }
  pdl_exit();
}

// explicit step: min over cells of h / (|U| + c + 2 nu / h), h = 3|Omega| / sum S
__global__ void __launch_bounds__(kCellBlock) k_dt(MeshT<double> m, ParamsT<double> P, const double *__restrict__ W,
                                                   unsigned long long *dt_bits) {
  pdl_enter();
  __shared__ double wmin[kCellBlock / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double d = INFINITY;
  if (i < m.nc) {
    const int n = m.nc;
    const double rho = W[i], ir = 1.0 / rho;
    const double u = W[n + i] * ir, v = W[2 * n + i] * ir, w = W[3 * n + i] * ir;
    const double p = (P.gamma - 1.0) * (W[4 * n + i] - 0.5 * rho * (u * u + v * v + w * w));
    const double hh = m.hdt[i];
    const double speed = sqrt(u * u + v * v + w * w) + sqrt(P.gamma * p * ir) + 2.0 * (P.mu * ir) / hh;
    d = hh / speed;
  }
  for (int o = 16; o > 0; o >>= 1) d = fmin(d, __shfl_down_sync(0xffffffffu, d, o));
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kCellBlock / 32; ++k) d = fmin(d, wmin[k]);
    if (d < INFINITY) atomicMin(dt_bits, static_cast<unsigned long long>(__double_as_longlong(d)));
  }
  pdl_exit();
}

// wall ghost of a state and its gradient (global), through the face frame
template <typename T>
__device__ __forceinline__ void wall_ghost(const ParamsT<T> &P, int tag, const D3::Frame<T> &F, const T w[NV],
                                           const T g[3][NV], T wg[NV], T gg[3][NV]) {
  T wl[NV], dl[3][NV], wgl[NV], dgl[3][NV];
  D3::rot_in(F, w, wl);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T t[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) t[v] = F.e[k][0] * g[0][v] + F.e[k][1] * g[1][v] + F.e[k][2] * g[2][v];
    D3::rot_in(F, t, dl[k]);
  }
  if (P.bc_kind[tag] == CGKS_BC_SLIP) {
    D3::ghost_slip(wl, dl, wgl, dgl);
  } else {
    T uw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      uw[a] = F.e[a][0] * P.bc_uw[3 * tag] + F.e[a][1] * P.bc_uw[3 * tag + 1] + F.e[a][2] * P.bc_uw[3 * tag + 2];
    D3::ghost_noslip(P.gamma, uw, wl, dl, wgl, dgl);
  }
  D3::rot_out(F, wgl, wg);
  T gk[3][NV];
#pragma unroll
  for (int k = 0; k < 3; ++k) D3::rot_out(F, dgl[k], gk[k]);
  // global gradient: grad_d = sum_k e_k[d] (derivative along e_k)
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < NV; ++v) gg[d][v] = F.e[0][d] * gk[0][v] + F.e[1][d] * gk[1][v] + F.e[2][d] * gk[2][v];
}

template <typename T>
__device__ __forceinline__ void farfield_ghost(const ParamsT<T> &P, int tag, const D3::Frame<T> &F, const T wl[NV],
                                               T wg[NV]) {
  T ue[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    ue[a] = F.e[a][0] * P.bc_u[3 * tag] + F.e[a][1] * P.bc_u[3 * tag + 1] + F.e[a][2] * P.bc_u[3 * tag + 2];
  D3::ghost_farfield(P.gamma, P.bc_rho[tag], ue, P.bc_p[tag], wl, wg);
}

// Compact WENO (conservative variables), 3-D form of the 2-D weno_combine:
// candidates P2 (c) and the nk linear polynomials h g.(xi, eta, zeta) of the
// mean gradients of the cell and its face neighbours (lin[k][d][v]).  beta:
// cell mean of the squared first derivatives (centroid value squared plus
// the quadratic form of the cell's second moments M = m2) plus the squared
// second derivatives, each multi-index once.  w ~ gamma / (beta + eps)^2,
// gamma_0 = g0, the rest (1 - g0)/nk; result
// (w_0 / gamma_0)(P2 - sum gamma_k P1_k) + sum w_k P1_k.
template <typename T>
__device__ __forceinline__ void weno_combine3(const ParamsT<T> &P, const T M[6], int nk, const T lin[7][3][NV],
                                              T c[kNM3][NV]) {
  const T g0 = P.weno_g0, eps = P.weno_eps;
  const T gk = (T(1) - g0) / T(nk);
  // symmetric M: xx xy xz yy yz zz
  const T Mx[3][3] = { { M[0], M[1], M[2] }, { M[1], M[3], M[4] }, { M[2], M[4], M[5] } };
  for (int v = 0; v < NV; ++v) {
    const T q[kNM3] = { c[0][v], c[1][v], c[2][v], c[3][v], c[4][v], c[5][v], c[6][v], c[7][v], c[8][v] };
    const T G[3][3] = { { T(2) * q[3], q[4], q[5] }, { q[4], T(2) * q[6], q[7] }, { q[5], q[7], T(2) * q[8] } };
    T b0 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    for (int d = 0; d < 3; ++d)
      for (int a = 0; a < 3; ++a)
        for (int e = 0; e < 3; ++e) b0 += G[d][a] * Mx[a][e] * G[d][e];
    b0 += T(4) * q[3] * q[3] + q[4] * q[4] + q[5] * q[5] + T(4) * q[6] * q[6] + q[7] * q[7] + T(4) * q[8] * q[8];
    const T w0 = g0 / ((b0 + eps) * (b0 + eps));
    T ws = w0, wk[7];
    T l[3] = { T(0), T(0), T(0) };
    for (int k = 0; k < 7; ++k) {
      if (k >= nk) break;
      const T b = lin[k][0][v] * lin[k][0][v] + lin[k][1][v] * lin[k][1][v] + lin[k][2][v] * lin[k][2][v];
      wk[k] = gk / ((b + eps) * (b + eps));
      ws += wk[k];
      for (int d = 0; d < 3; ++d) l[d] += gk * lin[k][d][v];
    }
    const T iws = T(1) / ws;
    const T f0 = w0 * iws / g0;
    T sel[3] = { T(0), T(0), T(0) };
    for (int k = 0; k < 7; ++k) {
      if (k >= nk) break;
      for (int d = 0; d < 3; ++d) sel[d] += wk[k] * iws * lin[k][d][v];
    }
    for (int d = 0; d < 3; ++d) c[d][v] = f0 * (q[d] - l[d]) + sel[d];
    for (int r = 3; r < kNM3; ++r) c[r][v] = f0 * q[r];
  }
}

// K1: compact quadratic per cell: coef[(q*5 + v)][n], 9 monomials
template <typename T, bool WENO>
__device__ __forceinline__ void recon_at(const MeshT<T> &m, const ParamsT<T> &P, const T *__restrict__ W,
                                         const T *__restrict__ Wx, T *__restrict__ coef,
                                         const unsigned char *__restrict__ wenok, const int i) {
  const int n = m.nc;
  T wi[NV], gi[3][NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    wi[v] = W[v * n + i];
#pragma unroll
    for (int d = 0; d < 3; ++d) gi[d][v] = Wx[(d * NV + v) * n + i];
  }
  T c[kNM3][NV];
#pragma unroll
  for (int q = 0; q < kNM3; ++q) {
    const T o0 = m.op[((4 * kMaxFace3) * kNM3 + q) * n + i];
    const T o1 = m.op[((4 * kMaxFace3 + 1) * kNM3 + q) * n + i];
    const T o2 = m.op[((4 * kMaxFace3 + 2) * kNM3 + q) * n + i];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[q][v] = o0 * gi[0][v] + o1 * gi[1][v] + o2 * gi[2][v];
  }
  T lin[WENO ? 7 : 1][3][NV];
  int nk = 1;
  if constexpr (WENO) {
    const T h = T(1) / m.ih[i];
    for (int v = 0; v < NV; ++v)
      for (int d = 0; d < 3; ++d) lin[0][d][v] = h * gi[d][v];
  }
  for (int s = 0; s < kMaxFace3; ++s) {
    const int fs = m.cface[s * n + i];
    if (fs == kNoFace) continue;
    const int j = m.cnbr[s * n + i];
    T b0[NV], b[3][NV];
    if (j >= 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        b0[v] = W[v * n + j] - wi[v];
#pragma unroll
        for (int d = 0; d < 3; ++d) b[d][v] = Wx[(d * NV + v) * n + j];
      }
      if constexpr (WENO) {
        const T h = T(1) / m.ih[i];
        for (int v = 0; v < NV; ++v)
          for (int d = 0; d < 3; ++d) lin[nk][d][v] = h * b[d][v];
        ++nk;
      }
    } else {
      const int f = fs >= 0 ? fs : ~fs;
      const int tag = -1 - m.fc1[f];
      if (P.bc_kind[tag] == CGKS_BC_FARFIELD) continue;
      const D3::Frame<T> F = frame_of(m, f);
      T wg[NV];
      wall_ghost(P, tag, F, wi, gi, wg, b);
#pragma unroll
      for (int v = 0; v < NV; ++v) b0[v] = wg[v] - wi[v];
    }
#pragma unroll
    for (int q = 0; q < kNM3; ++q) {
      const T o0 = m.op[((4 * s) * kNM3 + q) * n + i], o1 = m.op[((4 * s + 1) * kNM3 + q) * n + i];
      const T o2 = m.op[((4 * s + 2) * kNM3 + q) * n + i], o3 = m.op[((4 * s + 3) * kNM3 + q) * n + i];
#pragma unroll
      for (int v = 0; v < NV; ++v) c[q][v] += o0 * b0[v] + o1 * b[0][v] + o2 * b[1][v] + o3 * b[2][v];
    }
  }
  if constexpr (WENO) {
    if (wenok[i]) {
      const T M[6] = { m.m2[i], m.m2[n + i], m.m2[2 * n + i], m.m2[3 * n + i], m.m2[4 * n + i], m.m2[5 * n + i] };
      weno_combine3(P, M, nk, lin, c);
    }
  }
#pragma unroll
  for (int q = 0; q < kNM3; ++q)
#pragma unroll
    for (int v = 0; v < NV; ++v) coef[(q * NV + v) * n + i] = c[q][v];
}
template <typename T, int SH>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH))
    k_recon(MeshT<T> m, ParamsT<T> P, const T *__restrict__ W, const T *__restrict__ Wx, T *__restrict__ coef) {
  pdl_enter();
  for_items<SH>(m.nc, [&](int i) { recon_at<T, false>(m, P, W, Wx, coef, nullptr, i); });
  pdl_exit();
}
// with the compact WENO step; wenok[i] = 1 where the stencil gave a quadratic
template <typename T, int SH>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH))
    k_recon_weno(MeshT<T> m, ParamsT<T> P, const T *__restrict__ W, const T *__restrict__ Wx, T *__restrict__ coef,
                 const unsigned char *__restrict__ wenok) {
  pdl_enter();
  for_items<SH>(m.nc, [&](int i) { recon_at<T, true>(m, P, W, Wx, coef, wenok, i); });
  pdl_exit();
}

// value and gradient of cell i's quadratic at scaled offset x
template <typename T>
__device__ __forceinline__ void recon_point(const MeshT<T> &m, const T *__restrict__ W, const T *__restrict__ coef,
                                            int i, const T x[3], T val[NV], T g[3][NV]) {
  const int n = m.nc;
  const T ih = m.ih[i];
  const T a = x[0], b = x[1], e = x[2];
  const T p[6] = { a * a - m.m2[i], a * b - m.m2[n + i], a * e - m.m2[2 * n + i], b * b - m.m2[3 * n + i],
                   b * e - m.m2[4 * n + i], e * e - m.m2[5 * n + i] };
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T c[kNM3];
#pragma unroll
    for (int q = 0; q < kNM3; ++q) c[q] = coef[(q * NV + v) * n + i];
    val[v] = W[v * n + i] + c[0] * a + c[1] * b + c[2] * e + c[3] * p[0] + c[4] * p[1] + c[5] * p[2] + c[6] * p[3] +
             c[7] * p[4] + c[8] * p[5];
    g[0][v] = (c[0] + T(2) * c[3] * a + c[4] * b + c[5] * e) * ih;
    g[1][v] = (c[1] + c[4] * a + T(2) * c[6] * b + c[7] * e) * ih;
    g[2][v] = (c[2] + c[5] * a + c[7] * b + T(2) * c[8] * e) * ih;
  }
}

// K2: smooth GKS flux and interface state at the Gauss points of every face:
// out[f][k*5 + v], k = 0 F0, 1 F1, 2 Wc, 3 Wt, weighted sums, global frame:
// one run of kFO values per face (AoS), so that the cells gathering a face
// read it in one piece
template <typename T, bool FULL>
__device__ __forceinline__ void face_at(const MeshT<T> &m, const ParamsT<T> &P, const T *__restrict__ W,
                                        const T *__restrict__ coef, T *__restrict__ out, const Ctl *ctl,
                                        const unsigned long long *dt_bits, const int f) {
  const int nf = m.nf;
  T dt = T(0);
  if constexpr (FULL) dt = static_cast<T>(dt_of(ctl, dt_bits, static_cast<double>(P.cfl_hi)));
  const int c0 = m.fc0[f], c1 = m.fc1[f], ng = m.fng[f];
  const T ajump = m.fjump[f];
  const D3::Frame<T> F = frame_of(m, f);
  T acc[4][NV];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[k][v] = T(0);
  int tag = 0;
  bool farfield = false;
  T wff[NV];
  if (c1 < 0) {
    tag = -1 - c1;
    farfield = P.bc_kind[tag] == CGKS_BC_FARFIELD;
    if (farfield) {
      T wm[NV], wl[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) wm[v] = W[v * m.nc + c0];
      D3::rot_in(F, wm, wl);
      farfield_ghost(P, tag, F, wl, wff);
    }
  }
  for (int k = 0; k < ng; ++k) {
    T x0[3], wL[NV], gL[3][NV];
#pragma unroll
    for (int d = 0; d < 3; ++d) x0[d] = m.fxi[(3 * k + d) * nf + f];
    recon_point(m, W, coef, c0, x0, wL, gL);
    T wl[NV], dl[3][NV];
    D3::rot_in(F, wL, wl);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T t[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) t[v] = F.e[a][0] * gL[0][v] + F.e[a][1] * gL[1][v] + F.e[a][2] * gL[2][v];
      D3::rot_in(F, t, dl[a]);
    }
    T wr[NV], dr[3][NV];
    if (c1 >= 0) {
      T x1[3], wR[NV], gR[3][NV];
#pragma unroll
      for (int d = 0; d < 3; ++d) x1[d] = m.fxi[(12 + 3 * k + d) * nf + f];
      recon_point(m, W, coef, c1, x1, wR, gR);
      D3::rot_in(F, wR, wr);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T t[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) t[v] = F.e[a][0] * gR[0][v] + F.e[a][1] * gR[1][v] + F.e[a][2] * gR[2][v];
        D3::rot_in(F, t, dr[a]);
      }
    } else if (farfield) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        wr[v] = wff[v];
        dr[0][v] = dr[1][v] = dr[2][v] = T(0);
      }
    } else if (P.bc_kind[tag] == CGKS_BC_SLIP) {
      D3::ghost_slip(wl, dl, wr, dr);
    } else {
      T uw[3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
        uw[a] = F.e[a][0] * P.bc_uw[3 * tag] + F.e[a][1] * P.bc_uw[3 * tag + 1] + F.e[a][2] * P.bc_uw[3 * tag + 2];
      D3::ghost_noslip(P.gamma, uw, wl, dl, wr, dr);
    }
    T F0[NV], F1[NV], Wc[NV], Wt[NV];
    if constexpr (FULL)
      D3::gks_full_point_local(P.kc, P.mu, ajump, dt, P.tau_c1, P.tau_c2, wl, wr, dl, dr, F0, F1, Wc, Wt);
    else
      D3::gks_point_local(P.kc, P.mu, ajump, wl, wr, dl, dr, F0, F1, Wc, Wt);
    const T wk = m.fw[k * nf + f];
    T gq[NV];
    D3::rot_out(F, F0, gq);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[0][v] += wk * gq[v];
    D3::rot_out(F, F1, gq);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[1][v] += wk * gq[v];
    D3::rot_out(F, Wc, gq);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[2][v] += wk * gq[v];
    D3::rot_out(F, Wt, gq);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[3][v] += wk * gq[v];
  }
  T o[kFO];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int v = 0; v < NV; ++v) o[k * NV + v] = acc[k][v];
  vstore<T, kFO>(out + static_cast<size_t>(f) * kFO, o);
}
template <typename T, int SH>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH))
    k_face(MeshT<T> m, ParamsT<T> P, const T *__restrict__ W, const T *__restrict__ coef, T *__restrict__ out) {
  pdl_enter();
  for_items<SH>(m.nf, [&](int f) { face_at<T, false>(m, P, W, coef, out, nullptr, nullptr, f); });
  pdl_exit();
}
// the full flux of Eq. (2nd-flux): the same face loop, with the step's dt
template <typename T, int SH>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH))
    k_face_full(MeshT<T> m, ParamsT<T> P, const T *__restrict__ W, const T *__restrict__ coef, T *__restrict__ out,
                const Ctl *ctl, const unsigned long long *dt_bits) {
  pdl_enter();
  for_items<SH>(m.nf, [&](int f) { face_at<T, true>(m, P, W, coef, out, ctl, dt_bits, f); });
  pdl_exit();
}

enum UpdMode { kS1O2 = 0, kS2O4Stage = 1, kS2O4Final = 2, kResidual = 3 };

// K3: per cell gather of the face sums in FP64 (see the 2-D k_update):
//   R = -sum sgn S (a0 F0A + a1 F1(A, B));  W_out = W_base + dt/|Omega| R;
//   Wx_out = 1/|Omega| sum sgn S n (WcA + b1 Wt)
// The mode is a template argument so that each variant holds only the runs
// it reads: the residual reads F0 and F1 of one buffer, the stages one
// whole run, the final S2O4 stage two.
template <typename TF, int mode>
__global__ void __launch_bounds__(kCellBlock) k_update(MeshT<double> m, ParamsT<double> P,
                                                       const double *__restrict__ Wbase, const TF *__restrict__ FA,
                                                       const TF *__restrict__ FB, const Ctl *ctl,
                                                       const unsigned long long *dt_bits, int *status,
                                                       double *__restrict__ Wout, double *__restrict__ Wxout,
                                                       double *__restrict__ partial, double *__restrict__ Rout,
                                                       TF *__restrict__ Wout_m, TF *__restrict__ Wxout_m) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = m.nc;
  double num = 0.0, den = 0.0;
  if (i < n) {
    const double dt = dt_of(ctl, dt_bits, P.cfl_hi);
    double a0, a1, b1;
    switch (mode) {
      case kS1O2: a0 = 1.0; a1 = 0.5 * dt; b1 = dt; break;
      case kS2O4Stage: a0 = 0.5; a1 = 0.125 * dt; b1 = 0.5 * dt; break;
      case kS2O4Final: a0 = 1.0; a1 = dt / 6.0; b1 = dt; break;
      default: a0 = 1.0; a1 = 0.5 * dt; b1 = 0.0; break;
    }
    double R[NV] = { 0, 0, 0, 0, 0 }, g[3][NV] = { { 0 } };
    for (int s = 0; s < kMaxFace3; ++s) {
      const int fs = m.cface[s * n + i];
      if (fs == kNoFace) continue;
      const int f = fs >= 0 ? fs : ~fs;
      const double sg = fs >= 0 ? 1.0 : -1.0;
      // the slot's area and outward normal from the per-cell slot arrays
      // (coalesced; the same values as S_f and sg n_f, exactly)
      const double S = 2.0 * m.shs[s * n + i];
      const double nx = sg * m.sn[(3 * s) * n + i], ny = sg * m.sn[(3 * s + 1) * n + i],
                   nz = sg * m.sn[(3 * s + 2) * n + i];
      // the face's run of F0, F1, Wc, Wt (and the second stage's, when used);
      // the residual reads the leading F0, F1 part only
      constexpr int kRes = (2 * NV + VecOf<TF>::W - 1) / VecOf<TF>::W * VecOf<TF>::W;
      TF a[kFO], b[kFO];
      if constexpr (mode == kResidual) vload<TF, kRes>(FA + static_cast<size_t>(f) * kFO, a);
      else vload<TF, kFO>(FA + static_cast<size_t>(f) * kFO, a);
      if constexpr (mode == kS2O4Final) vload<TF, kFO>(FB + static_cast<size_t>(f) * kFO, b);
      const TF *wt = mode == kS2O4Final ? b : a;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double f1 = static_cast<double>(a[NV + v]);
        if constexpr (mode == kS2O4Final) f1 += 2.0 * static_cast<double>(b[NV + v]);
        R[v] -= sg * S * (a0 * static_cast<double>(a[v]) + a1 * f1);
        if constexpr (mode != kResidual) {
          const double wp = static_cast<double>(a[2 * NV + v]) + b1 * static_cast<double>(wt[3 * NV + v]);
          g[0][v] += sg * S * nx * wp;
          g[1][v] += sg * S * ny * wp;
          g[2][v] += sg * S * nz * wp;
        }
      }
    }
    if (Rout)
#pragma unroll
      for (int v = 0; v < NV; ++v) Rout[v * n + i] = R[v];
    if constexpr (mode != kResidual) {
      const double iv = m.ivol[i];
      double w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        w[v] = Wbase[v * n + i] + dt / m.vol[i] * R[v];
        Wout[v * n + i] = w[v];
        if (Wout_m) Wout_m[v * n + i] = static_cast<TF>(w[v]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          Wxout[(d * NV + v) * n + i] = g[d][v] * iv;
          if (Wxout_m) Wxout_m[(d * NV + v) * n + i] = static_cast<TF>(g[d][v] * iv);
        }
      }
      if (!state_ok(P.gamma, w)) atomicOr(status, kBadState);
      num = fabs(w[0] - Wbase[i]);
      den = Wbase[i];
    }
  }
  if (partial) block_sum2(num, den, &partial[2 * blockIdx.x]);
  pdl_exit();
}

__global__ void k_res_final(const double *__restrict__ partial, int nblocks, Ctl *ctl, double *hist, int cap,
                            double *last) {
  pdl_enter();
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) { a += partial[2 * k]; b += partial[2 * k + 1]; }
  __shared__ double tot[2];
  block_sum2(a, b, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double r = tot[0] / tot[1];
    last[0] = r; last[1] = tot[0]; last[2] = tot[1];
    const int c = ctl->res_ctr;
    if (hist && c < cap) hist[c] = r;
    ctl->res_ctr = c + 1;
  }
  pdl_exit();
}

// ---------------------------- low-order level ----------------------------
// Cell record of the low level, one per cell and implicit step: the
// conservative state U in the flux precision and its primitives, 16 values
// in one aligned run, so a neighbour's data costs one or two cache sectors
// instead of one sector per value:
//   [0..4] U, [5] u, [6] v, [7] w, [8] p, [9] rho, [10] 1/(2 lambda),
//   [11] sqrt(lambda), [12] 1/sqrt(pi lambda), [13] c, [14] 1/rho, [15] 0.
// A sweep reads only the first 8 (U and the velocity: 32 bytes in FP32).
// The increments dU are stored the same way, 8 values per cell ([0..4],
// then zeros).
constexpr int kRec = 16, kDU = 8;
template <typename T>
__device__ __forceinline__ D3::Prim<T> rec_prim(const T r[kRec]) {
  D3::Prim<T> q;
  q.u = r[5]; q.v = r[6]; q.w = r[7]; q.p = r[8]; q.rho = r[9];
  q.i2l = r[10]; q.sl = r[11]; q.isp = r[12]; q.c = r[13]; q.ir = r[14];
  return q;
}

// U^{k+1} = U^k + dU (FP64), cell record of U^{k+1}; first: U = W_p0
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_lo_cell(int n, ParamsT<TF> P, int first, const double *__restrict__ Wp0,
                                                        double *__restrict__ U, const TF *__restrict__ dU,
                                                        TF *__restrict__ rec) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  TF d[kDU];
  if (!first) vload<TF, kDU>(dU + static_cast<size_t>(i) * kDU, d);
  TF w[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double u = first ? Wp0[v * n + i] : U[v * n + i] + static_cast<double>(d[v]);
    U[v * n + i] = u;
    w[v] = static_cast<TF>(u);
  }
  const D3::Prim<TF> q = D3::prim_of(w, P.gamma, P.kc);
  const TF r[kRec] = { w[0], w[1], w[2], w[3], w[4], q.u, q.v, q.w, q.p, q.rho, q.i2l, q.sl, q.isp, q.c, q.ir, TF(0) };
  vstore<TF, kRec>(rec + static_cast<size_t>(i) * kRec, r);
  pdl_exit();
}

// ghost of a cell-mean state (zero gradients), global
template <typename T>
__device__ __forceinline__ void lo_ghost(const ParamsT<T> &P, int tag, const D3::Frame<T> &F, const T w[NV],
                                         T wg[NV]) {
  T wl[NV], wgl[NV];
  D3::rot_in(F, w, wl);
  const int kind = P.bc_kind[tag];
  if (kind == CGKS_BC_FARFIELD) {
    farfield_ghost(P, tag, F, wl, wgl);
  } else {
    T z[3][NV], dz[3][NV];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) z[k][v] = T(0);
    if (kind == CGKS_BC_SLIP) {
      D3::ghost_slip(wl, z, wgl, dz);
    } else {
      T uw[3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
        uw[a] = F.e[a][0] * P.bc_uw[3 * tag] + F.e[a][1] * P.bc_uw[3 * tag + 1] + F.e[a][2] * P.bc_uw[3 * tag + 2];
      D3::ghost_noslip(P.gamma, uw, wl, z, wgl, dz);
    }
  }
  D3::rot_out(F, wgl, wg);
}

// KFVS flux, lambda_p = max of both sides, Euler flux cache (FP64 mode)
template <typename T>
__device__ __forceinline__ void lo_face_at(const MeshT<T> &m, const ParamsT<T> &P, const T *__restrict__ rec,
                                           T *__restrict__ Flo, T *__restrict__ E0,
                                           T *__restrict__ E1, const int f) {
  const int nf = m.nf;
  const int c0 = m.fc0[f], c1 = m.fc1[f];
  const T S = m.fS[f];
  const D3::Frame<T> F = frame_of(m, f);
  T ra[kRec], rb[kRec];
  vload<T, kRec>(rec + static_cast<size_t>(c0) * kRec, ra);
  D3::Prim<T> a = rec_prim(ra), b;
  T ivb;
  if (c1 >= 0) {
    vload<T, kRec>(rec + static_cast<size_t>(c1) * kRec, rb);
    b = rec_prim(rb);
    ivb = m.ivol[c1];
  } else {
    T wg[NV];
    lo_ghost(P, -1 - c1, F, ra, wg);
#pragma unroll
    for (int v = 0; v < NV; ++v) rb[v] = wg[v];
    b = D3::prim_of(wg, P.gamma, P.kc);
    ivb = m.ivol[c0];
  }
  T la3[3], lb3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    la3[k] = a.u * F.e[k][0] + a.v * F.e[k][1] + a.w * F.e[k][2];
    lb3[k] = b.u * F.e[k][0] + b.v * F.e[k][1] + b.w * F.e[k][2];
  }
  const T la = fabs(la3[0]) + a.c + T(2) * (P.mu * a.ir) * S * m.ivol[c0];
  const T lb = fabs(lb3[0]) + b.c + T(2) * (P.mu * b.ir) * S * ivb;
  const T lmax = la > lb ? la : lb;
  // Euler normal fluxes of the two sides (the L-F flux, the FP64 cache)
  const T nx = F.e[0][0], ny = F.e[0][1], nz = F.e[0][2];
  const T una = la3[0], unb = lb3[0];
  T Fa[NV], Fb[NV];
  Fa[0] = a.rho * una; Fa[1] = ra[1] * una + a.p * nx; Fa[2] = ra[2] * una + a.p * ny;
  Fa[3] = ra[3] * una + a.p * nz; Fa[4] = (ra[4] + a.p) * una;
  Fb[0] = b.rho * unb; Fb[1] = rb[1] * unb + b.p * nx; Fb[2] = rb[2] * unb + b.p * ny;
  Fb[3] = rb[3] * unb + b.p * nz; Fb[4] = (rb[4] + b.p) * unb;
  T Fg[NV];
  if (P.flux_lo == CGKS_FLUX_LF) {
    // Lax-Friedrichs alternative of Section 3 with the implicit operator's
    // lambda_p: (F_n(U_l) + F_n(U_r)) / 2 - lambda_p (U_r - U_l) / 2
#pragma unroll
    for (int v = 0; v < NV; ++v) Fg[v] = T(0.5) * (Fa[v] + Fb[v]) - T(0.5) * lmax * (rb[v] - ra[v]);
  } else {
    T Fl[NV];
    D3::kfvs(P.K, a.rho, la3[0], la3[1], la3[2], a.i2l, a.sl, a.isp, b.rho, lb3[0], lb3[1], lb3[2], b.i2l, b.sl,
             b.isp, Fl);
    D3::rot_out(F, Fl, Fg);
  }
  if (P.lo_viscous && P.mu > T(0)) {
    // first-order viscous flux: normal gradients from the two cell states
    // over the centre distance delta, Stokes' hypothesis, Pr = 1 heat flux
    //   tau.n = mu / delta (du + (n.du) n / 3),  q.n = -kappa (T_r - T_l) / delta
    const T md = P.mu * m.fidl[f];
    const T du[3] = { b.u - a.u, b.v - a.v, b.w - a.w };
    const T nn[3] = { nx, ny, nz };
    const T dn = (du[0] * nx + du[1] * ny + du[2] * nz) / T(3);
    const T um[3] = { T(0.5) * (a.u + b.u), T(0.5) * (a.v + b.v), T(0.5) * (a.w + b.w) };
    T work = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T tau = md * (du[d] + dn * nn[d]);
      Fg[1 + d] -= tau;
      work += tau * um[d];
    }
    const T qn = -md * P.gamma / (P.gamma - T(1)) * (b.p * b.ir - a.p * a.ir);
    Fg[4] -= work - qn;
  }
  // one run per face (AoS): the flux and lambda_p, read together by the
  // right-hand side of each cell
  T o[kLo];
#pragma unroll
  for (int v = 0; v < NV; ++v) o[v] = Fg[v];
  o[NV] = lmax;
  o[NV + 1] = o[NV + 2] = T(0);
  vstore<T, kLo>(Flo + static_cast<size_t>(f) * kLo, o);
  if constexpr (!is_f32<T>())
  if (E0) {   // the FP64 path's cache (the mixed path has none)
    T e[kEu];
    e[NV] = T(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) e[v] = Fa[v];
    vstore<T, kEu>(E0 + static_cast<size_t>(f) * kEu, e);
    if (c1 >= 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) e[v] = Fb[v];
      vstore<T, kEu>(E1 + static_cast<size_t>(f) * kEu, e);
    }
  }
}
template <typename T, int SH>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH))
    k_lo_face(MeshT<T> m, ParamsT<T> P, const T *__restrict__ rec, T *__restrict__ Flo,
              T *__restrict__ E0, T *__restrict__ E1) {
  pdl_enter();
  for_items<SH>(m.nf, [&](int f) { lo_face_at(m, P, rec, Flo, E0, E1, f); });
  pdl_exit();
}

// right-hand side R^k = R_lo + S (FP64 sums), 1/D_i (FP64), lambda per slot,
// first colour pass (dU = R / D on colour 0, zero elsewhere)
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_lo_rhs(MeshT<double> m, ParamsT<double> P, int first, int colour0_end,
                                                       const TF *__restrict__ Flo,
                                                       const double *__restrict__ Rp0, double *__restrict__ Src,
                                                       TF *__restrict__ Rk, TF *__restrict__ invD, TF *__restrict__ dU,
                                                       TF *__restrict__ lamS) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.nc) return;
  const int n = m.nc;
  double R[NV] = { 0, 0, 0, 0, 0 }, sum = 0.0;
  for (int s = 0; s < kMaxFace3; ++s) {
    const int fs = m.cface[s * n + i];
    if (fs == kNoFace) { lamS[s * n + i] = TF(0); continue; }
    const int f = fs >= 0 ? fs : ~fs;
    const double sg = fs >= 0 ? 1.0 : -1.0;
    const double S = 2.0 * m.shs[s * n + i];   // S_f, from the per-cell slot array (coalesced)
    TF fl[kLo];
    vload<TF, kLo>(Flo + static_cast<size_t>(f) * kLo, fl);   // flux and lambda_p
#pragma unroll
    for (int v = 0; v < NV; ++v) R[v] -= sg * S * static_cast<double>(fl[v]);
    const TF l = fl[NV];
    lamS[s * n + i] = l;
    sum += static_cast<double>(l) * S;
  }
  const double id = 1.0 / (sum / P.cfl_lo + 0.5 * sum);
  invD[i] = static_cast<TF>(id);
  const bool c0 = i < colour0_end;
  TF d[kDU];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double src;
    if (first) { src = Rp0[v * n + i] - R[v]; Src[v * n + i] = src; }
    else src = Src[v * n + i];
    const double r = R[v] + src;
    Rk[v * n + i] = static_cast<TF>(r);
    d[v] = c0 ? static_cast<TF>(r * id) : TF(0);
  }
#pragma unroll
  for (int v = NV; v < kDU; ++v) d[v] = TF(0);
  vstore<TF, kDU>(dU + static_cast<size_t>(i) * kDU, d);
  pdl_exit();
}

// point relaxation of the cells [begin, begin + count) of one colour, Eq.
// (implicit-local): 8 lanes per cell, one per face slot (6 used); the five
// terms are summed over the lane group by shuffles, lane v writes
// component v.
// static (mesh) data of one lane of a sweep: neighbour across face slot s
// of cell i and the slot geometry; read before the kernel waits on its
// predecessor, since no kernel of a cycle writes it
template <typename T>
struct SweepGeo {
  int j, f;
  bool is0;
  T nn[3], hS;
};
template <typename T>
__device__ __forceinline__ SweepGeo<T> sweep_geo(const MeshT<T> &m, const int i, const int s) {
  const int n = m.nc;
  SweepGeo<T> g;
  g.j = (i >= 0 && s < kMaxFace3) ? m.cnbr[s * n + i] : -1;
  g.f = 0;
  g.is0 = true;
  g.nn[0] = g.nn[1] = g.nn[2] = g.hS = T(0);
  if (g.j >= 0) {
    g.nn[0] = m.sn[(3 * s) * n + i];
    g.nn[1] = m.sn[(3 * s + 1) * n + i];
    g.nn[2] = m.sn[(3 * s + 2) * n + i];
    g.hS = m.shs[s * n + i];
    if constexpr (!is_f32<T>()) {
      const int fs = m.cface[s * n + i];
      g.is0 = fs >= 0;
      g.f = g.is0 ? fs : ~fs;
    }
  }
  return g;
}
template <typename T>
__device__ __forceinline__ void sweep_cell(const MeshT<T> &m, const ParamsT<T> &P, const SweepGeo<T> &g,
                                           const int i, const int s, const T *__restrict__ rec,
                                           const T *__restrict__ Rk, const T *__restrict__ invD,
                                           const T *__restrict__ lamS, const T *__restrict__ E0,
                                           const T *__restrict__ E1, T *__restrict__ dU) {
  const int n = m.nc, nf = m.nf;
  const int j = g.j;
  T c[NV] = { T(0), T(0), T(0), T(0), T(0) };
  if (j >= 0) {
    const T hS = g.hS, lp = lamS[s * n + i];
    // the neighbour's U and velocity (the first 8 values of its record; 6
    // in FP64, which needs U only) and its increment
    constexpr int kUsed = is_f32<T>() ? 8 : 6;
    T rj[kUsed], dj[kDU];
    vload<T, kUsed>(rec + static_cast<size_t>(j) * kRec, rj);
    vload<T, kDU>(dU + static_cast<size_t>(j) * kDU, dj);
    T uj[NV], du[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { uj[v] = rj[v]; du[v] = dj[v]; }
    if constexpr (is_f32<T>()) {
      T dF[NV];
      // pressure of U_j, the expression of its primitives
      const T pj = (P.gamma - T(1)) * (uj[4] - T(0.5) * uj[0] * (rj[5] * rj[5] + rj[6] * rj[6] + rj[7] * rj[7]));
      D3::euler_flux_delta(P.gamma, uj, rj[5], rj[6], rj[7], pj, du, g.nn, dF);
#pragma unroll
      for (int v = 0; v < NV; ++v) c[v] = hS * (dF[v] - lp * du[v]);
    } else {
      const int f = g.f;
      T up[NV], fa[NV], e[kEu];
      vload<T, kEu>((g.is0 ? E1 : E0) + static_cast<size_t>(f) * kEu, e);
#pragma unroll
      for (int v = 0; v < NV; ++v) up[v] = uj[v] + du[v];
      D3::euler_flux(P.gamma, up, g.nn, fa);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T fb = g.is0 ? e[v] : -e[v];
        c[v] = hS * ((fa[v] - fb) - lp * du[v]);   // (U + dU) - U = dU
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    c[v] += __shfl_xor_sync(0xffffffffu, c[v], 1);
    c[v] += __shfl_xor_sync(0xffffffffu, c[v], 2);
    c[v] += __shfl_xor_sync(0xffffffffu, c[v], 4);
  }
  if (i >= 0 && s < NV) {
    const T mine = s == 0 ? c[0] : s == 1 ? c[1] : s == 2 ? c[2] : s == 3 ? c[3] : c[4];
    dU[static_cast<size_t>(i) * kDU + s] = (Rk[s * n + i] - mine) * invD[i];
  }
}
// cells per block of a sweep launch of shape SH
__host__ __device__ constexpr int sweep_cpb(int sh) { return shape_bs(sh) / kSweepLanes * shape_ipt(sh); }
template <typename T, int SH>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH))
    k_sweep(MeshT<T> m, ParamsT<T> P, int begin, int count, const T *__restrict__ rec,
            const T *__restrict__ Rk, const T *__restrict__ invD, const T *__restrict__ lamS,
            const T *__restrict__ E0, const T *__restrict__ E1, T *__restrict__ dU) {
  constexpr int kGroups = shape_bs(SH) / kSweepLanes, kIpt = shape_ipt(SH);
  const int s = threadIdx.x & (kSweepLanes - 1);
  // one copy of the per-cell code for every shape (the same arithmetic);
  // the first item's mesh data is read before the wait, later items' after
#pragma unroll 1
  for (int k = 0; k < kIpt; ++k) {
    const int g = (static_cast<int>(blockIdx.x) * kIpt + k) * kGroups + static_cast<int>(threadIdx.x) / kSweepLanes;
    const int i = g < count ? begin + g : -1;
    const SweepGeo<T> geo = sweep_geo(m, i, s);
    pdl_enter();
    sweep_cell(m, P, geo, i, s, rec, Rk, invD, lamS, E0, E1, dU);
  }
  pdl_exit();
}

// W = W_p0 + (U - W_p0), density residual partials, state check
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_prolong(MeshT<double> m, ParamsT<double> P, double *__restrict__ W,
                                                        const double *__restrict__ Wp0, const double *__restrict__ U,
                                                        int *status, double *__restrict__ partial,
                                                        TF *__restrict__ Wm) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = m.nc;
  double num = 0.0, den = 0.0;
  if (i < n) {
    double w[NV];
    const double old = W[i];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double wp = Wp0[v * n + i];
      w[v] = wp + (U[v * n + i] - wp);
      W[v * n + i] = w[v];
      if (Wm) Wm[v * n + i] = static_cast<TF>(w[v]);
    }
    if (!state_ok(P.gamma, w)) atomicOr(status, kBadState);
    num = fabs(w[0] - old);
    den = old;
  }
  block_sum2(num, den, &partial[2 * blockIdx.x]);
  pdl_exit();
}

// caller AoS <-> internal SoA
__global__ void k_gather_state(int n, const int *__restrict__ perm, const double *__restrict__ Wa,
                               const double *__restrict__ Wxa, double *__restrict__ W, double *__restrict__ Wx,
                               float *__restrict__ W32, float *__restrict__ Wx32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = perm[i];
  for (int v = 0; v < NV; ++v) {
    const double w = Wa[NV * c + v];
    W[v * n + i] = w;
    if (W32) W32[v * n + i] = static_cast<float>(w);
  }
  for (int q = 0; q < 3 * NV; ++q) {
    const double g = Wxa ? Wxa[3 * NV * c + q] : 0.0;
    Wx[q * n + i] = g;
    if (Wx32) Wx32[q * n + i] = static_cast<float>(g);
  }
}
__global__ void k_scatter_state(int n, const int *__restrict__ perm, const double *__restrict__ W,
                                const double *__restrict__ Wx, double *__restrict__ Wa, double *__restrict__ Wxa) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = perm[i];
  if (Wa) for (int v = 0; v < NV; ++v) Wa[NV * c + v] = W[v * n + i];
  if (Wxa) for (int q = 0; q < 3 * NV; ++q) Wxa[3 * NV * c + q] = Wx[q * n + i];
}

}  // namespace kern3
}  // namespace cgks
