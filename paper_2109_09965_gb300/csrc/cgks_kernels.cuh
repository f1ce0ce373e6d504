// Kernels of the batched hot path (included by cgks_device.cu only).
//
// Index space: a batch holds one or more solves in slots.  Each solve owns
// a contiguous range of cells (padded to a multiple of kCellBlock with
// inert cells, csid = -1) and a contiguous range of faces; space no solve
// holds is inert too (csid / fsid = -1).  Within a solve, cells are
// colour-major with reverse Cuthill-McKee order inside a colour.  Boundary
// faces store -1 - (16 * slot + tag) in fc1, so one table holds every
// solve's boundary conditions.  Per-solve values (viscosity, time step,
// status, residual) are indexed by the slot.  Arrays are strided by the
// batch capacity (m.nc cells, m.nf faces).
//
// Precision: kernels that evaluate fluxes are templated on the flux type
// TF.  FP64 mode runs everything in double.  Mixed mode keeps the
// conservative variables (W, W_x, U) and every accumulation into them, the
// residuals and the diagonal inversion in double, and runs reconstruction,
// face fluxes and relaxation sweeps in float on float mirrors of the state.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "cgks_internal.h"
#include "cgks_physics.cuh"
#include "cgks_pdl.cuh"
#include "cgks_shapes.h"

namespace cgks {
namespace kern {

namespace D = cgks::dev;

constexpr int kCellBlock = 256;
constexpr int kTagsPerSolve = CGKS_MAX_BC;
constexpr int kBadState = 1;   // bit of a solve's status word

template <typename T>
__host__ __device__ constexpr bool is_f32() { return std::is_same<T, float>::value; }

// Shared model constants and pointers to per-solve / per-tag tables.
template <typename T>
struct ParamsT {
  T gamma, K, cfl_hi, cfl_lo;
  D::KC<T> kc;
  const T *mu;                   // [S] dynamic viscosity per solve
  const int *bc_kind;            // [16 S] boundary kind per global tag
  const T *bc_uw;                // [16 S][2] wall velocity
  const T *bc_rho, *bc_u, *bc_p; // [16 S], [16 S][2], [16 S] far-field free stream
  int flux_lo;                   // low-level flux: CGKS_FLUX_KFVS or CGKS_FLUX_LF
  int flux_hi;                   // high-level flux: CGKS_FLUX_SMOOTH or CGKS_FLUX_FULL
  T tau_c1, tau_c2;              // numerical collision time constants of the full flux
  T weno_eps, weno_g0;           // compact WENO epsilon (0: linear weights), linear weight of P2
  int weno_vars;                 // CGKS_WENO_CONSERVATIVE (per cell) or CGKS_WENO_CHARACTERISTIC (per face side)
  // [S] per solve: 1 = limited (full flux + compact WENO), 0 = smooth flux,
  // linear weights; null when every solve of the batch takes the batch-wide
  // flux.  With it each instantiation of k_recon / k_face treats only the
  // solves of its own class.
  const int *slim;
  int lo_viscous;                // 1: the low-order residual carries a first-order viscous flux
};

template <typename T>
struct MeshT {
  int nc, nf;                                // padded cells, faces
  const T *vol, *ivol, *per, *ih, *m2;       // ih = 1/h; m2: [3][nc]
  const T *op;                               // [kNCol*kNM][nc]
  const T *fn, *fS, *fjump, *fxi;            // fn [2][nf], fjump = alpha/delta, fxi [8][nf]
  const T *fidl;                             // 1/delta: the centre distance along n (boundary: twice to the face)
  const T *snx, *sny, *shs;                  // [4][nc] per face slot: outward normal of the cell, S/2
  const int *cface, *cnbr;                   // [4][nc]
  const int *fc0, *fc1;
  const int *csid, *fsid;                    // solve of each cell (-1: padding) and face
  const unsigned char *ccol;                 // colour of each cell (255: padding)
  const unsigned char *wenok;                // 1: least-squares quadratic (WENO may limit it)
};

// per-batch control words on the device
struct Ctl {
  double dt_fixed;   // > 0: prescribed step for every solve
  int res_ctr;       // next slot of solve 0's residual history
  int pad_;
};

__device__ __forceinline__ double dt_of(const Ctl *ctl, const unsigned long long *dt_bits, int sid, double cfl) {
  if (ctl->dt_fixed > 0.0) return ctl->dt_fixed;
  return cfl * __longlong_as_double(static_cast<long long>(dt_bits[sid]));
}

__device__ __forceinline__ bool state_ok(double gamma, const double w[4]) {
  double p = (gamma - 1.0) * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0]);
  return w[0] > 0.0 && p > 0.0 && isfinite(w[0]) && isfinite(p) && isfinite(w[1]) && isfinite(w[2]);
}

// Block reduction of two doubles in a fixed order; thread 0 writes them.
__device__ __forceinline__ void block_sum2(double a, double b, double *out2) {
  __shared__ double sa[32], sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { out2[0] = a; out2[1] = b; }
  }
}

// ------------------------------------------------------------------
// K0: reset the per-solve time steps
__global__ void k_reset_dt(Ctl *ctl, unsigned long long *dt_bits, int S, double dt_fixed) {
  pdl_enter();
  for (int s = threadIdx.x; s < S; s += blockDim.x) dt_bits[s] = 0x7ff0000000000000ull;  // +inf
  if (threadIdx.x == 0) ctl->dt_fixed = dt_fixed;
  pdl_exit();
}

// K4: local explicit step per cell, per-solve min by atomicMin on the bits
// (min is order independent).  h = 2|Omega|/perimeter, speed |U| + c + 2 nu / h.
// Solves are padded to whole blocks, so a block never spans two solves and
// its first cell is a real one: one atomic per block.
__global__ void __launch_bounds__(kCellBlock) k_dt(MeshT<double> m, ParamsT<double> P, const double *__restrict__ W,
                                                   unsigned long long *dt_bits) {
  pdl_enter();
  __shared__ double wmin[kCellBlock / 32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double d = INFINITY;
  int sid = i < m.nc ? m.csid[i] : -1;
  if (sid >= 0) {
    int n = m.nc;
    double rho = W[i], mx = W[n + i], my = W[2 * n + i], E = W[3 * n + i];
    double u = mx / rho, v = my / rho;
    double p = (P.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    double a = sqrt(P.gamma * p / rho);
    double hh = 2.0 * m.vol[i] / m.per[i];
    double speed = sqrt(u * u + v * v) + a + 2.0 * (P.mu[sid] / rho) / hh;
    d = hh / speed;
  }
  for (int o = 16; o > 0; o >>= 1) d = fmin(d, __shfl_down_sync(0xffffffffu, d, o));
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kCellBlock / 32; ++w) d = fmin(d, wmin[w]);
    const int s0 = blockIdx.x * blockDim.x < m.nc ? m.csid[blockIdx.x * blockDim.x] : -1;
    if (s0 >= 0 && d < INFINITY) atomicMin(&dt_bits[s0], static_cast<unsigned long long>(__double_as_longlong(d)));
  }
  pdl_exit();
}

// Wall ghost of a state and its gradient (global frame), through the face frame.
template <typename T>
__device__ __forceinline__ void wall_ghost_global(const ParamsT<T> &P, int tag, T nx, T ny, const T w[4],
                                                  const T gx[4], const T gy[4], T wg[4], T ggx[4], T ggy[4]) {
  T wl[4], dn[4], dt[4], tn[4], tt[4];
  D::rot_in(nx, ny, w, wl);
  for (int v = 0; v < 4; ++v) { tn[v] = nx * gx[v] + ny * gy[v]; tt[v] = -ny * gx[v] + nx * gy[v]; }
  D::rot_in(nx, ny, tn, dn);
  D::rot_in(nx, ny, tt, dt);
  T wgl[4], dng[4], dtg[4];
  if (P.bc_kind[tag] == CGKS_BC_SLIP) {
    D::ghost_slip(wl, dn, dt, wgl, dng, dtg);
  } else {
    T wn = P.bc_uw[2 * tag] * nx + P.bc_uw[2 * tag + 1] * ny;
    T wt = -P.bc_uw[2 * tag] * ny + P.bc_uw[2 * tag + 1] * nx;
    D::ghost_noslip(P.gamma, wn, wt, wl, dn, dt, wgl, dng, dtg);
  }
  T gn[4], gt[4];
  D::rot_out(nx, ny, wgl, wg);
  D::rot_out(nx, ny, dng, gn);
  D::rot_out(nx, ny, dtg, gt);
  for (int v = 0; v < 4; ++v) { ggx[v] = nx * gn[v] - ny * gt[v]; ggy[v] = ny * gn[v] + nx * gt[v]; }
}

template <typename T>
__device__ __forceinline__ void farfield_ghost(const ParamsT<T> &P, int tag, T nx, T ny, const T wl[4], T wg[4]) {
  T une = P.bc_u[2 * tag] * nx + P.bc_u[2 * tag + 1] * ny;
  T ute = -P.bc_u[2 * tag] * ny + P.bc_u[2 * tag + 1] * nx;
  D::ghost_farfield(P.gamma, P.bc_rho[tag], une, ute, P.bc_p[tag], wl, wg);
}

// prescribed state of a Dirichlet boundary in the face frame
template <typename T>
__device__ __forceinline__ void dirichlet_ghost(const ParamsT<T> &P, int tag, T nx, T ny, T wg[4]) {
  const T r = P.bc_rho[tag], p = P.bc_p[tag];
  const T un = P.bc_u[2 * tag] * nx + P.bc_u[2 * tag + 1] * ny;
  const T ut = -P.bc_u[2 * tag] * ny + P.bc_u[2 * tag + 1] * nx;
  wg[0] = r; wg[1] = r * un; wg[2] = r * ut;
  wg[3] = p / (P.gamma - T(1)) + T(0.5) * r * (un * un + ut * ut);
}

__host__ __device__ __forceinline__ bool is_wall_kind(int k) { return k == CGKS_BC_SLIP || k == CGKS_BC_NOSLIP; }

// Compact WENO with nonlinear weights (Section 4, transonic and supersonic
// cases; the scheme is the cited one, read as follows).  Candidates: the
// compact quadratic P2 (scaled coefficients c[q][v]) and the m linear
// polynomials W_i + h g.(xi, eta), g the cell-mean gradient of the cell
// itself and of each face neighbour (h g given in lin[k][0..1][v]).
// Smoothness: the cell mean of (h D P)^2 over first and second derivative
// multi-indices; with the centroid at the origin and the cell's second
// moments M = (xi^2, xi eta, eta^2) means m2 this is, for
// P_xi = c0 + 2 c2 xi + c3 eta, P_eta = c1 + c3 xi + 2 c4 eta,
//   c0^2 + c1^2 + (4 c2^2 + c3^2) M_xx + (c3^2 + 4 c4^2) M_yy
//   + (4 c2 c3 + 4 c3 c4) M_xy + 4 c2^2 + c3^2 + 4 c4^2.
// Weights w_k ~ gamma_k / (beta_k + eps)^2 (gamma_0 = g0, the rest
// (1 - g0) / m); result (w_0/gamma_0)(P2 - sum gamma_k P1_k) + sum w_k P1_k.
template <typename T>
__device__ __forceinline__ void weno_combine(const ParamsT<T> &P, T mxx, T mxy, T myy, int nk, const T lin[5][2][4],
                                             T c[kNM][4]) {
  const T g0 = P.weno_g0, eps = P.weno_eps;
  const T gk = (T(1) - g0) / T(nk);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const T c0 = c[0][v], c1 = c[1][v], c2 = c[2][v], c3 = c[3][v], c4 = c[4][v];
    const T b0 = c0 * c0 + c1 * c1 + (T(4) * c2 * c2 + c3 * c3) * mxx + (c3 * c3 + T(4) * c4 * c4) * myy +
                 (T(4) * c2 * c3 + T(4) * c3 * c4) * mxy + T(4) * c2 * c2 + c3 * c3 + T(4) * c4 * c4;
    T w0 = g0 / ((b0 + eps) * (b0 + eps));
    T wk[5], ws = w0;
    T lin0 = T(0), lin1 = T(0);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      if (k < nk) {
        const T a0 = lin[k][0][v], a1 = lin[k][1][v];
        const T b = a0 * a0 + a1 * a1;
        wk[k] = gk / ((b + eps) * (b + eps));
        ws += wk[k];
        lin0 += gk * a0;
        lin1 += gk * a1;
      }
    }
    const T iws = T(1) / ws;
    const T f0 = w0 * iws / g0;
    T sel0 = T(0), sel1 = T(0);
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (k < nk) {
        sel0 += wk[k] * iws * lin[k][0][v];
        sel1 += wk[k] * iws * lin[k][1][v];
      }
    c[0][v] = f0 * (c0 - lin0) + sel0;
    c[1][v] = f0 * (c1 - lin1) + sel1;
    c[2][v] = f0 * c2;
    c[3][v] = f0 * c3;
    c[4][v] = f0 * c4;
  }
}

// K1: compact least-squares quadratic of every cell.
//   coef[(q*4 + v)*nc + i], q over (xi, eta, xi^2, xi eta, eta^2).
template <typename T, bool WENO>
__device__ __forceinline__ void recon_at(const MeshT<T> &m, const ParamsT<T> &P, const T *__restrict__ W,
                                         const T *__restrict__ Wx, T *__restrict__ coef, const int i) {
  const int n = m.nc;
  T wi[4], gxi[4], gyi[4];
  for (int v = 0; v < 4; ++v) { wi[v] = W[v * n + i]; gxi[v] = Wx[v * n + i]; gyi[v] = Wx[(4 + v) * n + i]; }
  T c[kNM][4];
  for (int q = 0; q < kNM; ++q) {
    T o0 = m.op[((kNCol - 2) * kNM + q) * n + i], o1 = m.op[((kNCol - 1) * kNM + q) * n + i];
    for (int v = 0; v < 4; ++v) c[q][v] = o0 * gxi[v] + o1 * gyi[v];
  }
  // linear WENO candidates: h times the cell-mean gradients of the cell and its face neighbours
  T lin[WENO ? 5 : 1][2][4];
  int nk = 1;
  if constexpr (WENO) {
    const T hi = T(1) / m.ih[i];
    for (int v = 0; v < 4; ++v) { lin[0][0][v] = hi * gxi[v]; lin[0][1][v] = hi * gyi[v]; }
  }
  for (int s = 0; s < kMaxFace; ++s) {
    int fs = m.cface[s * n + i];
    if (fs == kNoFace) continue;
    int j = m.cnbr[s * n + i];
    T b0[4], b1[4], b2[4];
    if (j >= 0) {
      for (int v = 0; v < 4; ++v) {
        b0[v] = W[v * n + j] - wi[v];
        b1[v] = Wx[v * n + j];
        b2[v] = Wx[(4 + v) * n + j];
      }
      if constexpr (WENO) {
        const T hi = T(1) / m.ih[i];
        for (int v = 0; v < 4; ++v) { lin[nk][0][v] = hi * b1[v]; lin[nk][1][v] = hi * b2[v]; }
        ++nk;
      }
    } else {
      int f = fs >= 0 ? fs : ~fs;
      int tag = -1 - m.fc1[f];
      if (!is_wall_kind(P.bc_kind[tag])) continue;
      T wg[4];
      wall_ghost_global(P, tag, m.fn[f], m.fn[m.nf + f], wi, gxi, gyi, wg, b1, b2);
      for (int v = 0; v < 4; ++v) b0[v] = wg[v] - wi[v];
    }
    for (int q = 0; q < kNM; ++q) {
      T o0 = m.op[((3 * s) * kNM + q) * n + i];
      T o1 = m.op[((3 * s + 1) * kNM + q) * n + i];
      T o2 = m.op[((3 * s + 2) * kNM + q) * n + i];
      for (int v = 0; v < 4; ++v) c[q][v] += o0 * b0[v] + o1 * b1[v] + o2 * b2[v];
    }
  }
  // cells whose stencil fell back to the linear polynomial of their own
  // gradient (too few neighbours, rank deficiency) carry no quadratic terms
  // in the operator and keep it; the others may be limited
  if constexpr (WENO)
    if (m.wenok[i]) weno_combine(P, m.m2[i], m.m2[n + i], m.m2[2 * n + i], nk, lin, c);
  for (int q = 0; q < kNM; ++q)
    for (int v = 0; v < 4; ++v) coef[(q * 4 + v) * n + i] = c[q][v];
}
template <typename T, int SH, bool WENO = false>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH)) k_recon(MeshT<T> m, ParamsT<T> P,
                                                                        const T *__restrict__ W,
                                                                        const T *__restrict__ Wx,
                                                                        T *__restrict__ coef) {
  pdl_enter();
  for_items<SH>(m.nc, [&](int i) {
    if (P.slim) {
      const int sid = m.csid[i];
      if (sid >= 0 && (P.slim[sid] != 0) != WENO) return;
    }
    recon_at<T, WENO>(m, P, W, Wx, coef, i);
  });
  pdl_exit();
}

// value and gradient of the quadratic of cell i at scaled offset (x, y)
template <typename T>
__device__ __forceinline__ void recon_point(const MeshT<T> &m, const T *__restrict__ W, const T *__restrict__ coef,
                                            int i, T x, T y, T val[4], T gx[4], T gy[4]) {
  const int n = m.nc;
  T ih = m.ih[i];
  T p2 = x * x - m.m2[i], p3 = x * y - m.m2[n + i], p4 = y * y - m.m2[2 * n + i];
  for (int v = 0; v < 4; ++v) {
    T c0 = coef[(0 * 4 + v) * n + i], c1 = coef[(1 * 4 + v) * n + i], c2 = coef[(2 * 4 + v) * n + i];
    T c3 = coef[(3 * 4 + v) * n + i], c4 = coef[(4 * 4 + v) * n + i];
    val[v] = W[v * n + i] + c0 * x + c1 * y + c2 * p2 + c3 * p3 + c4 * p4;
    gx[v] = (c0 + T(2) * c2 * x + c3 * y) * ih;
    gy[v] = (c1 + c3 * x + T(2) * c4 * y) * ih;
  }
}

// value and gradient at scaled offset (x, y) of a polynomial of cell i with
// the given coefficients c[q][v]
template <typename T>
__device__ __forceinline__ void poly_point(const MeshT<T> &m, const T *__restrict__ W, const T c[kNM][4], int i, T x,
                                           T y, T val[4], T gx[4], T gy[4]) {
  const int n = m.nc;
  T ih = m.ih[i];
  T p2 = x * x - m.m2[i], p3 = x * y - m.m2[n + i], p4 = y * y - m.m2[2 * n + i];
  for (int v = 0; v < 4; ++v) {
    val[v] = W[v * n + i] + c[0][v] * x + c[1][v] * y + c[2][v] * p2 + c[3][v] * p3 + c[4][v] * p4;
    gx[v] = (c[0][v] + T(2) * c[2][v] * x + c[3][v] * y) * ih;
    gy[v] = (c[1][v] + c[3][v] * x + T(2) * c[4][v] * y) * ih;
  }
}

// Compact WENO on characteristic variables (Section 4, shock reflection),
// for the side of a face held by cell i: the candidates of cell i (its
// linear-weight quadratic from coef, h times the mean gradients of the cell
// and its face neighbours) are projected on the left eigenvectors of the
// Euler flux Jacobian along the face normal n at the state wref (the mean
// of the two cell averages; the cell's own on a boundary face), combined by
// weno_combine per characteristic field and projected back.  Right
// eigenvectors (columns): u_n - c, entropy, shear, u_n + c; the left ones
// in closed form with b1 = (gamma - 1)/c^2, b2 = b1 |u|^2 / 2.
template <typename T>
__device__ void char_side(const MeshT<T> &m, const ParamsT<T> &P, const T *__restrict__ W, const T *__restrict__ Wx,
                          const T *__restrict__ coef, int i, const T wref[4], T nx, T ny, T out[kNM][4]) {
  const int n = m.nc;
  const T g = P.gamma;
  const T ir = T(1) / wref[0];
  const T u = wref[1] * ir, v = wref[2] * ir;
  const T q2 = u * u + v * v;
  const T p = (g - T(1)) * (wref[3] - T(0.5) * wref[0] * q2);
  const T c = D::d_sqrt(g * p * ir), ic = T(1) / c;
  const T H = (wref[3] + p) * ir;
  const T un = u * nx + v * ny, ut = -u * ny + v * nx;
  const T b1 = (g - T(1)) * ic * ic, b2 = T(0.5) * b1 * q2;
  const T R[4][4] = { { T(1), T(1), T(0), T(1) },
                      { u - c * nx, u, -ny, u + c * nx },
                      { v - c * ny, v, nx, v + c * ny },
                      { H - c * un, T(0.5) * q2, ut, H + c * un } };
  const T L[4][4] = { { T(0.5) * (b2 + un * ic), T(0.5) * (-b1 * u - nx * ic), T(0.5) * (-b1 * v - ny * ic),
                        T(0.5) * b1 },
                      { T(1) - b2, b1 * u, b1 * v, -b1 },
                      { -ut, -ny, nx, T(0) },
                      { T(0.5) * (b2 - un * ic), T(0.5) * (-b1 * u + nx * ic), T(0.5) * (-b1 * v + ny * ic),
                        T(0.5) * b1 } };
  const T h = T(1) / m.ih[i];
  T lin[5][2][4];
  int nk = 0;
  auto add = [&](int j) {
    T gx[4], gy[4];
    for (int a = 0; a < 4; ++a) { gx[a] = Wx[a * n + j]; gy[a] = Wx[(4 + a) * n + j]; }
    for (int a = 0; a < 4; ++a) {
      T sx = T(0), sy = T(0);
      for (int b = 0; b < 4; ++b) { sx += L[a][b] * gx[b]; sy += L[a][b] * gy[b]; }
      lin[nk][0][a] = h * sx;
      lin[nk][1][a] = h * sy;
    }
    ++nk;
  };
  add(i);
  for (int sl = 0; sl < kMaxFace; ++sl) {
    if (m.cface[sl * n + i] == kNoFace) continue;
    const int j = m.cnbr[sl * n + i];
    if (j >= 0) add(j);
  }
  T cq[kNM][4];
  for (int q = 0; q < kNM; ++q) {
    T cv[4];
    for (int b = 0; b < 4; ++b) cv[b] = coef[(q * 4 + b) * n + i];
    for (int a = 0; a < 4; ++a) {
      T acc = T(0);
      for (int b = 0; b < 4; ++b) acc += L[a][b] * cv[b];
      cq[q][a] = acc;
    }
  }
  weno_combine(P, m.m2[i], m.m2[n + i], m.m2[2 * n + i], nk, lin, cq);
  for (int q = 0; q < kNM; ++q)
    for (int b = 0; b < 4; ++b) {
      T acc = T(0);
      for (int a = 0; a < 4; ++a) acc += R[b][a] * cq[q][a];
      out[q][b] = acc;
    }
}

// ghost of a cell-mean state (zero gradients)
template <typename T>
__device__ __forceinline__ void lo_ghost(const ParamsT<T> &P, int tag, T nx, T ny, const T w[4], T wg[4]) {
  T wl[4], z[4] = { T(0), T(0), T(0), T(0) }, wgl[4], a[4], b[4];
  D::rot_in(nx, ny, w, wl);
  int kind = P.bc_kind[tag];
  if (kind == CGKS_BC_FARFIELD) {
    farfield_ghost(P, tag, nx, ny, wl, wgl);
  } else if (kind == CGKS_BC_DIRICHLET) {
    dirichlet_ghost(P, tag, nx, ny, wgl);
  } else if (kind == CGKS_BC_OUTFLOW) {
    for (int v = 0; v < 4; ++v) wgl[v] = wl[v];
  } else if (kind == CGKS_BC_SLIP) {
    D::ghost_slip(wl, z, z, wgl, a, b);
  } else {
    T wn = P.bc_uw[2 * tag] * nx + P.bc_uw[2 * tag + 1] * ny;
    T wt = -P.bc_uw[2 * tag] * ny + P.bc_uw[2 * tag + 1] * nx;
    D::ghost_noslip(P.gamma, wn, wt, wl, z, z, wgl, a, b);
  }
  D::rot_out(nx, ny, wgl, wg);
}

// K2: gas-kinetic flux and interface state at the two Gauss points of every
// face; writes the weighted sums F0, F1, Wc, Wt (global frame) per face:
//   out[(k*4 + v)*nf + f], k = 0 F0, 1 F1, 2 Wc, 3 Wt.
template <typename T, bool FULL, bool CHAR>
__device__ __forceinline__ void face_at(const MeshT<T> &m, const ParamsT<T> &P, const T *__restrict__ W,
                                        const T *__restrict__ Wx, const T *__restrict__ coef, T *__restrict__ out,
                                        const Ctl *ctl, const unsigned long long *dt_bits, const int f) {
  const int sid = m.fsid[f];
  if (sid < 0) return;   // free face space of a batch
  if (P.slim && (P.slim[sid] != 0) != FULL) return;   // the other flux class's launch
  const int nf = m.nf;
  const int c0 = m.fc0[f], c1 = m.fc1[f];
  const T nx = m.fn[f], ny = m.fn[nf + f], ajump = m.fjump[f];
  const T mu = P.mu[sid];
  // the full flux integrates over the step: it needs the step's dt
  T dt = T(0);
  if constexpr (FULL) dt = static_cast<T>(dt_of(ctl, dt_bits, sid, static_cast<double>(P.cfl_hi)));
  T acc[4][4];
  for (int k = 0; k < 4; ++k) for (int v = 0; v < 4; ++v) acc[k][v] = T(0);
  T wff[4];
  bool farfield = false;
  int tag = 0, kind = -1;
  if (c1 < 0) {
    tag = -1 - c1;
    kind = P.bc_kind[tag];
    farfield = kind == CGKS_BC_FARFIELD || kind == CGKS_BC_DIRICHLET;
    if (kind == CGKS_BC_FARFIELD) {
      // Riemann-invariant state from the cell mean and the free stream
      T wm[4], wl[4];
      for (int v = 0; v < 4; ++v) wm[v] = W[v * m.nc + c0];
      D::rot_in(nx, ny, wm, wl);
      farfield_ghost(P, tag, nx, ny, wl, wff);
    } else if (kind == CGKS_BC_DIRICHLET) {
      dirichlet_ghost(P, tag, nx, ny, wff);
    }
  }
  // characteristic WENO: the two sides' polynomials limited for this face
  T cs0[CHAR ? kNM : 1][4], cs1[CHAR ? kNM : 1][4];
  bool lim0 = false, lim1 = false;
  if constexpr (CHAR) {
    T wref[4];
    for (int v = 0; v < 4; ++v)
      wref[v] = c1 >= 0 ? T(0.5) * (W[v * m.nc + c0] + W[v * m.nc + c1]) : W[v * m.nc + c0];
    lim0 = m.wenok[c0] != 0;
    if (lim0) char_side(m, P, W, Wx, coef, c0, wref, nx, ny, cs0);
    lim1 = c1 >= 0 && m.wenok[c1] != 0;
    if (lim1) char_side(m, P, W, Wx, coef, c1, wref, nx, ny, cs1);
  }
  for (int k = 0; k < 2; ++k) {
    T wL[4], gxL[4], gyL[4];
    if (CHAR && lim0)
      poly_point(m, W, cs0, c0, m.fxi[(2 * k) * nf + f], m.fxi[(2 * k + 1) * nf + f], wL, gxL, gyL);
    else
      recon_point(m, W, coef, c0, m.fxi[(2 * k) * nf + f], m.fxi[(2 * k + 1) * nf + f], wL, gxL, gyL);
    T wl[4], dnl[4], dtl[4], t0[4], t1[4];
    D::rot_in(nx, ny, wL, wl);
    for (int v = 0; v < 4; ++v) { t0[v] = nx * gxL[v] + ny * gyL[v]; t1[v] = -ny * gxL[v] + nx * gyL[v]; }
    D::rot_in(nx, ny, t0, dnl);
    D::rot_in(nx, ny, t1, dtl);
    T wr[4], dnr[4], dtr[4];
    if (c1 >= 0) {
      T wR[4], gxR[4], gyR[4];
      if (CHAR && lim1)
        poly_point(m, W, cs1, c1, m.fxi[(4 + 2 * k) * nf + f], m.fxi[(5 + 2 * k) * nf + f], wR, gxR, gyR);
      else
        recon_point(m, W, coef, c1, m.fxi[(4 + 2 * k) * nf + f], m.fxi[(5 + 2 * k) * nf + f], wR, gxR, gyR);
      D::rot_in(nx, ny, wR, wr);
      for (int v = 0; v < 4; ++v) { t0[v] = nx * gxR[v] + ny * gyR[v]; t1[v] = -ny * gxR[v] + nx * gyR[v]; }
      D::rot_in(nx, ny, t0, dnr);
      D::rot_in(nx, ny, t1, dtr);
    } else if (farfield) {
      for (int v = 0; v < 4; ++v) { wr[v] = wff[v]; dnr[v] = T(0); dtr[v] = T(0); }
    } else if (kind == CGKS_BC_OUTFLOW) {
      for (int v = 0; v < 4; ++v) { wr[v] = wl[v]; dnr[v] = dnl[v]; dtr[v] = dtl[v]; }
    } else if (kind == CGKS_BC_SLIP) {
      D::ghost_slip(wl, dnl, dtl, wr, dnr, dtr);
    } else {
      T wn = P.bc_uw[2 * tag] * nx + P.bc_uw[2 * tag + 1] * ny;
      T wt = -P.bc_uw[2 * tag] * ny + P.bc_uw[2 * tag + 1] * nx;
      D::ghost_noslip(P.gamma, wn, wt, wl, dnl, dtl, wr, dnr, dtr);
    }
    T F0[4], F1[4], Wc[4], Wt[4];
    if constexpr (FULL)
      D::gks_full_point_local(P.kc, mu, ajump, dt, P.tau_c1, P.tau_c2, wl, wr, dnl, dtl, dnr, dtr, F0, F1, Wc, Wt);
    else
      D::gks_point_local(P.kc, mu, ajump, wl, wr, dnl, dtl, dnr, dtr, F0, F1, Wc, Wt);
    T g[4];
    D::rot_out(nx, ny, F0, g); for (int v = 0; v < 4; ++v) acc[0][v] += T(0.5) * g[v];
    D::rot_out(nx, ny, F1, g); for (int v = 0; v < 4; ++v) acc[1][v] += T(0.5) * g[v];
    D::rot_out(nx, ny, Wc, g); for (int v = 0; v < 4; ++v) acc[2][v] += T(0.5) * g[v];
    D::rot_out(nx, ny, Wt, g); for (int v = 0; v < 4; ++v) acc[3][v] += T(0.5) * g[v];
  }
  for (int k = 0; k < 4; ++k)
    for (int v = 0; v < 4; ++v) out[(k * 4 + v) * nf + f] = acc[k][v];
}
template <typename T, int SH, bool FULL = false, bool CHAR = false>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH)) k_face(MeshT<T> m, ParamsT<T> P,
                                                                       const T *__restrict__ W,
                                                                       const T *__restrict__ Wx,
                                                                       const T *__restrict__ coef,
                                                                       T *__restrict__ out, const Ctl *ctl,
                                                                       const unsigned long long *dt_bits) {
  pdl_enter();
  for_items<SH>(m.nf, [&](int f) { face_at<T, FULL, CHAR>(m, P, W, Wx, coef, out, ctl, dt_bits, f); });
  pdl_exit();
}

// K3 modes
enum UpdMode { kS1O2 = 0, kS2O4Stage = 1, kS2O4Final = 2, kResidual = 3 };

// K3: gather the face sums of each cell (accumulated in FP64).
//   net flux   R  = -sum_p sgn S_p (a0 F0A + a1 F1A + a2 F1B)
//   W_out = W_base + dt/|Omega| R   (not in kResidual mode)
//   Wx_out = 1/|Omega| sum_p sgn S_p n_p (WcA + b1 WtX)
// optional outputs: R itself, float mirrors of W_out / Wx_out, the
// per-block density-residual partial sums; plus the state check.
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_update(MeshT<double> m, ParamsT<double> P, int mode,
                                                       const double *__restrict__ Wbase, const TF *__restrict__ FA,
                                                       const TF *__restrict__ FB, const Ctl *ctl,
                                                       const unsigned long long *dt_bits, int *status,
                                                       double *__restrict__ Wout, double *__restrict__ Wxout,
                                                       double *__restrict__ partial, double *__restrict__ Rout,
                                                       TF *__restrict__ Wout_m, TF *__restrict__ Wxout_m) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = m.nc, nf = m.nf;
  double num = 0.0, den = 0.0;
  const int sid = i < n ? m.csid[i] : -1;
  if (sid >= 0) {
    double dt = dt_of(ctl, dt_bits, sid, P.cfl_hi);
    double a0, a1, b1;
    const TF *FW = FA;   // where Wt is taken from
    switch (mode) {
      case kS1O2: a0 = 1.0; a1 = 0.5 * dt; b1 = dt; break;
      case kS2O4Stage: a0 = 0.5; a1 = 0.125 * dt; b1 = 0.5 * dt; break;
      case kS2O4Final: a0 = 1.0; a1 = dt / 6.0; b1 = dt; FW = FB; break;
      default: a0 = 1.0; a1 = 0.5 * dt; b1 = 0.0; break;
    }
    double R[4] = { 0, 0, 0, 0 }, gx[4] = { 0, 0, 0, 0 }, gy[4] = { 0, 0, 0, 0 };
    for (int s = 0; s < kMaxFace; ++s) {
      int fs = m.cface[s * n + i];
      if (fs == kNoFace) continue;
      int f = fs >= 0 ? fs : ~fs;
      double sg = fs >= 0 ? 1.0 : -1.0;
      double S = m.fS[f], nx = m.fn[f], ny = m.fn[nf + f];
      for (int v = 0; v < 4; ++v) {
        double f1 = static_cast<double>(FA[(4 + v) * nf + f]);
        if (mode == kS2O4Final) f1 += 2.0 * static_cast<double>(FB[(4 + v) * nf + f]);
        double fl = S * (a0 * static_cast<double>(FA[v * nf + f]) + a1 * f1);
        R[v] -= sg * fl;
        if (mode != kResidual) {
          double wp = static_cast<double>(FA[(8 + v) * nf + f]) + b1 * static_cast<double>(FW[(12 + v) * nf + f]);
          gx[v] += sg * S * nx * wp;
          gy[v] += sg * S * ny * wp;
        }
      }
    }
    if (Rout)
      for (int v = 0; v < 4; ++v) Rout[v * n + i] = R[v];
    if (mode != kResidual) {
      double iv = m.ivol[i];
      double w[4];
      for (int v = 0; v < 4; ++v) {
        w[v] = Wbase[v * n + i] + dt / m.vol[i] * R[v];
        Wout[v * n + i] = w[v];
        Wxout[v * n + i] = gx[v] * iv;
        Wxout[(4 + v) * n + i] = gy[v] * iv;
        if (Wout_m) {
          Wout_m[v * n + i] = static_cast<TF>(w[v]);
          Wxout_m[v * n + i] = static_cast<TF>(gx[v] * iv);
          Wxout_m[(4 + v) * n + i] = static_cast<TF>(gy[v] * iv);
        }
      }
      if (!state_ok(P.gamma, w)) atomicOr(&status[sid], kBadState);
      num = fabs(w[0] - Wbase[i]);
      den = Wbase[i];
    }
  }
  if (partial) block_sum2(num, den, &partial[2 * blockIdx.x]);
  pdl_exit();
}

// Sum each solve's block partials in a fixed order (one block per solve
// slot; blk[2s], blk[2s+1] its cell blocks): Res_s = num / den.  Slot 0
// also appends to the residual history.
__global__ void k_res_final(const double *__restrict__ partial, const int *__restrict__ blk, Ctl *ctl,
                            double *__restrict__ res, double *hist, int cap, double *last) {
  pdl_enter();
  const int s = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int k = blk[2 * s] + threadIdx.x; k < blk[2 * s + 1]; k += blockDim.x) {
    a += partial[2 * k];
    b += partial[2 * k + 1];
  }
  __shared__ double tot[2];
  block_sum2(a, b, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = tot[0] / tot[1];
    res[s] = r;
    if (s == 0) {
      last[0] = r; last[1] = tot[0]; last[2] = tot[1];
      int c = ctl->res_ctr;
      if (hist && c < cap) hist[c] = r;
      ctl->res_ctr = c + 1;
    }
  }
  pdl_exit();
}

// ---------------------------- low-order level ----------------------------
// K5a: per-cell start of an implicit step: U = W_p0 (first step) or
// U += dU (Algorithm 1's update, in FP64), then the primitives of U (and
// its float mirror in mixed mode).
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_lo_cell(int n, ParamsT<TF> P, int first, const double *__restrict__ Wp0,
                                                        double *__restrict__ U, const TF *__restrict__ dU,
                                                        TF *__restrict__ prim, TF *__restrict__ Um) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  TF w[4];
  for (int v = 0; v < 4; ++v) {
    double u = first ? Wp0[v * n + i] : U[v * n + i] + static_cast<double>(dU[v * n + i]);
    U[v * n + i] = u;
    w[v] = static_cast<TF>(u);
    if (Um) Um[v * n + i] = w[v];
  }
  D::Prim<TF> q = D::prim_of(w, P.gamma, P.kc);
  prim[0 * n + i] = q.rho; prim[1 * n + i] = q.u; prim[2 * n + i] = q.v; prim[3 * n + i] = q.p;
  prim[4 * n + i] = q.i2l; prim[5 * n + i] = q.sl; prim[6 * n + i] = q.isp; prim[7 * n + i] = q.c;
  prim[8 * n + i] = q.ir;
  pdl_exit();
}

template <typename T>
__device__ __forceinline__ D::Prim<T> load_prim(const T *__restrict__ prim, int n, int i) {
  D::Prim<T> q;
  q.rho = prim[0 * n + i]; q.u = prim[1 * n + i]; q.v = prim[2 * n + i]; q.p = prim[3 * n + i];
  q.i2l = prim[4 * n + i]; q.sl = prim[5 * n + i]; q.isp = prim[6 * n + i]; q.c = prim[7 * n + i];
  q.ir = prim[8 * n + i];
  return q;
}

// K5b: first-order KFVS flux, spectral radius lambda_p = max of both sides,
// and (FP64 mode) the Euler normal fluxes F_n(U_c0), F_n(U_c1) the
// relaxation reuses.
template <typename T>
struct LoFaceGeo {
  int sid, c0, c1;
  T nx, ny, S, mu, iva, ivb;
};
// mesh and per-solve data of face f (nothing in a cycle writes them)
template <typename T>
__device__ __forceinline__ LoFaceGeo<T> lo_face_geo(const MeshT<T> &m, const ParamsT<T> &P, const int f) {
  LoFaceGeo<T> g;
  g.sid = m.fsid[f];
  g.c0 = g.c1 = 0;
  g.nx = g.ny = g.S = g.mu = g.iva = g.ivb = T(0);
  if (g.sid < 0) return g;
  const int nf = m.nf;
  g.c0 = m.fc0[f];
  g.c1 = m.fc1[f];
  g.nx = m.fn[f];
  g.ny = m.fn[nf + f];
  g.S = m.fS[f];
  g.mu = P.mu[g.sid];
  g.iva = m.ivol[g.c0];
  g.ivb = g.c1 >= 0 ? m.ivol[g.c1] : g.iva;
  return g;
}
template <typename T>
__device__ __forceinline__ void lo_face_at(const MeshT<T> &m, const ParamsT<T> &P, const LoFaceGeo<T> &g,
                                           const T *__restrict__ U, const T *__restrict__ prim,
                                           T *__restrict__ Flo, T *__restrict__ lam, T *__restrict__ E0,
                                           T *__restrict__ E1, const int f) {
  if (g.sid < 0) return;   // free face space of a batch
  const int n = m.nc, nf = m.nf;
  const int c0 = g.c0, c1 = g.c1;
  const T nx = g.nx, ny = g.ny, S = g.S;
  const T mu = g.mu;
  D::Prim<T> a = load_prim(prim, n, c0), b;
  const T ivb = g.ivb;
  T wa[4], wb[4];   // states of the two sides (global frame); wb is the ghost on a boundary
  const bool need_w = P.flux_lo == CGKS_FLUX_LF || E0 != nullptr;
  if (c1 >= 0) {
    b = load_prim(prim, n, c1);
    if (need_w)
      for (int v = 0; v < 4; ++v) { wa[v] = U[v * n + c0]; wb[v] = U[v * n + c1]; }
  } else {
    for (int v = 0; v < 4; ++v) wa[v] = U[v * n + c0];
    lo_ghost(P, -1 - c1, nx, ny, wa, wb);
    b = D::prim_of(wb, P.gamma, P.kc);
  }
  const T una = a.u * nx + a.v * ny, uta = -a.u * ny + a.v * nx;
  const T unb = b.u * nx + b.v * ny, utb = -b.u * ny + b.v * nx;
  const T la = fabs(una) + a.c + T(2) * (mu * a.ir) * S * g.iva;
  const T lb = fabs(unb) + b.c + T(2) * (mu * b.ir) * S * ivb;
  const T lmax = la > lb ? la : lb;
  lam[f] = lmax;
  // Euler normal fluxes of the two sides (the L-F flux, the FP64 cache)
  T Fa[4], Fb[4];
  if (need_w) {
    Fa[0] = a.rho * una; Fa[1] = wa[1] * una + a.p * nx; Fa[2] = wa[2] * una + a.p * ny; Fa[3] = (wa[3] + a.p) * una;
    Fb[0] = b.rho * unb; Fb[1] = wb[1] * unb + b.p * nx; Fb[2] = wb[2] * unb + b.p * ny; Fb[3] = (wb[3] + b.p) * unb;
  }
  T F[4];
  if (P.flux_lo == CGKS_FLUX_LF) {
    // Lax-Friedrichs alternative of Section 3 with the implicit operator's
    // lambda_p: (F_n(U_l) + F_n(U_r)) / 2 - lambda_p (U_r - U_l) / 2
    for (int v = 0; v < 4; ++v) F[v] = T(0.5) * (Fa[v] + Fb[v]) - T(0.5) * lmax * (wb[v] - wa[v]);
  } else {
    T Fl[4];
    D::kfvs_prims(P.K, a.rho, una, uta, a.i2l, a.sl, a.isp, b.rho, unb, utb, b.i2l, b.sl, b.isp, Fl);
    D::rot_out(nx, ny, Fl, F);
  }
  if (P.lo_viscous && mu > T(0)) {
    // first-order viscous flux: normal gradients from the two cell states
    // over the centre distance delta, Stokes' hypothesis, Pr = 1 heat flux
    //   tau.n = mu / delta (du + (n.du) n / 3),  q.n = -kappa (T_r - T_l) / delta
    const T md = mu * m.fidl[f];
    const T dux = b.u - a.u, duy = b.v - a.v;
    const T dn = (dux * nx + duy * ny) / T(3);
    const T tx = md * (dux + dn * nx), ty = md * (duy + dn * ny);
    const T qn = -md * P.gamma / (P.gamma - T(1)) * (b.p * b.ir - a.p * a.ir);
    F[1] -= tx;
    F[2] -= ty;
    F[3] -= tx * (T(0.5) * (a.u + b.u)) + ty * (T(0.5) * (a.v + b.v)) - qn;
  }
  for (int v = 0; v < 4; ++v) Flo[v * nf + f] = F[v];
  if (E0) {
    // Euler normal flux of the cell means (interior faces: both sides)
    for (int v = 0; v < 4; ++v) E0[v * nf + f] = Fa[v];
    if (c1 >= 0)
      for (int v = 0; v < 4; ++v) E1[v * nf + f] = Fb[v];
  }
}
template <typename T, int SH>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH)) k_lo_face(MeshT<T> m, ParamsT<T> P,
                                                                          const T *__restrict__ U,
                                                                          const T *__restrict__ prim,
                                                                          T *__restrict__ Flo, T *__restrict__ lam,
                                                                          T *__restrict__ E0, T *__restrict__ E1) {
  for_items_pdl<SH>(m.nf, [&](int f) { return lo_face_geo(m, P, f); },
                    [&](int f, const LoFaceGeo<T> &g) { lo_face_at(m, P, g, U, prim, Flo, lam, E0, E1, f); });
  pdl_exit();
}

// K6: low-order right-hand side R^k = R_lo(U^k) + S (FP64 sums), 1/D_i
// (FP64 inversion), each slot's lambda for the sweeps, and the first colour
// pass of the relaxation: with dU = 0 everywhere the update of a colour-0
// cell reduces to R_i / D_i; all other cells start at 0.  first: also
// forms the forcing S = R_p0 - R_lo(W_p0) (Section 3, step 3).
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_lo_rhs(MeshT<double> m, ParamsT<double> P, int first, int colour0,
                                                       const TF *__restrict__ Flo, const TF *__restrict__ lam,
                                                       const double *__restrict__ Rp0, double *__restrict__ Src,
                                                       TF *__restrict__ Rk, TF *__restrict__ invD, TF *__restrict__ dU,
                                                       TF *__restrict__ lamS) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.nc) { pdl_enter(); return; }
  const int n = m.nc, nf = m.nf;
  // mesh data first (nothing in a cycle writes it), then wait for the predecessor
  int fsl[kMaxFace];
  double Sl[kMaxFace];
#pragma unroll
  for (int s = 0; s < kMaxFace; ++s) {
    fsl[s] = m.cface[s * n + i];
    Sl[s] = fsl[s] == kNoFace ? 0.0 : m.fS[fsl[s] >= 0 ? fsl[s] : ~fsl[s]];
  }
  const bool c0 = colour0 && m.ccol[i] == 0;
  pdl_enter();
  double R[4] = { 0, 0, 0, 0 }, sum = 0.0;
#pragma unroll
  for (int s = 0; s < kMaxFace; ++s) {
    int fs = fsl[s];
    if (fs == kNoFace) { lamS[s * n + i] = TF(0); continue; }
    int f = fs >= 0 ? fs : ~fs;
    double sg = fs >= 0 ? 1.0 : -1.0;
    double S = Sl[s];
    for (int v = 0; v < 4; ++v) R[v] -= sg * S * static_cast<double>(Flo[v * nf + f]);
    TF l = lam[f];
    lamS[s * n + i] = l;
    sum += static_cast<double>(l) * S;
  }
  // dt_i = CFL_lo |Omega| / sum;  D_i = |Omega| / dt_i + sum / 2 (padding cells: 0)
  const double id = sum > 0.0 ? 1.0 / (sum / P.cfl_lo + 0.5 * sum) : 0.0;
  invD[i] = static_cast<TF>(id);
  for (int v = 0; v < 4; ++v) {
    double src;
    if (first) { src = Rp0[v * n + i] - R[v]; Src[v * n + i] = src; }
    else src = Src[v * n + i];
    double r = R[v] + src;
    Rk[v * n + i] = static_cast<TF>(r);
    dU[v * n + i] = c0 ? static_cast<TF>(r * id) : TF(0);
  }
  pdl_exit();
}

// The cells of one colour form one contiguous range per solve.  A sweep
// launch covers up to kMaxRanges ranges, carried in the kernel parameters
// (constant bank) so no dependent global load precedes the cell's own
// loads: block b works on range r with blk[r] <= b < blk[r+1].
constexpr int kMaxRanges = 64;
struct Ranges {
  int n;
  int blk[kMaxRanges + 1];
  int begin[kMaxRanges], end[kMaxRanges];
};

// cell of local index cl (cells per block: cpb) in the block's range, or -1
__device__ __forceinline__ int range_cell(const Ranges &R, int cl, int cpb) {
  int r = 0;
  if (R.n > 1) {
    int lo = 0, hi = R.n - 1;   // largest r with blk[r] <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (R.blk[mid] <= static_cast<int>(blockIdx.x)) lo = mid; else hi = mid - 1;
    }
    r = lo;
  }
  const int i = R.begin[r] + (static_cast<int>(blockIdx.x) - R.blk[r]) * cpb + cl;
  return i < R.end[r] ? i : -1;
}

// K7: point relaxation of the cells of one colour (ranges or a list
// spanning every solve of the batch), Eq. (implicit-local):
//   dU_i = (R_i - sum_p S_p [F^-(U_ip + dU_ip) - F^-(U_ip)]) / D_i,
//   F^-(U) = (F_n(U) - lambda_p U) / 2, ghost increments zero.
// FP64: F_n(U_ip) from the face cache of this implicit step.  Mixed: the
// difference F_n(U_ip + dU_ip) - F_n(U_ip) in the exact increment form.
// Four lanes per cell, one per face slot: each lane evaluates its
// neighbour's term, the four terms are summed by shuffles within the lane
// group, and lane v writes component v.  Cells of one colour never
// neighbour each other, so the dU_ip read here are not written by this
// launch.
// static (mesh) data of one lane of a sweep: the neighbour across face
// slot s of cell i and the slot geometry; read before the kernel waits on
// its predecessor, since no kernel of a cycle writes it
template <typename T>
struct SweepGeo {
  int j, f;
  bool is0;
  T nx, ny, hS;
};
template <typename T>
__device__ __forceinline__ SweepGeo<T> sweep_geo(const MeshT<T> &m, const int i, const int s) {
  const int n = m.nc;
  SweepGeo<T> g;
  g.j = i >= 0 ? m.cnbr[s * n + i] : -1;
  g.f = 0;
  g.is0 = true;
  g.nx = g.ny = g.hS = T(0);
  if (g.j >= 0) {
    g.nx = m.snx[s * n + i];
    g.ny = m.sny[s * n + i];
    g.hS = m.shs[s * n + i];
    if constexpr (!is_f32<T>()) {
      const int fs = m.cface[s * n + i];
      g.is0 = fs >= 0;
      g.f = g.is0 ? fs : ~fs;
    }
  }
  return g;
}
// The relaxation of cell i by its 4-lane group; the neighbour's increment
// is read from dn (through L2 when l2 is set: values another CTA of the
// launch wrote), the cell's new increment written to dU.
template <typename T>
__device__ __forceinline__ void sweep_cell_from(const MeshT<T> &m, const ParamsT<T> &P, const SweepGeo<T> &g,
                                                const int i, const int s, const T *__restrict__ U,
                                                const T *__restrict__ prim, const T *__restrict__ Rk,
                                                const T *__restrict__ invD, const T *__restrict__ lamS,
                                                const T *__restrict__ E0, const T *__restrict__ E1,
                                                const T *dn, const bool l2, T *dU) {
  const int n = m.nc, nf = m.nf;
  const int j = g.j;
  // every lane stays to the shuffles; lanes of absent cells or slots add 0
  T c[4] = { T(0), T(0), T(0), T(0) };
  if (j >= 0) {
    const T nx = g.nx, ny = g.ny, hS = g.hS, lp = lamS[s * n + i];
    T uj[4], du[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      uj[v] = U[v * n + j];
      du[v] = l2 ? __ldcg(&dn[v * n + j]) : dn[v * n + j];
    }
    if constexpr (is_f32<T>()) {
      T dF[4];
      D::euler_flux_delta(P.gamma, uj, prim[1 * n + j], prim[2 * n + j], prim[3 * n + j], du, nx, ny, dF);
#pragma unroll
      for (int v = 0; v < 4; ++v) c[v] = hS * (dF[v] - lp * du[v]);
    } else {
      const int f = g.f;
      T up[4], fa[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) up[v] = uj[v] + du[v];
      D::euler_flux(P.gamma, up, nx, ny, fa);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const T fb = g.is0 ? E1[v * nf + f] : -E0[v * nf + f];
        c[v] = hS * ((fa[v] - fb) - lp * du[v]);   // (U + dU) - U = dU
      }
    }
  }
  // lane s needs component s summed over the group: a transposing
  // reduction (3 additions per lane instead of an all-reduce of 4 values)
  const bool b0 = s & 1, b1 = s & 2;
  const T k0 = (b0 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b0 ? c[0] : c[1], 1);   // component b0
  const T k1 = (b0 ? c[3] : c[2]) + __shfl_xor_sync(0xffffffffu, b0 ? c[2] : c[3], 1);   // component b0 + 2
  const T mine = (b1 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, b1 ? k0 : k1, 2);
  if (i >= 0) dU[s * n + i] = (Rk[s * n + i] - mine) * invD[i];
}
template <typename T>
__device__ __forceinline__ void sweep_cell(const MeshT<T> &m, const ParamsT<T> &P, const SweepGeo<T> &g,
                                           const int i, const int s, const T *__restrict__ U,
                                           const T *__restrict__ prim, const T *__restrict__ Rk,
                                           const T *__restrict__ invD, const T *__restrict__ lamS,
                                           const T *__restrict__ E0, const T *__restrict__ E1, T *dU) {
  sweep_cell_from(m, P, g, i, s, U, prim, Rk, invD, lamS, E0, E1, dU, false, dU);
}
// cells per block of a sweep launch of shape SH
__host__ __device__ constexpr int sweep_cpb(int sh) { return shape_bs(sh) / kMaxFace * shape_ipt(sh); }
template <typename T, int SH>
__global__ void __launch_bounds__(shape_bs(SH), shape_minb(SH)) k_sweep(MeshT<T> m, ParamsT<T> P,
                                                                        const __grid_constant__ Ranges R,
                                                                        const int *__restrict__ list, int count,
                                                                        const T *__restrict__ U,
                                                                        const T *__restrict__ prim,
                                                                        const T *__restrict__ Rk,
                                                                        const T *__restrict__ invD,
                                                                        const T *__restrict__ lamS,
                                                                        const T *__restrict__ E0,
                                                                        const T *__restrict__ E1, T *__restrict__ dU) {
  constexpr int kGroups = shape_bs(SH) / kMaxFace, kCpb = sweep_cpb(SH), kIpt = shape_ipt(SH);
  const int s = threadIdx.x & (kMaxFace - 1);
  // one copy of the per-cell code for every shape (the same arithmetic);
  // the first item's mesh data is read before the wait, later items' after
#pragma unroll 1
  for (int k = 0; k < kIpt; ++k) {
    const int cl = k * kGroups + static_cast<int>(threadIdx.x) / kMaxFace;
    int i;
    if (list) {
      const int g = static_cast<int>(blockIdx.x) * kCpb + cl;
      i = g < count ? list[g] : -1;
    } else {
      i = range_cell(R, cl, kCpb);
    }
    const SweepGeo<T> geo = sweep_geo(m, i, s);
    pdl_enter();
    sweep_cell(m, P, geo, i, s, U, prim, Rk, invD, lamS, E0, E1, dU);
  }
  pdl_exit();
}

// ---- the partitioned sweep (CGKS_SWEEP_PARTITIONED) ----
// One launch is one sweep of Algorithm 1 -- a forward pass over the
// colours, then a backward pass -- over every partition at once.  A
// thread-block cluster owns one partition: its CTAs share out each
// colour's cells of the partition, and a cluster barrier (release /
// acquire at cluster scope) separates consecutive colours, so a cell sees
// the increments its partition's earlier colours just wrote to dU_out
// (read through L2).  Neighbours in other partitions, and cells of this
// partition not yet relaxed in this sweep, are read from dU_in, the
// increments at the start of the sweep: partitions exchange once per
// sweep, lagged, like the paper's threads.  Every cell of every partition
// is written to dU_out.  The colour C-1 ending the forward pass is not
// relaxed again at the start of the backward pass: with its inputs
// unchanged it would recompute the same values.
constexpr int kPartBlock = 256;        // threads per CTA: 64 cells per pass of a CTA
constexpr int kPartCluster = 8;        // CTAs per partition (portable cluster size)
constexpr int kMaxPartColours = 16;

__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; orders the global writes before
// it (release) before the reads after it (acquire), cluster scope
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ptab [Q][C][2]: first and end cell (internal index) of colour c in
// partition q; C colours
template <typename T>
__global__ void __launch_bounds__(kPartBlock) k_sweep_part(MeshT<T> m, ParamsT<T> P, const int *__restrict__ ptab,
                                                           int C, const T *__restrict__ U,
                                                           const T *__restrict__ prim, const T *__restrict__ Rk,
                                                           const T *__restrict__ invD,
                                                           const T *__restrict__ lamS, const T *__restrict__ E0,
                                                           const T *__restrict__ E1, const T *__restrict__ dU_in,
                                                           T *dU_out) {
  __shared__ int sb[kMaxPartColours], se[kMaxPartColours];
  const unsigned K = cluster_nctarank(), rank = cluster_ctarank();
  const int q = static_cast<int>(blockIdx.x / K);
  if (static_cast<int>(threadIdx.x) < C) {
    sb[threadIdx.x] = ptab[2 * (q * C + threadIdx.x)];
    se[threadIdx.x] = ptab[2 * (q * C + threadIdx.x) + 1];
  }
  __syncthreads();
  constexpr int G = kPartBlock / kMaxFace;          // cells per pass of a CTA
  const int s = threadIdx.x & (kMaxFace - 1);
  const int cl = static_cast<int>(threadIdx.x) / kMaxFace;
  pdl_enter();
  const int steps = 2 * C - 1;
  for (int step = 0; step < steps; ++step) {
    const bool fwd = step < C;
    const int c = fwd ? step : 2 * C - 2 - step;
    const int b = sb[c], e = se[c];
    // the CTA's passes are uniform over its threads (the shuffles need
    // whole lane groups)
    for (int base = b + static_cast<int>(rank) * G; base < e; base += static_cast<int>(K) * G) {
      const int i = base + cl < e ? base + cl : -1;
      const SweepGeo<T> g = sweep_geo(m, i, s);
      bool fresh = false;
      if (g.j >= 0) {
        const int cj = m.ccol[g.j];
        fresh = cj < C && g.j >= sb[cj] && g.j < se[cj] && (!fwd || cj < c);
      }
      sweep_cell_from(m, P, g, i, s, U, prim, Rk, invD, lamS, E0, E1, fresh ? dU_out : dU_in, fresh, dU_out);
    }
    if (step + 1 < steps) cluster_sync();
  }
  pdl_exit();
}

// K9: prolongation W = W_p0 + (U - W_p0) (Section 3, step 5), density
// residual against the state at the start of the cycle, state check.
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_prolong(MeshT<double> m, ParamsT<double> P, double *__restrict__ W,
                                                        const double *__restrict__ Wp0, const double *__restrict__ U,
                                                        int *status, double *__restrict__ partial,
                                                        TF *__restrict__ Wm) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = m.nc;
  double num = 0.0, den = 0.0;
  const int sid = i < n ? m.csid[i] : -1;
  if (i < n) {
    double w[4];
    double old_rho = W[i];
    for (int v = 0; v < 4; ++v) {
      double wp = Wp0[v * n + i];
      w[v] = wp + (U[v * n + i] - wp);
      W[v * n + i] = w[v];
      if (Wm) Wm[v * n + i] = static_cast<TF>(w[v]);
    }
    if (sid >= 0) {
      if (!state_ok(P.gamma, w)) atomicOr(&status[sid], kBadState);
      num = fabs(w[0] - old_rho);
      den = old_rho;
    }
  }
  block_sum2(num, den, &partial[2 * blockIdx.x]);
  pdl_exit();
}

// Caller AoS order <-> internal SoA order for the n cells of one solve
// starting at internal offset off (perm: internal within solve -> caller).
__global__ void k_gather_state(int ns, int off, int N, const int *__restrict__ perm, const double *__restrict__ Wa,
                               const double *__restrict__ Wxa, double *__restrict__ W, double *__restrict__ Wx,
                               float *__restrict__ W32, float *__restrict__ Wx32) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  int c = perm[k], i = off + k;
  for (int v = 0; v < 4; ++v) {
    double w = Wa[4 * c + v];
    W[v * N + i] = w;
    if (W32) W32[v * N + i] = static_cast<float>(w);
  }
  for (int q = 0; q < 8; ++q) {
    double g = Wxa ? Wxa[8 * c + q] : 0.0;
    Wx[q * N + i] = g;
    if (Wx32) Wx32[q * N + i] = static_cast<float>(g);
  }
}
__global__ void k_scatter_state(int ns, int off, int N, const int *__restrict__ perm, const double *__restrict__ W,
                                const double *__restrict__ Wx, double *__restrict__ Wa, double *__restrict__ Wxa) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  int c = perm[k], i = off + k;
  if (Wa) for (int v = 0; v < 4; ++v) Wa[4 * c + v] = W[v * N + i];
  if (Wxa) for (int q = 0; q < 8; ++q) Wxa[8 * c + q] = Wx[q * N + i];
}
// Inert cells (padding, free space of a batch): no faces, no neighbours,
// no solve, no colour, and a valid uniform state so that the arithmetic the
// cell kernels still do for them stays finite.
__global__ void k_clear_cells(int c0, int c1, int N, int *__restrict__ csid, unsigned char *__restrict__ ccol,
                              int *__restrict__ cface, int *__restrict__ cnbr, double *__restrict__ W,
                              double *__restrict__ Wx, double *__restrict__ Wn, double *__restrict__ Ws,
                              double *__restrict__ Wxs, float *__restrict__ W32, float *__restrict__ Wx32,
                              float *__restrict__ Wn32, float *__restrict__ Ws32, float *__restrict__ Wxs32) {
  const int i = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c1) return;
  csid[i] = -1;
  ccol[i] = 255;
  for (int s = 0; s < kMaxFace; ++s) { cface[s * N + i] = kNoFace; cnbr[s * N + i] = -1; }
  const double w[4] = { 1.0, 0.0, 0.0, 2.5 };
  for (int v = 0; v < 4; ++v) {
    W[v * N + i] = w[v]; Wn[v * N + i] = w[v]; Ws[v * N + i] = w[v];
    if (W32) { W32[v * N + i] = static_cast<float>(w[v]); Wn32[v * N + i] = static_cast<float>(w[v]);
               Ws32[v * N + i] = static_cast<float>(w[v]); }
  }
  for (int q = 0; q < 8; ++q) {
    Wx[q * N + i] = 0.0; Wxs[q * N + i] = 0.0;
    if (Wx32) { Wx32[q * N + i] = 0.0f; Wxs32[q * N + i] = 0.0f; }
  }
}

}  // namespace kern
}  // namespace cgks
