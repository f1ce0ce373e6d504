// libcgks device runtime: kernels of the high-order level (compact
// reconstruction, gas-kinetic face flux, S1O2 / S2O4 update with
// Gauss-Green gradients), of the low-order level (KFVS residual, L-F
// diagonal, coloured point relaxation) and of the two-level V-cycle of
// Ji, Shyy & Xu (arXiv:2109.09965), plus the C ABI declared in cgks.h.
//
// Layout: structure-of-arrays in the library's cell order (colour-major,
// reverse Cuthill-McKee inside a colour).  One thread per cell or face.
// The cell update gathers the face sums through each cell's face slots
// (no atomics, deterministic); reductions use a fixed block tree.
//
// Precision: kernels that evaluate fluxes are templated on the flux type
// TF.  FP64 mode runs everything in double.  Mixed mode keeps the
// conservative variables (W, W_x, U) and every accumulation into them, the
// residuals and the diagonal inversion in double, and runs reconstruction,
// face fluxes and relaxation sweeps in float on float mirrors of the state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "cgks_internal.h"
#include "cgks_physics.cuh"

using namespace cgks;
namespace D = cgks::dev;

namespace {

constexpr int kCellBlock = 256;
constexpr int kFaceBlock = 128;
constexpr int kSweepBlock = 128;

// status bits of the device status word
constexpr int kBadState = 1;

template <typename T>
struct ParamsT {
  T gamma, K, mu, cfl_hi, cfl_lo;
  D::KC<T> kc;
  int bc_kind[CGKS_MAX_BC];
  T bc_uw[CGKS_MAX_BC][2];
  T bc_rho[CGKS_MAX_BC], bc_u[CGKS_MAX_BC][2], bc_p[CGKS_MAX_BC];
};

template <typename T>
struct MeshT {
  int nc, nf;
  const T *vol, *ivol, *per, *ih, *m2;       // ih = 1/h; m2: [3][nc]
  const T *op;                               // [kNCol*kNM][nc]
  const T *fn, *fS, *fjump, *fxi;            // fn [2][nf], fjump = alpha/delta, fxi [8][nf]
  const T *snx, *sny, *shs;                  // [4][nc] per face slot: outward normal of the cell, S/2
  const int *cface, *cnbr;                   // [4][nc]
  const int *fc0, *fc1;
};

// arrays in the flux type TF (in FP64 mode the state entries alias the
// double state, in mixed mode they are float mirrors)
template <typename T>
struct Bufs {
  T *W = nullptr, *Wx = nullptr, *Wn = nullptr, *Ws = nullptr, *Wxs = nullptr, *U = nullptr;
  T *coef = nullptr, *FA = nullptr, *FB = nullptr;
  T *prim = nullptr, *Flo = nullptr, *lam = nullptr, *E0 = nullptr, *E1 = nullptr;
  T *Rk = nullptr, *invD = nullptr, *dU = nullptr, *lamS = nullptr;
};

struct Scalars {
  unsigned long long dt_bits;   // min over cells of the local explicit step (bits of a positive double)
  int status;
  int res_ctr;                  // next slot of the residual history
  double dt_fixed;              // > 0: prescribed step
};

template <typename T>
__host__ __device__ constexpr bool is_f32() { return std::is_same<T, float>::value; }

__device__ __forceinline__ double dt_value(const Scalars *sc, double cfl) {
  if (sc->dt_fixed > 0.0) return sc->dt_fixed;
  return cfl * __longlong_as_double(static_cast<long long>(sc->dt_bits));
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
// K0: reset per-step scalars
__global__ void k_reset_dt(Scalars *sc, double dt_fixed) {
  sc->dt_bits = 0x7ff0000000000000ull;  // +inf
  sc->dt_fixed = dt_fixed;
}

// K4: local explicit step per cell, global min by atomicMin on the bits
// (min is order independent).  h = 2|Omega|/perimeter, speed |U| + c + 2 nu / h.
__global__ void k_dt(MeshT<double> m, ParamsT<double> P, const double *__restrict__ W, Scalars *sc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double d = INFINITY;
  if (i < m.nc) {
    int n = m.nc;
    double rho = W[i], mx = W[n + i], my = W[2 * n + i], E = W[3 * n + i];
    double u = mx / rho, v = my / rho;
    double p = (P.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    double a = sqrt(P.gamma * p / rho);
    double hh = 2.0 * m.vol[i] / m.per[i];
    double speed = sqrt(u * u + v * v) + a + 2.0 * (P.mu / rho) / hh;
    d = hh / speed;
  }
  for (int o = 16; o > 0; o >>= 1) d = fmin(d, __shfl_down_sync(0xffffffffu, d, o));
  if ((threadIdx.x & 31) == 0 && d < INFINITY)
    atomicMin(&sc->dt_bits, static_cast<unsigned long long>(__double_as_longlong(d)));
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
    T wn = P.bc_uw[tag][0] * nx + P.bc_uw[tag][1] * ny;
    T wt = -P.bc_uw[tag][0] * ny + P.bc_uw[tag][1] * nx;
    D::ghost_noslip(P.gamma, wn, wt, wl, dn, dt, wgl, dng, dtg);
  }
  T gn[4], gt[4];
  D::rot_out(nx, ny, wgl, wg);
  D::rot_out(nx, ny, dng, gn);
  D::rot_out(nx, ny, dtg, gt);
  for (int v = 0; v < 4; ++v) { ggx[v] = nx * gn[v] - ny * gt[v]; ggy[v] = ny * gn[v] + nx * gt[v]; }
}

// K1: compact least-squares quadratic of every cell.
//   coef[(q*4 + v)*nc + i], q over (xi, eta, xi^2, xi eta, eta^2).
template <typename T>
__global__ void __launch_bounds__(kCellBlock) k_recon(MeshT<T> m, ParamsT<T> P, const T *__restrict__ W,
                                                      const T *__restrict__ Wx, T *__restrict__ coef) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.nc) return;
  const int n = m.nc;
  T wi[4], gxi[4], gyi[4];
  for (int v = 0; v < 4; ++v) { wi[v] = W[v * n + i]; gxi[v] = Wx[v * n + i]; gyi[v] = Wx[(4 + v) * n + i]; }
  T c[kNM][4];
  for (int q = 0; q < kNM; ++q) {
    T o0 = m.op[((kNCol - 2) * kNM + q) * n + i], o1 = m.op[((kNCol - 1) * kNM + q) * n + i];
    for (int v = 0; v < 4; ++v) c[q][v] = o0 * gxi[v] + o1 * gyi[v];
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
    } else {
      int f = fs >= 0 ? fs : ~fs;
      int tag = -1 - m.fc1[f];
      if (P.bc_kind[tag] == CGKS_BC_FARFIELD) continue;
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
  for (int q = 0; q < kNM; ++q)
    for (int v = 0; v < 4; ++v) coef[(q * 4 + v) * n + i] = c[q][v];
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

template <typename T>
__device__ __forceinline__ void lo_ghost(const ParamsT<T> &P, int tag, T nx, T ny, const T w[4], T wg[4]) {
  T wl[4], z[4] = { T(0), T(0), T(0), T(0) }, wgl[4], a[4], b[4];
  D::rot_in(nx, ny, w, wl);
  int kind = P.bc_kind[tag];
  if (kind == CGKS_BC_FARFIELD) {
    T une = P.bc_u[tag][0] * nx + P.bc_u[tag][1] * ny;
    T ute = -P.bc_u[tag][0] * ny + P.bc_u[tag][1] * nx;
    D::ghost_farfield(P.gamma, P.bc_rho[tag], une, ute, P.bc_p[tag], wl, wgl);
  } else if (kind == CGKS_BC_SLIP) {
    D::ghost_slip(wl, z, z, wgl, a, b);
  } else {
    T wn = P.bc_uw[tag][0] * nx + P.bc_uw[tag][1] * ny;
    T wt = -P.bc_uw[tag][0] * ny + P.bc_uw[tag][1] * nx;
    D::ghost_noslip(P.gamma, wn, wt, wl, z, z, wgl, a, b);
  }
  D::rot_out(nx, ny, wgl, wg);
}

// K2: gas-kinetic flux and interface state at the two Gauss points of every
// face; writes the weighted sums F0, F1, Wc, Wt (global frame) per face:
//   out[(k*4 + v)*nf + f], k = 0 F0, 1 F1, 2 Wc, 3 Wt.
template <typename T>
__global__ void __launch_bounds__(kFaceBlock) k_face(MeshT<T> m, ParamsT<T> P, const T *__restrict__ W,
                                                     const T *__restrict__ coef, T *__restrict__ out) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m.nf) return;
  const int nf = m.nf;
  const int c0 = m.fc0[f], c1 = m.fc1[f];
  const T nx = m.fn[f], ny = m.fn[nf + f], ajump = m.fjump[f];
  T acc[4][4];
  for (int k = 0; k < 4; ++k) for (int v = 0; v < 4; ++v) acc[k][v] = T(0);
  T wff[4];
  bool farfield = false;
  int tag = 0;
  if (c1 < 0) {
    tag = -1 - c1;
    farfield = P.bc_kind[tag] == CGKS_BC_FARFIELD;
    if (farfield) {
      // Riemann-invariant state from the cell mean and the free stream
      T wm[4], wl[4];
      for (int v = 0; v < 4; ++v) wm[v] = W[v * m.nc + c0];
      D::rot_in(nx, ny, wm, wl);
      T une = P.bc_u[tag][0] * nx + P.bc_u[tag][1] * ny;
      T ute = -P.bc_u[tag][0] * ny + P.bc_u[tag][1] * nx;
      D::ghost_farfield(P.gamma, P.bc_rho[tag], une, ute, P.bc_p[tag], wl, wff);
    }
  }
  for (int k = 0; k < 2; ++k) {
    T wL[4], gxL[4], gyL[4];
    recon_point(m, W, coef, c0, m.fxi[(2 * k) * nf + f], m.fxi[(2 * k + 1) * nf + f], wL, gxL, gyL);
    T wl[4], dnl[4], dtl[4], t0[4], t1[4];
    D::rot_in(nx, ny, wL, wl);
    for (int v = 0; v < 4; ++v) { t0[v] = nx * gxL[v] + ny * gyL[v]; t1[v] = -ny * gxL[v] + nx * gyL[v]; }
    D::rot_in(nx, ny, t0, dnl);
    D::rot_in(nx, ny, t1, dtl);
    T wr[4], dnr[4], dtr[4];
    if (c1 >= 0) {
      T wR[4], gxR[4], gyR[4];
      recon_point(m, W, coef, c1, m.fxi[(4 + 2 * k) * nf + f], m.fxi[(5 + 2 * k) * nf + f], wR, gxR, gyR);
      D::rot_in(nx, ny, wR, wr);
      for (int v = 0; v < 4; ++v) { t0[v] = nx * gxR[v] + ny * gyR[v]; t1[v] = -ny * gxR[v] + nx * gyR[v]; }
      D::rot_in(nx, ny, t0, dnr);
      D::rot_in(nx, ny, t1, dtr);
    } else if (farfield) {
      for (int v = 0; v < 4; ++v) { wr[v] = wff[v]; dnr[v] = T(0); dtr[v] = T(0); }
    } else if (P.bc_kind[tag] == CGKS_BC_SLIP) {
      D::ghost_slip(wl, dnl, dtl, wr, dnr, dtr);
    } else {
      T wn = P.bc_uw[tag][0] * nx + P.bc_uw[tag][1] * ny;
      T wt = -P.bc_uw[tag][0] * ny + P.bc_uw[tag][1] * nx;
      D::ghost_noslip(P.gamma, wn, wt, wl, dnl, dtl, wr, dnr, dtr);
    }
    T F0[4], F1[4], Wc[4], Wt[4];
    D::gks_point_local(P.kc, P.mu, ajump, wl, wr, dnl, dtl, dnr, dtr, F0, F1, Wc, Wt);
    T g[4];
    D::rot_out(nx, ny, F0, g); for (int v = 0; v < 4; ++v) acc[0][v] += T(0.5) * g[v];
    D::rot_out(nx, ny, F1, g); for (int v = 0; v < 4; ++v) acc[1][v] += T(0.5) * g[v];
    D::rot_out(nx, ny, Wc, g); for (int v = 0; v < 4; ++v) acc[2][v] += T(0.5) * g[v];
    D::rot_out(nx, ny, Wt, g); for (int v = 0; v < 4; ++v) acc[3][v] += T(0.5) * g[v];
  }
  for (int k = 0; k < 4; ++k)
    for (int v = 0; v < 4; ++v) out[(k * 4 + v) * nf + f] = acc[k][v];
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
                                                       const TF *__restrict__ FB, Scalars *sc,
                                                       double *__restrict__ Wout, double *__restrict__ Wxout,
                                                       double *__restrict__ partial, double *__restrict__ Rout,
                                                       TF *__restrict__ Wout_m, TF *__restrict__ Wxout_m) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = m.nc, nf = m.nf;
  double num = 0.0, den = 0.0;
  if (i < n) {
    double dt = dt_value(sc, P.cfl_hi);
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
      if (!state_ok(P.gamma, w)) atomicOr(&sc->status, kBadState);
      num = fabs(w[0] - Wbase[i]);
      den = Wbase[i];
    }
  }
  if (partial) block_sum2(num, den, &partial[2 * blockIdx.x]);
}

// Sum the block partials in a fixed order; Res = num / den into hist[ctr++].
__global__ void k_res_final(const double *__restrict__ partial, int nblocks, Scalars *sc, double *hist, int cap,
                            double *last) {
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) { a += partial[2 * k]; b += partial[2 * k + 1]; }
  block_sum2(a, b, last + 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = last[1] / last[2];
    last[0] = r;
    int c = sc->res_ctr;
    if (hist && c < cap) hist[c] = r;
    sc->res_ctr = c + 1;
  }
}

// ---------------------------- low-order level ----------------------------
// K5a: per-cell start of an implicit step: U = W_p0 (first step) or
// U += dU (Algorithm 1's update, in FP64), then the primitives of U (and
// its float mirror in mixed mode).
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_lo_cell(int n, ParamsT<TF> P, int first, const double *__restrict__ Wp0,
                                                        double *__restrict__ U, const TF *__restrict__ dU,
                                                        TF *__restrict__ prim, TF *__restrict__ Um) {
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
__global__ void __launch_bounds__(kCellBlock) k_lo_face(MeshT<T> m, ParamsT<T> P, const T *__restrict__ U,
                                                        const T *__restrict__ prim, T *__restrict__ Flo,
                                                        T *__restrict__ lam, T *__restrict__ E0, T *__restrict__ E1) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= m.nf) return;
  const int n = m.nc, nf = m.nf;
  const int c0 = m.fc0[f], c1 = m.fc1[f];
  const T nx = m.fn[f], ny = m.fn[nf + f], S = m.fS[f];
  D::Prim<T> a = load_prim(prim, n, c0), b;
  T ivb;
  if (c1 >= 0) {
    b = load_prim(prim, n, c1);
    ivb = m.ivol[c1];
  } else {
    T w0[4], wg[4];
    for (int v = 0; v < 4; ++v) w0[v] = U[v * n + c0];
    lo_ghost(P, -1 - c1, nx, ny, w0, wg);
    b = D::prim_of(wg, P.gamma, P.kc);
    ivb = m.ivol[c0];
  }
  const T una = a.u * nx + a.v * ny, uta = -a.u * ny + a.v * nx;
  const T unb = b.u * nx + b.v * ny, utb = -b.u * ny + b.v * nx;
  T Fl[4], F[4];
  D::kfvs_prims(P.K, a.rho, una, uta, a.i2l, a.sl, a.isp, b.rho, unb, utb, b.i2l, b.sl, b.isp, Fl);
  D::rot_out(nx, ny, Fl, F);
  for (int v = 0; v < 4; ++v) Flo[v * nf + f] = F[v];
  const T la = fabs(una) + a.c + T(2) * (P.mu * a.ir) * S * m.ivol[c0];
  const T lb = fabs(unb) + b.c + T(2) * (P.mu * b.ir) * S * ivb;
  lam[f] = la > lb ? la : lb;
  if (E0) {
    // Euler normal flux of the cell means (interior faces: both sides)
    E0[0 * nf + f] = a.rho * una;
    E0[1 * nf + f] = U[1 * n + c0] * una + a.p * nx;
    E0[2 * nf + f] = U[2 * n + c0] * una + a.p * ny;
    E0[3 * nf + f] = (U[3 * n + c0] + a.p) * una;
    if (c1 >= 0) {
      E1[0 * nf + f] = b.rho * unb;
      E1[1 * nf + f] = U[1 * n + c1] * unb + b.p * nx;
      E1[2 * nf + f] = U[2 * n + c1] * unb + b.p * ny;
      E1[3 * nf + f] = (U[3 * n + c1] + b.p) * unb;
    }
  }
}

// K6: low-order right-hand side R^k = R_lo(U^k) + S (FP64 sums), 1/D_i
// (FP64 inversion), and the first colour pass of the relaxation: with
// dU = 0 everywhere the update of a colour-0 cell reduces to R_i / D_i; all
// other cells start at 0.  first: also forms the forcing S = R_p0 -
// R_lo(W_p0) (Section 3, step 3).
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_lo_rhs(MeshT<double> m, ParamsT<double> P, int first, int colour0_end,
                                                       const TF *__restrict__ Flo, const TF *__restrict__ lam,
                                                       const double *__restrict__ Rp0, double *__restrict__ Src,
                                                       TF *__restrict__ Rk, TF *__restrict__ invD, TF *__restrict__ dU,
                                                       TF *__restrict__ lamS) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m.nc) return;
  const int n = m.nc, nf = m.nf;
  double R[4] = { 0, 0, 0, 0 }, sum = 0.0;
  for (int s = 0; s < kMaxFace; ++s) {
    int fs = m.cface[s * n + i];
    if (fs == kNoFace) { lamS[s * n + i] = TF(0); continue; }
    int f = fs >= 0 ? fs : ~fs;
    double sg = fs >= 0 ? 1.0 : -1.0;
    double S = m.fS[f];
    for (int v = 0; v < 4; ++v) R[v] -= sg * S * static_cast<double>(Flo[v * nf + f]);
    TF l = lam[f];
    lamS[s * n + i] = l;
    sum += static_cast<double>(l) * S;
  }
  // dt_i = CFL_lo |Omega| / sum;  D_i = |Omega| / dt_i + sum / 2
  const double id = 1.0 / (sum / P.cfl_lo + 0.5 * sum);
  invD[i] = static_cast<TF>(id);
  for (int v = 0; v < 4; ++v) {
    double src;
    if (first) { src = Rp0[v * n + i] - R[v]; Src[v * n + i] = src; }
    else src = Src[v * n + i];
    double r = R[v] + src;
    Rk[v * n + i] = static_cast<TF>(r);
    dU[v * n + i] = i < colour0_end ? static_cast<TF>(r * id) : TF(0);
  }
}

// K7: point relaxation of the cells of one colour, Eq. (implicit-local):
//   dU_i = (R_i - sum_p S_p [F^-(U_ip + dU_ip) - F^-(U_ip)]) / D_i,
//   F^-(U) = (F_n(U) - lambda_p U) / 2, ghost increments zero.
// FP64: F_n(U_ip) from the face cache of this implicit step.  Mixed: the
// difference F_n(U_ip + dU_ip) - F_n(U_ip) in the exact increment form.
// All neighbour loads are issued up front (absent slots read the cell
// itself and contribute nothing) so they overlap.
template <typename T>
__global__ void __launch_bounds__(kSweepBlock) k_sweep(MeshT<T> m, ParamsT<T> P, int begin, int end,
                                                       const T *__restrict__ U, const T *__restrict__ prim,
                                                       const T *__restrict__ Rk, const T *__restrict__ invD,
                                                       const T *__restrict__ lamS, const T *__restrict__ E0,
                                                       const T *__restrict__ E1, T *__restrict__ dU) {
  int i = begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= end) return;
  const int n = m.nc, nf = m.nf;
  int jn[kMaxFace];
#pragma unroll
  for (int s = 0; s < kMaxFace; ++s) jn[s] = m.cnbr[s * n + i];
  T acc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) acc[v] = Rk[v * n + i];
#pragma unroll
  for (int s = 0; s < kMaxFace; ++s) {
    const bool ok = jn[s] >= 0;
    const int j = ok ? jn[s] : i;
    const T w = ok ? T(1) : T(0);
    const T nx = m.snx[s * n + i], ny = m.sny[s * n + i], hS = w * m.shs[s * n + i], lp = lamS[s * n + i];
    T uj[4], du[4], dF[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { uj[v] = U[v * n + j]; du[v] = dU[v * n + j]; }
    if constexpr (is_f32<T>()) {
      D::euler_flux_delta(P.gamma, uj, prim[1 * n + j], prim[2 * n + j], prim[3 * n + j], du, nx, ny, dF);
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] -= hS * (dF[v] - lp * du[v]);
    } else {
      const int fs = m.cface[s * n + i];
      const bool is0 = fs >= 0;
      const int f = ok ? (is0 ? fs : ~fs) : 0;
      T up[4], fa[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) up[v] = uj[v] + du[v];
      D::euler_flux(P.gamma, up, nx, ny, fa);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const T fb = is0 ? E1[v * nf + f] : -E0[v * nf + f];
        acc[v] -= hS * ((fa[v] - fb) - lp * (up[v] - uj[v]));
      }
    }
  }
  const T id = invD[i];
#pragma unroll
  for (int v = 0; v < 4; ++v) dU[v * n + i] = acc[v] * id;
}

// K9: prolongation W = W_p0 + (U - W_p0) (Section 3, step 5), density
// residual against the state at the start of the cycle, state check.
template <typename TF>
__global__ void __launch_bounds__(kCellBlock) k_prolong(MeshT<double> m, ParamsT<double> P, double *__restrict__ W,
                                                        const double *__restrict__ Wp0, const double *__restrict__ U,
                                                        Scalars *sc, double *__restrict__ partial, TF *__restrict__ Wm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = m.nc;
  double num = 0.0, den = 0.0;
  if (i < n) {
    double w[4];
    double old_rho = W[i];
    for (int v = 0; v < 4; ++v) {
      double wp = Wp0[v * n + i];
      w[v] = wp + (U[v * n + i] - wp);
      W[v * n + i] = w[v];
      if (Wm) Wm[v * n + i] = static_cast<TF>(w[v]);
    }
    if (!state_ok(P.gamma, w)) atomicOr(&sc->status, kBadState);
    num = fabs(w[0] - old_rho);
    den = old_rho;
  }
  block_sum2(num, den, &partial[2 * blockIdx.x]);
}

// AoS caller order <-> SoA internal order
__global__ void k_gather_state(int n, const int *__restrict__ perm, const double *__restrict__ Wa,
                               const double *__restrict__ Wxa, double *__restrict__ W, double *__restrict__ Wx,
                               float *__restrict__ W32, float *__restrict__ Wx32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = perm[i];
  for (int v = 0; v < 4; ++v) {
    double w = Wa[4 * c + v];
    W[v * n + i] = w;
    if (W32) W32[v * n + i] = static_cast<float>(w);
  }
  for (int k = 0; k < 8; ++k) {
    double g = Wxa ? Wxa[8 * c + k] : 0.0;
    Wx[k * n + i] = g;
    if (Wx32) Wx32[k * n + i] = static_cast<float>(g);
  }
}
__global__ void k_scatter_state(int n, const int *__restrict__ perm, const double *__restrict__ W,
                                const double *__restrict__ Wx, double *__restrict__ Wa, double *__restrict__ Wxa) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = perm[i];
  if (Wa) for (int v = 0; v < 4; ++v) Wa[4 * c + v] = W[v * n + i];
  if (Wxa) for (int k = 0; k < 8; ++k) Wxa[8 * c + k] = Wx[k * n + i];
}

// kernel ids for the per-kernel timers
enum KernelId { KI_DT = 0, KI_RECON, KI_FACE, KI_UPDATE, KI_RESFIN, KI_LOFACE, KI_LORHS, KI_SWEEP, KI_LOCELL,
                KI_PROLONG, KI_COUNT };
const char *kKernelNames[KI_COUNT] = { "k_dt", "k_recon", "k_face", "k_update", "k_res_final", "k_lo_face",
                                       "k_lo_rhs", "k_sweep", "k_lo_cell", "k_prolong" };

inline int nblk(int n, int b) { return (n + b - 1) / b; }

}  // namespace

// ------------------------------------------------------------------------
struct cgks_solver {
  HostMesh hm;                  // host copy (ordering and permutations)
  cgks_params params{};
  bool mixed = false;
  ParamsT<double> dp{};
  ParamsT<float> fp{};
  MeshT<double> dm{};
  MeshT<float> fm{};
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_user = nullptr, ev_done = nullptr;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  int device = 0;
  // FP64 state and accumulation arrays (device)
  double *W = nullptr, *Wx = nullptr, *Wn = nullptr, *Ws = nullptr, *Wxs = nullptr;
  double *U = nullptr, *Rp0 = nullptr, *Src = nullptr;
  double *partial = nullptr, *last = nullptr;
  // flux-type arrays
  Bufs<double> bd;
  Bufs<float> bf;
  std::vector<int> sweep_colours;   // colour sequence of the relaxation after the first pass
  double *hist = nullptr;
  int hist_cap = 0;
  double *stage_aos = nullptr;  // [12 n] staging for set/get state
  int *perm = nullptr;
  Scalars *sc = nullptr;
  int nblk_cell = 0;
  // graphs
  cudaGraphExec_t g_cycle = nullptr, g_step = nullptr;
  // timers
  bool timing = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> tev;
  double t_ms[KI_COUNT] = { 0 };
  long long t_cnt[KI_COUNT] = { 0 };
  long long launches = 0;
  int status_cache = 0;
};

namespace {

void *dev_alloc(cgks_solver *s, size_t bytes) {
  if (s->params.alloc) return s->params.alloc(bytes, s->params.alloc_ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}
void dev_free(cgks_solver *s, void *p) {
  if (!p) return;
  if (s->params.alloc && s->params.free) s->params.free(p, s->params.alloc_ctx);
  else if (!s->params.alloc) cudaFree(p);
}

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return CGKS_ECUDA;   \
  } while (0)

// launch helper with optional timing
template <typename Kern, typename... Args>
void launch(cgks_solver *s, int id, Kern kern, dim3 grid, dim3 block, Args... args) {
  if (grid.x == 0) return;
  cudaEvent_t a = nullptr, b = nullptr;
  if (s->timing) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s->stream);
  }
  kern<<<grid, block, 0, s->stream>>>(args...);
  if (s->timing) {
    cudaEventRecord(b, s->stream);
    s->tev.push_back({ id, { a, b } });
  }
  s->launches++;
}

template <typename TF> Bufs<TF> &bufs(cgks_solver *s);
template <> Bufs<double> &bufs<double>(cgks_solver *s) { return s->bd; }
template <> Bufs<float> &bufs<float>(cgks_solver *s) { return s->bf; }
template <typename TF> const MeshT<TF> &fmesh(cgks_solver *s);
template <> const MeshT<double> &fmesh<double>(cgks_solver *s) { return s->dm; }
template <> const MeshT<float> &fmesh<float>(cgks_solver *s) { return s->fm; }
template <typename TF> const ParamsT<TF> &fparams(cgks_solver *s);
template <> const ParamsT<double> &fparams<double>(cgks_solver *s) { return s->dp; }
template <> const ParamsT<float> &fparams<float>(cgks_solver *s) { return s->fp; }
// float mirror of a flux-type array, or null when the flux type is double
template <typename TF> TF *mirror(TF *p) { return is_f32<TF>() ? p : nullptr; }

// ---- building blocks of a step / cycle ----
void enqueue_dt(cgks_solver *s, double dt_fixed) {
  launch(s, KI_DT, k_reset_dt, dim3(1), dim3(1), s->sc, dt_fixed);
  if (!(dt_fixed > 0.0))
    launch(s, KI_DT, k_dt, dim3(s->nblk_cell), dim3(kCellBlock), s->dm, s->dp, (const double *)s->W, s->sc);
}

template <typename TF>
void enqueue_hi_eval(cgks_solver *s, const TF *W, const TF *Wx, TF *Fout) {
  Bufs<TF> &B = bufs<TF>(s);
  launch(s, KI_RECON, k_recon<TF>, dim3(s->nblk_cell), dim3(kCellBlock), fmesh<TF>(s), fparams<TF>(s), W, Wx, B.coef);
  launch(s, KI_FACE, k_face<TF>, dim3(nblk(s->dm.nf, kFaceBlock)), dim3(kFaceBlock), fmesh<TF>(s), fparams<TF>(s), W,
         (const TF *)B.coef, Fout);
}

// high-order step from (W, Wx) into (Wout, Wx): Wx updated in place.
template <typename TF>
void enqueue_hi_step(cgks_solver *s, double *Wout, TF *Wout_m, bool want_res) {
  Bufs<TF> &B = bufs<TF>(s);
  double *part = want_res ? s->partial : nullptr;
  enqueue_hi_eval<TF>(s, B.W, B.Wx, B.FA);
  if (s->params.time_scheme == CGKS_S1O2) {
    launch(s, KI_UPDATE, k_update<TF>, dim3(s->nblk_cell), dim3(kCellBlock), s->dm, s->dp, (int)kS1O2,
           (const double *)s->W, (const TF *)B.FA, (const TF *)B.FA, s->sc, Wout, s->Wx, part, s->Rp0, Wout_m,
           mirror<TF>(B.Wx));
  } else {
    launch(s, KI_UPDATE, k_update<TF>, dim3(s->nblk_cell), dim3(kCellBlock), s->dm, s->dp, (int)kS2O4Stage,
           (const double *)s->W, (const TF *)B.FA, (const TF *)B.FA, s->sc, s->Ws, s->Wxs, (double *)nullptr,
           (double *)nullptr, mirror<TF>(B.Ws), mirror<TF>(B.Wxs));
    enqueue_hi_eval<TF>(s, B.Ws, B.Wxs, B.FB);
    launch(s, KI_UPDATE, k_update<TF>, dim3(s->nblk_cell), dim3(kCellBlock), s->dm, s->dp, (int)kS2O4Final,
           (const double *)s->W, (const TF *)B.FA, (const TF *)B.FB, s->sc, Wout, s->Wx, part, s->Rp0, Wout_m,
           mirror<TF>(B.Wx));
  }
  if (want_res)
    launch(s, KI_RESFIN, k_res_final, dim3(1), dim3(256), (const double *)s->partial, s->nblk_cell, s->sc, s->hist,
           s->hist_cap, s->last);
}

// low-order solve from U = W_p0 (= s->Wn), R_p0 in s->Rp0; result in s->U.
// Per implicit step: cell primitives (and U += dU), KFVS faces, right-hand
// side with the first colour pass, then the remaining colour passes.
template <typename TF>
void enqueue_lo_solve(cgks_solver *s) {
  Bufs<TF> &B = bufs<TF>(s);
  const int n = s->dm.nc, nf = s->dm.nf;
  const int c0_end = s->params.n_sweeps > 0 ? s->hm.colour_start[1] : 0;
  for (int k = 0; k < s->params.n_implicit; ++k) {
    launch(s, KI_LOCELL, k_lo_cell<TF>, dim3(s->nblk_cell), dim3(kCellBlock), n, fparams<TF>(s), k == 0 ? 1 : 0,
           (const double *)s->Wn, s->U, (const TF *)B.dU, B.prim, mirror<TF>(B.U));
    launch(s, KI_LOFACE, k_lo_face<TF>, dim3(nblk(nf, kCellBlock)), dim3(kCellBlock), fmesh<TF>(s), fparams<TF>(s),
           (const TF *)B.U, (const TF *)B.prim, B.Flo, B.lam, B.E0, B.E1);
    launch(s, KI_LORHS, k_lo_rhs<TF>, dim3(s->nblk_cell), dim3(kCellBlock), s->dm, s->dp, k == 0 ? 1 : 0, c0_end,
           (const TF *)B.Flo, (const TF *)B.lam, (const double *)s->Rp0, s->Src, B.Rk, B.invD, B.dU, B.lamS);
    for (int c : s->sweep_colours) {
      int b = s->hm.colour_start[c], e = s->hm.colour_start[c + 1];
      launch(s, KI_SWEEP, k_sweep<TF>, dim3(nblk(e - b, kSweepBlock)), dim3(kSweepBlock), fmesh<TF>(s),
             fparams<TF>(s), b, e, (const TF *)B.U, (const TF *)B.prim, (const TF *)B.Rk, (const TF *)B.invD,
             (const TF *)B.lamS, (const TF *)B.E0, (const TF *)B.E1, B.dU);
    }
  }
  // U^{n_implicit} = U + dU of the last step
  if (s->params.n_implicit > 0)
    launch(s, KI_LOCELL, k_lo_cell<TF>, dim3(s->nblk_cell), dim3(kCellBlock), n, fparams<TF>(s), 0,
           (const double *)s->Wn, s->U, (const TF *)B.dU, B.prim, mirror<TF>(B.U));
  else
    cudaMemcpyAsync(s->U, s->Wn, sizeof(double) * 4 * n, cudaMemcpyDeviceToDevice, s->stream);
}

template <typename TF>
void enqueue_prolong(cgks_solver *s) {
  launch(s, KI_PROLONG, k_prolong<TF>, dim3(s->nblk_cell), dim3(kCellBlock), s->dm, s->dp, s->W,
         (const double *)s->Wn, (const double *)s->U, s->sc, s->partial, mirror<TF>(bufs<TF>(s).W));
  launch(s, KI_RESFIN, k_res_final, dim3(1), dim3(256), (const double *)s->partial, s->nblk_cell, s->sc, s->hist,
         s->hist_cap, s->last);
}

template <typename TF>
void enqueue_cycle_t(cgks_solver *s) {
  Bufs<TF> &B = bufs<TF>(s);
  enqueue_dt(s, -1.0);
  // 1: high-order step into W_p0 = Wn (W keeps W^n for the residual)
  enqueue_hi_step<TF>(s, s->Wn, mirror<TF>(B.Wn), false);
  // 2: R_p0 = time-averaged high-order net flux at W^{n+1}
  enqueue_hi_eval<TF>(s, B.Wn, B.Wx, B.FB);
  launch(s, KI_UPDATE, k_update<TF>, dim3(s->nblk_cell), dim3(kCellBlock), s->dm, s->dp, (int)kResidual,
         (const double *)s->Wn, (const TF *)B.FB, (const TF *)B.FB, s->sc, (double *)nullptr, (double *)nullptr,
         (double *)nullptr, s->Rp0, (TF *)nullptr, (TF *)nullptr);
  // 3-4: forcing and implicit low-order solve
  enqueue_lo_solve<TF>(s);
  // 5: correction and residual
  enqueue_prolong<TF>(s);
}

void enqueue_cycle(cgks_solver *s) {
  if (s->mixed) enqueue_cycle_t<float>(s);
  else enqueue_cycle_t<double>(s);
}

void enqueue_explicit_step(cgks_solver *s, double dt_fixed) {
  enqueue_dt(s, dt_fixed);
  if (s->mixed) enqueue_hi_step<float>(s, s->W, s->bf.W, true);
  else enqueue_hi_step<double>(s, s->W, nullptr, true);
}

void enqueue_lo_smooth(cgks_solver *s) {
  cudaMemcpyAsync(s->Wn, s->W, sizeof(double) * 4 * s->dm.nc, cudaMemcpyDeviceToDevice, s->stream);
  if (s->mixed) { enqueue_lo_solve<float>(s); enqueue_prolong<float>(s); }
  else { enqueue_lo_solve<double>(s); enqueue_prolong<double>(s); }
}

int ensure_hist(cgks_solver *s, int n) {
  if (n <= s->hist_cap) return CGKS_OK;
  // grow: graphs captured with the old pointer must be rebuilt
  double *p = static_cast<double *>(dev_alloc(s, sizeof(double) * n));
  if (!p) return CGKS_ENOMEM;
  if (s->hist) { cudaStreamSynchronize(s->stream); dev_free(s, s->hist); }
  s->hist = p;
  s->hist_cap = n;
  if (s->g_cycle) { cudaGraphExecDestroy(s->g_cycle); s->g_cycle = nullptr; }
  if (s->g_step) { cudaGraphExecDestroy(s->g_step); s->g_step = nullptr; }
  return CGKS_OK;
}

int begin_call(cgks_solver *s) {
  CK(cudaSetDevice(s->device));
  CK(cudaEventRecord(s->ev_user, s->user_stream));
  CK(cudaStreamWaitEvent(s->stream, s->ev_user, 0));
  return CGKS_OK;
}
int end_call(cgks_solver *s) {
  CK(cudaEventRecord(s->ev_done, s->stream));
  CK(cudaStreamWaitEvent(s->user_stream, s->ev_done, 0));
  return CGKS_OK;
}

int capture(cgks_solver *s, bool cycle, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  bool t = s->timing;
  s->timing = false;
  long long l0 = s->launches;
  CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  if (cycle) enqueue_cycle(s);
  else enqueue_explicit_step(s, -1.0);
  cudaError_t e = cudaStreamEndCapture(s->stream, &g);
  s->launches = l0;
  s->timing = t;
  if (e != cudaSuccess) return CGKS_ECUDA;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? CGKS_OK : CGKS_ECUDA;
}

long long count_launches(cgks_solver *s, bool cycle) {
  // number of kernels one cycle / step enqueues
  long long per_eval = 2;
  long long hi = per_eval + 1 + (s->params.time_scheme == CGKS_S2O4 ? per_eval + 1 : 0);
  long long dt = 2;
  if (!cycle) return dt + hi + 1;
  long long lo = s->params.n_implicit * (3 + static_cast<long long>(s->sweep_colours.size())) +
                 (s->params.n_implicit > 0 ? 1 : 0);
  return dt + hi + per_eval + 1 + lo + 2;
}

int read_status(cgks_solver *s) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, &s->sc->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->status_cache = st;
  return st ? CGKS_EDIVERGED : CGKS_OK;
}

void collect_timing(cgks_solver *s) {
  for (auto &e : s->tev) {
    float ms = 0.f;
    cudaEventSynchronize(e.second.second);
    cudaEventElapsedTime(&ms, e.second.first, e.second.second);
    s->t_ms[e.first] += ms;
    s->t_cnt[e.first] += 1;
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  s->tev.clear();
}

template <typename T>
void fill_params(const cgks_params *p, ParamsT<T> &P) {
  double K = (4.0 - 2.0 * p->gamma) / (p->gamma - 1.0);
  P.gamma = static_cast<T>(p->gamma);
  P.K = static_cast<T>(K);
  P.mu = static_cast<T>(p->mu);
  P.cfl_hi = static_cast<T>(p->cfl_hi);
  P.cfl_lo = static_cast<T>(p->cfl_lo);
  P.kc.K = static_cast<T>(K);
  P.kc.c2K = static_cast<T>(2.0 / (K + 2.0));
  P.kc.c4K = static_cast<T>(4.0 / (K + 2.0));
  for (int b = 0; b < CGKS_MAX_BC; ++b) {
    const cgks_bc &bc = p->bc[b];
    P.bc_kind[b] = b < p->n_bc ? bc.kind : CGKS_BC_SLIP;
    P.bc_uw[b][0] = static_cast<T>(bc.u_wall[0]);
    P.bc_uw[b][1] = static_cast<T>(bc.u_wall[1]);
    P.bc_rho[b] = static_cast<T>(bc.rho);
    P.bc_u[b][0] = static_cast<T>(bc.u[0]);
    P.bc_u[b][1] = static_cast<T>(bc.u[1]);
    P.bc_p[b] = static_cast<T>(bc.p);
  }
}

}  // namespace

// =============================== C ABI ===================================
extern "C" {

void cgks_default_params(cgks_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->gamma = 1.4;
  p->mu = 0.0;
  p->alpha = 0.5;
  p->cfl_hi = 0.4;
  p->cfl_lo = 1000.0;
  p->n_implicit = 6;
  p->n_sweeps = 2;
  p->time_scheme = CGKS_S1O2;
  p->precision = CGKS_FP64;
  p->use_graph = 1;
}

const char *cgks_strerror(int st) {
  switch (st) {
    case CGKS_OK: return "ok";
    case CGKS_EINVAL: return "invalid argument";
    case CGKS_ENOMEM: return "out of memory";
    case CGKS_EMESH: return "mesh rejected";
    case CGKS_ECUDA: return "CUDA error or no device";
    case CGKS_EDIVERGED: return "solution diverged (non-positive or non-finite density / pressure)";
    case CGKS_ETIMEOUT: return "timeout";
    case CGKS_EBUDGET: return "memory budget exceeded";
    default: return "unknown status";
  }
}

int cgks_mesh_create(int dim, int64_t n_nodes, const double *xyz, int64_t n_cells, const uint8_t *cell_type,
                     const int64_t *cell_ptr, const int64_t *cell_nodes, int64_t n_bfaces, const int64_t *bface_ptr,
                     const int64_t *bface_nodes, const int32_t *bface_tag, cgks_mesh **out) {
  if (!out) return CGKS_EINVAL;
  *out = nullptr;
  if (dim != 2) return CGKS_EINVAL;
  cgks_mesh *m = new (std::nothrow) cgks_mesh();
  if (!m) return CGKS_ENOMEM;
  int rc;
  try {
    rc = build_host_mesh(n_nodes, xyz, n_cells, cell_type, cell_ptr, cell_nodes, n_bfaces, bface_ptr, bface_nodes,
                         bface_tag, m->h);
  } catch (const std::bad_alloc &) {
    rc = CGKS_ENOMEM;
  }
  if (rc != CGKS_OK) { delete m; return rc; }
  *out = m;
  return CGKS_OK;
}

// device bytes of a solver: FP64 state/accumulation + geometry + the flux
// arrays in the flux type (doubles in FP64 mode, floats in mixed mode with
// float mirrors of the state and of the geometry)
static size_t solver_bytes(int64_t nc, int64_t nf, bool mixed) {
  const size_t d_cells = 4 * 5 + 8 * 2 + 4 * 3 + 12 + 6 + 3 + kNCol * kNM;  // W..Wxs, U, Rp0, Src, stage, geometry, op
  const size_t d_faces = 2 + 1 + 1 + 8;                                   // fn, fS, fjump, fxi
  const size_t d_slots = 3 * kMaxFace;                                    // slot normals, S/2
  const size_t t_cells = 4 + 8 + 4 + 4 + 8 + 4 + 20 + D::NPRIM + 4 + 1 + 4;  // mirrors, coef, prim, Rk, invD, dU
  const size_t t_faces = 16 * 2 + 4 + 1 + (mixed ? 0 : 8);               // FA, FB, Flo, lam, E0/E1
  const size_t f_geo_c = mixed ? (1 + 1 + 3 + kNCol * kNM + 3 * kMaxFace) : 0;  // float ivol, ih, m2, op, slots
  const size_t f_geo_f = mixed ? 12 : 0;
  const size_t tsz = mixed ? sizeof(float) : sizeof(double);
  return sizeof(double) * ((d_cells + d_slots) * nc + d_faces * nf) + tsz * ((t_cells + kMaxFace) * nc + t_faces * nf) +
         sizeof(float) * (f_geo_c * nc + f_geo_f * nf) + sizeof(int) * (8 * nc + 2 * nf + nc) +
         sizeof(double) * (2 * ((nc + kCellBlock - 1) / kCellBlock) + 16) + 64 * 256 + sizeof(Scalars);
}

int cgks_mesh_info(const cgks_mesh *m, cgks_mesh_info_t *out) {
  if (!m || !out) return CGKS_EINVAL;
  out->n_cells = m->h.n_cells;
  out->n_faces = m->h.n_faces;
  out->n_bfaces = m->h.n_bfaces;
  out->n_colours = m->h.n_colours;
  out->dim = m->h.dim;
  out->device_bytes = static_cast<int64_t>(solver_bytes(m->h.n_cells, m->h.n_faces, false));
  return CGKS_OK;
}

int cgks_mesh_ordering(const cgks_mesh *m, int64_t *rcm, int32_t *colour) {
  if (!m) return CGKS_EINVAL;
  if (rcm) std::copy(m->h.rcm.begin(), m->h.rcm.end(), rcm);
  if (colour) std::copy(m->h.colour.begin(), m->h.colour.end(), colour);
  return CGKS_OK;
}

int cgks_mesh_destroy(cgks_mesh *m) {
  delete m;
  return CGKS_OK;
}

int cgks_solver_destroy(cgks_solver *s) {
  if (!s) return CGKS_OK;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  collect_timing(s);
  if (s->g_cycle) cudaGraphExecDestroy(s->g_cycle);
  if (s->g_step) cudaGraphExecDestroy(s->g_step);
  dev_free(s, s->hist);
  dev_free(s, s->arena);
  if (s->ev_user) cudaEventDestroy(s->ev_user);
  if (s->ev_done) cudaEventDestroy(s->ev_done);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return CGKS_OK;
}

int cgks_solver_create(const cgks_mesh *m, const cgks_params *p, cgks_solver **out) {
  if (!m || !p || !out) return CGKS_EINVAL;
  *out = nullptr;
  if (!(p->gamma > 1.0) || p->mu < 0.0 || !(p->cfl_hi > 0.0) || !(p->cfl_lo > 0.0) || p->n_implicit < 0 ||
      p->n_sweeps < 0 || (p->time_scheme != CGKS_S1O2 && p->time_scheme != CGKS_S2O4) || p->n_bc < 0 ||
      p->n_bc > CGKS_MAX_BC || (p->precision != CGKS_FP64 && p->precision != CGKS_MIXED))
    return CGKS_EINVAL;
  for (int t : m->h.bface_tags_used)
    if (t >= p->n_bc) return CGKS_EINVAL;
  for (int b = 0; b < p->n_bc; ++b) {
    int k = p->bc[b].kind;
    if (k != CGKS_BC_SLIP && k != CGKS_BC_NOSLIP && k != CGKS_BC_FARFIELD) return CGKS_EINVAL;
    if (k == CGKS_BC_FARFIELD && !(p->bc[b].rho > 0.0 && p->bc[b].p > 0.0)) return CGKS_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return CGKS_ECUDA;
  cgks_solver *s = new (std::nothrow) cgks_solver();
  if (!s) return CGKS_ENOMEM;
  s->hm = m->h;
  s->params = *p;
  s->mixed = p->precision == CGKS_MIXED;
  cudaGetDevice(&s->device);
  s->user_stream = static_cast<cudaStream_t>(p->stream);
  auto fail = [&](int rc) { cgks_solver_destroy(s); return rc; };
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(CGKS_ECUDA);
  if (cudaEventCreateWithFlags(&s->ev_user, cudaEventDisableTiming) != cudaSuccess) return fail(CGKS_ECUDA);
  if (cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming) != cudaSuccess) return fail(CGKS_ECUDA);
  fill_params(p, s->dp);
  fill_params(p, s->fp);
  // operators depend on which tags are walls
  std::vector<char> wall(CGKS_MAX_BC, 0);
  for (int b = 0; b < p->n_bc; ++b) wall[b] = p->bc[b].kind != CGKS_BC_FARFIELD;
  std::vector<double> op;
  try {
    build_operator(s->hm, wall, op);
  } catch (const std::bad_alloc &) {
    return fail(CGKS_ENOMEM);
  }
  const int64_t nc = s->hm.n_cells, nf = s->hm.n_faces;
  s->nblk_cell = nblk(static_cast<int>(nc), kCellBlock);
  // carve one arena
  struct Piece { void **dst; size_t bytes; };
  std::vector<Piece> pieces;
  auto D8 = [&](double **d, int64_t cnt) { pieces.push_back({ reinterpret_cast<void **>(d), sizeof(double) * cnt }); };
  auto F4 = [&](float **d, int64_t cnt) { pieces.push_back({ reinterpret_cast<void **>(d), sizeof(float) * cnt }); };
  auto I4 = [&](int **d, int64_t cnt) { pieces.push_back({ reinterpret_cast<void **>(d), sizeof(int) * cnt }); };
  double *vol, *ivol, *per, *ih, *m2, *opd, *fn, *fS, *fjump, *fxi, *snx, *sny, *shs;
  int *cface, *cnbr, *fc0, *fc1;
  D8(&s->W, 4 * nc); D8(&s->Wx, 8 * nc); D8(&s->Wn, 4 * nc); D8(&s->Ws, 4 * nc); D8(&s->Wxs, 8 * nc);
  D8(&s->U, 4 * nc); D8(&s->Rp0, 4 * nc); D8(&s->Src, 4 * nc);
  D8(&s->partial, 2 * std::max(s->nblk_cell, 1)); D8(&s->last, 4); D8(&s->stage_aos, 12 * nc);
  D8(&vol, nc); D8(&ivol, nc); D8(&per, nc); D8(&ih, nc); D8(&m2, 3 * nc); D8(&opd, kNCol * kNM * nc);
  D8(&fn, 2 * nf); D8(&fS, nf); D8(&fjump, nf); D8(&fxi, 8 * nf);
  D8(&snx, kMaxFace * nc); D8(&sny, kMaxFace * nc); D8(&shs, kMaxFace * nc);
  I4(&cface, kMaxFace * nc); I4(&cnbr, kMaxFace * nc); I4(&fc0, nf); I4(&fc1, nf); I4(&s->perm, nc);
  float *f_ivol = nullptr, *f_ih = nullptr, *f_m2 = nullptr, *f_op = nullptr, *f_fn = nullptr, *f_fS = nullptr,
        *f_fjump = nullptr, *f_fxi = nullptr, *f_snx = nullptr, *f_sny = nullptr, *f_shs = nullptr;
  if (!s->mixed) {
    Bufs<double> &B = s->bd;
    D8(&B.coef, 20 * nc); D8(&B.FA, 16 * nf); D8(&B.FB, 16 * nf);
    D8(&B.prim, D::NPRIM * nc); D8(&B.Flo, 4 * nf); D8(&B.lam, nf); D8(&B.E0, 4 * nf); D8(&B.E1, 4 * nf);
    D8(&B.Rk, 4 * nc); D8(&B.invD, nc); D8(&B.dU, 4 * nc); D8(&B.lamS, kMaxFace * nc);
  } else {
    Bufs<float> &B = s->bf;
    F4(&B.W, 4 * nc); F4(&B.Wx, 8 * nc); F4(&B.Wn, 4 * nc); F4(&B.Ws, 4 * nc); F4(&B.Wxs, 8 * nc); F4(&B.U, 4 * nc);
    F4(&B.coef, 20 * nc); F4(&B.FA, 16 * nf); F4(&B.FB, 16 * nf);
    F4(&B.prim, D::NPRIM * nc); F4(&B.Flo, 4 * nf); F4(&B.lam, nf);
    F4(&B.Rk, 4 * nc); F4(&B.invD, nc); F4(&B.dU, 4 * nc); F4(&B.lamS, kMaxFace * nc);
    F4(&f_ivol, nc); F4(&f_ih, nc); F4(&f_m2, 3 * nc); F4(&f_op, kNCol * kNM * nc);
    F4(&f_fn, 2 * nf); F4(&f_fS, nf); F4(&f_fjump, nf); F4(&f_fxi, 8 * nf);
    F4(&f_snx, kMaxFace * nc); F4(&f_sny, kMaxFace * nc); F4(&f_shs, kMaxFace * nc);
  }
  pieces.push_back({ reinterpret_cast<void **>(&s->sc), sizeof(Scalars) });
  size_t total = 0;
  for (auto &pc : pieces) total += (pc.bytes + 255) & ~size_t(255);
  s->arena = dev_alloc(s, total);
  if (!s->arena) return fail(CGKS_ENOMEM);
  s->arena_bytes = total;
  {
    char *cur = static_cast<char *>(s->arena);
    for (auto &pc : pieces) { *pc.dst = cur; cur += (pc.bytes + 255) & ~size_t(255); }
  }
  if (!s->mixed) {
    Bufs<double> &B = s->bd;
    B.W = s->W; B.Wx = s->Wx; B.Wn = s->Wn; B.Ws = s->Ws; B.Wxs = s->Wxs; B.U = s->U;
  }
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream) == cudaSuccess;
  };
  const HostMesh &hm = s->hm;
  // derived per-solver arrays: reciprocals and the jump coefficient alpha/delta
  std::vector<double> h_ivol(nc), h_ih(nc), h_jump(nf);
  for (int64_t i = 0; i < nc; ++i) { h_ivol[i] = 1.0 / hm.vol[i]; h_ih[i] = 1.0 / hm.h[i]; }
  for (int64_t f = 0; f < nf; ++f) h_jump[f] = hm.fdelta[f] > 0.0 ? p->alpha / hm.fdelta[f] : 0.0;
  // per face slot: the cell's outward unit normal and half the face length
  std::vector<double> h_snx(kMaxFace * nc, 0.0), h_sny(kMaxFace * nc, 0.0), h_shs(kMaxFace * nc, 0.0);
  for (int64_t i = 0; i < nc; ++i)
    for (int sl = 0; sl < kMaxFace; ++sl) {
      int32_t fs = hm.cface[sl * nc + i];
      if (fs == kNoFace) continue;
      int32_t f = fs >= 0 ? fs : ~fs;
      double sg = fs >= 0 ? 1.0 : -1.0;
      h_snx[sl * nc + i] = sg * hm.fn[f];
      h_sny[sl * nc + i] = sg * hm.fn[nf + f];
      h_shs[sl * nc + i] = 0.5 * hm.fS[f];
    }
  bool ok = up(vol, hm.vol.data(), 8 * nc) && up(ivol, h_ivol.data(), 8 * nc) && up(per, hm.per.data(), 8 * nc) &&
            up(ih, h_ih.data(), 8 * nc) && up(m2, hm.m2.data(), 8 * 3 * nc) && up(opd, op.data(), 8 * op.size()) &&
            up(fn, hm.fn.data(), 8 * 2 * nf) && up(fS, hm.fS.data(), 8 * nf) && up(fjump, h_jump.data(), 8 * nf) &&
            up(fxi, hm.fxi.data(), 8 * 8 * nf) && up(cface, hm.cface.data(), 4 * kMaxFace * nc) &&
            up(cnbr, hm.cnbr.data(), 4 * kMaxFace * nc) && up(fc0, hm.fc0.data(), 4 * nf) &&
            up(fc1, hm.fc1.data(), 4 * nf) && up(s->perm, hm.perm.data(), 4 * nc) &&
            up(snx, h_snx.data(), 8 * kMaxFace * nc) && up(sny, h_sny.data(), 8 * kMaxFace * nc) &&
            up(shs, h_shs.data(), 8 * kMaxFace * nc);
  std::vector<float> tmp;
  auto upf = [&](float *dst, const double *src, size_t cnt) {
    tmp.assign(src, src + cnt);
    bool r = cudaMemcpyAsync(dst, tmp.data(), 4 * cnt, cudaMemcpyHostToDevice, s->stream) == cudaSuccess;
    return r && cudaStreamSynchronize(s->stream) == cudaSuccess;   // tmp is reused
  };
  if (ok && s->mixed)
    ok = upf(f_ivol, h_ivol.data(), nc) && upf(f_ih, h_ih.data(), nc) && upf(f_m2, hm.m2.data(), 3 * nc) &&
         upf(f_op, op.data(), op.size()) && upf(f_fn, hm.fn.data(), 2 * nf) && upf(f_fS, hm.fS.data(), nf) &&
         upf(f_fjump, h_jump.data(), nf) && upf(f_fxi, hm.fxi.data(), 8 * nf) &&
         upf(f_snx, h_snx.data(), kMaxFace * nc) && upf(f_sny, h_sny.data(), kMaxFace * nc) &&
         upf(f_shs, h_shs.data(), kMaxFace * nc);
  if (!ok) return fail(CGKS_ECUDA);
  if (cudaMemsetAsync(s->sc, 0, sizeof(Scalars), s->stream) != cudaSuccess) return fail(CGKS_ECUDA);
  if (cudaMemsetAsync(s->W, 0, sizeof(double) * 12 * nc, s->stream) != cudaSuccess) return fail(CGKS_ECUDA);
  if (cudaMemsetAsync(s->Rp0, 0, sizeof(double) * 4 * nc, s->stream) != cudaSuccess) return fail(CGKS_ECUDA);
  if (s->mixed) {
    if (cudaMemsetAsync(s->bf.dU, 0, sizeof(float) * 4 * nc, s->stream) != cudaSuccess) return fail(CGKS_ECUDA);
    if (cudaMemsetAsync(s->bf.W, 0, sizeof(float) * 4 * nc, s->stream) != cudaSuccess) return fail(CGKS_ECUDA);
    if (cudaMemsetAsync(s->bf.Wx, 0, sizeof(float) * 8 * nc, s->stream) != cudaSuccess) return fail(CGKS_ECUDA);
  } else if (cudaMemsetAsync(s->bd.dU, 0, sizeof(double) * 4 * nc, s->stream) != cudaSuccess) {
    return fail(CGKS_ECUDA);
  }
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(CGKS_ECUDA);
  MeshT<double> &dm = s->dm;
  dm.nc = static_cast<int>(nc); dm.nf = static_cast<int>(nf);
  dm.vol = vol; dm.ivol = ivol; dm.per = per; dm.ih = ih; dm.m2 = m2; dm.op = opd;
  dm.fn = fn; dm.fS = fS; dm.fjump = fjump; dm.fxi = fxi; dm.snx = snx; dm.sny = sny; dm.shs = shs;
  dm.cface = cface; dm.cnbr = cnbr; dm.fc0 = fc0; dm.fc1 = fc1;
  MeshT<float> &fm = s->fm;
  fm.nc = dm.nc; fm.nf = dm.nf;
  fm.vol = nullptr; fm.per = nullptr; fm.ivol = f_ivol; fm.ih = f_ih; fm.m2 = f_m2; fm.op = f_op;
  fm.fn = f_fn; fm.fS = f_fS; fm.fjump = f_fjump; fm.fxi = f_fxi; fm.snx = f_snx; fm.sny = f_sny; fm.shs = f_shs;
  fm.cface = cface; fm.cnbr = cnbr; fm.fc0 = fc0; fm.fc1 = fc1;
  // Colour sequence of Algorithm 1 with colour classes: n_sweeps x (0..C-1,
  // C-1..0).  A colour repeated back to back recomputes identical values
  // (its cells read only other colours), and the first pass is done by
  // k_lo_rhs, so both are dropped.
  {
    std::vector<int> seq;
    const int C = s->hm.n_colours;
    for (int sw = 0; sw < p->n_sweeps; ++sw) {
      for (int c = 0; c < C; ++c) if (seq.empty() || seq.back() != c) seq.push_back(c);
      for (int c = C - 1; c >= 0; --c) if (seq.empty() || seq.back() != c) seq.push_back(c);
    }
    if (!seq.empty()) seq.erase(seq.begin());
    s->sweep_colours = seq;
  }
  if (ensure_hist(s, 1024) != CGKS_OK) return fail(CGKS_ENOMEM);
  *out = s;
  return CGKS_OK;
}

static int set_state_impl(cgks_solver *s, const double *W, const double *Wx, bool device) {
  if (!s || !W) return CGKS_EINVAL;
  const int n = s->dm.nc;
  int rc = begin_call(s);
  if (rc) return rc;
  double *wa = s->stage_aos, *wxa = s->stage_aos + 4 * n;
  cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(wa, W, sizeof(double) * 4 * n, kind, s->stream));
  if (Wx) CK(cudaMemcpyAsync(wxa, Wx, sizeof(double) * 8 * n, kind, s->stream));
  k_gather_state<<<nblk(n, kCellBlock), kCellBlock, 0, s->stream>>>(n, s->perm, wa, Wx ? wxa : nullptr, s->W, s->Wx,
                                                                    s->mixed ? s->bf.W : nullptr,
                                                                    s->mixed ? s->bf.Wx : nullptr);
  s->launches++;
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(&s->sc->status, 0, sizeof(int), s->stream));
  s->status_cache = 0;
  return end_call(s);
}

int cgks_set_state(cgks_solver *s, const double *W, const double *Wx) { return set_state_impl(s, W, Wx, false); }
int cgks_set_state_device(cgks_solver *s, const double *W, const double *Wx) { return set_state_impl(s, W, Wx, true); }

static int get_state_impl(cgks_solver *s, double *W, double *Wx, bool device) {
  if (!s) return CGKS_EINVAL;
  const int n = s->dm.nc;
  int rc = begin_call(s);
  if (rc) return rc;
  double *wa = s->stage_aos, *wxa = s->stage_aos + 4 * n;
  k_scatter_state<<<nblk(n, kCellBlock), kCellBlock, 0, s->stream>>>(n, s->perm, s->W, s->Wx, wa, wxa);
  s->launches++;
  CK(cudaGetLastError());
  cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (W) CK(cudaMemcpyAsync(W, wa, sizeof(double) * 4 * n, kind, s->stream));
  if (Wx) CK(cudaMemcpyAsync(Wx, wxa, sizeof(double) * 8 * n, kind, s->stream));
  if (!device) CK(cudaStreamSynchronize(s->stream));
  return end_call(s);
}

int cgks_get_state(cgks_solver *s, double *W, double *Wx) { return get_state_impl(s, W, Wx, false); }
int cgks_get_state_device(cgks_solver *s, double *W, double *Wx) { return get_state_impl(s, W, Wx, true); }

int cgks_highorder_step(cgks_solver *s, double dt, double *dt_used) {
  if (!s) return CGKS_EINVAL;
  if (s->status_cache) return CGKS_EDIVERGED;
  int rc = begin_call(s);
  if (rc) return rc;
  CK(cudaMemsetAsync(&s->sc->res_ctr, 0, sizeof(int), s->stream));
  enqueue_explicit_step(s, dt);
  CK(cudaGetLastError());
  Scalars h;
  CK(cudaMemcpyAsync(&h, s->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (s->timing) collect_timing(s);
  if (dt_used) *dt_used = h.dt_fixed > 0.0 ? h.dt_fixed : s->params.cfl_hi * __builtin_bit_cast(double, h.dt_bits);
  s->status_cache = h.status;
  rc = end_call(s);
  if (rc) return rc;
  return h.status ? CGKS_EDIVERGED : CGKS_OK;
}

static int run_many(cgks_solver *s, int n, double *res_hist, bool cycle) {
  if (!s || n < 0) return CGKS_EINVAL;
  if (s->status_cache) return CGKS_EDIVERGED;
  if (n == 0) return CGKS_OK;
  int rc = ensure_hist(s, n);
  if (rc) return rc;
  rc = begin_call(s);
  if (rc) return rc;
  CK(cudaMemsetAsync(&s->sc->res_ctr, 0, sizeof(int), s->stream));
  bool graph = s->params.use_graph && !s->timing;
  cudaGraphExec_t *ge = cycle ? &s->g_cycle : &s->g_step;
  if (graph && !*ge) {
    rc = capture(s, cycle, ge);
    if (rc) return rc;
  }
  long long per = count_launches(s, cycle);
  for (int k = 0; k < n; ++k) {
    if (graph) {
      CK(cudaGraphLaunch(*ge, s->stream));
      s->launches += per;
    } else if (cycle) {
      enqueue_cycle(s);
    } else {
      enqueue_explicit_step(s, -1.0);
    }
  }
  CK(cudaGetLastError());
  if (res_hist) CK(cudaMemcpyAsync(res_hist, s->hist, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  rc = read_status(s);
  if (s->timing) collect_timing(s);
  int rc2 = end_call(s);
  return rc ? rc : rc2;
}

int cgks_explicit_steps(cgks_solver *s, int n, double *res_hist) { return run_many(s, n, res_hist, false); }
int cgks_pmg_cycle(cgks_solver *s, int n_cycles, double *res_hist) { return run_many(s, n_cycles, res_hist, true); }

int cgks_loworder_smooth(cgks_solver *s) {
  if (!s) return CGKS_EINVAL;
  if (s->status_cache) return CGKS_EDIVERGED;
  int rc = begin_call(s);
  if (rc) return rc;
  CK(cudaMemsetAsync(&s->sc->res_ctr, 0, sizeof(int), s->stream));
  enqueue_lo_smooth(s);
  CK(cudaGetLastError());
  rc = read_status(s);
  if (s->timing) collect_timing(s);
  int rc2 = end_call(s);
  return rc ? rc : rc2;
}

int cgks_residual(cgks_solver *s, double *res, double *r_l2) {
  if (!s) return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  double last[3];
  CK(cudaMemcpyAsync(last, s->last, sizeof(double) * 3, cudaMemcpyDeviceToHost, s->stream));
  std::vector<double> R;
  if (r_l2) {
    R.resize(4 * static_cast<size_t>(s->dm.nc));
    CK(cudaMemcpyAsync(R.data(), s->Rp0, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  if (res) *res = last[0];
  if (r_l2) {
    const int n = s->dm.nc;
    for (int v = 0; v < 4; ++v) {
      double a = 0.0;
      for (int i = 0; i < n; ++i) a += R[v * n + i] * R[v * n + i];
      r_l2[v] = std::sqrt(a);
    }
  }
  return end_call(s);
}

int cgks_get_rp0(cgks_solver *s, double *Rp0) {
  if (!s || !Rp0) return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  const int n = s->dm.nc;
  std::vector<double> R(4 * static_cast<size_t>(n));
  CK(cudaMemcpyAsync(R.data(), s->Rp0, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  for (int i = 0; i < n; ++i) {
    int c = s->hm.perm[i];
    for (int v = 0; v < 4; ++v) Rp0[4 * c + v] = R[v * n + i];
  }
  return end_call(s);
}

// ---- instrumentation (not in the paper): per-kernel CUDA-event timers and
// the count of kernels this solver has launched ----
int cgks_set_timing(cgks_solver *s, int on) {
  if (!s) return CGKS_EINVAL;
  cudaStreamSynchronize(s->stream);
  collect_timing(s);
  s->timing = on != 0;
  return CGKS_OK;
}

int cgks_get_timing(cgks_solver *s, int max, const char **names, double *total_ms, int64_t *count) {
  if (!s) return CGKS_EINVAL;
  cudaStreamSynchronize(s->stream);
  collect_timing(s);
  int k = 0;
  for (; k < KI_COUNT && k < max; ++k) {
    if (names) names[k] = kKernelNames[k];
    if (total_ms) total_ms[k] = s->t_ms[k];
    if (count) count[k] = s->t_cnt[k];
  }
  return k;
}

int cgks_reset_timing(cgks_solver *s) {
  if (!s) return CGKS_EINVAL;
  cudaStreamSynchronize(s->stream);
  collect_timing(s);
  for (int k = 0; k < KI_COUNT; ++k) { s->t_ms[k] = 0.0; s->t_cnt[k] = 0; }
  return CGKS_OK;
}

int64_t cgks_launch_count(const cgks_solver *s) { return s ? s->launches : -1; }

int cgks_launches_per_call(const cgks_solver *s, int cycle) {
  return s ? static_cast<int>(count_launches(const_cast<cgks_solver *>(s), cycle != 0)) : -1;
}

}  // extern "C"
