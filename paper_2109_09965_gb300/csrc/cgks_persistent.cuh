// Persistent fused low-order solve (included by cgks_device.cu only).
//
// One cooperative launch runs the whole low-order level of a V-cycle
// (Section 3, steps 3-4): n_implicit backward-Euler steps, each = cell
// primitives (and U += dU), KFVS faces, right-hand side with the first
// colour pass, then the remaining colour passes of Algorithm 1, and the
// final U += dU.  Phases are separated by a grid barrier instead of kernel
// boundaries.  Every value produced inside the launch is read with
// ld.global.cg (L2, never a stale L1 line); the arithmetic of each phase is
// the same as in the per-phase kernels of cgks_kernels.cuh.
//
// Measured on GB300 (57k-cell cylinder V-cycle): slower than the per-phase
// kernels replayed from a CUDA graph (FP64 2.22 vs 1.89 ms, mixed 0.54 vs
// 0.42 ms): the resident grid holds fewer warps per SM than the separate
// launches and the graph already hides their launch gaps, so the library
// uses it only when asked (cgks_params.low_order_fused).
//
// The barrier spins with a bound: past the launch's spin limit (kSpinLimit
// unless the caller sets one) a block records kBarrierTimeout in the status
// word of every slot of the batch and leaves; every other block then times
// out at its next barrier, so the launch always ends.  The host clears the
// barrier before every launch, so a launch that timed out leaves nothing
// behind for the next one.
#pragma once

#include "cgks_kernels.cuh"

namespace cgks {
namespace kern {

constexpr int kPersistBlock = 256;
constexpr int kBarrierTimeout = 2;              // bit of the status word
constexpr long long kSpinLimit = 1ll << 22;     // ~4M polls of ~0.1-1 us: seconds, far above any phase

struct GridBarrier {
  unsigned int count, gen;
};

template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// a load that observes other blocks' writes (acquire, GPU scope)
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// all blocks of the grid; returns false after a timeout (status bit set in
// each of the n_err status words)
__device__ __forceinline__ bool grid_barrier(GridBarrier *gb, long long spin_limit, int *err, int n_err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned my_gen = ld_acquire(&gb->gen);
    const unsigned arrived = atomicAdd(&gb->count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      long long it = 0;
      while (ld_acquire(&gb->gen) == my_gen) {
        if (++it > spin_limit) {
          for (int k = 0; k < n_err; ++k) atomicOr(&err[k], kBadState | kBarrierTimeout);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// per-colour cell ranges of the batch in device memory (any number of solves)
struct ColourRanges {
  const int *rstart;   // [C + 1] first range of each colour
  const int *rbegin;   // [R] first cell of each range
  const int *rpre;     // [R + C] cells of the colour before each range (per colour, R_c + 1 entries)
};

template <typename TF>
struct LoArgs {
  MeshT<double> dm;
  MeshT<TF> fm;
  ParamsT<double> dp;
  ParamsT<TF> fp;
  int n_implicit, colour0, n_seq;
  int n_cells, n_faces;              // extents of the solves present (arrays are strided by capacity)
  int seq[48];                       // colour order after the first pass (n_sweeps x 2 x colours)
  ColourRanges cr;
  const double *Wp0, *Rp0;
  double *U, *Src;
  TF *dU, *prim, *Um, *Flo, *lam, *E0, *E1, *Rk, *invD, *lamS;
  GridBarrier *gb;
  long long spin_limit;              // polls per barrier wait before giving up
  int *err;                          // [n_err] status words of the batch's slots
  int n_err;
};

template <typename TF>
__device__ __forceinline__ void lo_cell_at(const LoArgs<TF> &a, int i, int first) {
  const int n = a.dm.nc;
  TF w[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double u = first ? a.Wp0[v * n + i] : ldcg(&a.U[v * n + i]) + static_cast<double>(ldcg(&a.dU[v * n + i]));
    a.U[v * n + i] = u;
    w[v] = static_cast<TF>(u);
    if (a.Um) a.Um[v * n + i] = w[v];
  }
  const D::Prim<TF> q = D::prim_of(w, a.fp.gamma, a.fp.kc);
  TF *pr = a.prim;
  pr[0 * n + i] = q.rho; pr[1 * n + i] = q.u; pr[2 * n + i] = q.v; pr[3 * n + i] = q.p;
  pr[4 * n + i] = q.i2l; pr[5 * n + i] = q.sl; pr[6 * n + i] = q.isp; pr[7 * n + i] = q.c; pr[8 * n + i] = q.ir;
}

template <typename T>
__device__ __forceinline__ D::Prim<T> ldcg_prim(const T *prim, int n, int i) {
  D::Prim<T> q;
  q.rho = ldcg(&prim[0 * n + i]); q.u = ldcg(&prim[1 * n + i]); q.v = ldcg(&prim[2 * n + i]);
  q.p = ldcg(&prim[3 * n + i]); q.i2l = ldcg(&prim[4 * n + i]); q.sl = ldcg(&prim[5 * n + i]);
  q.isp = ldcg(&prim[6 * n + i]); q.c = ldcg(&prim[7 * n + i]); q.ir = ldcg(&prim[8 * n + i]);
  return q;
}

template <typename TF>
__device__ __forceinline__ void lo_face_at(const LoArgs<TF> &a, int f) {
  const MeshT<TF> &m = a.fm;
  const ParamsT<TF> &P = a.fp;
  const int sid = m.fsid[f];
  if (sid < 0) return;
  const int n = m.nc, nf = m.nf;
  const int c0 = m.fc0[f], c1 = m.fc1[f];
  const TF nx = m.fn[f], ny = m.fn[nf + f], S = m.fS[f];
  const TF mu = P.mu[sid];
  // the float mirror of U is written in this launch: read it through L2
  const TF *Uf = a.Um ? a.Um : reinterpret_cast<const TF *>(a.U);
  D::Prim<TF> pa = ldcg_prim(a.prim, n, c0), pb;
  TF ivb;
  if (c1 >= 0) {
    pb = ldcg_prim(a.prim, n, c1);
    ivb = m.ivol[c1];
  } else {
    TF w0[4], wg[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) w0[v] = ldcg(&Uf[v * n + c0]);
    lo_ghost(P, -1 - c1, nx, ny, w0, wg);
    pb = D::prim_of(wg, P.gamma, P.kc);
    ivb = m.ivol[c0];
  }
  const TF una = pa.u * nx + pa.v * ny, uta = -pa.u * ny + pa.v * nx;
  const TF unb = pb.u * nx + pb.v * ny, utb = -pb.u * ny + pb.v * nx;
  TF Fl[4], F[4];
  D::kfvs_prims(P.K, pa.rho, una, uta, pa.i2l, pa.sl, pa.isp, pb.rho, unb, utb, pb.i2l, pb.sl, pb.isp, Fl);
  D::rot_out(nx, ny, Fl, F);
#pragma unroll
  for (int v = 0; v < 4; ++v) a.Flo[v * nf + f] = F[v];
  const TF la = fabs(una) + pa.c + TF(2) * (mu * pa.ir) * S * m.ivol[c0];
  const TF lb = fabs(unb) + pb.c + TF(2) * (mu * pb.ir) * S * ivb;
  a.lam[f] = la > lb ? la : lb;
  if (a.E0) {
    a.E0[0 * nf + f] = pa.rho * una;
    a.E0[1 * nf + f] = ldcg(&Uf[1 * n + c0]) * una + pa.p * nx;
    a.E0[2 * nf + f] = ldcg(&Uf[2 * n + c0]) * una + pa.p * ny;
    a.E0[3 * nf + f] = (ldcg(&Uf[3 * n + c0]) + pa.p) * una;
    if (c1 >= 0) {
      a.E1[0 * nf + f] = pb.rho * unb;
      a.E1[1 * nf + f] = ldcg(&Uf[1 * n + c1]) * unb + pb.p * nx;
      a.E1[2 * nf + f] = ldcg(&Uf[2 * n + c1]) * unb + pb.p * ny;
      a.E1[3 * nf + f] = (ldcg(&Uf[3 * n + c1]) + pb.p) * unb;
    }
  }
}

template <typename TF>
__device__ __forceinline__ void lo_rhs_at(const LoArgs<TF> &a, int i, int first) {
  const MeshT<double> &m = a.dm;
  const int n = m.nc, nf = m.nf;
  double R[4] = { 0, 0, 0, 0 }, sum = 0.0;
  for (int s = 0; s < kMaxFace; ++s) {
    const int fs = m.cface[s * n + i];
    if (fs == kNoFace) { a.lamS[s * n + i] = TF(0); continue; }
    const int f = fs >= 0 ? fs : ~fs;
    const double sg = fs >= 0 ? 1.0 : -1.0;
    const double S = m.fS[f];
#pragma unroll
    for (int v = 0; v < 4; ++v) R[v] -= sg * S * static_cast<double>(ldcg(&a.Flo[v * nf + f]));
    const TF l = ldcg(&a.lam[f]);
    a.lamS[s * n + i] = l;
    sum += static_cast<double>(l) * S;
  }
  const double id = sum > 0.0 ? 1.0 / (sum / a.dp.cfl_lo + 0.5 * sum) : 0.0;
  a.invD[i] = static_cast<TF>(id);
  const bool c0 = a.colour0 && m.ccol[i] == 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double src;
    if (first) { src = a.Rp0[v * n + i] - R[v]; a.Src[v * n + i] = src; }
    else src = ldcg(&a.Src[v * n + i]);
    const double r = R[v] + src;
    a.Rk[v * n + i] = static_cast<TF>(r);
    a.dU[v * n + i] = c0 ? static_cast<TF>(r * id) : TF(0);
  }
}

// point relaxation of cell i by the 4-lane group (lane s = face slot)
template <typename TF>
__device__ __forceinline__ void sweep_at(const LoArgs<TF> &a, int i, int s) {
  const MeshT<TF> &m = a.fm;
  const int n = m.nc, nf = m.nf;
  const int j = i >= 0 ? m.cnbr[s * n + i] : -1;
  TF c[4] = { TF(0), TF(0), TF(0), TF(0) };
  if (j >= 0) {
    const TF nx = m.snx[s * n + i], ny = m.sny[s * n + i], hS = m.shs[s * n + i];
    const TF lp = ldcg(&a.lamS[s * n + i]);
    const TF *Uf = a.Um ? a.Um : reinterpret_cast<const TF *>(a.U);
    TF uj[4], du[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) { uj[v] = ldcg(&Uf[v * n + j]); du[v] = ldcg(&a.dU[v * n + j]); }
    if constexpr (is_f32<TF>()) {
      TF dF[4];
      D::euler_flux_delta(a.fp.gamma, uj, ldcg(&a.prim[1 * n + j]), ldcg(&a.prim[2 * n + j]),
                          ldcg(&a.prim[3 * n + j]), du, nx, ny, dF);
#pragma unroll
      for (int v = 0; v < 4; ++v) c[v] = hS * (dF[v] - lp * du[v]);
    } else {
      const int fs = m.cface[s * n + i];
      const bool is0 = fs >= 0;
      const int f = is0 ? fs : ~fs;
      TF up[4], fa[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) up[v] = uj[v] + du[v];
      D::euler_flux(a.fp.gamma, up, nx, ny, fa);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const TF fb = is0 ? ldcg(&a.E1[v * nf + f]) : -ldcg(&a.E0[v * nf + f]);
        c[v] = hS * ((fa[v] - fb) - lp * du[v]);   // (U + dU) - U = dU
      }
    }
  }
  const bool b0 = s & 1, b1 = s & 2;
  const TF k0 = (b0 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b0 ? c[0] : c[1], 1);
  const TF k1 = (b0 ? c[3] : c[2]) + __shfl_xor_sync(0xffffffffu, b0 ? c[2] : c[3], 1);
  const TF mine = (b1 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, b1 ? k0 : k1, 2);
  if (i >= 0) a.dU[s * n + i] = (ldcg(&a.Rk[s * n + i]) - mine) * ldcg(&a.invD[i]);
}

// cell of the g-th position of colour c, or -1 past its end
__device__ __forceinline__ int colour_cell(const ColourRanges &cr, int c, int g) {
  const int r0 = cr.rstart[c], r1 = cr.rstart[c + 1];
  const int *pre = cr.rpre + r0 + c;            // r1 - r0 + 1 prefix entries
  if (g >= pre[r1 - r0]) return -1;
  int lo = 0, hi = r1 - r0 - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return cr.rbegin[r0 + lo] + (g - pre[lo]);
}

template <typename TF>
__global__ void __launch_bounds__(kPersistBlock, 2) k_lo_solve(const __grid_constant__ LoArgs<TF> a) {
  const int n = a.n_cells, nf = a.n_faces;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  const int lane4 = threadIdx.x & 3;
  const int grp = tid >> 2, ngrp = nth >> 2;
  for (int k = 0; k < a.n_implicit; ++k) {
    for (int i = tid; i < n; i += nth) lo_cell_at(a, i, k == 0);
    if (!grid_barrier(a.gb, a.spin_limit, a.err, a.n_err)) return;
    for (int f = tid; f < nf; f += nth) lo_face_at(a, f);
    if (!grid_barrier(a.gb, a.spin_limit, a.err, a.n_err)) return;
    for (int i = tid; i < n; i += nth) lo_rhs_at(a, i, k == 0);
    if (!grid_barrier(a.gb, a.spin_limit, a.err, a.n_err)) return;
    for (int q = 0; q < a.n_seq; ++q) {
      const int c = a.seq[q];
      const int total = a.cr.rpre[a.cr.rstart[c + 1] + c];
      // whole 4-lane groups iterate together so the shuffles stay converged
      for (int g0 = grp - (grp % 8); g0 < total; g0 += ngrp) {
        const int g = g0 + (grp % 8);
        const int i = g < total ? colour_cell(a.cr, c, g) : -1;
        sweep_at(a, i, lane4);
      }
      if (!grid_barrier(a.gb, a.spin_limit, a.err, a.n_err)) return;
    }
  }
  if (a.n_implicit > 0)
    for (int i = tid; i < n; i += nth) lo_cell_at(a, i, 0);
}

}  // namespace kern
}  // namespace cgks
