// libcgks device runtime and C ABI.
//
// A Batch holds one or more steady solves in one concatenated index space
// (see cgks_kernels.cuh) and runs the two-level V-cycle of Ji, Shyy & Xu
// (arXiv:2109.09965, Section 3) or the explicit high-order step (Section
// 2.4) for all of them with one launch per kernel, captured in a CUDA
// graph.  cgks_solver is a batch of one solve; cgks_server admits and
// retires solves and rebuilds its batch when the active set changes.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "cgks_internal.h"
#include "cgks_kernels.cuh"
#include "cgks_persistent.cuh"
#include "cgks_runtime.h"

using namespace cgks;
using namespace cgks::kern;
namespace D = cgks::dev;

namespace {

inline int nblk(int64_t n, int b) { return static_cast<int>((n + b - 1) / b); }

// arrays in the flux type TF (in FP64 mode the state entries alias the
// double state, in mixed mode they are float mirrors)
template <typename T>
struct Bufs {
  T *W = nullptr, *Wx = nullptr, *Wn = nullptr, *Ws = nullptr, *Wxs = nullptr, *U = nullptr;
  T *coef = nullptr, *FA = nullptr, *FB = nullptr;
  T *prim = nullptr, *Flo = nullptr, *lam = nullptr, *E0 = nullptr, *E1 = nullptr;
  T *Rk = nullptr, *invD = nullptr, *dU = nullptr, *lamS = nullptr;
  T *dU2 = nullptr;   // second increment buffer of the partitioned sweep (ping-pong with dU)
};

// batch-wide settings (every solve of a batch shares them)
struct Shared {
  double gamma = 1.4, cfl_hi = 0.4, cfl_lo = 1000.0;
  int n_implicit = 6, n_sweeps = 2, time_scheme = CGKS_S1O2, precision = CGKS_FP64, use_graph = 1, lo_fused = 0;
  int autotune = 1, pdl = 1, flux_lo = CGKS_FLUX_KFVS, flux_hi = CGKS_FLUX_SMOOTH;
  double tau_c1 = 0.01, tau_c2 = 1.0, weno_eps = 0.0, weno_g0 = 0.95;
  int weno_vars = CGKS_WENO_CONSERVATIVE;
  long long spin_limit = 0;      // grid-barrier polls of the persistent launch (0: kSpinLimit)
  int sweep_order = CGKS_SWEEP_COLOUR, part_cells = 2048;
  int lo_viscous = 0;            // first-order viscous flux on the low-order level
  // serving batches: a per-solve flux class (smooth / limited) instead of
  // the batch-wide flux_hi and weno_eps; the limited class takes the full
  // flux with conservative compact WENO and the constants above
  bool per_slot_flux = false;
  cgks_alloc_fn alloc = nullptr;
  cgks_free_fn free = nullptr;
  void *alloc_ctx = nullptr;
};

// One solve of a batch: its mesh, its parameters and where it sits.
struct Member {
  std::shared_ptr<const HostMesh> mesh;
  cgks_params params{};
  int64_t cell_off = 0, n_pad = 0, face_off = 0;
  bool active = false;
};

// device tables of a batch (views into its arena)
struct DevArrays {
  double *vol, *ivol, *per, *ih, *m2, *op, *fn, *fS, *fjump, *fxi, *snx, *sny, *shs, *fidl = nullptr;
  double *mu, *bcuw, *bcrho, *bcu, *bcp;
  int *cface, *cnbr, *fc0, *fc1, *csid, *fsid, *bckind;
  unsigned char *ccol, *wenok;
  float *f_ivol = nullptr, *f_ih = nullptr, *f_m2 = nullptr, *f_op = nullptr, *f_fn = nullptr, *f_fS = nullptr,
        *f_fjump = nullptr, *f_fidl = nullptr, *f_fxi = nullptr, *f_snx = nullptr, *f_sny = nullptr, *f_shs = nullptr, *f_mu = nullptr,
        *f_bcuw = nullptr, *f_bcrho = nullptr, *f_bcu = nullptr, *f_bcp = nullptr;
};

// A batch is a slot table over one device arena: capacity for Ncap cells,
// Fcap faces and S solve slots.  A solve occupies a contiguous cell range
// (a multiple of kCellBlock) and a contiguous face range; cells and faces
// outside every solve are inert (csid / fsid = -1, no faces, a valid
// uniform state).  Kernels run over [0, N) cells and [0, F) faces, the
// extents of the solves present; arrays are strided by the capacity.
struct Batch {
  Shared sh;
  DevArrays d{};
  std::vector<Member> mem;     // [S] slots
  int S = 0;
  int64_t Ncap = 0, Fcap = 0;  // capacity (array strides)
  int64_t N = 0, F = 0;        // launch extents
  bool mixed = false;
  int n_colours = 0;
  std::vector<int> sweep_seq;        // colour order after the first pass
  std::vector<int> list_off;         // [n_colours + 1] offsets into the sweep cell list
  std::vector<Ranges> ranges[kNShape];  // per sweep shape, per colour: per-solve cell ranges (n = 0: the list)
  ParamsT<double> dp{};
  ParamsT<float> fp{};
  MeshT<double> dm{};
  MeshT<float> fm{};
  cudaStream_t stream = nullptr;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  // FP64 state and accumulation arrays
  double *W = nullptr, *Wx = nullptr, *Wn = nullptr, *Ws = nullptr, *Wxs = nullptr;
  double *U = nullptr, *Rp0 = nullptr, *Src = nullptr, *partial = nullptr, *last = nullptr, *stage = nullptr;
  Bufs<double> bd;
  Bufs<float> bf;
  int *list = nullptr, *perm = nullptr, *blk = nullptr;   // blk: [S][2] residual block range per slot
  Ctl *ctl = nullptr;
  unsigned long long *dt_bits = nullptr;
  int *status = nullptr;
  double *res = nullptr;               // [S] residual of the last update
  double *hist = nullptr;              // solve 0's residual history
  int hist_cap = 0;
  cudaGraphExec_t g_cycle = nullptr, g_step = nullptr;
  Timer *timer = nullptr;              // owned by the caller
  long long launches = 0;
  // persistent low-order level: barrier, per-colour ranges, grid size
  GridBarrier *gb = nullptr;
  int *r_start = nullptr, *r_begin = nullptr, *r_pre = nullptr;
  int *ptab = nullptr;               // partitioned sweep: [n_parts][n_colours][2] cell ranges
  int *slim = nullptr;               // [S] flux class per slot (per_slot_flux batches)
  std::vector<int> slim_host;
  int n_lim = 0, n_smooth = 0;       // active solves of each class
  int64_t ptab_cap = 0;              // ints ptab holds
  int n_parts = 0;
  int lo_grid = 0;
  bool lo_fused_ok = false;
  Tuner tune;                          // launch shapes of the tunable kernels
};

constexpr int kMaxColFused = 16;     // colours the fused path handles

void *dev_alloc(const Shared &sh, size_t bytes) {
  if (sh.alloc) return sh.alloc(bytes, sh.alloc_ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}
void dev_free(const Shared &sh, void *p) {
  if (!p) return;
  if (sh.alloc) { if (sh.free) sh.free(p, sh.alloc_ctx); }
  else cudaFree(p);
}

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return CGKS_ECUDA;   \
  } while (0)

// ------------------------------------------------------------------------
// launch helper with optional per-kernel timing
template <typename Kern, typename... Args>
void launch(Batch *b, int id, Kern kern, dim3 grid, dim3 block, Args... args) {
  if (grid.x == 0) return;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool t = b->timer && b->timer->on;
  if (t) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
  }
  launch_on(b->stream, b->sh.pdl != 0, kern, grid, block, args...);
  if (t) {
    cudaEventRecord(e1, b->stream);
    b->timer->ev.push_back({ id, { e0, e1 } });
  }
  b->launches++;
}

// launch with thread-block clusters of cluster_x CTAs along x
template <typename Kern, typename... Args>
void launch_cluster(Batch *b, int id, Kern kern, dim3 grid, dim3 block, int cluster_x, Args... args) {
  if (grid.x == 0) return;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool t = b->timer && b->timer->on;
  if (t) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster_x;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = b->sh.pdl != 0 ? 2 : 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
  if (t) {
    cudaEventRecord(e1, b->stream);
    b->timer->ev.push_back({ id, { e0, e1 } });
  }
  b->launches++;
}

template <typename TF> Bufs<TF> &bufs(Batch *b);
template <> Bufs<double> &bufs<double>(Batch *b) { return b->bd; }
template <> Bufs<float> &bufs<float>(Batch *b) { return b->bf; }
template <typename TF> const MeshT<TF> &fmesh(Batch *b);
template <> const MeshT<double> &fmesh<double>(Batch *b) { return b->dm; }
template <> const MeshT<float> &fmesh<float>(Batch *b) { return b->fm; }
template <typename TF> const ParamsT<TF> &fparams(Batch *b);
template <> const ParamsT<double> &fparams<double>(Batch *b) { return b->dp; }
template <> const ParamsT<float> &fparams<float>(Batch *b) { return b->fp; }
// float mirror of a flux-type array, or null when the flux type is double
template <typename TF> TF *mirror(TF *p) { return is_f32<TF>() ? p : nullptr; }

void enqueue_dt(Batch *b, double dt_fixed) {
  launch(b, KI_DT, k_reset_dt, dim3(1), dim3(256), b->ctl, b->dt_bits, b->S, dt_fixed);
  if (!(dt_fixed > 0.0))
    launch(b, KI_DT, k_dt, dim3(nblk(b->N, kCellBlock)), dim3(kCellBlock), b->dm, b->dp, (const double *)b->W, b->dt_bits);
}

void enqueue_res(Batch *b) {
  launch(b, KI_RESFIN, k_res_final, dim3(b->S), dim3(256), (const double *)b->partial, (const int *)b->blk,
         b->ctl, b->res, b->hist, b->hist_cap, b->last);
}

template <typename TF>
void enqueue_hi_eval(Batch *b, const TF *W, const TF *Wx, TF *Fout) {
  Bufs<TF> &B = bufs<TF>(b);
  // the nonlinear WENO weights and the full flux are separate instantiations,
  // so the default (linear weights, smooth flux) kernels stay as lean as before
  const bool chr = b->sh.weno_eps > 0.0 && b->sh.weno_vars == CGKS_WENO_CHARACTERISTIC;
  const bool weno = b->sh.weno_eps > 0.0 && !chr, full = b->sh.flux_hi == CGKS_FLUX_FULL;
  if (b->sh.per_slot_flux) {
    // one launch per flux class present; each skips the other class's solves
    tuned_launch(b->tune, TK_RECON, b->stream, [&] {
      with_shape(b->tune.shape(TK_RECON), [&](auto sh) {
        constexpr int S = decltype(sh)::value;
        const dim3 g(nblk(b->N, shape_bs(S) * shape_ipt(S))), blk(shape_bs(S));
        if (b->n_smooth) launch(b, KI_RECON, k_recon<TF, S, false>, g, blk, fmesh<TF>(b), fparams<TF>(b), W, Wx, B.coef);
        if (b->n_lim) launch(b, KI_RECON, k_recon<TF, S, true>, g, blk, fmesh<TF>(b), fparams<TF>(b), W, Wx, B.coef);
      });
    });
    tuned_launch(b->tune, TK_FACE, b->stream, [&] {
      with_shape(b->tune.shape(TK_FACE), [&](auto sh) {
        constexpr int S = decltype(sh)::value;
        const dim3 g(nblk(b->F, shape_bs(S) * shape_ipt(S))), blk(shape_bs(S));
        auto go = [&](auto kern) {
          launch(b, KI_FACE, kern, g, blk, fmesh<TF>(b), fparams<TF>(b), W, Wx, (const TF *)B.coef, Fout,
                 (const Ctl *)b->ctl, (const unsigned long long *)b->dt_bits);
        };
        if (b->n_smooth) go(k_face<TF, S, false, false>);
        if (b->n_lim) go(k_face<TF, S, true, false>);
      });
    });
    return;
  }
  tuned_launch(b->tune, TK_RECON, b->stream, [&] {
    with_shape(b->tune.shape(TK_RECON), [&](auto sh) {
      constexpr int S = decltype(sh)::value;
      const dim3 g(nblk(b->N, shape_bs(S) * shape_ipt(S))), blk(shape_bs(S));
      if (weno) launch(b, KI_RECON, k_recon<TF, S, true>, g, blk, fmesh<TF>(b), fparams<TF>(b), W, Wx, B.coef);
      else launch(b, KI_RECON, k_recon<TF, S, false>, g, blk, fmesh<TF>(b), fparams<TF>(b), W, Wx, B.coef);
    });
  });
  tuned_launch(b->tune, TK_FACE, b->stream, [&] {
    with_shape(b->tune.shape(TK_FACE), [&](auto sh) {
      constexpr int S = decltype(sh)::value;
      const dim3 g(nblk(b->F, shape_bs(S) * shape_ipt(S))), blk(shape_bs(S));
      auto go = [&](auto kern) {
        launch(b, KI_FACE, kern, g, blk, fmesh<TF>(b), fparams<TF>(b), W, Wx, (const TF *)B.coef, Fout,
               (const Ctl *)b->ctl, (const unsigned long long *)b->dt_bits);
      };
      if (full && chr) go(k_face<TF, S, true, true>);
      else if (full) go(k_face<TF, S, true, false>);
      else if (chr) go(k_face<TF, S, false, true>);
      else go(k_face<TF, S, false, false>);
    });
  });
}

// high-order step from (W, Wx) into (Wout, Wx): Wx updated in place.
template <typename TF>
void enqueue_hi_step(Batch *b, double *Wout, TF *Wout_m, bool want_res) {
  Bufs<TF> &B = bufs<TF>(b);
  double *part = want_res ? b->partial : nullptr;
  const dim3 g(nblk(b->N, kCellBlock)), blk(kCellBlock);
  enqueue_hi_eval<TF>(b, B.W, B.Wx, B.FA);
  if (b->sh.time_scheme == CGKS_S1O2) {
    launch(b, KI_UPDATE, k_update<TF>, g, blk, b->dm, b->dp, (int)kS1O2, (const double *)b->W, (const TF *)B.FA,
           (const TF *)B.FA, (const Ctl *)b->ctl, (const unsigned long long *)b->dt_bits, b->status, Wout, b->Wx,
           part, b->Rp0, Wout_m, mirror<TF>(B.Wx));
  } else {
    launch(b, KI_UPDATE, k_update<TF>, g, blk, b->dm, b->dp, (int)kS2O4Stage, (const double *)b->W, (const TF *)B.FA,
           (const TF *)B.FA, (const Ctl *)b->ctl, (const unsigned long long *)b->dt_bits, b->status, b->Ws, b->Wxs,
           (double *)nullptr, (double *)nullptr, mirror<TF>(B.Ws), mirror<TF>(B.Wxs));
    enqueue_hi_eval<TF>(b, B.Ws, B.Wxs, B.FB);
    launch(b, KI_UPDATE, k_update<TF>, g, blk, b->dm, b->dp, (int)kS2O4Final, (const double *)b->W, (const TF *)B.FA,
           (const TF *)B.FB, (const Ctl *)b->ctl, (const unsigned long long *)b->dt_bits, b->status, Wout, b->Wx,
           part, b->Rp0, Wout_m, mirror<TF>(B.Wx));
  }
  if (want_res) enqueue_res(b);
}

// low-order solve from U = W_p0 (= Wn), R_p0 in Rp0; result in U.  Per
// implicit step: cell primitives (and U += dU), KFVS faces, right-hand side
// with the first colour pass, then the remaining colour passes.
template <typename TF>
void enqueue_lo_fused(Batch *b) {
  Bufs<TF> &B = bufs<TF>(b);
  LoArgs<TF> a;
  std::memset(&a, 0, sizeof(a));
  a.dm = b->dm; a.fm = fmesh<TF>(b); a.dp = b->dp; a.fp = fparams<TF>(b);
  a.n_implicit = b->sh.n_implicit;
  a.colour0 = b->sh.n_sweeps > 0 ? 1 : 0;
  a.n_seq = static_cast<int>(b->sweep_seq.size());
  a.n_cells = static_cast<int>(b->N);
  a.n_faces = static_cast<int>(b->F);
  for (int q = 0; q < a.n_seq; ++q) a.seq[q] = b->sweep_seq[q];
  a.cr.rstart = b->r_start; a.cr.rbegin = b->r_begin; a.cr.rpre = b->r_pre;
  a.Wp0 = b->Wn; a.Rp0 = b->Rp0; a.U = b->U; a.Src = b->Src;
  a.dU = B.dU; a.prim = B.prim; a.Um = mirror<TF>(B.U); a.Flo = B.Flo; a.lam = B.lam; a.E0 = B.E0; a.E1 = B.E1;
  a.Rk = B.Rk; a.invD = B.invD; a.lamS = B.lamS;
  a.gb = b->gb; a.err = b->status; a.n_err = static_cast<int>(b->S);
  a.spin_limit = b->sh.spin_limit > 0 ? b->sh.spin_limit : kSpinLimit;
  // a launch that timed out leaves the barrier's arrival count behind: start
  // every launch from a cleared barrier (a memset node when captured)
  cudaMemsetAsync(b->gb, 0, sizeof(GridBarrier), b->stream);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->lo_grid);
  cfg.blockDim = dim3(kPersistBlock);
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool t = b->timer && b->timer->on;
  if (t) { cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventRecord(e0, b->stream); }
  cudaLaunchKernelEx(&cfg, k_lo_solve<TF>, a);
  if (t) { cudaEventRecord(e1, b->stream); b->timer->ev.push_back({ KI_LOSOLVE, { e0, e1 } }); }
  b->launches++;
}

template <typename TF>
void enqueue_lo_solve(Batch *b) {
  if (b->lo_fused_ok) {
    enqueue_lo_fused<TF>(b);
    return;
  }
  Bufs<TF> &B = bufs<TF>(b);
  const dim3 gc(nblk(b->N, kCellBlock)), blk(kCellBlock);
  const bool part = b->sh.sweep_order == CGKS_SWEEP_PARTITIONED;
  // colour sweeps: k_lo_rhs relaxes colour 0 of the first pass.  Partitioned:
  // k_lo_rhs zeroes the increments, the sweeps ping-pong between dU and
  // dU2 starting so that the last one writes dU
  const int colour0 = !part && b->sh.n_sweeps > 0 ? 1 : 0;
  TF *dU0 = part && (b->sh.n_sweeps & 1) ? B.dU2 : B.dU;
  for (int k = 0; k < b->sh.n_implicit; ++k) {
    launch(b, KI_LOCELL, k_lo_cell<TF>, gc, blk, static_cast<int>(b->Ncap), fparams<TF>(b), k == 0 ? 1 : 0,
           (const double *)b->Wn, b->U, (const TF *)B.dU, B.prim, mirror<TF>(B.U));
    tuned_launch(b->tune, TK_LOFACE, b->stream, [&] {
      with_shape(b->tune.shape(TK_LOFACE), [&](auto sh) {
        constexpr int S = decltype(sh)::value;
        launch(b, KI_LOFACE, k_lo_face<TF, S>, dim3(nblk(b->F, shape_bs(S) * shape_ipt(S))), dim3(shape_bs(S)),
               fmesh<TF>(b), fparams<TF>(b), (const TF *)B.U, (const TF *)B.prim, B.Flo, B.lam, B.E0, B.E1);
      });
    });
    launch(b, KI_LORHS, k_lo_rhs<TF>, gc, blk, b->dm, b->dp, k == 0 ? 1 : 0, colour0, (const TF *)B.Flo,
           (const TF *)B.lam, (const double *)b->Rp0, b->Src, B.Rk, B.invD, dU0, B.lamS);
    if (part) {
      TF *in = dU0, *out = dU0 == B.dU ? B.dU2 : B.dU;
      for (int sw = 0; sw < b->sh.n_sweeps; ++sw) {
        launch_cluster(b, KI_SWEEP, k_sweep_part<TF>, dim3(b->n_parts * kPartCluster), dim3(kPartBlock),
                       kPartCluster, fmesh<TF>(b), fparams<TF>(b), (const int *)b->ptab, b->n_colours,
                       (const TF *)B.U, (const TF *)B.prim, (const TF *)B.Rk, (const TF *)B.invD,
                       (const TF *)B.lamS, (const TF *)B.E0, (const TF *)B.E1, (const TF *)in, out);
        std::swap(in, out);
      }
      continue;
    }
    const int ssh = b->tune.shape(TK_SWEEP);
    for (int c : b->sweep_seq) {
      const int cnt = b->list_off[c + 1] - b->list_off[c];
      const Ranges &R = b->ranges[ssh][c];
      const bool use_list = R.n == 0;
      const int grid = use_list ? nblk(cnt, sweep_cpb(ssh)) : R.blk[R.n];
      tuned_launch(b->tune, TK_SWEEP, b->stream, [&] {
        with_shape(ssh, [&](auto sh) {
          constexpr int S = decltype(sh)::value;
          launch(b, KI_SWEEP, k_sweep<TF, S>, dim3(grid), dim3(shape_bs(S)), fmesh<TF>(b), fparams<TF>(b), R,
                 use_list ? (const int *)b->list + b->list_off[c] : (const int *)nullptr, cnt, (const TF *)B.U,
                 (const TF *)B.prim, (const TF *)B.Rk, (const TF *)B.invD, (const TF *)B.lamS,
                 (const TF *)B.E0, (const TF *)B.E1, B.dU);
        });
      });
    }
  }
  // U^{n_implicit} = U + dU of the last step
  if (b->sh.n_implicit > 0)
    launch(b, KI_LOCELL, k_lo_cell<TF>, gc, blk, static_cast<int>(b->Ncap), fparams<TF>(b), 0, (const double *)b->Wn, b->U,
           (const TF *)B.dU, B.prim, mirror<TF>(B.U));
  else
    cudaMemcpyAsync(b->U, b->Wn, sizeof(double) * 4 * b->Ncap, cudaMemcpyDeviceToDevice, b->stream);
}

template <typename TF>
void enqueue_prolong(Batch *b) {
  launch(b, KI_PROLONG, k_prolong<TF>, dim3(nblk(b->N, kCellBlock)), dim3(kCellBlock), b->dm, b->dp, b->W,
         (const double *)b->Wn, (const double *)b->U, b->status, b->partial, mirror<TF>(bufs<TF>(b).W));
  enqueue_res(b);
}

template <typename TF>
void enqueue_cycle_t(Batch *b) {
  Bufs<TF> &B = bufs<TF>(b);
  enqueue_dt(b, -1.0);
  // 1: high-order step into W_p0 = Wn (W keeps W^n for the residual)
  enqueue_hi_step<TF>(b, b->Wn, mirror<TF>(B.Wn), false);
  // 2: R_p0 = time-averaged high-order net flux at W^{n+1}
  enqueue_hi_eval<TF>(b, B.Wn, B.Wx, B.FB);
  launch(b, KI_UPDATE, k_update<TF>, dim3(nblk(b->N, kCellBlock)), dim3(kCellBlock), b->dm, b->dp, (int)kResidual,
         (const double *)b->Wn, (const TF *)B.FB, (const TF *)B.FB, (const Ctl *)b->ctl,
         (const unsigned long long *)b->dt_bits, b->status, (double *)nullptr, (double *)nullptr, (double *)nullptr,
         b->Rp0, (TF *)nullptr, (TF *)nullptr);
  // 3-4: forcing and implicit low-order solve
  enqueue_lo_solve<TF>(b);
  // 5: correction and residual
  enqueue_prolong<TF>(b);
}

void enqueue_cycle(Batch *b) {
  if (b->mixed) enqueue_cycle_t<float>(b);
  else enqueue_cycle_t<double>(b);
}

void enqueue_explicit_step(Batch *b, double dt_fixed) {
  enqueue_dt(b, dt_fixed);
  if (b->mixed) enqueue_hi_step<float>(b, b->W, b->bf.W, true);
  else enqueue_hi_step<double>(b, b->W, nullptr, true);
}

void enqueue_lo_smooth(Batch *b) {
  cudaMemcpyAsync(b->Wn, b->W, sizeof(double) * 4 * b->Ncap, cudaMemcpyDeviceToDevice, b->stream);
  if (b->mixed) { enqueue_lo_solve<float>(b); enqueue_prolong<float>(b); }
  else { enqueue_lo_solve<double>(b); enqueue_prolong<double>(b); }
}

long long count_launches(const Batch *b, bool cycle) {
  long long per_eval = b->sh.per_slot_flux ? 2 * ((b->n_smooth > 0) + (b->n_lim > 0)) : 2;
  long long hi = per_eval + 1 + (b->sh.time_scheme == CGKS_S2O4 ? per_eval + 1 : 0);
  long long dt = 2;
  if (!cycle) return dt + hi + 1;
  const long long sweeps = b->sh.sweep_order == CGKS_SWEEP_PARTITIONED
                               ? static_cast<long long>(b->sh.n_sweeps)
                               : static_cast<long long>(b->sweep_seq.size());
  long long lo = b->lo_fused_ok ? 1 : b->sh.n_implicit * (3 + sweeps) + (b->sh.n_implicit > 0 ? 1 : 0);
  return dt + hi + per_eval + 1 + lo + 2;
}

void drop_graphs(Batch *b) {
  if (b->g_cycle) { cudaGraphExecDestroy(b->g_cycle); b->g_cycle = nullptr; }
  if (b->g_step) { cudaGraphExecDestroy(b->g_step); b->g_step = nullptr; }
}

int ensure_hist(Batch *b, int n) {
  if (n <= b->hist_cap) return CGKS_OK;
  double *p = static_cast<double *>(dev_alloc(b->sh, sizeof(double) * n));
  if (!p) return CGKS_ENOMEM;
  if (b->hist) { cudaStreamSynchronize(b->stream); dev_free(b->sh, b->hist); }
  b->hist = p;
  b->hist_cap = n;
  drop_graphs(b);   // graphs hold the old pointer
  return CGKS_OK;
}

int capture(Batch *b, bool cycle, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  Timer *t = b->timer;
  b->timer = nullptr;
  long long l0 = b->launches;
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  if (cycle) enqueue_cycle(b);
  else enqueue_explicit_step(b, -1.0);
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  b->launches = l0;
  b->timer = t;
  if (e != cudaSuccess) return CGKS_ECUDA;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? CGKS_OK : CGKS_ECUDA;
}

// n cycles (or explicit steps) without host synchronisation, except that
// the autotuner's units read their events back (once per call)
int run_many(Batch *b, int n, bool cycle) {
  if (n <= 0) return CGKS_OK;
  CK(cudaMemsetAsync(&b->ctl->res_ctr, 0, sizeof(int), b->stream));
  const bool graph = b->sh.use_graph && !(b->timer && b->timer->on);
  cudaGraphExec_t *ge = cycle ? &b->g_cycle : &b->g_step;
  const long long per = count_launches(b, cycle);
  int k = 0;
  if (b->tune.eager(cycle)) {
    for (; k < n && b->tune.eager(cycle); ++k) {
      b->tune.begin_unit();
      if (cycle) enqueue_cycle(b);
      else enqueue_explicit_step(b, -1.0);
      b->tune.end_unit(cycle);
    }
    if (b->tune.collect()) drop_graphs(b);
  }
  if (graph && k < n && !*ge) {
    int rc = capture(b, cycle, ge);
    if (rc) return rc;
  }
  for (; k < n; ++k) {
    if (graph) {
      CK(cudaGraphLaunch(*ge, b->stream));
      b->launches += per;
    } else if (cycle) {
      enqueue_cycle(b);
    } else {
      enqueue_explicit_step(b, -1.0);
    }
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}

template <typename T>
void fill_shared_params(const Shared &sh, ParamsT<T> &P) {
  double K = (4.0 - 2.0 * sh.gamma) / (sh.gamma - 1.0);
  P.gamma = static_cast<T>(sh.gamma);
  P.K = static_cast<T>(K);
  P.cfl_hi = static_cast<T>(sh.cfl_hi);
  P.cfl_lo = static_cast<T>(sh.cfl_lo);
  P.kc.K = static_cast<T>(K);
  P.kc.c2K = static_cast<T>(2.0 / (K + 2.0));
  P.kc.c4K = static_cast<T>(4.0 / (K + 2.0));
  P.flux_lo = sh.flux_lo;
  P.flux_hi = sh.flux_hi;
  P.tau_c1 = static_cast<T>(sh.tau_c1);
  P.tau_c2 = static_cast<T>(sh.tau_c2);
  P.weno_eps = static_cast<T>(sh.weno_eps);
  P.weno_g0 = static_cast<T>(sh.weno_g0);
  P.weno_vars = sh.weno_vars;
  P.lo_viscous = sh.lo_viscous;
}

// The device arena of a batch: one allocation carved into 256-byte aligned
// pieces.  plan_arena lists the pieces for N padded cells, F faces, S
// solves and L cells in the sweep lists; arena_total is the exact size.
struct Piece { void **dst; size_t bytes; };

size_t arena_total(const std::vector<Piece> &pieces) {
  size_t total = 0;
  for (auto &pc : pieces) total += (pc.bytes + 255) & ~size_t(255);
  return total;
}

void plan_arena(Batch *b, int64_t N, int64_t F, int S, int64_t L, bool mixed, std::vector<Piece> &pieces) {
  DevArrays &d = b->d;
  auto P8 = [&](double **x, int64_t cnt) { pieces.push_back({ reinterpret_cast<void **>(x), sizeof(double) * cnt }); };
  auto P4 = [&](float **x, int64_t cnt) { pieces.push_back({ reinterpret_cast<void **>(x), sizeof(float) * cnt }); };
  auto PI = [&](int **x, int64_t cnt) { pieces.push_back({ reinterpret_cast<void **>(x), sizeof(int) * cnt }); };
  auto PV = [&](void **x, size_t bytes) { pieces.push_back({ x, bytes }); };
  const int64_t T = kTagsPerSolve * static_cast<int64_t>(S);
  P8(&b->W, 4 * N); P8(&b->Wx, 8 * N); P8(&b->Wn, 4 * N); P8(&b->Ws, 4 * N); P8(&b->Wxs, 8 * N);
  P8(&b->U, 4 * N); P8(&b->Rp0, 4 * N); P8(&b->Src, 4 * N); P8(&b->stage, 12 * N);
  P8(&b->partial, 2 * std::max<int64_t>(N / kCellBlock, 1)); P8(&b->last, 4); P8(&b->res, S);
  P8(&d.vol, N); P8(&d.ivol, N); P8(&d.per, N); P8(&d.ih, N); P8(&d.m2, 3 * N); P8(&d.op, kNCol * kNM * N);
  P8(&d.snx, kMaxFace * N); P8(&d.sny, kMaxFace * N); P8(&d.shs, kMaxFace * N);
  P8(&d.fn, 2 * F); P8(&d.fS, F); P8(&d.fjump, F); P8(&d.fxi, 8 * F); P8(&d.fidl, F);
  P8(&d.mu, S); P8(&d.bcuw, 2 * T); P8(&d.bcrho, T); P8(&d.bcu, 2 * T); P8(&d.bcp, T);
  PI(&d.cface, kMaxFace * N); PI(&d.cnbr, kMaxFace * N); PI(&d.fc0, F); PI(&d.fc1, F); PI(&d.csid, N); PI(&d.fsid, F);
  PI(&d.bckind, T); PI(&b->list, std::max<int64_t>(L, 1)); PI(&b->perm, N); PI(&b->blk, 2 * S);
  PV(reinterpret_cast<void **>(&d.ccol), N);
  PV(reinterpret_cast<void **>(&d.wenok), N);
  PV(reinterpret_cast<void **>(&b->ctl), sizeof(Ctl));
  PV(reinterpret_cast<void **>(&b->dt_bits), sizeof(unsigned long long) * S);
  PI(&b->status, S);
  PV(reinterpret_cast<void **>(&b->gb), sizeof(GridBarrier));
  PI(&b->slim, S);
  PI(&b->r_start, kMaxColFused + 1); PI(&b->r_begin, kMaxColFused * static_cast<int64_t>(S));
  PI(&b->r_pre, kMaxColFused * static_cast<int64_t>(S) + kMaxColFused);
  if (b->sh.sweep_order == CGKS_SWEEP_PARTITIONED) {
    // at most N / part_cells + S partitions (one partial per solve)
    b->ptab_cap = 2 * kMaxPartColours * (N / std::max(b->sh.part_cells, 1) + S);
    PI(&b->ptab, b->ptab_cap);
  }
  if (!mixed) {
    Bufs<double> &X = b->bd;
    P8(&X.coef, 20 * N); P8(&X.FA, 16 * F); P8(&X.FB, 16 * F);
    P8(&X.prim, D::NPRIM * N); P8(&X.Flo, 4 * F); P8(&X.lam, F); P8(&X.E0, 4 * F); P8(&X.E1, 4 * F);
    P8(&X.Rk, 4 * N); P8(&X.invD, N); P8(&X.dU, 4 * N); P8(&X.lamS, kMaxFace * N);
    if (b->sh.sweep_order == CGKS_SWEEP_PARTITIONED) P8(&X.dU2, 4 * N);
  } else {
    Bufs<float> &X = b->bf;
    P4(&X.W, 4 * N); P4(&X.Wx, 8 * N); P4(&X.Wn, 4 * N); P4(&X.Ws, 4 * N); P4(&X.Wxs, 8 * N); P4(&X.U, 4 * N);
    P4(&X.coef, 20 * N); P4(&X.FA, 16 * F); P4(&X.FB, 16 * F);
    P4(&X.prim, D::NPRIM * N); P4(&X.Flo, 4 * F); P4(&X.lam, F);
    P4(&X.Rk, 4 * N); P4(&X.invD, N); P4(&X.dU, 4 * N); P4(&X.lamS, kMaxFace * N);
    if (b->sh.sweep_order == CGKS_SWEEP_PARTITIONED) P4(&X.dU2, 4 * N);
    P4(&d.f_ivol, N); P4(&d.f_ih, N); P4(&d.f_m2, 3 * N); P4(&d.f_op, kNCol * kNM * N);
    P4(&d.f_snx, kMaxFace * N); P4(&d.f_sny, kMaxFace * N); P4(&d.f_shs, kMaxFace * N);
    P4(&d.f_fn, 2 * F); P4(&d.f_fS, F); P4(&d.f_fjump, F); P4(&d.f_fxi, 8 * F); P4(&d.f_fidl, F);
    P4(&d.f_mu, S); P4(&d.f_bcuw, 2 * T); P4(&d.f_bcrho, T); P4(&d.f_bcu, 2 * T); P4(&d.f_bcp, T);
  }
}

constexpr int kHistDefault = 1024;

// Device bytes one solve of n cells and nf faces takes in a batch: the
// arena pieces for its padded cells and faces and one solve slot, plus a
// residual history.
size_t solve_footprint(int64_t n, int64_t nf, bool mixed) {
  const int64_t np = (n + kCellBlock - 1) / kCellBlock * kCellBlock;
  Batch tmp;
  std::vector<Piece> pieces;
  plan_arena(&tmp, np, nf, 1, n, mixed, pieces);
  return arena_total(pieces) + sizeof(double) * kHistDefault;
}

int64_t pad_cells(int64_t n) { return (n + kCellBlock - 1) / kCellBlock * kCellBlock; }

void destroy_batch(Batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  dev_free(b->sh, b->hist);
  dev_free(b->sh, b->arena);
  delete b;
}

// Make cells [c0, c1) inert: no faces, no solve, no colour, uniform state.
void clear_cells(Batch *b, int64_t c0, int64_t c1) {
  if (c1 <= c0) return;
  k_clear_cells<<<nblk(c1 - c0, kCellBlock), kCellBlock, 0, b->stream>>>(
      static_cast<int>(c0), static_cast<int>(c1), static_cast<int>(b->Ncap), b->d.csid, b->d.ccol, b->d.cface,
      b->d.cnbr, b->W, b->Wx, b->Wn, b->Ws, b->Wxs, b->mixed ? b->bf.W : nullptr, b->mixed ? b->bf.Wx : nullptr,
      b->mixed ? b->bf.Wn : nullptr, b->mixed ? b->bf.Ws : nullptr, b->mixed ? b->bf.Wxs : nullptr);
  // the second increment buffer of the partitioned sweep is written only at
  // partition cells: clear it (and the first) where cells become inert
  for (int v = 0; v < 4; ++v) {
    if (b->bd.dU2) {
      cudaMemsetAsync(b->bd.dU + v * b->Ncap + c0, 0, sizeof(double) * (c1 - c0), b->stream);
      cudaMemsetAsync(b->bd.dU2 + v * b->Ncap + c0, 0, sizeof(double) * (c1 - c0), b->stream);
    }
    if (b->bf.dU2) {
      cudaMemsetAsync(b->bf.dU + v * b->Ncap + c0, 0, sizeof(float) * (c1 - c0), b->stream);
      cudaMemsetAsync(b->bf.dU2 + v * b->Ncap + c0, 0, sizeof(float) * (c1 - c0), b->stream);
    }
  }
}

// Allocate a batch with capacity for Ncap cells, Fcap faces and S slots;
// every cell and face starts inert.
int create_batch(const Shared &sh, int64_t Ncap, int64_t Fcap, int S, cudaStream_t st, Batch **out) {
  *out = nullptr;
  if (S < 1 || Ncap < kCellBlock || Ncap % kCellBlock || Fcap < 1) return CGKS_EINVAL;
  if (Ncap * kNCol * kNM > INT32_MAX || Fcap * 16 > INT32_MAX) return CGKS_EINVAL;
  std::unique_ptr<Batch> B(new (std::nothrow) Batch());
  if (!B) return CGKS_ENOMEM;
  Batch *b = B.get();
  b->sh = sh;
  b->tune.on = sh.autotune != 0;
  b->S = S;
  b->mem.assign(S, Member{});
  b->Ncap = Ncap; b->Fcap = Fcap;
  b->mixed = sh.precision == CGKS_MIXED;
  b->stream = st;
  DevArrays &d = b->d;
  std::vector<Piece> pieces;
  plan_arena(b, Ncap, Fcap, S, Ncap, b->mixed, pieces);
  const size_t total = arena_total(pieces);
  b->arena = dev_alloc(sh, total);
  if (!b->arena) return CGKS_ENOMEM;
  b->arena_bytes = total;
  {
    char *cur = static_cast<char *>(b->arena);
    for (auto &pc : pieces) { *pc.dst = cur; cur += (pc.bytes + 255) & ~size_t(255); }
  }
  if (!b->mixed) {
    Bufs<double> &X = b->bd;
    X.W = b->W; X.Wx = b->Wx; X.Wn = b->Wn; X.Ws = b->Ws; X.Wxs = b->Wxs; X.U = b->U;
  }
  // kernel-side views
  fill_shared_params(sh, b->dp);
  fill_shared_params(sh, b->fp);
  b->dp.mu = d.mu; b->dp.bc_kind = d.bckind; b->dp.bc_uw = d.bcuw; b->dp.bc_rho = d.bcrho; b->dp.bc_u = d.bcu;
  b->dp.bc_p = d.bcp;
  b->fp.mu = d.f_mu; b->fp.bc_kind = d.bckind; b->fp.bc_uw = d.f_bcuw; b->fp.bc_rho = d.f_bcrho; b->fp.bc_u = d.f_bcu;
  b->fp.bc_p = d.f_bcp;
  b->dp.slim = sh.per_slot_flux ? b->slim : nullptr;
  b->fp.slim = sh.per_slot_flux ? b->slim : nullptr;
  b->slim_host.assign(S, 0);
  MeshT<double> &dm = b->dm;
  dm.nc = static_cast<int>(Ncap); dm.nf = static_cast<int>(Fcap);
  dm.vol = d.vol; dm.ivol = d.ivol; dm.per = d.per; dm.ih = d.ih; dm.m2 = d.m2; dm.op = d.op;
  dm.fn = d.fn; dm.fS = d.fS; dm.fjump = d.fjump; dm.fxi = d.fxi; dm.snx = d.snx; dm.sny = d.sny; dm.shs = d.shs;
  dm.fidl = d.fidl;
  dm.cface = d.cface; dm.cnbr = d.cnbr; dm.fc0 = d.fc0; dm.fc1 = d.fc1; dm.csid = d.csid; dm.fsid = d.fsid;
  dm.ccol = d.ccol; dm.wenok = d.wenok;
  MeshT<float> &fm = b->fm;
  fm.nc = dm.nc; fm.nf = dm.nf;
  fm.vol = nullptr; fm.per = nullptr; fm.ivol = d.f_ivol; fm.ih = d.f_ih; fm.m2 = d.f_m2; fm.op = d.f_op;
  fm.fn = d.f_fn; fm.fS = d.f_fS; fm.fjump = d.f_fjump; fm.fxi = d.f_fxi; fm.snx = d.f_snx; fm.sny = d.f_sny;
  fm.fidl = d.f_fidl;
  fm.shs = d.f_shs;
  fm.cface = d.cface; fm.cnbr = d.cnbr; fm.fc0 = d.fc0; fm.fc1 = d.fc1; fm.csid = d.csid; fm.fsid = d.fsid;
  fm.ccol = d.ccol; fm.wenok = d.wenok;
  bool ok = cudaMemsetAsync(b->ctl, 0, sizeof(Ctl), st) == cudaSuccess &&
            cudaMemsetAsync(b->status, 0, sizeof(int) * S, st) == cudaSuccess &&
            cudaMemsetAsync(b->res, 0, sizeof(double) * S, st) == cudaSuccess &&
            cudaMemsetAsync(b->blk, 0, sizeof(int) * 2 * S, st) == cudaSuccess &&
            cudaMemsetAsync(b->last, 0, sizeof(double) * 4, st) == cudaSuccess &&
            cudaMemsetAsync(b->Rp0, 0, sizeof(double) * 4 * Ncap, st) == cudaSuccess &&
            cudaMemsetAsync(d.fsid, 0xff, sizeof(int) * Fcap, st) == cudaSuccess &&
            cudaMemsetAsync(d.bckind, 0, sizeof(int) * kTagsPerSolve * S, st) == cudaSuccess &&
            cudaMemsetAsync(b->gb, 0, sizeof(GridBarrier), st) == cudaSuccess &&
            cudaMemsetAsync(b->slim, 0, sizeof(int) * S, st) == cudaSuccess;
  if (ok) {
    if (b->mixed) ok = cudaMemsetAsync(b->bf.dU, 0, sizeof(float) * 4 * Ncap, st) == cudaSuccess;
    else ok = cudaMemsetAsync(b->bd.dU, 0, sizeof(double) * 4 * Ncap, st) == cudaSuccess;
    if (ok && b->bf.dU2) ok = cudaMemsetAsync(b->bf.dU2, 0, sizeof(float) * 4 * Ncap, st) == cudaSuccess;
    if (ok && b->bd.dU2) ok = cudaMemsetAsync(b->bd.dU2, 0, sizeof(double) * 4 * Ncap, st) == cudaSuccess;
  }
  if (ok) {
    clear_cells(b, 0, Ncap);
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  }
  if (!ok) { destroy_batch(B.release()); return CGKS_ECUDA; }
  int rc = ensure_hist(b, kHistDefault);
  if (rc) { destroy_batch(B.release()); return rc; }
  // grid of the persistent low-order launch: every block resident at once
  {
    int dev = 0, coop = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (b->mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lo_solve<float>, kPersistBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lo_solve<double>, kPersistBlock, 0);
    b->lo_grid = coop ? per_sm * nsm : 0;
    cudaGetLastError();
  }
  *out = B.release();
  return CGKS_OK;
}

// Upload solve m into slot s at cells [cell_off, cell_off + n_pad) and
// faces [face_off, face_off + n_faces).  Its state is set separately.
int insert_solve(Batch *b, int s, const Member &m, int64_t cell_off, int64_t face_off) {
  const HostMesh &hm = *m.mesh;
  const cgks_params &p = m.params;
  const int64_t nc = hm.n_cells, nf = hm.n_faces, np = pad_cells(nc), co = cell_off, fo = face_off;
  const int64_t N = b->Ncap, F = b->Fcap;
  if (s < 0 || s >= b->S || b->mem[s].active || co % kCellBlock || co + np > N || fo + nf > F) return CGKS_EINVAL;
  cudaStream_t st = b->stream;
  clear_cells(b, co, co + np);
  if (cudaGetLastError() != cudaSuccess) return CGKS_ECUDA;
  // local tables (np cells, nf faces) with global indices
  std::vector<double> vol(np, 1.0), ivol(np, 1.0), per(np, 4.0), ih(np, 1.0), m2(3 * np, 0.0),
      op(kNCol * kNM * np, 0.0), snx(kMaxFace * np, 0.0), sny(kMaxFace * np, 0.0), shs(kMaxFace * np, 0.0);
  std::vector<double> fn(2 * nf), fS(nf), fjump(nf), fxi(8 * nf), fidl(nf);
  std::vector<int> cface(kMaxFace * np, kNoFace), cnbr(kMaxFace * np, -1), csid(np, -1), perm(np, 0), fc0(nf),
      fc1(nf), fsid(nf, s);
  std::vector<unsigned char> ccol(np, 255), wenok(np, 0);
  std::vector<char> wall(kTagsPerSolve, 0);
  for (int t = 0; t < p.n_bc; ++t) wall[t] = is_wall_kind(p.bc[t].kind);
  std::vector<double> ops;
  std::vector<unsigned char> qok;
  build_operator(hm, wall, ops, &qok);
  for (int64_t i = 0; i < nc; ++i) wenok[i] = qok[i];
  for (int64_t i = 0; i < nc; ++i) {
    vol[i] = hm.vol[i]; ivol[i] = 1.0 / hm.vol[i]; per[i] = hm.per[i]; ih[i] = 1.0 / hm.h[i];
    for (int q = 0; q < 3; ++q) m2[q * np + i] = hm.m2[q * nc + i];
    for (int q = 0; q < kNCol * kNM; ++q) op[q * np + i] = ops[q * nc + i];
    csid[i] = s;
    perm[i] = hm.perm[i];
    for (int sl = 0; sl < kMaxFace; ++sl) {
      const int32_t fs = hm.cface[sl * nc + i];
      if (fs == kNoFace) continue;
      const int32_t f = fs >= 0 ? fs : ~fs;
      const double sg = fs >= 0 ? 1.0 : -1.0;
      cface[sl * np + i] = fs >= 0 ? static_cast<int>(f + fo) : ~static_cast<int>(f + fo);
      const int32_t j = hm.cnbr[sl * nc + i];
      cnbr[sl * np + i] = j >= 0 ? static_cast<int>(j + co) : -1;
      snx[sl * np + i] = sg * hm.fn[f];
      sny[sl * np + i] = sg * hm.fn[nf + f];
      shs[sl * np + i] = 0.5 * hm.fS[f];
    }
  }
  for (int c = 0; c < hm.n_colours; ++c)
    for (int32_t i = hm.colour_start[c]; i < hm.colour_start[c + 1]; ++i) ccol[i] = static_cast<unsigned char>(c);
  for (int64_t f = 0; f < nf; ++f) {
    fc0[f] = static_cast<int>(hm.fc0[f] + co);
    const int32_t c1 = hm.fc1[f];
    fc1[f] = c1 >= 0 ? static_cast<int>(c1 + co) : -1 - (s * kTagsPerSolve + (-1 - c1));
    fn[f] = hm.fn[f]; fn[nf + f] = hm.fn[nf + f];
    fS[f] = hm.fS[f];
    fjump[f] = hm.fdelta[f] > 0.0 ? p.alpha / hm.fdelta[f] : 0.0;
    fidl[f] = hm.fdelta[f] > 0.0 ? 1.0 / hm.fdelta[f] : 0.0;
    for (int q = 0; q < 8; ++q) fxi[q * nf + f] = hm.fxi[q * nf + f];
  }
  std::vector<double> mu(1, p.mu), bc_uw(2 * kTagsPerSolve, 0.0), bc_rho(kTagsPerSolve, 1.0),
      bc_u(2 * kTagsPerSolve, 0.0), bc_p(kTagsPerSolve, 1.0);
  std::vector<int> bc_kind(kTagsPerSolve, CGKS_BC_SLIP);
  for (int t = 0; t < kTagsPerSolve; ++t) {
    const cgks_bc &bc = p.bc[t];
    bc_kind[t] = t < p.n_bc ? bc.kind : CGKS_BC_SLIP;
    bc_uw[2 * t] = bc.u_wall[0]; bc_uw[2 * t + 1] = bc.u_wall[1];
    bc_rho[t] = bc.rho; bc_u[2 * t] = bc.u[0]; bc_u[2 * t + 1] = bc.u[1]; bc_p[t] = bc.p;
  }
  // component-sliced uploads: host [comps][len] -> device [comps][stride] at off
  bool ok = true;
  auto up = [&](auto *dst, const auto &src, int64_t len, int64_t stride, int64_t off) {
    using E = typename std::decay_t<decltype(src)>::value_type;
    const int64_t comps = static_cast<int64_t>(src.size()) / std::max<int64_t>(len, 1);
    for (int64_t q = 0; q < comps && ok && len > 0; ++q)
      ok = cudaMemcpyAsync(dst + q * stride + off, src.data() + q * len, sizeof(E) * len, cudaMemcpyHostToDevice,
                           st) == cudaSuccess;
  };
  DevArrays &d = b->d;
  const int64_t T = kTagsPerSolve;
  up(d.vol, vol, np, N, co); up(d.ivol, ivol, np, N, co); up(d.per, per, np, N, co); up(d.ih, ih, np, N, co);
  up(d.m2, m2, np, N, co); up(d.op, op, np, N, co); up(d.snx, snx, np, N, co); up(d.sny, sny, np, N, co);
  up(d.shs, shs, np, N, co); up(d.cface, cface, np, N, co); up(d.cnbr, cnbr, np, N, co);
  up(d.csid, csid, np, N, co); up(b->perm, perm, np, N, co); up(d.ccol, ccol, np, N, co);
  up(d.wenok, wenok, np, N, co);
  up(d.fn, fn, nf, F, fo); up(d.fS, fS, nf, F, fo); up(d.fjump, fjump, nf, F, fo); up(d.fxi, fxi, nf, F, fo);
  up(d.fidl, fidl, nf, F, fo);
  up(d.fc0, fc0, nf, F, fo); up(d.fc1, fc1, nf, F, fo); up(d.fsid, fsid, nf, F, fo);
  up(d.mu, mu, 1, 1, s); up(d.bcuw, bc_uw, 2 * T, 0, 2 * T * s); up(d.bcrho, bc_rho, T, 0, T * s);
  up(d.bcu, bc_u, 2 * T, 0, 2 * T * s); up(d.bcp, bc_p, T, 0, T * s); up(d.bckind, bc_kind, T, 0, T * s);
  if (ok && b->mixed) {
    auto f32 = [](const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); };
    std::vector<std::vector<float>> keep;   // alive until the stream syncs
    auto upf = [&](float *dst, const std::vector<double> &src, int64_t len, int64_t stride, int64_t off) {
      keep.push_back(f32(src));
      up(dst, keep.back(), len, stride, off);
    };
    upf(d.f_ivol, ivol, np, N, co); upf(d.f_ih, ih, np, N, co); upf(d.f_m2, m2, np, N, co);
    upf(d.f_op, op, np, N, co); upf(d.f_snx, snx, np, N, co); upf(d.f_sny, sny, np, N, co);
    upf(d.f_shs, shs, np, N, co);
    upf(d.f_fn, fn, nf, F, fo); upf(d.f_fS, fS, nf, F, fo); upf(d.f_fjump, fjump, nf, F, fo);
    upf(d.f_fidl, fidl, nf, F, fo);
    upf(d.f_fxi, fxi, nf, F, fo);
    upf(d.f_mu, mu, 1, 1, s); upf(d.f_bcuw, bc_uw, 2 * T, 0, 2 * T * s); upf(d.f_bcrho, bc_rho, T, 0, T * s);
    upf(d.f_bcu, bc_u, 2 * T, 0, 2 * T * s); upf(d.f_bcp, bc_p, T, 0, T * s);
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
  }
  ok = ok && cudaMemsetAsync(b->status + s, 0, sizeof(int), st) == cudaSuccess &&
       cudaStreamSynchronize(st) == cudaSuccess;   // host tables go out of scope
  if (!ok) return CGKS_ECUDA;
  Member &M = b->mem[s];
  M = m;
  M.cell_off = co; M.n_pad = np; M.face_off = fo; M.active = true;
  return CGKS_OK;
}

// Take solve s out: its cells and faces become inert.
int remove_solve(Batch *b, int s) {
  Member &M = b->mem[s];
  if (!M.active) return CGKS_EINVAL;
  clear_cells(b, M.cell_off, M.cell_off + M.n_pad);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(b->d.fsid + M.face_off, 0xff, sizeof(int) * M.mesh->n_faces, b->stream));
  M.active = false;
  M.mesh.reset();
  return CGKS_OK;
}

// After inserts and removals: launch extents, colour sequence, sweep
// ranges (or cell lists beyond kMaxRanges solves), residual block ranges.
int finalize_batch(Batch *b) {
  int64_t N = 0, F = 0;
  int C = 0;
  std::vector<int> order;   // active slots by cell offset
  for (int s = 0; s < b->S; ++s) {
    const Member &M = b->mem[s];
    if (!M.active) continue;
    order.push_back(s);
    N = std::max(N, M.cell_off + M.n_pad);
    F = std::max(F, M.face_off + M.mesh->n_faces);
    C = std::max(C, M.mesh->n_colours);
  }
  std::sort(order.begin(), order.end(), [&](int x, int y) { return b->mem[x].cell_off < b->mem[y].cell_off; });
  b->N = N; b->F = F; b->n_colours = C;
  // flux class per slot (serving batches): smooth, or limited (full flux +
  // conservative compact WENO); the class constants are batch-wide
  b->n_lim = b->n_smooth = 0;
  if (b->sh.per_slot_flux) {
    for (int s = 0; s < b->S; ++s) {
      const Member &M = b->mem[s];
      b->slim_host[s] = M.active && M.params.flux_hi == CGKS_FLUX_FULL ? 1 : 0;
      if (M.active) (b->slim_host[s] ? b->n_lim : b->n_smooth)++;
    }
    CK(cudaMemcpyAsync(b->slim, b->slim_host.data(), sizeof(int) * b->S, cudaMemcpyHostToDevice, b->stream));
    fill_shared_params(b->sh, b->dp);
    fill_shared_params(b->sh, b->fp);
  }
  std::vector<int> blk(2 * b->S, 0);
  for (int s : order) {
    blk[2 * s] = static_cast<int>(b->mem[s].cell_off / kCellBlock);
    blk[2 * s + 1] = static_cast<int>((b->mem[s].cell_off + b->mem[s].n_pad) / kCellBlock);
  }
  CK(cudaMemcpyAsync(b->blk, blk.data(), sizeof(int) * blk.size(), cudaMemcpyHostToDevice, b->stream));
  // colour sequence of Algorithm 1 with colour classes: n_sweeps x (0..C-1,
  // C-1..0).  A colour repeated back to back recomputes identical values
  // (its cells read only other colours), and the first pass is done by
  // k_lo_rhs, so both are dropped.
  std::vector<int> seq;
  for (int sw = 0; sw < b->sh.n_sweeps; ++sw) {
    for (int c = 0; c < C; ++c) if (seq.empty() || seq.back() != c) seq.push_back(c);
    for (int c = C - 1; c >= 0; --c) if (seq.empty() || seq.back() != c) seq.push_back(c);
  }
  if (!seq.empty()) seq.erase(seq.begin());
  b->sweep_seq = seq;
  for (auto &rs : b->ranges) rs.assign(C, Ranges{});
  b->list_off.assign(C + 1, 0);
  std::vector<int> list;
  bool need_list = false;
  for (int c = 0; c < C; ++c) {
    for (int sh = 0; sh < kNShape; ++sh) {
      Ranges &R = b->ranges[sh][c];
      std::memset(&R, 0, sizeof(R));
      int nr = 0, blocks = 0;
      for (int s : order) {
        const Member &M = b->mem[s];
        const HostMesh &hm = *M.mesh;
        if (c >= hm.n_colours) continue;
        const int beg = static_cast<int>(M.cell_off) + hm.colour_start[c];
        const int end = static_cast<int>(M.cell_off) + hm.colour_start[c + 1];
        if (end == beg) continue;
        if (sh == 0)
          for (int i = beg; i < end; ++i) list.push_back(i);
        if (nr == kMaxRanges) { nr = -1; continue; }
        if (nr < 0) continue;
        R.blk[nr] = blocks;
        R.begin[nr] = beg;
        R.end[nr] = end;
        blocks += nblk(end - beg, sweep_cpb(sh));
        ++nr;
      }
      if (nr >= 0) { R.n = nr; R.blk[nr] = blocks; }
      else { std::memset(&R, 0, sizeof(R)); need_list = true; }
    }
    b->list_off[c + 1] = static_cast<int>(list.size());
  }
  if (need_list && !list.empty())
    CK(cudaMemcpyAsync(b->list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, b->stream));
  // partitioned sweep: each solve's RCM order cut into ceil(n / part_cells)
  // partitions (RCM position k in partition floor(k P / n)); inside a
  // colour's internal range (RCM order) a partition is a contiguous run
  b->n_parts = 0;
  if (b->sh.sweep_order == CGKS_SWEEP_PARTITIONED) {
    if (C > kMaxPartColours) return CGKS_EMESH;
    std::vector<int> tab;
    for (int s : order) {
      const Member &M = b->mem[s];
      const HostMesh &hm = *M.mesh;
      const int64_t n = hm.n_cells;
      const int64_t P = (n + b->sh.part_cells - 1) / b->sh.part_cells;
      std::vector<int64_t> pos(n);
      for (int64_t k = 0; k < n; ++k) pos[hm.rcm[k]] = k;
      const size_t q0 = tab.size() / (2 * C);
      tab.resize(tab.size() + static_cast<size_t>(2 * C * P), 0);
      for (int c = 0; c < C; ++c) {
        const int beg = c < hm.n_colours ? hm.colour_start[c] : 0;
        const int end = c < hm.n_colours ? hm.colour_start[c + 1] : 0;
        // first internal index of each partition in this colour's range
        int cur = beg;
        for (int64_t q = 0; q < P; ++q) {
          int e = cur;
          while (e < end && (pos[hm.perm[e]] * P) / n == q) ++e;
          int *t = &tab[2 * ((q0 + q) * C + c)];
          t[0] = static_cast<int>(M.cell_off) + cur;
          t[1] = static_cast<int>(M.cell_off) + e;
          cur = e;
        }
        if (cur != end) return CGKS_EMESH;   // not monotone in RCM position: never for this layout
      }
    }
    b->n_parts = static_cast<int>(tab.size() / (2 * std::max(C, 1)));
    if (static_cast<int64_t>(tab.size()) > b->ptab_cap) return CGKS_EINVAL;
    if (!tab.empty())
      CK(cudaMemcpyAsync(b->ptab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, b->stream));
    // the colour-launch shapes are not used: nothing to tune for the sweep
    b->tune.unit[TK_SWEEP] = Tuner::kRounds * kNShape;
    b->tune.decided[TK_SWEEP] = true;
  }
  // the fused low-order launch: per-colour ranges of every active solve
  b->lo_fused_ok = false;
  // (the fused launch implements the KFVS low level only)
  if (b->sh.lo_fused && b->sh.flux_lo == CGKS_FLUX_KFVS && !b->sh.lo_viscous && b->lo_grid > 0 && C <= kMaxColFused &&
      b->sweep_seq.size() <= 48 && N > 0) {
    std::vector<int> rstart(kMaxColFused + 1, 0), rbegin, rpre;
    for (int c = 0; c < C; ++c) {
      rstart[c] = static_cast<int>(rbegin.size());
      int acc = 0;
      for (int s : order) {
        const Member &M = b->mem[s];
        const HostMesh &hm = *M.mesh;
        if (c >= hm.n_colours) continue;
        const int beg = static_cast<int>(M.cell_off) + hm.colour_start[c];
        const int cnt = hm.colour_start[c + 1] - hm.colour_start[c];
        if (cnt == 0) continue;
        rbegin.push_back(beg);
        rpre.push_back(acc);
        acc += cnt;
      }
      rpre.push_back(acc);
    }
    for (int c = C; c <= kMaxColFused; ++c) rstart[c] = static_cast<int>(rbegin.size());
    if (rbegin.empty()) rbegin.push_back(0);
    CK(cudaMemcpyAsync(b->r_start, rstart.data(), sizeof(int) * rstart.size(), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->r_begin, rbegin.data(), sizeof(int) * rbegin.size(), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->r_pre, rpre.data(), sizeof(int) * rpre.size(), cudaMemcpyHostToDevice, b->stream));
    b->lo_fused_ok = true;
  }
  CK(cudaStreamSynchronize(b->stream));
  drop_graphs(b);
  return CGKS_OK;
}

// A batch holding exactly the given solves, packed from offset 0.
int build_batch(const Shared &sh, std::vector<Member> mem, cudaStream_t st, Batch **out) {
  *out = nullptr;
  if (mem.empty()) return CGKS_EINVAL;
  int64_t N = 0, F = 0;
  for (auto &m : mem) { N += pad_cells(m.mesh->n_cells); F += m.mesh->n_faces; }
  Batch *b = nullptr;
  int rc = create_batch(sh, N, std::max<int64_t>(F, 1), static_cast<int>(mem.size()), st, &b);
  if (rc) return rc;
  int64_t co = 0, fo = 0;
  for (size_t s = 0; s < mem.size() && !rc; ++s) {
    rc = insert_solve(b, static_cast<int>(s), mem[s], co, fo);
    co += pad_cells(mem[s].mesh->n_cells);
    fo += mem[s].mesh->n_faces;
  }
  if (!rc) rc = finalize_batch(b);
  if (rc) { destroy_batch(b); return rc; }
  *out = b;
  return CGKS_OK;
}

// state of member s from caller-order AoS (host or device staging)
int load_state(Batch *b, int s, const double *W, const double *Wx, bool device) {
  const Member &M = b->mem[s];
  const int64_t n = M.mesh->n_cells;
  double *wa = b->stage, *wxa = b->stage + 4 * n;
  cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(wa, W, sizeof(double) * 4 * n, kind, b->stream));
  if (Wx) CK(cudaMemcpyAsync(wxa, Wx, sizeof(double) * 8 * n, kind, b->stream));
  k_gather_state<<<nblk(n, kCellBlock), kCellBlock, 0, b->stream>>>(
      static_cast<int>(n), static_cast<int>(M.cell_off), static_cast<int>(b->Ncap), b->perm + M.cell_off, wa,
      Wx ? wxa : nullptr, b->W, b->Wx, b->mixed ? b->bf.W : nullptr, b->mixed ? b->bf.Wx : nullptr);
  b->launches++;
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(b->status + s, 0, sizeof(int), b->stream));
  return CGKS_OK;
}

int store_state(Batch *b, int s, double *W, double *Wx, bool device) {
  const Member &M = b->mem[s];
  const int64_t n = M.mesh->n_cells;
  double *wa = b->stage, *wxa = b->stage + 4 * n;
  k_scatter_state<<<nblk(n, kCellBlock), kCellBlock, 0, b->stream>>>(
      static_cast<int>(n), static_cast<int>(M.cell_off), static_cast<int>(b->Ncap), b->perm + M.cell_off, b->W, b->Wx, wa,
      wxa);
  b->launches++;
  CK(cudaGetLastError());
  cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (W) CK(cudaMemcpyAsync(W, wa, sizeof(double) * 4 * n, kind, b->stream));
  if (Wx) CK(cudaMemcpyAsync(Wx, wxa, sizeof(double) * 8 * n, kind, b->stream));
  if (!device) CK(cudaStreamSynchronize(b->stream));
  return CGKS_OK;
}

Shared shared_from(const cgks_params *p) {
  Shared sh;
  sh.gamma = p->gamma; sh.cfl_hi = p->cfl_hi; sh.cfl_lo = p->cfl_lo;
  sh.n_implicit = p->n_implicit; sh.n_sweeps = p->n_sweeps; sh.time_scheme = p->time_scheme;
  sh.precision = p->precision; sh.use_graph = p->use_graph; sh.lo_fused = p->low_order_fused;
  sh.autotune = p->autotune;
  sh.pdl = p->programmatic_launch;
  sh.flux_lo = p->flux_lo;
  sh.flux_hi = p->flux_hi;
  sh.tau_c1 = p->tau_c1; sh.tau_c2 = p->tau_c2; sh.weno_eps = p->weno_eps; sh.weno_g0 = p->weno_g0;
  sh.weno_vars = p->weno_vars;
  sh.sweep_order = p->sweep_order;
  sh.lo_viscous = p->lo_viscous;
  sh.part_cells = p->sweep_part_cells > 0 ? p->sweep_part_cells : 2048;
  sh.alloc = p->alloc; sh.free = p->free; sh.alloc_ctx = p->alloc_ctx;
  return sh;
}

int validate_params_tags(const cgks_params *p, const std::vector<int32_t> &tags_used) {
  if (!(p->gamma > 1.0) || p->mu < 0.0 || !(p->cfl_hi > 0.0) || !(p->cfl_lo > 0.0) || p->n_implicit < 0 ||
      p->n_sweeps < 0 || (p->time_scheme != CGKS_S1O2 && p->time_scheme != CGKS_S2O4) || p->n_bc < 0 ||
      p->n_bc > CGKS_MAX_BC || (p->precision != CGKS_FP64 && p->precision != CGKS_MIXED) || !(p->alpha >= 0.0) ||
      (p->flux_lo != CGKS_FLUX_KFVS && p->flux_lo != CGKS_FLUX_LF) ||
      (p->flux_hi != CGKS_FLUX_SMOOTH && p->flux_hi != CGKS_FLUX_FULL) || !(p->tau_c1 >= 0.0) ||
      !(p->tau_c2 >= 0.0) || !(p->weno_eps >= 0.0) || (p->weno_eps > 0.0 && !(p->weno_g0 > 0.0 && p->weno_g0 < 1.0)) ||
      (p->weno_vars != CGKS_WENO_CONSERVATIVE && p->weno_vars != CGKS_WENO_CHARACTERISTIC) ||
      (p->sweep_order != CGKS_SWEEP_COLOUR && p->sweep_order != CGKS_SWEEP_PARTITIONED) ||
      (p->sweep_order == CGKS_SWEEP_PARTITIONED && p->low_order_fused) ||
      (p->sweep_part_cells != 0 && p->sweep_part_cells < 64) || (p->lo_viscous != 0 && p->lo_viscous != 1))
    return CGKS_EINVAL;
  for (int t : tags_used)
    if (t >= p->n_bc) return CGKS_EINVAL;
  for (int b = 0; b < p->n_bc; ++b) {
    int k = p->bc[b].kind;
    if (k != CGKS_BC_SLIP && k != CGKS_BC_NOSLIP && k != CGKS_BC_FARFIELD && k != CGKS_BC_DIRICHLET &&
        k != CGKS_BC_OUTFLOW)
      return CGKS_EINVAL;
    if ((k == CGKS_BC_FARFIELD || k == CGKS_BC_DIRICHLET) && !(p->bc[b].rho > 0.0 && p->bc[b].p > 0.0))
      return CGKS_EINVAL;
  }
  return CGKS_OK;
}

int validate_params(const cgks_params *p, const HostMesh &hm) { return validate_params_tags(p, hm.bface_tags_used); }

}  // namespace

// ------------------------------------------------------------------------
struct cgks_solver {
  Batch *b = nullptr;
  Solver3 *s3 = nullptr;       // 3-D meshes
  cgks_params params{};
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_user = nullptr, ev_done = nullptr;
  int device = 0;
  Timer timer;
  int status_cache = 0;
};

// First-fit allocator of ranges [0, cap) in units of `align`.
struct RangeAlloc {
  std::map<int64_t, int64_t> free_;   // offset -> length
  void reset(int64_t cap) { free_.clear(); if (cap > 0) free_[0] = cap; }
  int64_t alloc(int64_t len) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < len) continue;
      const int64_t off = it->first, rest = it->second - len;
      free_.erase(it);
      if (rest > 0) free_[off + len] = rest;
      return off;
    }
    return -1;
  }
  void release(int64_t off, int64_t len) {
    if (len <= 0) return;
    auto it = free_.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && off + len == nx->first) { it->second += nx->second; free_.erase(nx); }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
    }
  }
};

struct cgks_server {
  struct Req {
    int64_t id;
    std::shared_ptr<const HostMesh> mesh;
    cgks_params params;
    std::vector<double> W0;
    double drop;
    int max_cycles;
    cgks_req_status st;
    std::vector<double> result;      // final state, caller order
    size_t footprint;
  };
  Shared sh;
  int max_active = 64, max_cycles = 20000;
  size_t budget = 0, used = 0;
  int64_t Ncap = 0, Fcap = 0;      // batch capacity the budget allows
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_user = nullptr, ev_done = nullptr;
  int device = 0;
  int64_t next_id = 1;
  std::map<int64_t, std::unique_ptr<Req>> reqs;
  std::deque<int64_t> queue;
  std::vector<int64_t> slot_req;   // request in each slot of the batch, -1 free
  bool lim_set = false;            // the limited class's constants are fixed (sh)
  RangeAlloc cells, faces;
  Batch *b = nullptr;              // created at the first admission
  std::chrono::steady_clock::time_point t0;
  std::vector<double> res_host;
  std::vector<int> status_host;
};

namespace {

int begin_call(cudaStream_t user, cudaStream_t own, cudaEvent_t ev, int device) {
  CK(cudaSetDevice(device));
  CK(cudaEventRecord(ev, user));
  CK(cudaStreamWaitEvent(own, ev, 0));
  return CGKS_OK;
}
int end_call(cudaStream_t user, cudaStream_t own, cudaEvent_t ev) {
  CK(cudaEventRecord(ev, own));
  CK(cudaStreamWaitEvent(user, ev, 0));
  return CGKS_OK;
}
int begin_call(cgks_solver *s) { return begin_call(s->user_stream, s->stream, s->ev_user, s->device); }
int end_call(cgks_solver *s) { return end_call(s->user_stream, s->stream, s->ev_done); }

int solver_status(cgks_solver *s) {
  int st = 0;
  if (s->s3) {
    int rc = s3_status(s->s3, &st);
    if (rc) return rc;
  } else {
    CK(cudaMemcpyAsync(&st, s->b->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  s->status_cache = st;
  if (st & kBarrierTimeout) return CGKS_ETIMEOUT;
  return st ? CGKS_EDIVERGED : CGKS_OK;
}

double now_s(const cgks_server *v) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - v->t0).count();
}

}  // namespace

// =============================== C ABI ===================================
// Momentum flux through the boundary faces of one tag at the current state
// (post-processing; see include/cgks.h).
template <typename TF>
int wall_loads_t(cgks_solver *s, int32_t tag, int64_t max_faces, int64_t *n_faces, double *x, double *nrm,
                 double *S, double *traction) {
  Batch *b = s->b;
  const HostMesh &hm = *b->mem[0].mesh;
  Bufs<TF> &B = bufs<TF>(b);
  if (b->sh.flux_hi == CGKS_FLUX_FULL) enqueue_dt(b, -1.0);   // the full flux integrates over a step
  enqueue_hi_eval<TF>(b, B.W, B.Wx, B.FA);
  const int64_t F = b->F, nf = hm.n_faces, off = b->mem[0].face_off;
  std::vector<TF> F0(4 * static_cast<size_t>(F));
  for (int v = 0; v < 4; ++v)
    CK(cudaMemcpyAsync(F0.data() + v * F, B.FA + v * F, sizeof(TF) * F, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  int64_t k = 0;
  for (int64_t f = 0; f < nf; ++f) {
    if (hm.fc1[f] != -1 - tag) continue;
    if (k < max_faces) {
      const int c0 = hm.fc0[f];
      const double h = hm.h[c0];
      // face midpoint: the mean of its two Gauss points (offsets from c0 scaled by 1/h)
      x[2 * k] = hm.xc[c0] + 0.5 * h * (hm.fxi[0 * nf + f] + hm.fxi[2 * nf + f]);
      x[2 * k + 1] = hm.xc[hm.n_cells + c0] + 0.5 * h * (hm.fxi[1 * nf + f] + hm.fxi[3 * nf + f]);
      nrm[2 * k] = hm.fn[f];
      nrm[2 * k + 1] = hm.fn[nf + f];
      S[k] = hm.fS[f];
      traction[2 * k] = static_cast<double>(F0[1 * F + off + f]);
      traction[2 * k + 1] = static_cast<double>(F0[2 * F + off + f]);
    }
    ++k;
  }
  *n_faces = k;
  return k <= max_faces ? CGKS_OK : CGKS_EINVAL;
}

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
  p->low_order_fused = 0;
  p->autotune = 1;
  p->programmatic_launch = 1;
  p->flux_hi = CGKS_FLUX_SMOOTH;
  p->tau_c1 = 0.01;
  p->tau_c2 = 1.0;
  p->weno_eps = 0.0;
  p->weno_g0 = 0.95;
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
  if (dim != 2 && dim != 3) return CGKS_EINVAL;
  cgks_mesh *m = new (std::nothrow) cgks_mesh();
  if (!m) return CGKS_ENOMEM;
  m->dim = dim;
  int rc;
  try {
    if (dim == 2)
      rc = build_host_mesh(n_nodes, xyz, n_cells, cell_type, cell_ptr, cell_nodes, n_bfaces, bface_ptr, bface_nodes,
                           bface_tag, m->h);
    else
      rc = build_host_mesh3(n_nodes, xyz, n_cells, cell_type, cell_ptr, cell_nodes, n_bfaces, bface_ptr,
                            bface_nodes, bface_tag, m->h3);
  } catch (const std::bad_alloc &) {
    rc = CGKS_ENOMEM;
  }
  if (rc != CGKS_OK) { delete m; return rc; }
  *out = m;
  return CGKS_OK;
}

int cgks_mesh_info(const cgks_mesh *m, cgks_mesh_info_t *out) {
  if (!m || !out) return CGKS_EINVAL;
  if (m->dim == 3) {
    out->n_cells = m->h3.n_cells;
    out->n_faces = m->h3.n_faces;
    out->n_bfaces = m->h3.n_bfaces;
    out->n_colours = m->h3.n_colours;
    out->dim = 3;
    out->device_bytes = static_cast<int64_t>(s3_footprint(m->h3.n_cells, m->h3.n_faces, false));
    return CGKS_OK;
  }
  out->n_cells = m->h.n_cells;
  out->n_faces = m->h.n_faces;
  out->n_bfaces = m->h.n_bfaces;
  out->n_colours = m->h.n_colours;
  out->dim = m->h.dim;
  out->device_bytes = static_cast<int64_t>(solve_footprint(m->h.n_cells, m->h.n_faces, false));
  return CGKS_OK;
}

int cgks_mesh_ordering(const cgks_mesh *m, int64_t *rcm, int32_t *colour) {
  if (!m) return CGKS_EINVAL;
  const std::vector<int64_t> &r = m->dim == 3 ? m->h3.rcm : m->h.rcm;
  const std::vector<int32_t> &c = m->dim == 3 ? m->h3.colour : m->h.colour;
  if (rcm) std::copy(r.begin(), r.end(), rcm);
  if (colour) std::copy(c.begin(), c.end(), colour);
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
  collect_timing(&s->timer);
  destroy_batch(s->b);
  s3_destroy(s->s3);
  if (s->ev_user) cudaEventDestroy(s->ev_user);
  if (s->ev_done) cudaEventDestroy(s->ev_done);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return CGKS_OK;
}

int cgks_solver_create(const cgks_mesh *m, const cgks_params *p, cgks_solver **out) {
  if (!m || !p || !out) return CGKS_EINVAL;
  *out = nullptr;
  int rc = validate_params_tags(p, m->dim == 3 ? m->h3.bface_tags_used : m->h.bface_tags_used);
  if (rc) return rc;
  if (m->dim == 3) {
    // the 3-D path has walls and far field, and WENO on conservative variables
    if (p->weno_eps > 0.0 && p->weno_vars != CGKS_WENO_CONSERVATIVE) return CGKS_EINVAL;
    if (p->sweep_order != CGKS_SWEEP_COLOUR) return CGKS_EINVAL;   // the partitioned sweep is 2-D
    for (int b = 0; b < p->n_bc; ++b)
      if (p->bc[b].kind != CGKS_BC_SLIP && p->bc[b].kind != CGKS_BC_NOSLIP && p->bc[b].kind != CGKS_BC_FARFIELD)
        return CGKS_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return CGKS_ECUDA;
  cgks_solver *s = new (std::nothrow) cgks_solver();
  if (!s) return CGKS_ENOMEM;
  s->params = *p;
  cudaGetDevice(&s->device);
  s->user_stream = static_cast<cudaStream_t>(p->stream);
  auto fail = [&](int r) { cgks_solver_destroy(s); return r; };
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(CGKS_ECUDA);
  if (cudaEventCreateWithFlags(&s->ev_user, cudaEventDisableTiming) != cudaSuccess) return fail(CGKS_ECUDA);
  if (cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming) != cudaSuccess) return fail(CGKS_ECUDA);
  if (m->dim == 3) {
    try {
      rc = s3_create(m->h3, p, s->stream, &s->timer, &s->s3);
    } catch (const std::bad_alloc &) {
      rc = CGKS_ENOMEM;
    }
    if (rc) return fail(rc);
    *out = s;
    return CGKS_OK;
  }
  std::vector<Member> mem(1);
  try {
    mem[0].mesh = std::make_shared<HostMesh>(m->h);
  } catch (const std::bad_alloc &) {
    return fail(CGKS_ENOMEM);
  }
  mem[0].params = *p;
  rc = build_batch(shared_from(p), std::move(mem), s->stream, &s->b);
  if (rc) return fail(rc);
  s->b->timer = &s->timer;
  *out = s;
  return CGKS_OK;
}

static int set_state_impl(cgks_solver *s, const double *W, const double *Wx, bool device) {
  if (!s || !W) return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  rc = s->s3 ? s3_set_state(s->s3, W, Wx, device) : load_state(s->b, 0, W, Wx, device);
  if (rc) return rc;
  s->status_cache = 0;
  return end_call(s);
}

int cgks_set_state(cgks_solver *s, const double *W, const double *Wx) { return set_state_impl(s, W, Wx, false); }
int cgks_set_state_device(cgks_solver *s, const double *W, const double *Wx) { return set_state_impl(s, W, Wx, true); }

static int get_state_impl(cgks_solver *s, double *W, double *Wx, bool device) {
  if (!s) return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  rc = s->s3 ? s3_get_state(s->s3, W, Wx, device) : store_state(s->b, 0, W, Wx, device);
  if (rc) return rc;
  return end_call(s);
}

int cgks_get_state(cgks_solver *s, double *W, double *Wx) { return get_state_impl(s, W, Wx, false); }
int cgks_get_state_device(cgks_solver *s, double *W, double *Wx) { return get_state_impl(s, W, Wx, true); }

int cgks_highorder_step(cgks_solver *s, double dt, double *dt_used) {
  if (!s) return CGKS_EINVAL;
  if (s->status_cache) return CGKS_EDIVERGED;
  int rc = begin_call(s);
  if (rc) return rc;
  if (s->s3) {
    int st = 0;
    rc = s3_highorder_step(s->s3, dt, dt_used, &st);
    if (rc) return rc;
    collect_timing(&s->timer);
    s->status_cache = st;
    rc = end_call(s);
    if (rc) return rc;
    return st ? CGKS_EDIVERGED : CGKS_OK;
  }
  Batch *b = s->b;
  CK(cudaMemsetAsync(&b->ctl->res_ctr, 0, sizeof(int), s->stream));
  enqueue_explicit_step(b, dt);
  CK(cudaGetLastError());
  Ctl c;
  unsigned long long bits = 0;
  int st = 0;
  CK(cudaMemcpyAsync(&c, b->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(&bits, b->dt_bits, sizeof(bits), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  collect_timing(&s->timer);
  if (dt_used) *dt_used = c.dt_fixed > 0.0 ? c.dt_fixed : s->params.cfl_hi * __builtin_bit_cast(double, bits);
  s->status_cache = st;
  rc = end_call(s);
  if (rc) return rc;
  return st ? CGKS_EDIVERGED : CGKS_OK;
}

static int solver_run(cgks_solver *s, int n, double *res_hist, bool cycle) {
  if (!s || n < 0) return CGKS_EINVAL;
  if (s->status_cache) return CGKS_EDIVERGED;
  if (n == 0) return CGKS_OK;
  if (s->s3) {
    int rc = begin_call(s);
    if (rc) return rc;
    rc = s3_run(s->s3, n, cycle);
    if (rc) return rc;
    if (res_hist) { rc = s3_history(s->s3, res_hist, n); if (rc) return rc; }
    rc = solver_status(s);
    collect_timing(&s->timer);
    int rc2 = end_call(s);
    return rc ? rc : rc2;
  }
  Batch *b = s->b;
  int rc = ensure_hist(b, n);
  if (rc) return rc;
  rc = begin_call(s);
  if (rc) return rc;
  rc = run_many(b, n, cycle);
  if (rc) return rc;
  if (res_hist) CK(cudaMemcpyAsync(res_hist, b->hist, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  rc = solver_status(s);
  collect_timing(&s->timer);
  int rc2 = end_call(s);
  return rc ? rc : rc2;
}

int cgks_explicit_steps(cgks_solver *s, int n, double *res_hist) { return solver_run(s, n, res_hist, false); }
int cgks_pmg_cycle(cgks_solver *s, int n_cycles, double *res_hist) { return solver_run(s, n_cycles, res_hist, true); }

int cgks_loworder_smooth(cgks_solver *s) {
  if (!s) return CGKS_EINVAL;
  if (s->status_cache) return CGKS_EDIVERGED;
  int rc = begin_call(s);
  if (rc) return rc;
  if (s->s3) {
    rc = s3_loworder_smooth(s->s3);
    if (rc) return rc;
  } else {
    CK(cudaMemsetAsync(&s->b->ctl->res_ctr, 0, sizeof(int), s->stream));
    enqueue_lo_smooth(s->b);
    CK(cudaGetLastError());
  }
  rc = solver_status(s);
  collect_timing(&s->timer);
  int rc2 = end_call(s);
  return rc ? rc : rc2;
}

int cgks_residual(cgks_solver *s, double *res, double *r_l2) {
  if (!s) return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  if (s->s3) {
    rc = s3_residual(s->s3, res, r_l2);
    if (rc) return rc;
    return end_call(s);
  }
  Batch *b = s->b;
  double last[3];
  CK(cudaMemcpyAsync(last, b->last, sizeof(double) * 3, cudaMemcpyDeviceToHost, s->stream));
  std::vector<double> R;
  if (r_l2) {
    R.resize(4 * static_cast<size_t>(b->Ncap));
    CK(cudaMemcpyAsync(R.data(), b->Rp0, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  if (res) *res = last[0];
  if (r_l2) {
    const int64_t n = b->mem[0].mesh->n_cells, N = b->Ncap;
    for (int v = 0; v < 4; ++v) {
      double a = 0.0;
      for (int64_t i = 0; i < n; ++i) a += R[v * N + i] * R[v * N + i];
      r_l2[v] = std::sqrt(a);
    }
  }
  return end_call(s);
}

int cgks_wall_loads(cgks_solver *s, int32_t tag, int64_t max_faces, int64_t *n_faces, double *x, double *nrm,
                    double *S, double *traction) {
  if (!s || !n_faces || tag < 0 || tag >= CGKS_MAX_BC || max_faces < 0 ||
      (max_faces > 0 && (!x || !nrm || !S || !traction)))
    return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  if (s->s3) rc = s3_wall_loads(s->s3, tag, max_faces, n_faces, x, nrm, S, traction);
  else if (s->b->mixed) rc = wall_loads_t<float>(s, tag, max_faces, n_faces, x, nrm, S, traction);
  else rc = wall_loads_t<double>(s, tag, max_faces, n_faces, x, nrm, S, traction);
  const int rc2 = end_call(s);
  return rc ? rc : rc2;
}

int cgks_get_rp0(cgks_solver *s, double *Rp0) {
  if (!s || !Rp0) return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  if (s->s3) {
    rc = s3_get_rp0(s->s3, Rp0);
    if (rc) return rc;
    return end_call(s);
  }
  Batch *b = s->b;
  const int64_t N = b->Ncap, n = b->mem[0].mesh->n_cells;
  std::vector<double> R(4 * static_cast<size_t>(N));
  CK(cudaMemcpyAsync(R.data(), b->Rp0, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  const HostMesh &hm = *b->mem[0].mesh;
  for (int64_t i = 0; i < n; ++i) {
    int c = hm.perm[i];
    for (int v = 0; v < 4; ++v) Rp0[4 * c + v] = R[v * N + i];
  }
  return end_call(s);
}

// ---- instrumentation (not in the paper): per-kernel CUDA-event timers and
// the count of kernels this solver has launched ----
int cgks_set_timing(cgks_solver *s, int on) {
  if (!s) return CGKS_EINVAL;
  cudaStreamSynchronize(s->stream);
  collect_timing(&s->timer);
  s->timer.on = on != 0;
  return CGKS_OK;
}

int cgks_get_timing(cgks_solver *s, int max, const char **names, double *total_ms, int64_t *count) {
  if (!s) return CGKS_EINVAL;
  cudaStreamSynchronize(s->stream);
  collect_timing(&s->timer);
  int k = 0;
  for (; k < KI_COUNT && k < max; ++k) {
    if (names) names[k] = kernel_name(k);
    if (total_ms) total_ms[k] = s->timer.ms[k];
    if (count) count[k] = s->timer.cnt[k];
  }
  return k;
}

int cgks_reset_timing(cgks_solver *s) {
  if (!s) return CGKS_EINVAL;
  cudaStreamSynchronize(s->stream);
  collect_timing(&s->timer);
  for (int k = 0; k < KI_COUNT; ++k) { s->timer.ms[k] = 0.0; s->timer.cnt[k] = 0; }
  return CGKS_OK;
}

int64_t cgks_launch_count(const cgks_solver *s) {
  if (!s) return -1;
  return s->s3 ? s3_launches(s->s3) : s->b->launches;
}

int cgks_launches_per_call(const cgks_solver *s, int cycle) {
  if (!s) return -1;
  return s->s3 ? s3_launches_per_call(s->s3, cycle != 0) : static_cast<int>(count_launches(s->b, cycle != 0));
}

int cgks_tune_shape(int32_t shape, int32_t *block, int32_t *per_thread, int32_t *min_blocks) {
  if (shape < 0 || shape >= kNShape) return CGKS_EINVAL;
  if (block) *block = shape_bs(shape);
  if (per_thread) *per_thread = shape_ipt(shape);
  if (min_blocks) *min_blocks = shape_minb(shape);
  return CGKS_OK;
}

int cgks_get_tuning(cgks_solver *s, cgks_tuning *t) {
  if (!s || !t) return CGKS_EINVAL;
  if (s->s3) return s3_tuner(s->s3)->report(t), CGKS_OK;
  s->b->tune.report(t);
  return CGKS_OK;
}

int cgks_set_barrier_spin_limit(cgks_solver *s, int64_t polls) {
  if (!s || polls < 0 || s->s3) return CGKS_EINVAL;
  s->b->sh.spin_limit = polls;
  drop_graphs(s->b);   // the limit is a launch argument baked into captured graphs
  return CGKS_OK;
}

int cgks_set_tuning(cgks_solver *s, const int32_t shape[CGKS_TUNE_KERNELS]) {
  if (!s || !shape) return CGKS_EINVAL;
  int shp[TK_COUNT];
  for (int k = 0; k < TK_COUNT; ++k) {
    if (shape[k] < 0 || shape[k] >= kNShape) return CGKS_EINVAL;
    shp[k] = shape[k];
  }
  if (s->s3) return s3_set_tuning(s->s3, shp);
  s->b->tune.set(shp);
  drop_graphs(s->b);
  return CGKS_OK;
}

// ================================ serving ================================
void cgks_server_default_opts(cgks_server_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = CGKS_FP64;
  o->time_scheme = CGKS_S1O2;
  o->cfl_hi = 0.4;
  o->cfl_lo = 1000.0;
  o->n_implicit = 6;
  o->n_sweeps = 2;
  o->max_active = 64;
  o->max_cycles = 20000;
  o->use_graph = 1;
  o->low_order_fused = 0;
  o->autotune = 1;
  o->programmatic_launch = 1;
}

// Faces per cell the batch capacity provides for (2-D: triangles 1.5,
// quads 2, plus boundary faces of small meshes).
constexpr double kFacesPerCell = 2.5;

int cgks_server_create(size_t hbm_budget, const cgks_server_opts *o, cgks_server **out) {
  if (!o || !out || hbm_budget == 0 || o->max_active < 1 || o->max_cycles < 1 || !(o->cfl_hi > 0.0) ||
      !(o->cfl_lo > 0.0) || o->n_implicit < 0 || o->n_sweeps < 0 ||
      (o->precision != CGKS_FP64 && o->precision != CGKS_MIXED) ||
      (o->time_scheme != CGKS_S1O2 && o->time_scheme != CGKS_S2O4) ||
      (o->flux_lo != CGKS_FLUX_KFVS && o->flux_lo != CGKS_FLUX_LF) || (o->lo_viscous != 0 && o->lo_viscous != 1))
    return CGKS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return CGKS_ECUDA;
  cgks_server *v = new (std::nothrow) cgks_server();
  if (!v) return CGKS_ENOMEM;
  v->sh.cfl_hi = o->cfl_hi; v->sh.cfl_lo = o->cfl_lo; v->sh.n_implicit = o->n_implicit; v->sh.n_sweeps = o->n_sweeps;
  v->sh.time_scheme = o->time_scheme; v->sh.precision = o->precision; v->sh.use_graph = o->use_graph;
  v->sh.lo_fused = o->low_order_fused;
  v->sh.autotune = o->autotune;
  v->sh.pdl = o->programmatic_launch;
  v->sh.flux_lo = o->flux_lo;
  v->sh.lo_viscous = o->lo_viscous;
  v->sh.per_slot_flux = true;
  v->sh.weno_vars = CGKS_WENO_CONSERVATIVE;
  v->sh.alloc = o->alloc; v->sh.free = o->free; v->sh.alloc_ctx = o->alloc_ctx;
  v->max_active = o->max_active;
  v->max_cycles = o->max_cycles;
  v->budget = hbm_budget;
  v->slot_req.assign(o->max_active, -1);
  // capacity: the arena of Ncap cells and kFacesPerCell * Ncap faces within the budget
  {
    const bool mixed = o->precision == CGKS_MIXED;
    const int64_t U = 1 << 20;
    auto total = [&](int64_t N, int64_t F) {
      Batch tmp;
      std::vector<Piece> pc;
      plan_arena(&tmp, N, F, o->max_active, N, mixed, pc);
      return static_cast<double>(arena_total(pc));
    };
    const double c0 = total(kCellBlock, 1);
    const double cc = (total(kCellBlock + U, 1) - c0) / U, cf = (total(kCellBlock, 1 + U) - c0) / U;
    const double room = static_cast<double>(hbm_budget) - c0 - sizeof(double) * kHistDefault - 64.0 * 256;
    int64_t N = room > 0 ? static_cast<int64_t>(room / (cc + kFacesPerCell * cf)) : 0;
    N = std::min<int64_t>(N, (INT32_MAX / (kNCol * kNM)) & ~int64_t(kCellBlock - 1));
    N = N / kCellBlock * kCellBlock;
    v->Ncap = N;
    v->Fcap = static_cast<int64_t>(kFacesPerCell * N);
    v->cells.reset(v->Ncap);
    v->faces.reset(v->Fcap);
  }
  v->user_stream = static_cast<cudaStream_t>(o->stream);
  cudaGetDevice(&v->device);
  v->t0 = std::chrono::steady_clock::now();
  if (cudaStreamCreateWithFlags(&v->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&v->ev_user, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&v->ev_done, cudaEventDisableTiming) != cudaSuccess) {
    cgks_server_destroy(v);
    return CGKS_ECUDA;
  }
  *out = v;
  return CGKS_OK;
}

int cgks_server_destroy(cgks_server *v) {
  if (!v) return CGKS_OK;
  cudaSetDevice(v->device);
  destroy_batch(v->b);
  if (v->ev_user) cudaEventDestroy(v->ev_user);
  if (v->ev_done) cudaEventDestroy(v->ev_done);
  if (v->stream) cudaStreamDestroy(v->stream);
  delete v;
  return CGKS_OK;
}

int cgks_server_submit(cgks_server *v, const cgks_mesh *m, const cgks_params *p, const double *W0, double res_drop,
                       int32_t max_cycles, int64_t *req_id) {
  if (!v || !m || !p || !W0 || !(res_drop > 0.0)) return CGKS_EINVAL;
  if (m->dim != 2) return CGKS_EINVAL;   // the serving path batches 2-D solves
  cgks_params q = *p;   // batch-wide fields come from the server
  q.cfl_hi = v->sh.cfl_hi; q.cfl_lo = v->sh.cfl_lo; q.n_implicit = v->sh.n_implicit; q.n_sweeps = v->sh.n_sweeps;
  q.time_scheme = v->sh.time_scheme; q.precision = v->sh.precision;
  q.lo_viscous = v->sh.lo_viscous; q.flux_lo = v->sh.flux_lo;
  int rc = validate_params(&q, m->h);
  if (rc) return rc;
  // two flux classes per batch: smooth flux with linear weights, or the
  // limited one (full flux with conservative compact WENO) whose constants
  // every limited request of the server shares
  const bool smooth = q.flux_hi == CGKS_FLUX_SMOOTH && q.weno_eps == 0.0;
  const bool limited = q.flux_hi == CGKS_FLUX_FULL && q.weno_eps > 0.0 && q.weno_vars == CGKS_WENO_CONSERVATIVE;
  if (!smooth && !limited) return CGKS_EINVAL;
  if (limited) {
    if (!v->lim_set) {
      v->sh.tau_c1 = q.tau_c1; v->sh.tau_c2 = q.tau_c2; v->sh.weno_eps = q.weno_eps; v->sh.weno_g0 = q.weno_g0;
      v->lim_set = true;
    } else if (q.tau_c1 != v->sh.tau_c1 || q.tau_c2 != v->sh.tau_c2 || q.weno_eps != v->sh.weno_eps ||
               q.weno_g0 != v->sh.weno_g0) {
      return CGKS_EINVAL;
    }
  }
  if (std::fabs(q.gamma - v->sh.gamma) > 1e-15) {
    if (v->reqs.empty()) v->sh.gamma = q.gamma;
    else return CGKS_EINVAL;   // every solve of a server shares gamma
  }
  std::unique_ptr<cgks_server::Req> r(new (std::nothrow) cgks_server::Req());
  if (!r) return CGKS_ENOMEM;
  try {
    r->mesh = std::make_shared<HostMesh>(m->h);
    r->W0.assign(W0, W0 + 4 * m->h.n_cells);
  } catch (const std::bad_alloc &) {
    return CGKS_ENOMEM;
  }
  r->id = v->next_id++;
  r->params = q;
  r->drop = res_drop;
  r->max_cycles = max_cycles > 0 ? std::min(max_cycles, v->max_cycles) : v->max_cycles;
  std::memset(&r->st, 0, sizeof(r->st));
  r->st.n_cells = m->h.n_cells;
  r->st.t_submit = now_s(v);
  r->footprint = solve_footprint(m->h.n_cells, m->h.n_faces, v->sh.precision == CGKS_MIXED);
  const int64_t id = r->id;
  if (req_id) *req_id = id;
  if (r->footprint > v->budget || pad_cells(m->h.n_cells) > v->Ncap || m->h.n_faces > v->Fcap) {
    r->st.state = CGKS_REQ_REJECTED;
    r->st.t_done = r->st.t_submit;
    v->reqs[id] = std::move(r);
    return CGKS_EBUDGET;
  }
  r->st.state = CGKS_REQ_QUEUED;
  v->reqs[id] = std::move(r);
  v->queue.push_back(id);
  return CGKS_OK;
}

// Retire finished solves, admit queued ones into free slots and free cell /
// face space, and refresh the batch's launch plan when the set changed.
static int server_update(cgks_server *v, double t, bool *changed) {
  *changed = false;
  Batch *b = v->b;
  for (int s = 0; s < v->max_active; ++s) {
    const int64_t id = v->slot_req[s];
    if (id < 0) continue;
    cgks_server::Req &r = *v->reqs[id];
    if (r.st.state == CGKS_REQ_ACTIVE) continue;
    const Member &M = b->mem[s];
    const int64_t co = M.cell_off, np = M.n_pad, fo = M.face_off, nf = M.mesh->n_faces;
    int rc = remove_solve(b, s);
    if (rc) return rc;
    v->cells.release(co, np);
    v->faces.release(fo, nf);
    v->used -= r.footprint;
    v->slot_req[s] = -1;
    *changed = true;
  }
  while (!v->queue.empty()) {
    cgks_server::Req &r = *v->reqs[v->queue.front()];
    int s = 0;
    while (s < v->max_active && v->slot_req[s] >= 0) ++s;
    if (s == v->max_active || v->used + r.footprint > v->budget) break;
    const int64_t np = pad_cells(r.mesh->n_cells), nf = r.mesh->n_faces;
    const int64_t co = v->cells.alloc(np);
    if (co < 0) break;
    const int64_t fo = v->faces.alloc(nf);
    if (fo < 0) { v->cells.release(co, np); break; }
    if (!v->b) {
      int rc = create_batch(v->sh, v->Ncap, v->Fcap, v->max_active, v->stream, &v->b);
      if (rc) { v->cells.release(co, np); v->faces.release(fo, nf); return rc; }
      b = v->b;
    }
    Member m;
    m.mesh = r.mesh;
    m.params = r.params;
    int rc = insert_solve(b, s, m, co, fo);
    if (!rc) rc = load_state(b, s, r.W0.data(), nullptr, false);
    if (rc) {
      // this request cannot be placed: reject it and leave the rest queued
      if (b->mem[s].active) remove_solve(b, s);
      v->cells.release(co, np);
      v->faces.release(fo, nf);
      r.st.state = CGKS_REQ_REJECTED;
      r.st.t_done = t;
      v->queue.pop_front();
      *changed = true;
      return rc;
    }
    v->slot_req[s] = r.id;
    v->used += r.footprint;
    r.st.state = CGKS_REQ_ACTIVE;
    r.st.t_admit = t;
    r.W0.clear();
    r.W0.shrink_to_fit();
    v->queue.pop_front();
    *changed = true;
  }
  if (*changed && b) {
    b->sh.tau_c1 = v->sh.tau_c1; b->sh.tau_c2 = v->sh.tau_c2;
    b->sh.weno_eps = v->sh.weno_eps; b->sh.weno_g0 = v->sh.weno_g0;
    return finalize_batch(b);
  }
  return CGKS_OK;
}

int cgks_server_step(cgks_server *v, int32_t *n_active) {
  if (!v) return CGKS_EINVAL;
  int rc = begin_call(v->user_stream, v->stream, v->ev_user, v->device);
  if (rc) return rc;
  bool changed = false;
  rc = server_update(v, now_s(v), &changed);
  if (rc) { end_call(v->user_stream, v->stream, v->ev_done); return rc; }
  int na = 0;
  for (int64_t id : v->slot_req) na += id >= 0;
  if (n_active) *n_active = na;
  if (na == 0) return end_call(v->user_stream, v->stream, v->ev_done);
  // one batched V-cycle
  Batch *b = v->b;
  rc = run_many(b, 1, true);
  if (rc) return rc;
  v->res_host.resize(b->S);
  v->status_host.resize(b->S);
  CK(cudaMemcpyAsync(v->res_host.data(), b->res, sizeof(double) * b->S, cudaMemcpyDeviceToHost, v->stream));
  CK(cudaMemcpyAsync(v->status_host.data(), b->status, sizeof(int) * b->S, cudaMemcpyDeviceToHost, v->stream));
  CK(cudaStreamSynchronize(v->stream));
  const double t1 = now_s(v);
  // convergence bookkeeping; finished states are copied out now and their
  // slots freed at the next step
  for (int s = 0; s < b->S; ++s) {
    if (v->slot_req[s] < 0) continue;
    cgks_server::Req &r = *v->reqs[v->slot_req[s]];
    const double res = v->res_host[s];
    r.st.cycles += 1;
    if (r.st.cycles == 1) r.st.res_first = res;
    r.st.res_last = res;
    int state = CGKS_REQ_ACTIVE;
    if (v->status_host[s] || !std::isfinite(res)) state = CGKS_REQ_DIVERGED;
    else if (r.st.cycles > 1 && res <= r.drop * r.st.res_first) state = CGKS_REQ_CONVERGED;
    else if (r.st.cycles >= r.max_cycles) state = CGKS_REQ_STOPPED;
    if (state != CGKS_REQ_ACTIVE) {
      try {
        r.result.resize(4 * r.mesh->n_cells);
      } catch (const std::bad_alloc &) {
        return CGKS_ENOMEM;
      }
      rc = store_state(b, s, r.result.data(), nullptr, false);
      if (rc) return rc;
      r.st.state = state;
      r.st.t_done = t1;
    }
  }
  return end_call(v->user_stream, v->stream, v->ev_done);
}

int cgks_server_poll(cgks_server *v, int64_t req_id, cgks_req_status *st, double *W_out, int timeout_ms) {
  if (!v) return CGKS_EINVAL;
  auto it = v->reqs.find(req_id);
  if (it == v->reqs.end()) return CGKS_EINVAL;
  cgks_server::Req &r = *it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms > 0 ? timeout_ms : 0);
  auto done = [&] { return r.st.state >= CGKS_REQ_CONVERGED; };
  while (timeout_ms > 0 && !done() && std::chrono::steady_clock::now() < deadline) {
    int rc = cgks_server_step(v, nullptr);
    if (rc) return rc;
  }
  if (st) *st = r.st;
  if (done()) {
    if (W_out && !r.result.empty()) std::copy(r.result.begin(), r.result.end(), W_out);
    return CGKS_OK;
  }
  return timeout_ms > 0 ? CGKS_ETIMEOUT : CGKS_OK;
}

int cgks_server_footprint(const cgks_server *v, const cgks_mesh *m, int64_t *bytes) {
  if (!v || !m || !bytes || m->dim != 2) return CGKS_EINVAL;
  *bytes = static_cast<int64_t>(solve_footprint(m->h.n_cells, m->h.n_faces, v->sh.precision == CGKS_MIXED));
  return CGKS_OK;
}

int cgks_server_info(cgks_server *v, int64_t *device_bytes, int32_t *n_queued, int32_t *n_active) {
  if (!v) return CGKS_EINVAL;
  if (device_bytes) *device_bytes = v->b ? static_cast<int64_t>(v->b->arena_bytes + sizeof(double) * v->b->hist_cap) : 0;
  if (n_queued) *n_queued = static_cast<int32_t>(v->queue.size());
  int na = 0;
  for (int64_t id : v->slot_req) na += id >= 0;
  if (n_active) *n_active = na;
  return CGKS_OK;
}

int cgks_server_get_tuning(cgks_server *v, cgks_tuning *t) {
  if (!v || !t) return CGKS_EINVAL;
  if (v->b) {
    v->b->tune.report(t);
  } else {
    Tuner fresh;   // no batch yet: nothing tuned
    fresh.on = v->sh.autotune != 0;
    fresh.report(t);
  }
  return CGKS_OK;
}

}  // extern "C"
