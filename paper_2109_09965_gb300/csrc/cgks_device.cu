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
};

// kernel ids for the per-kernel timers
enum KernelId { KI_DT = 0, KI_RECON, KI_FACE, KI_UPDATE, KI_RESFIN, KI_LOFACE, KI_LORHS, KI_SWEEP, KI_LOCELL,
                KI_PROLONG, KI_COUNT };
const char *kKernelNames[KI_COUNT] = { "k_dt", "k_recon", "k_face", "k_update", "k_res_final", "k_lo_face",
                                       "k_lo_rhs", "k_sweep", "k_lo_cell", "k_prolong" };

// batch-wide settings (every solve of a batch shares them)
struct Shared {
  double gamma = 1.4, cfl_hi = 0.4, cfl_lo = 1000.0;
  int n_implicit = 6, n_sweeps = 2, time_scheme = CGKS_S1O2, precision = CGKS_FP64, use_graph = 1;
  cgks_alloc_fn alloc = nullptr;
  cgks_free_fn free = nullptr;
  void *alloc_ctx = nullptr;
};

// One solve of a batch: its mesh, its parameters and where it sits.
struct Member {
  std::shared_ptr<const HostMesh> mesh;
  cgks_params params;
  int64_t cell_off = 0, n_pad = 0, face_off = 0;
};

struct Timer {
  bool on = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  double ms[KI_COUNT] = { 0 };
  long long cnt[KI_COUNT] = { 0 };
};

// device tables of a batch (views into its arena)
struct DevArrays {
  double *vol, *ivol, *per, *ih, *m2, *op, *fn, *fS, *fjump, *fxi, *snx, *sny, *shs;
  double *mu, *bcuw, *bcrho, *bcu, *bcp;
  int *cface, *cnbr, *fc0, *fc1, *csid, *fsid, *bckind;
  unsigned char *ccol;
  float *f_ivol = nullptr, *f_ih = nullptr, *f_m2 = nullptr, *f_op = nullptr, *f_fn = nullptr, *f_fS = nullptr,
        *f_fjump = nullptr, *f_fxi = nullptr, *f_snx = nullptr, *f_sny = nullptr, *f_shs = nullptr, *f_mu = nullptr,
        *f_bcuw = nullptr, *f_bcrho = nullptr, *f_bcu = nullptr, *f_bcp = nullptr;
};

struct Batch {
  Shared sh;
  DevArrays d{};
  std::vector<Member> mem;
  int S = 0;
  int64_t N = 0, F = 0;        // padded cells, faces
  bool mixed = false;
  int n_colours = 0;
  std::vector<int> sweep_seq;        // colour order after the first pass
  std::vector<int> list_off;         // [n_colours + 1] offsets into the sweep cell list
  std::vector<Ranges> ranges;        // per colour: per-solve cell ranges (n = 0: use the list)
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
  int *list = nullptr, *perm = nullptr, *blk_begin = nullptr;
  Ctl *ctl = nullptr;
  unsigned long long *dt_bits = nullptr;
  int *status = nullptr;
  double *res = nullptr;               // [S] residual of the last update
  double *hist = nullptr;              // solve 0's residual history
  int hist_cap = 0;
  cudaGraphExec_t g_cycle = nullptr, g_step = nullptr;
  Timer *timer = nullptr;              // owned by the caller
  long long launches = 0;
};

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
  kern<<<grid, block, 0, b->stream>>>(args...);
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
  launch(b, KI_RESFIN, k_res_final, dim3(b->S), dim3(256), (const double *)b->partial, (const int *)b->blk_begin,
         b->ctl, b->res, b->hist, b->hist_cap, b->last);
}

template <typename TF>
void enqueue_hi_eval(Batch *b, const TF *W, const TF *Wx, TF *Fout) {
  Bufs<TF> &B = bufs<TF>(b);
  launch(b, KI_RECON, k_recon<TF>, dim3(nblk(b->N, kCellBlock)), dim3(kCellBlock), fmesh<TF>(b), fparams<TF>(b), W, Wx,
         B.coef);
  launch(b, KI_FACE, k_face<TF>, dim3(nblk(b->F, kFaceBlock)), dim3(kFaceBlock), fmesh<TF>(b), fparams<TF>(b), W,
         (const TF *)B.coef, Fout);
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
void enqueue_lo_solve(Batch *b) {
  Bufs<TF> &B = bufs<TF>(b);
  const dim3 gc(nblk(b->N, kCellBlock)), gf(nblk(b->F, kCellBlock)), blk(kCellBlock);
  const int colour0 = b->sh.n_sweeps > 0 ? 1 : 0;
  for (int k = 0; k < b->sh.n_implicit; ++k) {
    launch(b, KI_LOCELL, k_lo_cell<TF>, gc, blk, static_cast<int>(b->N), fparams<TF>(b), k == 0 ? 1 : 0,
           (const double *)b->Wn, b->U, (const TF *)B.dU, B.prim, mirror<TF>(B.U));
    launch(b, KI_LOFACE, k_lo_face<TF>, gf, blk, fmesh<TF>(b), fparams<TF>(b), (const TF *)B.U, (const TF *)B.prim,
           B.Flo, B.lam, B.E0, B.E1);
    launch(b, KI_LORHS, k_lo_rhs<TF>, gc, blk, b->dm, b->dp, k == 0 ? 1 : 0, colour0, (const TF *)B.Flo,
           (const TF *)B.lam, (const double *)b->Rp0, b->Src, B.Rk, B.invD, B.dU, B.lamS);
    for (int c : b->sweep_seq) {
      const int cnt = b->list_off[c + 1] - b->list_off[c];
      const Ranges &R = b->ranges[c];
      const bool use_list = R.n == 0;
      const int grid = use_list ? nblk(cnt, kSweepCells) : R.blk[R.n];
      launch(b, KI_SWEEP, k_sweep<TF>, dim3(grid), dim3(kSweepBlock), fmesh<TF>(b), fparams<TF>(b), R,
             use_list ? (const int *)b->list + b->list_off[c] : (const int *)nullptr, cnt, (const TF *)B.U,
             (const TF *)B.prim, (const TF *)B.Rk, (const TF *)B.invD, (const TF *)B.lamS, (const TF *)B.E0,
             (const TF *)B.E1, B.dU);
    }
  }
  // U^{n_implicit} = U + dU of the last step
  if (b->sh.n_implicit > 0)
    launch(b, KI_LOCELL, k_lo_cell<TF>, gc, blk, static_cast<int>(b->N), fparams<TF>(b), 0, (const double *)b->Wn, b->U,
           (const TF *)B.dU, B.prim, mirror<TF>(B.U));
  else
    cudaMemcpyAsync(b->U, b->Wn, sizeof(double) * 4 * b->N, cudaMemcpyDeviceToDevice, b->stream);
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
  cudaMemcpyAsync(b->Wn, b->W, sizeof(double) * 4 * b->N, cudaMemcpyDeviceToDevice, b->stream);
  if (b->mixed) { enqueue_lo_solve<float>(b); enqueue_prolong<float>(b); }
  else { enqueue_lo_solve<double>(b); enqueue_prolong<double>(b); }
}

long long count_launches(const Batch *b, bool cycle) {
  long long per_eval = 2;
  long long hi = per_eval + 1 + (b->sh.time_scheme == CGKS_S2O4 ? per_eval + 1 : 0);
  long long dt = 2;
  if (!cycle) return dt + hi + 1;
  long long lo = b->sh.n_implicit * (3 + static_cast<long long>(b->sweep_seq.size())) + (b->sh.n_implicit > 0 ? 1 : 0);
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

// n cycles (or explicit steps) without host synchronisation
int run_many(Batch *b, int n, bool cycle) {
  if (n <= 0) return CGKS_OK;
  CK(cudaMemsetAsync(&b->ctl->res_ctr, 0, sizeof(int), b->stream));
  const bool graph = b->sh.use_graph && !(b->timer && b->timer->on);
  cudaGraphExec_t *ge = cycle ? &b->g_cycle : &b->g_step;
  if (graph && !*ge) {
    int rc = capture(b, cycle, ge);
    if (rc) return rc;
  }
  const long long per = count_launches(b, cycle);
  for (int k = 0; k < n; ++k) {
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

void collect_timing(Timer *t) {
  if (!t) return;
  for (auto &e : t->ev) {
    float ms = 0.f;
    cudaEventSynchronize(e.second.second);
    cudaEventElapsedTime(&ms, e.second.first, e.second.second);
    t->ms[e.first] += ms;
    t->cnt[e.first] += 1;
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  t->ev.clear();
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
  P8(&d.fn, 2 * F); P8(&d.fS, F); P8(&d.fjump, F); P8(&d.fxi, 8 * F);
  P8(&d.mu, S); P8(&d.bcuw, 2 * T); P8(&d.bcrho, T); P8(&d.bcu, 2 * T); P8(&d.bcp, T);
  PI(&d.cface, kMaxFace * N); PI(&d.cnbr, kMaxFace * N); PI(&d.fc0, F); PI(&d.fc1, F); PI(&d.csid, N); PI(&d.fsid, F);
  PI(&d.bckind, T); PI(&b->list, std::max<int64_t>(L, 1)); PI(&b->perm, N); PI(&b->blk_begin, S + 1);
  PV(reinterpret_cast<void **>(&d.ccol), N);
  PV(reinterpret_cast<void **>(&b->ctl), sizeof(Ctl));
  PV(reinterpret_cast<void **>(&b->dt_bits), sizeof(unsigned long long) * S);
  PI(&b->status, S);
  if (!mixed) {
    Bufs<double> &X = b->bd;
    P8(&X.coef, 20 * N); P8(&X.FA, 16 * F); P8(&X.FB, 16 * F);
    P8(&X.prim, D::NPRIM * N); P8(&X.Flo, 4 * F); P8(&X.lam, F); P8(&X.E0, 4 * F); P8(&X.E1, 4 * F);
    P8(&X.Rk, 4 * N); P8(&X.invD, N); P8(&X.dU, 4 * N); P8(&X.lamS, kMaxFace * N);
  } else {
    Bufs<float> &X = b->bf;
    P4(&X.W, 4 * N); P4(&X.Wx, 8 * N); P4(&X.Wn, 4 * N); P4(&X.Ws, 4 * N); P4(&X.Wxs, 8 * N); P4(&X.U, 4 * N);
    P4(&X.coef, 20 * N); P4(&X.FA, 16 * F); P4(&X.FB, 16 * F);
    P4(&X.prim, D::NPRIM * N); P4(&X.Flo, 4 * F); P4(&X.lam, F);
    P4(&X.Rk, 4 * N); P4(&X.invD, N); P4(&X.dU, 4 * N); P4(&X.lamS, kMaxFace * N);
    P4(&d.f_ivol, N); P4(&d.f_ih, N); P4(&d.f_m2, 3 * N); P4(&d.f_op, kNCol * kNM * N);
    P4(&d.f_snx, kMaxFace * N); P4(&d.f_sny, kMaxFace * N); P4(&d.f_shs, kMaxFace * N);
    P4(&d.f_fn, 2 * F); P4(&d.f_fS, F); P4(&d.f_fjump, F); P4(&d.f_fxi, 8 * F);
    P4(&d.f_mu, S); P4(&d.f_bcuw, 2 * T); P4(&d.f_bcrho, T); P4(&d.f_bcu, 2 * T); P4(&d.f_bcp, T);
  }
}

constexpr int kHistDefault = 1024;

// Device bytes one solve of n cells and nf faces adds to a batch: its
// share of the arena, the residual history and, for the serving rebuild,
// the stash of its state (12 doubles) and two move maps per cell.  The
// arena size is sub-additive over solves, so the footprints of a set of
// solves bound the batch they form.
size_t solve_footprint(int64_t n, int64_t nf, bool mixed) {
  const int64_t np = (n + kCellBlock - 1) / kCellBlock * kCellBlock;
  Batch tmp;
  std::vector<Piece> pieces;
  plan_arena(&tmp, np, nf, 1, n, mixed, pieces);
  return arena_total(pieces) + sizeof(double) * kHistDefault + (12 * sizeof(double) + 2 * sizeof(int)) * np + 3 * 256;
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

// Build a batch on stream st from members (mesh + per-solve parameters).
int build_batch(const Shared &sh, std::vector<Member> mem, cudaStream_t st, Batch **out) {
  *out = nullptr;
  std::unique_ptr<Batch> B(new (std::nothrow) Batch());
  if (!B) return CGKS_ENOMEM;
  Batch *b = B.get();
  b->sh = sh;
  b->mem = std::move(mem);
  b->S = static_cast<int>(b->mem.size());
  b->mixed = sh.precision == CGKS_MIXED;
  b->stream = st;
  if (b->S == 0) return CGKS_EINVAL;
  int64_t N = 0, F = 0;
  int C = 0;
  for (auto &m : b->mem) {
    m.cell_off = N;
    m.n_pad = pad_cells(m.mesh->n_cells);
    m.face_off = F;
    N += m.n_pad;
    F += m.mesh->n_faces;
    C = std::max(C, m.mesh->n_colours);
  }
  if (N > INT32_MAX / 32 || F > INT32_MAX / 32) return CGKS_EINVAL;
  b->N = N; b->F = F; b->n_colours = C;
  const int S = b->S;
  // ---- host arrays of the concatenated index space
  std::vector<double> vol(N, 1.0), ivol(N, 1.0), per(N, 4.0), ih(N, 1.0), m2(3 * N, 0.0), op(kNCol * kNM * N, 0.0);
  std::vector<double> snx(kMaxFace * N, 0.0), sny(kMaxFace * N, 0.0), shs(kMaxFace * N, 0.0);
  std::vector<double> fn(2 * F), fS(F), fjump(F), fxi(8 * F);
  std::vector<int> cface(kMaxFace * N, kNoFace), cnbr(kMaxFace * N, -1), fc0(F), fc1(F), csid(N, -1), fsid(F),
      perm(N, 0), blk(S + 1);
  std::vector<unsigned char> ccol(N, 255);
  std::vector<double> mu(S), bc_uw(2 * kTagsPerSolve * S, 0.0), bc_rho(kTagsPerSolve * S, 1.0),
      bc_u(2 * kTagsPerSolve * S, 0.0), bc_p(kTagsPerSolve * S, 1.0);
  std::vector<int> bc_kind(kTagsPerSolve * S, CGKS_BC_SLIP);
  std::vector<std::vector<int>> lists(C);
  for (int s = 0; s < S; ++s) {
    const Member &M = b->mem[s];
    const HostMesh &hm = *M.mesh;
    const cgks_params &p = M.params;
    const int64_t nc = hm.n_cells, nf = hm.n_faces, co = M.cell_off, fo = M.face_off;
    blk[s] = static_cast<int>(co / kCellBlock);
    mu[s] = p.mu;
    for (int t = 0; t < kTagsPerSolve; ++t) {
      const int g = s * kTagsPerSolve + t;
      const cgks_bc &bc = p.bc[t];
      bc_kind[g] = t < p.n_bc ? bc.kind : CGKS_BC_SLIP;
      bc_uw[2 * g] = bc.u_wall[0]; bc_uw[2 * g + 1] = bc.u_wall[1];
      bc_rho[g] = bc.rho; bc_u[2 * g] = bc.u[0]; bc_u[2 * g + 1] = bc.u[1]; bc_p[g] = bc.p;
    }
    std::vector<char> wall(kTagsPerSolve, 0);
    for (int t = 0; t < p.n_bc; ++t) wall[t] = p.bc[t].kind != CGKS_BC_FARFIELD;
    std::vector<double> ops;
    build_operator(hm, wall, ops);
    for (int64_t i = 0; i < nc; ++i) {
      const int64_t I = co + i;
      vol[I] = hm.vol[i]; ivol[I] = 1.0 / hm.vol[i]; per[I] = hm.per[i]; ih[I] = 1.0 / hm.h[i];
      for (int q = 0; q < 3; ++q) m2[q * N + I] = hm.m2[q * nc + i];
      for (int q = 0; q < kNCol * kNM; ++q) op[q * N + I] = ops[q * nc + i];
      csid[I] = s;
      perm[I] = hm.perm[i];
      for (int sl = 0; sl < kMaxFace; ++sl) {
        const int32_t fs = hm.cface[sl * nc + i];
        if (fs == kNoFace) continue;
        const int32_t f = fs >= 0 ? fs : ~fs;
        const double sg = fs >= 0 ? 1.0 : -1.0;
        cface[sl * N + I] = fs >= 0 ? static_cast<int>(f + fo) : ~static_cast<int>(f + fo);
        const int32_t j = hm.cnbr[sl * nc + i];
        cnbr[sl * N + I] = j >= 0 ? static_cast<int>(j + co) : -1;
        snx[sl * N + I] = sg * hm.fn[f];
        sny[sl * N + I] = sg * hm.fn[nf + f];
        shs[sl * N + I] = 0.5 * hm.fS[f];
      }
    }
    for (int c = 0; c < hm.n_colours; ++c)
      for (int32_t i = hm.colour_start[c]; i < hm.colour_start[c + 1]; ++i) {
        ccol[co + i] = static_cast<unsigned char>(c);
        lists[c].push_back(static_cast<int>(co + i));
      }
    for (int64_t f = 0; f < nf; ++f) {
      const int64_t G = fo + f;
      fc0[G] = static_cast<int>(hm.fc0[f] + co);
      const int32_t c1 = hm.fc1[f];
      fc1[G] = c1 >= 0 ? static_cast<int>(c1 + co) : -1 - (s * kTagsPerSolve + (-1 - c1));
      fsid[G] = s;
      fn[G] = hm.fn[f]; fn[F + G] = hm.fn[nf + f];
      fS[G] = hm.fS[f];
      fjump[G] = hm.fdelta[f] > 0.0 ? p.alpha / hm.fdelta[f] : 0.0;
      for (int q = 0; q < 8; ++q) fxi[q * F + G] = hm.fxi[q * nf + f];
    }
  }
  blk[S] = static_cast<int>(N / kCellBlock);
  std::vector<int> list;
  b->list_off.assign(C + 1, 0);
  for (int c = 0; c < C; ++c) {
    list.insert(list.end(), lists[c].begin(), lists[c].end());
    b->list_off[c + 1] = static_cast<int>(list.size());
  }
  if (list.empty()) list.push_back(0);
  // per-colour ranges for the sweeps (the list is used beyond kMaxRanges solves)
  b->ranges.assign(C, Ranges{});
  for (int c = 0; c < C; ++c) {
    Ranges &R = b->ranges[c];
    std::memset(&R, 0, sizeof(R));
    int nr = 0, blocks = 0;
    bool fits = true;
    for (int s = 0; s < S && fits; ++s) {
      const HostMesh &hm = *b->mem[s].mesh;
      if (c >= hm.n_colours) continue;
      const int beg = static_cast<int>(b->mem[s].cell_off) + hm.colour_start[c];
      const int end = static_cast<int>(b->mem[s].cell_off) + hm.colour_start[c + 1];
      if (end == beg) continue;
      if (nr == kMaxRanges) { fits = false; break; }
      R.blk[nr] = blocks;
      R.begin[nr] = beg;
      R.end[nr] = end;
      blocks += nblk(end - beg, kSweepCells);
      ++nr;
    }
    if (fits) { R.n = nr; R.blk[nr] = blocks; }
    else std::memset(&R, 0, sizeof(R));
  }
  // colour sequence of Algorithm 1 with colour classes: n_sweeps x (0..C-1,
  // C-1..0).  A colour repeated back to back recomputes identical values
  // (its cells read only other colours), and the first pass is done by
  // k_lo_rhs, so both are dropped.
  {
    std::vector<int> seq;
    for (int sw = 0; sw < sh.n_sweeps; ++sw) {
      for (int c = 0; c < C; ++c) if (seq.empty() || seq.back() != c) seq.push_back(c);
      for (int c = C - 1; c >= 0; --c) if (seq.empty() || seq.back() != c) seq.push_back(c);
    }
    if (!seq.empty()) seq.erase(seq.begin());
    b->sweep_seq = seq;
  }
  // ---- device arena
  DevArrays &d = b->d;
  std::vector<Piece> pieces;
  plan_arena(b, N, F, S, static_cast<int64_t>(list.size()), b->mixed, pieces);
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
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  bool ok = up(d.vol, vol.data(), 8 * N) && up(d.ivol, ivol.data(), 8 * N) && up(d.per, per.data(), 8 * N) &&
            up(d.ih, ih.data(), 8 * N) && up(d.m2, m2.data(), 8 * m2.size()) && up(d.op, op.data(), 8 * op.size()) &&
            up(d.snx, snx.data(), 8 * snx.size()) && up(d.sny, sny.data(), 8 * sny.size()) &&
            up(d.shs, shs.data(), 8 * shs.size()) && up(d.fn, fn.data(), 8 * fn.size()) && up(d.fS, fS.data(), 8 * F) &&
            up(d.fjump, fjump.data(), 8 * F) && up(d.fxi, fxi.data(), 8 * fxi.size()) && up(d.mu, mu.data(), 8 * S) &&
            up(d.bcuw, bc_uw.data(), 8 * bc_uw.size()) && up(d.bcrho, bc_rho.data(), 8 * bc_rho.size()) &&
            up(d.bcu, bc_u.data(), 8 * bc_u.size()) && up(d.bcp, bc_p.data(), 8 * bc_p.size()) &&
            up(d.cface, cface.data(), 4 * cface.size()) && up(d.cnbr, cnbr.data(), 4 * cnbr.size()) &&
            up(d.fc0, fc0.data(), 4 * F) && up(d.fc1, fc1.data(), 4 * F) && up(d.csid, csid.data(), 4 * N) &&
            up(d.fsid, fsid.data(), 4 * F) && up(d.bckind, bc_kind.data(), 4 * bc_kind.size()) &&
            up(b->list, list.data(), 4 * list.size()) && up(b->perm, perm.data(), 4 * N) &&
            up(b->blk_begin, blk.data(), 4 * (S + 1)) && up(d.ccol, ccol.data(), N);
  std::vector<float> tmp;
  auto upf = [&](float *dst, const std::vector<double> &src) {
    tmp.assign(src.begin(), src.end());
    bool r = cudaMemcpyAsync(dst, tmp.data(), 4 * tmp.size(), cudaMemcpyHostToDevice, st) == cudaSuccess;
    return r && cudaStreamSynchronize(st) == cudaSuccess;   // tmp is reused
  };
  if (ok && b->mixed)
    ok = upf(d.f_ivol, ivol) && upf(d.f_ih, ih) && upf(d.f_m2, m2) && upf(d.f_op, op) && upf(d.f_snx, snx) && upf(d.f_sny, sny) &&
         upf(d.f_shs, shs) && upf(d.f_fn, fn) && upf(d.f_fS, fS) && upf(d.f_fjump, fjump) && upf(d.f_fxi, fxi) &&
         upf(d.f_mu, mu) && upf(d.f_bcuw, bc_uw) && upf(d.f_bcrho, bc_rho) && upf(d.f_bcu, bc_u) && upf(d.f_bcp, bc_p);
  if (ok) ok = cudaMemsetAsync(b->ctl, 0, sizeof(Ctl), st) == cudaSuccess &&
               cudaMemsetAsync(b->status, 0, sizeof(int) * S, st) == cudaSuccess &&
               cudaMemsetAsync(b->Rp0, 0, sizeof(double) * 4 * N, st) == cudaSuccess &&
               cudaMemsetAsync(b->res, 0, sizeof(double) * S, st) == cudaSuccess &&
               cudaMemsetAsync(b->last, 0, sizeof(double) * 4, st) == cudaSuccess;
  if (ok) {
    if (b->mixed) ok = cudaMemsetAsync(b->bf.dU, 0, sizeof(float) * 4 * N, st) == cudaSuccess;
    else ok = cudaMemsetAsync(b->bd.dU, 0, sizeof(double) * 4 * N, st) == cudaSuccess;
  }
  if (ok) {
    k_fill_padding<<<nblk(N, kCellBlock), kCellBlock, 0, st>>>(static_cast<int>(N), d.csid, b->W, b->Wx,
                                                               b->mixed ? b->bf.W : nullptr,
                                                               b->mixed ? b->bf.Wx : nullptr);
    ok = cudaGetLastError() == cudaSuccess;
    // the stage and predictor states keep the same inert padding: the
    // update kernels never write padding cells
    ok = ok && cudaMemcpyAsync(b->Wn, b->W, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(b->Ws, b->W, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(b->Wxs, b->Wx, sizeof(double) * 8 * N, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    if (ok && b->mixed)
      ok = cudaMemcpyAsync(b->bf.Wn, b->bf.W, sizeof(float) * 4 * N, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(b->bf.Ws, b->bf.W, sizeof(float) * 4 * N, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(b->bf.Wxs, b->bf.Wx, sizeof(float) * 8 * N, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
  }
  if (!ok) { destroy_batch(B.release()); return CGKS_ECUDA; }
  // kernel-side views
  fill_shared_params(sh, b->dp);
  fill_shared_params(sh, b->fp);
  b->dp.mu = d.mu; b->dp.bc_kind = d.bckind; b->dp.bc_uw = d.bcuw; b->dp.bc_rho = d.bcrho; b->dp.bc_u = d.bcu;
  b->dp.bc_p = d.bcp;
  b->fp.mu = d.f_mu; b->fp.bc_kind = d.bckind; b->fp.bc_uw = d.f_bcuw; b->fp.bc_rho = d.f_bcrho; b->fp.bc_u = d.f_bcu;
  b->fp.bc_p = d.f_bcp;
  MeshT<double> &dm = b->dm;
  dm.nc = static_cast<int>(N); dm.nf = static_cast<int>(F);
  dm.vol = d.vol; dm.ivol = d.ivol; dm.per = d.per; dm.ih = d.ih; dm.m2 = d.m2; dm.op = d.op;
  dm.fn = d.fn; dm.fS = d.fS; dm.fjump = d.fjump; dm.fxi = d.fxi; dm.snx = d.snx; dm.sny = d.sny; dm.shs = d.shs;
  dm.cface = d.cface; dm.cnbr = d.cnbr; dm.fc0 = d.fc0; dm.fc1 = d.fc1; dm.csid = d.csid; dm.fsid = d.fsid;
  dm.ccol = d.ccol;
  MeshT<float> &fm = b->fm;
  fm.nc = dm.nc; fm.nf = dm.nf;
  fm.vol = nullptr; fm.per = nullptr; fm.ivol = d.f_ivol; fm.ih = d.f_ih; fm.m2 = d.f_m2; fm.op = d.f_op;
  fm.fn = d.f_fn; fm.fS = d.f_fS; fm.fjump = d.f_fjump; fm.fxi = d.f_fxi; fm.snx = d.f_snx; fm.sny = d.f_sny; fm.shs = d.f_shs;
  fm.cface = d.cface; fm.cnbr = d.cnbr; fm.fc0 = d.fc0; fm.fc1 = d.fc1; fm.csid = d.csid; fm.fsid = d.fsid;
  fm.ccol = d.ccol;
  int rc = ensure_hist(b, kHistDefault);
  if (rc) { destroy_batch(B.release()); return rc; }
  *out = B.release();
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
      static_cast<int>(n), static_cast<int>(M.cell_off), static_cast<int>(b->N), b->perm + M.cell_off, wa,
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
      static_cast<int>(n), static_cast<int>(M.cell_off), static_cast<int>(b->N), b->perm + M.cell_off, b->W, b->Wx, wa,
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
  sh.precision = p->precision; sh.use_graph = p->use_graph;
  sh.alloc = p->alloc; sh.free = p->free; sh.alloc_ctx = p->alloc_ctx;
  return sh;
}

int validate_params(const cgks_params *p, const HostMesh &hm) {
  if (!(p->gamma > 1.0) || p->mu < 0.0 || !(p->cfl_hi > 0.0) || !(p->cfl_lo > 0.0) || p->n_implicit < 0 ||
      p->n_sweeps < 0 || (p->time_scheme != CGKS_S1O2 && p->time_scheme != CGKS_S2O4) || p->n_bc < 0 ||
      p->n_bc > CGKS_MAX_BC || (p->precision != CGKS_FP64 && p->precision != CGKS_MIXED) || !(p->alpha >= 0.0))
    return CGKS_EINVAL;
  for (int t : hm.bface_tags_used)
    if (t >= p->n_bc) return CGKS_EINVAL;
  for (int b = 0; b < p->n_bc; ++b) {
    int k = p->bc[b].kind;
    if (k != CGKS_BC_SLIP && k != CGKS_BC_NOSLIP && k != CGKS_BC_FARFIELD) return CGKS_EINVAL;
    if (k == CGKS_BC_FARFIELD && !(p->bc[b].rho > 0.0 && p->bc[b].p > 0.0)) return CGKS_EINVAL;
  }
  return CGKS_OK;
}

}  // namespace

// ------------------------------------------------------------------------
struct cgks_solver {
  Batch *b = nullptr;
  cgks_params params{};
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_user = nullptr, ev_done = nullptr;
  int device = 0;
  Timer timer;
  int status_cache = 0;
};

struct cgks_server {
  struct Req {
    int64_t id;
    std::shared_ptr<const HostMesh> mesh;
    cgks_params params;
    std::vector<double> W0;
    double drop;
    cgks_req_status st;
    std::vector<double> result;      // final state, caller order
    size_t footprint;
  };
  Shared sh;
  int max_active = 64, max_cycles = 20000;
  size_t budget = 0;
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev_user = nullptr, ev_done = nullptr;
  int device = 0;
  int64_t next_id = 1;
  std::map<int64_t, std::unique_ptr<Req>> reqs;
  std::deque<int64_t> queue;
  std::vector<int64_t> active;     // member s of the batch runs request active[s]
  Batch *b = nullptr;
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
  CK(cudaMemcpyAsync(&st, s->b->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->status_cache = st;
  return st ? CGKS_EDIVERGED : CGKS_OK;
}

double now_s(const cgks_server *v) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - v->t0).count();
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

int cgks_mesh_info(const cgks_mesh *m, cgks_mesh_info_t *out) {
  if (!m || !out) return CGKS_EINVAL;
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
  collect_timing(&s->timer);
  destroy_batch(s->b);
  if (s->ev_user) cudaEventDestroy(s->ev_user);
  if (s->ev_done) cudaEventDestroy(s->ev_done);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return CGKS_OK;
}

int cgks_solver_create(const cgks_mesh *m, const cgks_params *p, cgks_solver **out) {
  if (!m || !p || !out) return CGKS_EINVAL;
  *out = nullptr;
  int rc = validate_params(p, m->h);
  if (rc) return rc;
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
  rc = load_state(s->b, 0, W, Wx, device);
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
  rc = store_state(s->b, 0, W, Wx, device);
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
  CK(cudaMemsetAsync(&s->b->ctl->res_ctr, 0, sizeof(int), s->stream));
  enqueue_lo_smooth(s->b);
  CK(cudaGetLastError());
  rc = solver_status(s);
  collect_timing(&s->timer);
  int rc2 = end_call(s);
  return rc ? rc : rc2;
}

int cgks_residual(cgks_solver *s, double *res, double *r_l2) {
  if (!s) return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  Batch *b = s->b;
  double last[3];
  CK(cudaMemcpyAsync(last, b->last, sizeof(double) * 3, cudaMemcpyDeviceToHost, s->stream));
  std::vector<double> R;
  if (r_l2) {
    R.resize(4 * static_cast<size_t>(b->N));
    CK(cudaMemcpyAsync(R.data(), b->Rp0, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  if (res) *res = last[0];
  if (r_l2) {
    const int64_t n = b->mem[0].mesh->n_cells, N = b->N;
    for (int v = 0; v < 4; ++v) {
      double a = 0.0;
      for (int64_t i = 0; i < n; ++i) a += R[v * N + i] * R[v * N + i];
      r_l2[v] = std::sqrt(a);
    }
  }
  return end_call(s);
}

int cgks_get_rp0(cgks_solver *s, double *Rp0) {
  if (!s || !Rp0) return CGKS_EINVAL;
  int rc = begin_call(s);
  if (rc) return rc;
  Batch *b = s->b;
  const int64_t N = b->N, n = b->mem[0].mesh->n_cells;
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
    if (names) names[k] = kKernelNames[k];
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

int64_t cgks_launch_count(const cgks_solver *s) { return s ? s->b->launches : -1; }

int cgks_launches_per_call(const cgks_solver *s, int cycle) {
  return s ? static_cast<int>(count_launches(s->b, cycle != 0)) : -1;
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
}

int cgks_server_create(size_t hbm_budget, const cgks_server_opts *o, cgks_server **out) {
  if (!o || !out || hbm_budget == 0 || o->max_active < 1 || o->max_cycles < 1 || !(o->cfl_hi > 0.0) ||
      !(o->cfl_lo > 0.0) || o->n_implicit < 0 || o->n_sweeps < 0 ||
      (o->precision != CGKS_FP64 && o->precision != CGKS_MIXED) ||
      (o->time_scheme != CGKS_S1O2 && o->time_scheme != CGKS_S2O4))
    return CGKS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return CGKS_ECUDA;
  cgks_server *v = new (std::nothrow) cgks_server();
  if (!v) return CGKS_ENOMEM;
  v->sh.cfl_hi = o->cfl_hi; v->sh.cfl_lo = o->cfl_lo; v->sh.n_implicit = o->n_implicit; v->sh.n_sweeps = o->n_sweeps;
  v->sh.time_scheme = o->time_scheme; v->sh.precision = o->precision; v->sh.use_graph = o->use_graph;
  v->sh.alloc = o->alloc; v->sh.free = o->free; v->sh.alloc_ctx = o->alloc_ctx;
  v->max_active = o->max_active;
  v->max_cycles = o->max_cycles;
  v->budget = hbm_budget;
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
                       int64_t *req_id) {
  if (!v || !m || !p || !W0 || !(res_drop > 0.0)) return CGKS_EINVAL;
  cgks_params q = *p;   // batch-wide fields come from the server
  q.cfl_hi = v->sh.cfl_hi; q.cfl_lo = v->sh.cfl_lo; q.n_implicit = v->sh.n_implicit; q.n_sweeps = v->sh.n_sweeps;
  q.time_scheme = v->sh.time_scheme; q.precision = v->sh.precision;
  int rc = validate_params(&q, m->h);
  if (rc) return rc;
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
  std::memset(&r->st, 0, sizeof(r->st));
  r->st.n_cells = m->h.n_cells;
  r->st.t_submit = now_s(v);
  r->footprint = solve_footprint(m->h.n_cells, m->h.n_faces, v->sh.precision == CGKS_MIXED);
  const int64_t id = r->id;
  if (req_id) *req_id = id;
  if (r->footprint > v->budget) {
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

// Replace the active batch by one running `next`.  Continuing solves keep
// their device state: it is stashed compactly, the old batch is freed, the
// new batch is built and the stash is moved in, so device memory never
// holds two batches at once.
static int server_rebuild(cgks_server *v, const std::vector<int64_t> &next) {
  Batch *old = v->b;
  v->b = nullptr;
  // continuing solves: (index in next, index in old)
  std::vector<std::pair<int, int>> cont;
  for (size_t s = 0; s < next.size(); ++s)
    for (size_t k = 0; k < v->active.size(); ++k)
      if (v->active[k] == next[s]) cont.push_back({ static_cast<int>(s), static_cast<int>(k) });
  int64_t n_st = 0;
  for (auto &c : cont) n_st += old->mem[c.second].mesh->n_cells;
  std::vector<int64_t> st_off(cont.size());
  char *stash = nullptr;
  double *sW = nullptr, *sWx = nullptr;
  int *smap = nullptr;
  int64_t N_new = 0;
  for (int64_t id : next) N_new += pad_cells(v->reqs[id]->mesh->n_cells);
  v->active.clear();
  if (n_st > 0) {
    const size_t bytes = sizeof(double) * 12 * n_st + sizeof(int) * std::max(n_st, N_new) + 512;
    stash = static_cast<char *>(dev_alloc(v->sh, bytes));
    if (!stash) { destroy_batch(old); return CGKS_ENOMEM; }
    sW = reinterpret_cast<double *>(stash);
    sWx = sW + 4 * n_st;
    smap = reinterpret_cast<int *>(sWx + 8 * n_st);
    std::vector<int> map(n_st);
    int64_t o = 0;
    for (size_t c = 0; c < cont.size(); ++c) {
      const Member &O = old->mem[cont[c].second];
      st_off[c] = o;
      for (int64_t i = 0; i < O.mesh->n_cells; ++i) map[o + i] = static_cast<int>(O.cell_off + i);
      o += O.mesh->n_cells;
    }
    CK(cudaMemcpyAsync(smap, map.data(), sizeof(int) * n_st, cudaMemcpyHostToDevice, v->stream));
    k_move_state<<<nblk(n_st, kCellBlock), kCellBlock, 0, v->stream>>>(
        static_cast<int>(n_st), static_cast<int>(old->N), smap, old->W, old->Wx, sW, sWx, nullptr, nullptr);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(v->stream));
  }
  destroy_batch(old);
  auto fail = [&](int rc) { dev_free(v->sh, stash); return rc; };
  if (next.empty()) return fail(CGKS_OK);
  std::vector<Member> mem(next.size());
  for (size_t s = 0; s < next.size(); ++s) {
    mem[s].mesh = v->reqs[next[s]]->mesh;
    mem[s].params = v->reqs[next[s]]->params;
  }
  Batch *nb = nullptr;
  int rc = build_batch(v->sh, std::move(mem), v->stream, &nb);
  if (rc) return fail(rc);
  if (n_st > 0) {
    std::vector<int> map(nb->N, -1);
    for (size_t c = 0; c < cont.size(); ++c) {
      const Member &M = nb->mem[cont[c].first];
      for (int64_t i = 0; i < M.mesh->n_cells; ++i) map[M.cell_off + i] = static_cast<int>(st_off[c] + i);
    }
    if (cudaMemcpyAsync(smap, map.data(), sizeof(int) * nb->N, cudaMemcpyHostToDevice, v->stream) != cudaSuccess) {
      destroy_batch(nb);
      return fail(CGKS_ECUDA);
    }
    k_move_state<<<nblk(nb->N, kCellBlock), kCellBlock, 0, v->stream>>>(
        static_cast<int>(nb->N), static_cast<int>(n_st), smap, sW, sWx, nb->W, nb->Wx,
        nb->mixed ? nb->bf.W : nullptr, nb->mixed ? nb->bf.Wx : nullptr);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(v->stream) != cudaSuccess) {
      destroy_batch(nb);
      return fail(CGKS_ECUDA);
    }
  }
  dev_free(v->sh, stash);
  for (size_t s = 0; s < next.size(); ++s) {
    bool is_cont = false;
    for (auto &c : cont) is_cont |= c.first == static_cast<int>(s);
    if (!is_cont) {
      rc = load_state(nb, static_cast<int>(s), v->reqs[next[s]]->W0.data(), nullptr, false);
      if (rc) { destroy_batch(nb); return rc; }
    }
  }
  CK(cudaStreamSynchronize(v->stream));
  v->b = nb;
  v->active = next;
  return CGKS_OK;
}

int cgks_server_step(cgks_server *v, int32_t *n_active) {
  if (!v) return CGKS_EINVAL;
  int rc = begin_call(v->user_stream, v->stream, v->ev_user, v->device);
  if (rc) return rc;
  const double t = now_s(v);
  // 1. drop finished solves (their states were copied out when they finished)
  std::vector<int64_t> next;
  for (int64_t id : v->active)
    if (v->reqs[id]->st.state == CGKS_REQ_ACTIVE) next.push_back(id);
  // 2. admit queued requests while the footprint fits
  size_t used = 0;
  for (int64_t id : next) used += v->reqs[id]->footprint;
  bool changed = next.size() != v->active.size();
  while (!v->queue.empty() && static_cast<int>(next.size()) < v->max_active) {
    cgks_server::Req &r = *v->reqs[v->queue.front()];
    if (used + r.footprint > v->budget) break;
    used += r.footprint;
    r.st.state = CGKS_REQ_ACTIVE;
    r.st.t_admit = t;
    next.push_back(r.id);
    v->queue.pop_front();
    changed = true;
  }
  if (changed) {
    rc = server_rebuild(v, next);
    if (rc) {
      // the batch could not be formed: its requests are rejected
      for (int64_t id : next) {
        cgks_server::Req &r = *v->reqs[id];
        r.st.state = CGKS_REQ_REJECTED;
        r.st.t_done = now_s(v);
      }
      return rc;
    }
  }
  if (n_active) *n_active = static_cast<int32_t>(v->active.size());
  if (v->active.empty()) return end_call(v->user_stream, v->stream, v->ev_done);
  // 3. one batched V-cycle
  Batch *b = v->b;
  rc = run_many(b, 1, true);
  if (rc) return rc;
  v->res_host.resize(b->S);
  v->status_host.resize(b->S);
  CK(cudaMemcpyAsync(v->res_host.data(), b->res, sizeof(double) * b->S, cudaMemcpyDeviceToHost, v->stream));
  CK(cudaMemcpyAsync(v->status_host.data(), b->status, sizeof(int) * b->S, cudaMemcpyDeviceToHost, v->stream));
  CK(cudaStreamSynchronize(v->stream));
  const double t1 = now_s(v);
  // 4. convergence bookkeeping
  for (int s = 0; s < b->S; ++s) {
    cgks_server::Req &r = *v->reqs[v->active[s]];
    const double res = v->res_host[s];
    r.st.cycles += 1;
    if (r.st.cycles == 1) r.st.res_first = res;
    r.st.res_last = res;
    int state = CGKS_REQ_ACTIVE;
    if (v->status_host[s] || !std::isfinite(res)) state = CGKS_REQ_DIVERGED;
    else if (r.st.cycles > 1 && res <= r.drop * r.st.res_first) state = CGKS_REQ_CONVERGED;
    else if (r.st.cycles >= v->max_cycles) state = CGKS_REQ_STOPPED;
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
  if (!v || !m || !bytes) return CGKS_EINVAL;
  *bytes = static_cast<int64_t>(solve_footprint(m->h.n_cells, m->h.n_faces, v->sh.precision == CGKS_MIXED));
  return CGKS_OK;
}

int cgks_server_info(cgks_server *v, int64_t *device_bytes, int32_t *n_queued, int32_t *n_active) {
  if (!v) return CGKS_EINVAL;
  if (device_bytes) *device_bytes = v->b ? static_cast<int64_t>(v->b->arena_bytes + sizeof(double) * v->b->hist_cap) : 0;
  if (n_queued) *n_queued = static_cast<int32_t>(v->queue.size());
  if (n_active) *n_active = static_cast<int32_t>(v->active.size());
  return CGKS_OK;
}

}  // extern "C"
