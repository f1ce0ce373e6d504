// libcgks 3-D device runtime: one solve on a polyhedral mesh, the V-cycle of
// Ji, Shyy & Xu (arXiv:2109.09965, Section 3) and the explicit high-order
// step (Section 2.4) in 3-D, FP64 or mixed FP32/FP64, CUDA graphs per call
// pattern.  The C ABI in cgks_device.cu dispatches here for 3-D meshes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "cgks_internal.h"
#include "cgks_kernels3.cuh"
#include "cgks_runtime.h"

namespace cgks {

using namespace kern3;
namespace D3 = cgks::dev3;

namespace {
inline int nblk(int64_t n, int b) { return static_cast<int>((n + b - 1) / b); }

template <typename T>
struct Bufs3 {
  T *W = nullptr, *Wx = nullptr, *Wn = nullptr, *Ws = nullptr, *Wxs = nullptr, *U = nullptr;
  T *coef = nullptr, *FA = nullptr, *FB = nullptr, *rec = nullptr;
  T *Flo = nullptr;   // [F][kLo]: low-level flux and lambda_p per face
  T *E0 = nullptr, *E1 = nullptr, *Rk = nullptr, *invD = nullptr, *dU = nullptr, *lamS = nullptr;
};

struct Geo3 {
  double *vol, *ivol, *ih, *hdt, *m2, *op, *fe, *fS, *fjump, *fw, *fxi, *sn, *shs, *bcuw, *bcrho, *bcu, *bcp;
  double *fidl = nullptr;
  float *f_ivol = nullptr, *f_ih = nullptr, *f_m2 = nullptr, *f_op = nullptr, *f_fe = nullptr, *f_fS = nullptr,
        *f_fjump = nullptr, *f_fidl = nullptr, *f_fw = nullptr, *f_fxi = nullptr, *f_sn = nullptr, *f_shs = nullptr,
        *f_bcuw = nullptr, *f_bcrho = nullptr, *f_bcu = nullptr, *f_bcp = nullptr;
  int *fng, *cface, *cnbr, *fc0, *fc1, *bckind;
  unsigned char *wenok;
};

struct Piece3 { void **dst; size_t bytes; };
}  // namespace

struct Solver3 {
  cgks_params P{};
  int64_t N = 0, F = 0;
  bool mixed = false;
  int n_colours = 0;
  std::vector<int32_t> colour_start;
  std::vector<int> sweep_seq;
  cudaStream_t stream = nullptr;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  Geo3 g{};
  ParamsT<double> dp{};
  ParamsT<float> fp{};
  MeshT<double> dm{};
  MeshT<float> fm{};
  double *W = nullptr, *Wx = nullptr, *Wn = nullptr, *Ws = nullptr, *Wxs = nullptr, *U = nullptr;
  double *Rp0 = nullptr, *Src = nullptr, *partial = nullptr, *last = nullptr, *stage = nullptr, *hist = nullptr;
  int hist_cap = 0;
  Bufs3<double> bd;
  Bufs3<float> bf;
  int *perm = nullptr, *status = nullptr;
  Ctl *ctl = nullptr;
  unsigned long long *dt_bits = nullptr;
  cudaGraphExec_t g_cycle = nullptr, g_step = nullptr;
  Timer *timer = nullptr;
  long long launches = 0;
  Tuner tune;                     // launch shapes of the tunable kernels
  // boundary faces (for the wall loads): internal face, tag, centre, normal, area
  std::vector<int32_t> bf_face, bf_tag;
  std::vector<double> bf_geo;     // [7] per boundary face
};

namespace {

void *alloc3(const cgks_params &P, size_t bytes) {
  if (P.alloc) return P.alloc(bytes, P.alloc_ctx);
  void *p = nullptr;
  return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}
void free3(const cgks_params &P, void *p) {
  if (!p) return;
  if (P.alloc) { if (P.free) P.free(p, P.alloc_ctx); }
  else cudaFree(p);
}

template <typename Kern, typename... Args>
void launch(Solver3 *s, int id, Kern kern, dim3 grid, dim3 block, Args... args) {
  if (grid.x == 0) return;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool t = s->timer && s->timer->on;
  if (t) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s->stream);
  }
  launch_on(s->stream, s->P.programmatic_launch != 0, kern, grid, block, args...);
  if (t) {
    cudaEventRecord(e1, s->stream);
    s->timer->ev.push_back({ id, { e0, e1 } });
  }
  s->launches++;
}

template <typename TF> Bufs3<TF> &bufs(Solver3 *s);
template <> Bufs3<double> &bufs<double>(Solver3 *s) { return s->bd; }
template <> Bufs3<float> &bufs<float>(Solver3 *s) { return s->bf; }
template <typename TF> const MeshT<TF> &fmesh(Solver3 *s);
template <> const MeshT<double> &fmesh<double>(Solver3 *s) { return s->dm; }
template <> const MeshT<float> &fmesh<float>(Solver3 *s) { return s->fm; }
template <typename TF> const ParamsT<TF> &fpar(Solver3 *s);
template <> const ParamsT<double> &fpar<double>(Solver3 *s) { return s->dp; }
template <> const ParamsT<float> &fpar<float>(Solver3 *s) { return s->fp; }
template <typename TF> TF *mirror(TF *p) { return is_f32<TF>() ? p : nullptr; }

void enqueue_dt(Solver3 *s, double dt_fixed) {
  launch(s, KI_DT, k_reset_dt, dim3(1), dim3(32), s->ctl, s->dt_bits, dt_fixed);
  if (!(dt_fixed > 0.0))
    launch(s, KI_DT, k_dt, dim3(nblk(s->N, kCellBlock)), dim3(kCellBlock), s->dm, s->dp, (const double *)s->W,
           s->dt_bits);
}
void enqueue_res(Solver3 *s) {
  launch(s, KI_RESFIN, k_res_final, dim3(1), dim3(256), (const double *)s->partial, nblk(s->N, kCellBlock), s->ctl,
         s->hist, s->hist_cap, s->last);
}

template <typename TF>
void hi_eval(Solver3 *s, const TF *W, const TF *Wx, TF *Fout) {
  Bufs3<TF> &B = bufs<TF>(s);
  // nonlinear weights and the full flux are separate instantiations (the
  // default kernels stay as before)
  const bool weno = s->P.weno_eps > 0.0, full = s->P.flux_hi == CGKS_FLUX_FULL;
  tuned_launch(s->tune, TK_RECON, s->stream, [&] {
    with_shape(s->tune.shape(TK_RECON), [&](auto sh) {
      constexpr int S = decltype(sh)::value;
      const dim3 gr(nblk(s->N, shape_bs(S) * shape_ipt(S))), blk(shape_bs(S));
      if (weno)
        launch(s, KI_RECON, k_recon_weno<TF, S>, gr, blk, fmesh<TF>(s), fpar<TF>(s), W, Wx, B.coef,
               (const unsigned char *)s->g.wenok);
      else launch(s, KI_RECON, k_recon<TF, S>, gr, blk, fmesh<TF>(s), fpar<TF>(s), W, Wx, B.coef);
    });
  });
  tuned_launch(s->tune, TK_FACE, s->stream, [&] {
    with_shape(s->tune.shape(TK_FACE), [&](auto sh) {
      constexpr int S = decltype(sh)::value;
      const dim3 gr(nblk(s->F, shape_bs(S) * shape_ipt(S))), blk(shape_bs(S));
      if (full)
        launch(s, KI_FACE, k_face_full<TF, S>, gr, blk, fmesh<TF>(s), fpar<TF>(s), W, (const TF *)B.coef, Fout,
               (const Ctl *)s->ctl, (const unsigned long long *)s->dt_bits);
      else
        launch(s, KI_FACE, k_face<TF, S>, gr, blk, fmesh<TF>(s), fpar<TF>(s), W, (const TF *)B.coef, Fout);
    });
  });
}

template <typename TF>
void hi_step(Solver3 *s, double *Wout, TF *Wout_m, bool want_res) {
  Bufs3<TF> &B = bufs<TF>(s);
  double *part = want_res ? s->partial : nullptr;
  const dim3 g(nblk(s->N, kCellBlock)), blk(kCellBlock);
  hi_eval<TF>(s, B.W, B.Wx, B.FA);
  if (s->P.time_scheme == CGKS_S1O2) {
    launch(s, KI_UPDATE, k_update<TF, kS1O2>, g, blk, s->dm, s->dp, (const double *)s->W, (const TF *)B.FA,
           (const TF *)B.FA, (const Ctl *)s->ctl, (const unsigned long long *)s->dt_bits, s->status, Wout, s->Wx,
           part, s->Rp0, Wout_m, mirror<TF>(B.Wx));
  } else {
    launch(s, KI_UPDATE, k_update<TF, kS2O4Stage>, g, blk, s->dm, s->dp, (const double *)s->W, (const TF *)B.FA,
           (const TF *)B.FA, (const Ctl *)s->ctl, (const unsigned long long *)s->dt_bits, s->status, s->Ws, s->Wxs,
           (double *)nullptr, (double *)nullptr, mirror<TF>(B.Ws), mirror<TF>(B.Wxs));
    hi_eval<TF>(s, B.Ws, B.Wxs, B.FB);
    launch(s, KI_UPDATE, k_update<TF, kS2O4Final>, g, blk, s->dm, s->dp, (const double *)s->W, (const TF *)B.FA,
           (const TF *)B.FB, (const Ctl *)s->ctl, (const unsigned long long *)s->dt_bits, s->status, Wout, s->Wx,
           part, s->Rp0, Wout_m, mirror<TF>(B.Wx));
  }
  if (want_res) enqueue_res(s);
}

template <typename TF>
void lo_solve(Solver3 *s) {
  Bufs3<TF> &B = bufs<TF>(s);
  const dim3 gc(nblk(s->N, kCellBlock)), blk(kCellBlock);
  const int colour0_end = s->P.n_sweeps > 0 ? s->colour_start[1] : 0;
  for (int k = 0; k < s->P.n_implicit; ++k) {
    launch(s, KI_LOCELL, k_lo_cell<TF>, gc, blk, static_cast<int>(s->N), fpar<TF>(s), k == 0 ? 1 : 0,
           (const double *)s->Wn, s->U, (const TF *)B.dU, B.rec);
    tuned_launch(s->tune, TK_LOFACE, s->stream, [&] {
      with_shape(s->tune.shape(TK_LOFACE), [&](auto sh) {
        constexpr int S = decltype(sh)::value;
        launch(s, KI_LOFACE, k_lo_face<TF, S>, dim3(nblk(s->F, shape_bs(S) * shape_ipt(S))), dim3(shape_bs(S)),
               fmesh<TF>(s), fpar<TF>(s), (const TF *)B.rec, B.Flo, B.E0, B.E1);
      });
    });
    launch(s, KI_LORHS, k_lo_rhs<TF>, gc, blk, s->dm, s->dp, k == 0 ? 1 : 0, colour0_end, (const TF *)B.Flo,
           (const double *)s->Rp0, s->Src, B.Rk, B.invD, B.dU, B.lamS);
    for (int c : s->sweep_seq) {
      const int beg = s->colour_start[c], cnt = s->colour_start[c + 1] - beg;
      tuned_launch(s->tune, TK_SWEEP, s->stream, [&] {
        with_shape(s->tune.shape(TK_SWEEP), [&](auto sh) {
          constexpr int S = decltype(sh)::value;
          launch(s, KI_SWEEP, k_sweep<TF, S>, dim3(nblk(cnt, sweep_cpb(S))), dim3(shape_bs(S)), fmesh<TF>(s),
                 fpar<TF>(s), beg, cnt, (const TF *)B.rec, (const TF *)B.Rk, (const TF *)B.invD,
                 (const TF *)B.lamS, (const TF *)B.E0, (const TF *)B.E1, B.dU);
        });
      });
    }
  }
  if (s->P.n_implicit > 0)
    launch(s, KI_LOCELL, k_lo_cell<TF>, gc, blk, static_cast<int>(s->N), fpar<TF>(s), 0, (const double *)s->Wn, s->U,
           (const TF *)B.dU, B.rec);
  else
    cudaMemcpyAsync(s->U, s->Wn, sizeof(double) * NV * s->N, cudaMemcpyDeviceToDevice, s->stream);
}

template <typename TF>
void prolong(Solver3 *s) {
  launch(s, KI_PROLONG, k_prolong<TF>, dim3(nblk(s->N, kCellBlock)), dim3(kCellBlock), s->dm, s->dp, s->W,
         (const double *)s->Wn, (const double *)s->U, s->status, s->partial, mirror<TF>(bufs<TF>(s).W));
  enqueue_res(s);
}

template <typename TF>
void cycle_t(Solver3 *s) {
  Bufs3<TF> &B = bufs<TF>(s);
  enqueue_dt(s, -1.0);
  hi_step<TF>(s, s->Wn, mirror<TF>(B.Wn), false);
  hi_eval<TF>(s, B.Wn, B.Wx, B.FB);
  launch(s, KI_UPDATE, k_update<TF, kResidual>, dim3(nblk(s->N, kCellBlock)), dim3(kCellBlock), s->dm, s->dp,
         (const double *)s->Wn, (const TF *)B.FB, (const TF *)B.FB, (const Ctl *)s->ctl,
         (const unsigned long long *)s->dt_bits, s->status, (double *)nullptr, (double *)nullptr, (double *)nullptr,
         s->Rp0, (TF *)nullptr, (TF *)nullptr);
  lo_solve<TF>(s);
  prolong<TF>(s);
}
void enqueue_cycle(Solver3 *s) { if (s->mixed) cycle_t<float>(s); else cycle_t<double>(s); }
void enqueue_step(Solver3 *s, double dt_fixed) {
  enqueue_dt(s, dt_fixed);
  if (s->mixed) hi_step<float>(s, s->W, s->bf.W, true);
  else hi_step<double>(s, s->W, nullptr, true);
}

long long count_launches(const Solver3 *s, bool cycle) {
  const long long hi = 3 + (s->P.time_scheme == CGKS_S2O4 ? 3 : 0);
  if (!cycle) return 2 + hi + 1;
  const long long lo = s->P.n_implicit * (3 + static_cast<long long>(s->sweep_seq.size())) + (s->P.n_implicit > 0);
  return 2 + hi + 3 + lo + 2;
}

void drop_graphs(Solver3 *s) {
  if (s->g_cycle) { cudaGraphExecDestroy(s->g_cycle); s->g_cycle = nullptr; }
  if (s->g_step) { cudaGraphExecDestroy(s->g_step); s->g_step = nullptr; }
}

int capture(Solver3 *s, bool cycle, cudaGraphExec_t *out) {
  cudaGraph_t gr = nullptr;
  Timer *t = s->timer;
  s->timer = nullptr;
  const long long l0 = s->launches;
  if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { s->timer = t; return CGKS_ECUDA; }
  if (cycle) enqueue_cycle(s);
  else enqueue_step(s, -1.0);
  cudaError_t e = cudaStreamEndCapture(s->stream, &gr);
  s->launches = l0;
  s->timer = t;
  if (e != cudaSuccess) return CGKS_ECUDA;
  e = cudaGraphInstantiate(out, gr, 0);
  cudaGraphDestroy(gr);
  return e == cudaSuccess ? CGKS_OK : CGKS_ECUDA;
}

void plan(Solver3 *s, std::vector<Piece3> &pc) {
  const int64_t N = s->N, F = s->F;
  Geo3 &g = s->g;
  auto P8 = [&](double **x, int64_t c) { pc.push_back({ reinterpret_cast<void **>(x), sizeof(double) * c }); };
  auto P4 = [&](float **x, int64_t c) { pc.push_back({ reinterpret_cast<void **>(x), sizeof(float) * c }); };
  auto PI = [&](int **x, int64_t c) { pc.push_back({ reinterpret_cast<void **>(x), sizeof(int) * c }); };
  P8(&s->W, NV * N); P8(&s->Wx, 3 * NV * N); P8(&s->Wn, NV * N); P8(&s->Ws, NV * N); P8(&s->Wxs, 3 * NV * N);
  P8(&s->U, NV * N); P8(&s->Rp0, NV * N); P8(&s->Src, NV * N); P8(&s->stage, 4 * NV * N);
  P8(&s->partial, 2 * std::max<int64_t>(nblk(N, kCellBlock), 1)); P8(&s->last, 4);
  P8(&g.vol, N); P8(&g.ivol, N); P8(&g.ih, N); P8(&g.hdt, N); P8(&g.m2, 6 * N); P8(&g.op, kNCol3 * kNM3 * N);
  P8(&g.fe, 9 * F); P8(&g.fS, F); P8(&g.fjump, F); P8(&g.fw, 4 * F); P8(&g.fxi, 24 * F); P8(&g.fidl, F);
  P8(&g.sn, 3 * kMaxFace3 * N); P8(&g.shs, kMaxFace3 * N);
  P8(&g.bcuw, 3 * CGKS_MAX_BC); P8(&g.bcrho, CGKS_MAX_BC); P8(&g.bcu, 3 * CGKS_MAX_BC); P8(&g.bcp, CGKS_MAX_BC);
  PI(&g.fng, F); PI(&g.cface, kMaxFace3 * N); PI(&g.cnbr, kMaxFace3 * N); PI(&g.fc0, F); PI(&g.fc1, F);
  PI(&g.bckind, CGKS_MAX_BC); PI(&s->perm, N); PI(&s->status, 1);
  pc.push_back({ reinterpret_cast<void **>(&g.wenok), static_cast<size_t>(N) });
  pc.push_back({ reinterpret_cast<void **>(&s->ctl), sizeof(Ctl) });
  pc.push_back({ reinterpret_cast<void **>(&s->dt_bits), sizeof(unsigned long long) });
  if (!s->mixed) {
    Bufs3<double> &X = s->bd;
    P8(&X.coef, kNM3 * NV * N); P8(&X.FA, 4 * NV * F); P8(&X.FB, 4 * NV * F); P8(&X.rec, kRec * N);
    P8(&X.Flo, kLo * F); P8(&X.E0, kEu * F); P8(&X.E1, kEu * F); P8(&X.Rk, NV * N); P8(&X.invD, N);
    P8(&X.dU, kDU * N); P8(&X.lamS, kMaxFace3 * N);
  } else {
    Bufs3<float> &X = s->bf;
    P4(&X.W, NV * N); P4(&X.Wx, 3 * NV * N); P4(&X.Wn, NV * N); P4(&X.Ws, NV * N); P4(&X.Wxs, 3 * NV * N);
    P4(&X.coef, kNM3 * NV * N); P4(&X.FA, 4 * NV * F); P4(&X.FB, 4 * NV * F);
    P4(&X.rec, kRec * N); P4(&X.Flo, kLo * F); P4(&X.Rk, NV * N); P4(&X.invD, N);
    P4(&X.dU, kDU * N); P4(&X.lamS, kMaxFace3 * N);
    P4(&g.f_ivol, N); P4(&g.f_ih, N); P4(&g.f_m2, 6 * N); P4(&g.f_op, kNCol3 * kNM3 * N); P4(&g.f_fe, 9 * F);
    P4(&g.f_fS, F); P4(&g.f_fjump, F); P4(&g.f_fw, 4 * F); P4(&g.f_fxi, 24 * F); P4(&g.f_fidl, F); P4(&g.f_sn, 3 * kMaxFace3 * N);
    P4(&g.f_shs, kMaxFace3 * N); P4(&g.f_bcuw, 3 * CGKS_MAX_BC); P4(&g.f_bcrho, CGKS_MAX_BC);
    P4(&g.f_bcu, 3 * CGKS_MAX_BC); P4(&g.f_bcp, CGKS_MAX_BC);
  }
}

size_t total_of(const std::vector<Piece3> &pc) {
  size_t t = 0;
  for (auto &p : pc) t += (p.bytes + 255) & ~size_t(255);
  return t;
}

template <typename T>
void fill_params(const cgks_params &p, ParamsT<T> &P) {
  const double K = (5.0 - 3.0 * p.gamma) / (p.gamma - 1.0);
  P.gamma = static_cast<T>(p.gamma);
  P.K = static_cast<T>(K);
  P.cfl_hi = static_cast<T>(p.cfl_hi);
  P.cfl_lo = static_cast<T>(p.cfl_lo);
  P.mu = static_cast<T>(p.mu);
  P.kc.K = static_cast<T>(K);
  P.kc.c2K = static_cast<T>(2.0 / (K + 3.0));
  P.kc.c4K = static_cast<T>(4.0 / (K + 3.0));
  P.flux_lo = p.flux_lo;
  P.tau_c1 = static_cast<T>(p.tau_c1);
  P.tau_c2 = static_cast<T>(p.tau_c2);
  P.weno_eps = static_cast<T>(p.weno_eps);
  P.weno_g0 = static_cast<T>(p.weno_g0);
  P.lo_viscous = p.lo_viscous;
}

#define CK3(x)                                  \
  do {                                          \
    if ((x) != cudaSuccess) return CGKS_ECUDA;  \
  } while (0)

}  // namespace

Tuner *s3_tuner(Solver3 *s) { return &s->tune; }

int s3_set_tuning(Solver3 *s, const int *shape) {
  s->tune.set(shape);
  drop_graphs(s);
  return CGKS_OK;
}

size_t s3_footprint(int64_t n_cells, int64_t n_faces, bool mixed) {
  Solver3 tmp;
  tmp.N = n_cells;
  tmp.F = n_faces;
  tmp.mixed = mixed;
  std::vector<Piece3> pc;
  plan(&tmp, pc);
  return total_of(pc);
}

void s3_destroy(Solver3 *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  drop_graphs(s);
  free3(s->P, s->hist);
  free3(s->P, s->arena);
  delete s;
}

int s3_create(const HostMesh3 &m, const cgks_params *p, cudaStream_t stream, Timer *timer, Solver3 **out) {
  *out = nullptr;
  std::unique_ptr<Solver3> S(new (std::nothrow) Solver3());
  if (!S) return CGKS_ENOMEM;
  Solver3 *s = S.get();
  s->P = *p;
  s->N = m.n_cells;
  s->F = m.n_faces;
  s->mixed = p->precision == CGKS_MIXED;
  s->n_colours = m.n_colours;
  s->colour_start = m.colour_start;
  for (int64_t f = 0; f < m.n_faces; ++f) {
    if (m.fc1[f] >= 0) continue;
    s->bf_face.push_back(static_cast<int32_t>(f));
    s->bf_tag.push_back(-1 - m.fc1[f]);
    const int64_t nf = m.n_faces;
    const double geo[7] = { m.fxf[f], m.fxf[nf + f], m.fxf[2 * nf + f], m.fn[f], m.fn[nf + f], m.fn[2 * nf + f],
                            m.fS[f] };
    s->bf_geo.insert(s->bf_geo.end(), geo, geo + 7);
  }
  s->stream = stream;
  s->timer = timer;
  s->tune.on = p->autotune != 0;
  if (s->N * kNCol3 * kNM3 > INT32_MAX || s->F * 24 > INT32_MAX) return CGKS_EINVAL;
  {
    std::vector<int> seq;
    const int C = m.n_colours;
    for (int sw = 0; sw < p->n_sweeps; ++sw) {
      for (int c = 0; c < C; ++c) if (seq.empty() || seq.back() != c) seq.push_back(c);
      for (int c = C - 1; c >= 0; --c) if (seq.empty() || seq.back() != c) seq.push_back(c);
    }
    if (!seq.empty()) seq.erase(seq.begin());
    s->sweep_seq = seq;
  }
  std::vector<Piece3> pc;
  plan(s, pc);
  s->arena_bytes = total_of(pc);
  s->arena = alloc3(s->P, s->arena_bytes);
  if (!s->arena) return CGKS_ENOMEM;
  {
    char *cur = static_cast<char *>(s->arena);
    for (auto &q : pc) { *q.dst = cur; cur += (q.bytes + 255) & ~size_t(255); }
  }
  if (!s->mixed) {
    Bufs3<double> &X = s->bd;
    X.W = s->W; X.Wx = s->Wx; X.Wn = s->Wn; X.Ws = s->Ws; X.Wxs = s->Wxs; X.U = s->U;
  }
  // ---- host tables
  const int64_t N = s->N, F = s->F;
  std::vector<char> wall(CGKS_MAX_BC, 0);
  for (int t = 0; t < p->n_bc; ++t) wall[t] = p->bc[t].kind != CGKS_BC_FARFIELD;
  std::vector<double> op;
  std::vector<unsigned char> wenok;
  build_operator3(m, wall, op, &wenok);
  std::vector<double> ivol(N), ih(N), hdt(N), fe(9 * F), fjump(F), fidl(F), sn(3 * kMaxFace3 * N, 0.0), shs(kMaxFace3 * N, 0.0);
  for (int64_t i = 0; i < N; ++i) {
    ivol[i] = 1.0 / m.vol[i];
    ih[i] = 1.0 / m.h[i];
    hdt[i] = 3.0 * m.vol[i] / m.asum[i];
  }
  for (int64_t f = 0; f < F; ++f) {
    const double n[3] = { m.fn[f], m.fn[F + f], m.fn[2 * F + f] };
    // tangents: t1 = normalised (a x n), a the axis least aligned with n; t2 = n x t1
    int k = 0;
    for (int d = 1; d < 3; ++d) if (std::fabs(n[d]) < std::fabs(n[k])) k = d;
    double a[3] = { 0, 0, 0 };
    a[k] = 1.0;
    double t1[3] = { a[1] * n[2] - a[2] * n[1], a[2] * n[0] - a[0] * n[2], a[0] * n[1] - a[1] * n[0] };
    const double l = std::sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int d = 0; d < 3; ++d) t1[d] /= l;
    const double t2[3] = { n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0] };
    for (int d = 0; d < 3; ++d) { fe[d * F + f] = n[d]; fe[(3 + d) * F + f] = t1[d]; fe[(6 + d) * F + f] = t2[d]; }
    fjump[f] = m.fdelta[f] > 0.0 ? p->alpha / m.fdelta[f] : 0.0;
    fidl[f] = m.fdelta[f] > 0.0 ? 1.0 / m.fdelta[f] : 0.0;
  }
  for (int64_t i = 0; i < N; ++i)
    for (int sl = 0; sl < kMaxFace3; ++sl) {
      const int32_t fs = m.cface[sl * N + i];
      if (fs == kNoFace) continue;
      const int32_t f = fs >= 0 ? fs : ~fs;
      const double sg = fs >= 0 ? 1.0 : -1.0;
      for (int d = 0; d < 3; ++d) sn[(3 * sl + d) * N + i] = sg * m.fn[d * F + f];
      shs[sl * N + i] = 0.5 * m.fS[f];
    }
  std::vector<double> bcuw(3 * CGKS_MAX_BC, 0.0), bcrho(CGKS_MAX_BC, 1.0), bcu(3 * CGKS_MAX_BC, 0.0),
      bcp(CGKS_MAX_BC, 1.0);
  std::vector<int> bckind(CGKS_MAX_BC, CGKS_BC_SLIP);
  for (int t = 0; t < CGKS_MAX_BC; ++t) {
    const cgks_bc &b = p->bc[t];
    bckind[t] = t < p->n_bc ? b.kind : CGKS_BC_SLIP;
    for (int d = 0; d < 3; ++d) { bcuw[3 * t + d] = b.u_wall[d]; bcu[3 * t + d] = b.u[d]; }
    bcrho[t] = b.rho;
    bcp[t] = b.p;
  }
  std::vector<int> perm(m.perm.begin(), m.perm.end());
  Geo3 &g = s->g;
  bool ok = true;
  auto up = [&](void *dst, const void *src, size_t bytes) {
    if (ok) ok = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream) == cudaSuccess;
  };
  up(g.vol, m.vol.data(), 8 * N); up(g.ivol, ivol.data(), 8 * N); up(g.ih, ih.data(), 8 * N);
  up(g.hdt, hdt.data(), 8 * N); up(g.m2, m.m2.data(), 8 * 6 * N); up(g.op, op.data(), 8 * op.size());
  up(g.fe, fe.data(), 8 * fe.size()); up(g.fS, m.fS.data(), 8 * F); up(g.fjump, fjump.data(), 8 * F);
  up(g.fidl, fidl.data(), 8 * F);
  up(g.fw, m.fw.data(), 8 * 4 * F); up(g.fxi, m.fxi.data(), 8 * 24 * F); up(g.sn, sn.data(), 8 * sn.size());
  up(g.shs, shs.data(), 8 * shs.size()); up(g.bcuw, bcuw.data(), 8 * bcuw.size());
  up(g.bcrho, bcrho.data(), 8 * bcrho.size()); up(g.bcu, bcu.data(), 8 * bcu.size());
  up(g.bcp, bcp.data(), 8 * bcp.size()); up(g.fng, m.fng.data(), 4 * F); up(g.cface, m.cface.data(), 4 * kMaxFace3 * N);
  up(g.cnbr, m.cnbr.data(), 4 * kMaxFace3 * N); up(g.fc0, m.fc0.data(), 4 * F); up(g.fc1, m.fc1.data(), 4 * F);
  up(g.bckind, bckind.data(), 4 * bckind.size()); up(s->perm, perm.data(), 4 * N);
  up(g.wenok, wenok.data(), N);
  std::vector<std::vector<float>> keep;
  auto upf = [&](float *dst, const std::vector<double> &src) {
    keep.emplace_back(src.begin(), src.end());
    up(dst, keep.back().data(), 4 * keep.back().size());
  };
  if (s->mixed) {
    upf(g.f_ivol, ivol); upf(g.f_ih, ih); upf(g.f_m2, m.m2); upf(g.f_op, op); upf(g.f_fe, fe);
    upf(g.f_fS, m.fS); upf(g.f_fjump, fjump); upf(g.f_fidl, fidl); upf(g.f_fw, m.fw); upf(g.f_fxi, m.fxi); upf(g.f_sn, sn);
    upf(g.f_shs, shs); upf(g.f_bcuw, bcuw); upf(g.f_bcrho, bcrho); upf(g.f_bcu, bcu); upf(g.f_bcp, bcp);
  }
  if (ok) ok = cudaMemsetAsync(s->ctl, 0, sizeof(Ctl), stream) == cudaSuccess &&
               cudaMemsetAsync(s->status, 0, sizeof(int), stream) == cudaSuccess &&
               cudaMemsetAsync(s->Rp0, 0, sizeof(double) * NV * N, stream) == cudaSuccess &&
               cudaMemsetAsync(s->last, 0, sizeof(double) * 4, stream) == cudaSuccess &&
               (s->mixed ? cudaMemsetAsync(s->bf.dU, 0, sizeof(float) * kDU * N, stream)
                         : cudaMemsetAsync(s->bd.dU, 0, sizeof(double) * kDU * N, stream)) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(stream) == cudaSuccess;
  if (!ok) { s3_destroy(S.release()); return CGKS_ECUDA; }
  fill_params(*p, s->dp);
  fill_params(*p, s->fp);
  s->dp.bc_kind = g.bckind; s->dp.bc_uw = g.bcuw; s->dp.bc_rho = g.bcrho; s->dp.bc_u = g.bcu; s->dp.bc_p = g.bcp;
  s->fp.bc_kind = g.bckind; s->fp.bc_uw = g.f_bcuw; s->fp.bc_rho = g.f_bcrho; s->fp.bc_u = g.f_bcu;
  s->fp.bc_p = g.f_bcp;
  MeshT<double> &dm = s->dm;
  dm.nc = static_cast<int>(N); dm.nf = static_cast<int>(F);
  dm.vol = g.vol; dm.ivol = g.ivol; dm.ih = g.ih; dm.hdt = g.hdt; dm.m2 = g.m2; dm.op = g.op;
  dm.fe = g.fe; dm.fS = g.fS; dm.fjump = g.fjump; dm.fw = g.fw; dm.fxi = g.fxi; dm.sn = g.sn; dm.shs = g.shs;
  dm.fidl = g.fidl;
  dm.fng = g.fng; dm.cface = g.cface; dm.cnbr = g.cnbr; dm.fc0 = g.fc0; dm.fc1 = g.fc1;
  MeshT<float> &fm = s->fm;
  fm.nc = dm.nc; fm.nf = dm.nf;
  fm.vol = nullptr; fm.hdt = nullptr; fm.ivol = g.f_ivol; fm.ih = g.f_ih; fm.m2 = g.f_m2; fm.op = g.f_op;
  fm.fe = g.f_fe; fm.fS = g.f_fS; fm.fjump = g.f_fjump; fm.fw = g.f_fw; fm.fxi = g.f_fxi; fm.sn = g.f_sn;
  fm.fidl = g.f_fidl;
  fm.shs = g.f_shs; fm.fng = g.fng; fm.cface = g.cface; fm.cnbr = g.cnbr; fm.fc0 = g.fc0; fm.fc1 = g.fc1;
  *out = S.release();
  return CGKS_OK;
}

int s3_set_state(Solver3 *s, const double *W, const double *Wx, bool device) {
  const int64_t n = s->N;
  double *wa = s->stage, *wxa = s->stage + NV * n;
  const cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK3(cudaMemcpyAsync(wa, W, sizeof(double) * NV * n, kind, s->stream));
  if (Wx) CK3(cudaMemcpyAsync(wxa, Wx, sizeof(double) * 3 * NV * n, kind, s->stream));
  k_gather_state<<<nblk(n, kCellBlock), kCellBlock, 0, s->stream>>>(
      static_cast<int>(n), s->perm, wa, Wx ? wxa : nullptr, s->W, s->Wx, s->mixed ? s->bf.W : nullptr,
      s->mixed ? s->bf.Wx : nullptr);
  s->launches++;
  CK3(cudaGetLastError());
  CK3(cudaMemsetAsync(s->status, 0, sizeof(int), s->stream));
  return CGKS_OK;
}

int s3_get_state(Solver3 *s, double *W, double *Wx, bool device) {
  const int64_t n = s->N;
  double *wa = s->stage, *wxa = s->stage + NV * n;
  k_scatter_state<<<nblk(n, kCellBlock), kCellBlock, 0, s->stream>>>(static_cast<int>(n), s->perm, s->W, s->Wx, wa,
                                                                     wxa);
  s->launches++;
  CK3(cudaGetLastError());
  const cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (W) CK3(cudaMemcpyAsync(W, wa, sizeof(double) * NV * n, kind, s->stream));
  if (Wx) CK3(cudaMemcpyAsync(Wx, wxa, sizeof(double) * 3 * NV * n, kind, s->stream));
  if (!device) CK3(cudaStreamSynchronize(s->stream));
  return CGKS_OK;
}

int s3_highorder_step(Solver3 *s, double dt, double *dt_used, int *status) {
  CK3(cudaMemsetAsync(&s->ctl->res_ctr, 0, sizeof(int), s->stream));
  enqueue_step(s, dt);
  CK3(cudaGetLastError());
  Ctl c;
  unsigned long long bits = 0;
  int st = 0;
  CK3(cudaMemcpyAsync(&c, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  CK3(cudaMemcpyAsync(&bits, s->dt_bits, sizeof(bits), cudaMemcpyDeviceToHost, s->stream));
  CK3(cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK3(cudaStreamSynchronize(s->stream));
  if (dt_used) {
    double d;
    std::memcpy(&d, &bits, sizeof d);
    *dt_used = c.dt_fixed > 0.0 ? c.dt_fixed : s->P.cfl_hi * d;
  }
  *status = st;
  return CGKS_OK;
}

int s3_run(Solver3 *s, int n, bool cycle) {
  if (n <= 0) return CGKS_OK;
  if (n > s->hist_cap) {
    double *h = static_cast<double *>(alloc3(s->P, sizeof(double) * n));
    if (!h) return CGKS_ENOMEM;
    if (s->hist) { cudaStreamSynchronize(s->stream); free3(s->P, s->hist); }
    s->hist = h;
    s->hist_cap = n;
    drop_graphs(s);   // the graphs hold the old pointer
  }
  CK3(cudaMemsetAsync(&s->ctl->res_ctr, 0, sizeof(int), s->stream));
  const bool graph = s->P.use_graph && !(s->timer && s->timer->on);
  cudaGraphExec_t *ge = cycle ? &s->g_cycle : &s->g_step;
  int k = 0;
  if (s->tune.eager(cycle)) {
    for (; k < n && s->tune.eager(cycle); ++k) {
      s->tune.begin_unit();
      if (cycle) enqueue_cycle(s);
      else enqueue_step(s, -1.0);
      s->tune.end_unit(cycle);
    }
    if (s->tune.collect()) drop_graphs(s);
  }
  if (graph && k < n && !*ge) {
    const int rc = capture(s, cycle, ge);
    if (rc) return rc;
  }
  const long long per = count_launches(s, cycle);
  for (; k < n; ++k) {
    if (graph) { CK3(cudaGraphLaunch(*ge, s->stream)); s->launches += per; }
    else if (cycle) enqueue_cycle(s);
    else enqueue_step(s, -1.0);
  }
  CK3(cudaGetLastError());
  return CGKS_OK;
}

int s3_loworder_smooth(Solver3 *s) {
  CK3(cudaMemsetAsync(&s->ctl->res_ctr, 0, sizeof(int), s->stream));
  CK3(cudaMemcpyAsync(s->Wn, s->W, sizeof(double) * NV * s->N, cudaMemcpyDeviceToDevice, s->stream));
  if (s->mixed) { lo_solve<float>(s); prolong<float>(s); }
  else { lo_solve<double>(s); prolong<double>(s); }
  CK3(cudaGetLastError());
  return CGKS_OK;
}

int s3_status(Solver3 *s, int *status) {
  CK3(cudaMemcpyAsync(status, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK3(cudaStreamSynchronize(s->stream));
  return CGKS_OK;
}

int s3_history(Solver3 *s, double *res_hist, int n) {
  if (n <= 0 || !res_hist) return CGKS_OK;
  CK3(cudaMemcpyAsync(res_hist, s->hist, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  CK3(cudaStreamSynchronize(s->stream));
  return CGKS_OK;
}

int s3_residual(Solver3 *s, double *res, double *r_l2) {
  double last[3];
  CK3(cudaMemcpyAsync(last, s->last, sizeof(double) * 3, cudaMemcpyDeviceToHost, s->stream));
  std::vector<double> R;
  if (r_l2) {
    R.resize(NV * static_cast<size_t>(s->N));
    CK3(cudaMemcpyAsync(R.data(), s->Rp0, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, s->stream));
  }
  CK3(cudaStreamSynchronize(s->stream));
  if (res) *res = last[0];
  if (r_l2)
    for (int v = 0; v < NV; ++v) {
      double a = 0.0;
      for (int64_t i = 0; i < s->N; ++i) a += R[v * s->N + i] * R[v * s->N + i];
      r_l2[v] = std::sqrt(a);
    }
  return CGKS_OK;
}

template <typename TF>
int s3_wall_loads_t(Solver3 *s, int32_t tag, int64_t max_faces, int64_t *n_faces, double *x, double *nrm,
                    double *S, double *traction) {
  Bufs3<TF> &B = bufs<TF>(s);
  if (s->P.flux_hi == CGKS_FLUX_FULL) enqueue_dt(s, -1.0);   // the full flux integrates over a step
  hi_eval<TF>(s, B.W, B.Wx, B.FA);
  const int64_t F = s->F;
  // the face outputs, one run of kFO values per face: F0 is the first NV
  std::vector<TF> FO(static_cast<size_t>(kFO) * F);
  CK3(cudaMemcpyAsync(FO.data(), B.FA, sizeof(TF) * FO.size(), cudaMemcpyDeviceToHost, s->stream));
  CK3(cudaStreamSynchronize(s->stream));
  int64_t k = 0;
  for (size_t b = 0; b < s->bf_face.size(); ++b) {
    if (s->bf_tag[b] != tag) continue;
    if (k < max_faces) {
      const double *g = &s->bf_geo[7 * b];
      const int64_t f = s->bf_face[b];
      for (int a = 0; a < 3; ++a) {
        x[3 * k + a] = g[a];
        nrm[3 * k + a] = g[3 + a];
        traction[3 * k + a] = static_cast<double>(FO[static_cast<size_t>(f) * kFO + 1 + a]);
      }
      S[k] = g[6];
    }
    ++k;
  }
  *n_faces = k;
  return k <= max_faces ? CGKS_OK : CGKS_EINVAL;
}

int s3_wall_loads(Solver3 *s, int32_t tag, int64_t max_faces, int64_t *n_faces, double *x, double *nrm, double *S,
                  double *traction) {
  return s->mixed ? s3_wall_loads_t<float>(s, tag, max_faces, n_faces, x, nrm, S, traction)
                  : s3_wall_loads_t<double>(s, tag, max_faces, n_faces, x, nrm, S, traction);
}

int s3_get_rp0(Solver3 *s, double *Rp0) {
  const int64_t N = s->N;
  std::vector<double> R(NV * N);
  std::vector<int> perm(N);
  CK3(cudaMemcpyAsync(R.data(), s->Rp0, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, s->stream));
  CK3(cudaMemcpyAsync(perm.data(), s->perm, sizeof(int) * N, cudaMemcpyDeviceToHost, s->stream));
  CK3(cudaStreamSynchronize(s->stream));
  for (int64_t i = 0; i < N; ++i)
    for (int v = 0; v < NV; ++v) Rp0[NV * perm[i] + v] = R[v * N + i];
  return CGKS_OK;
}

long long s3_launches(const Solver3 *s) { return s->launches; }
int s3_launches_per_call(const Solver3 *s, bool cycle) { return static_cast<int>(count_launches(s, cycle)); }

}  // namespace cgks
