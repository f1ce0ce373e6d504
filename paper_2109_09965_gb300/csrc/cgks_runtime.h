// Internal runtime pieces shared by the 2-D and 3-D device runtimes.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>
#include <vector>

#include "cgks_internal.h"
#include "cgks_shapes.h"

namespace cgks {

// kernel ids for the per-kernel timers
enum KernelId { KI_DT = 0, KI_RECON, KI_FACE, KI_UPDATE, KI_RESFIN, KI_LOFACE, KI_LORHS, KI_SWEEP, KI_LOCELL,
                KI_PROLONG, KI_LOSOLVE, KI_COUNT };
inline const char *kernel_name(int k) {
  static const char *names[KI_COUNT] = { "k_dt", "k_recon", "k_face", "k_update", "k_res_final", "k_lo_face",
                                         "k_lo_rhs", "k_sweep", "k_lo_cell", "k_prolong",
                                         "k_lo_solve" };
  return names[k];
}

// CUDA-event timer around every launch while on
struct Timer {
  bool on = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  double ms[KI_COUNT] = { 0 };
  long long cnt[KI_COUNT] = { 0 };
};

inline void collect_timing(Timer *t) {
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

// Launch a kernel on st; with pdl, as a programmatic dependent launch: the
// kernel may be scheduled while its predecessor on st still runs and orders
// itself after it on the device (every kernel launched this way calls
// pdl_enter() before touching global memory).
template <typename... Exp, typename... Act>
void launch_on(cudaStream_t st, bool pdl, void (*kern)(Exp...), dim3 grid, dim3 block, Act... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---- launch-shape autotuner ----
// Each tunable kernel's first kRounds x kNShape tuning units (eager cycles
// or explicit steps that launch it) use shape unit % kNShape; the first
// round only warms up (lazy module loading), the others are timed with CUDA
// events around each launch.  When a kernel's units are spent it keeps the
// shape of least mean launch time.  A unit runs eagerly (no graph) while a
// kernel that this kind of unit launched last time is still being tuned.
struct Tuner {
  static constexpr int kRounds = 3;
  bool on = false;
  int pick[TK_COUNT] = { kDefaultShape[0], kDefaultShape[1], kDefaultShape[2], kDefaultShape[3] };
  int unit[TK_COUNT] = { 0, 0, 0, 0 };
  bool used[TK_COUNT] = { false, false, false, false };
  bool seen[2][TK_COUNT] = { { true, true, true, true }, { true, true, true, true } };  // [cycle]
  bool in_unit = false;
  double ms[TK_COUNT][kNShape] = {};
  int cnt[TK_COUNT][kNShape] = {};
  struct Ev { int k, shape; cudaEvent_t e0, e1; };
  std::vector<Ev> ev;

  bool tuning(int k) const { return on && unit[k] < kRounds * kNShape; }
  int shape(int k) const { return tuning(k) ? unit[k] % kNShape : pick[k]; }
  bool timed(int k) const { return in_unit && tuning(k) && unit[k] >= kNShape; }
  // the next unit of this kind runs eagerly
  bool eager(bool cycle) const {
    for (int k = 0; k < TK_COUNT; ++k)
      if (seen[cycle][k] && tuning(k)) return true;
    return false;
  }
  void begin_unit() {
    in_unit = true;
    for (bool &u : used) u = false;
  }
  void end_unit(bool cycle) {
    in_unit = false;
    for (int k = 0; k < TK_COUNT; ++k) {
      seen[cycle][k] = used[k];
      if (used[k] && tuning(k)) ++unit[k];
    }
  }
  // read the pending events (synchronises on the last); kernels whose
  // units are spent take the fastest shape.  Returns true if a pick changed.
  bool collect() {
    for (auto &e : ev) {
      float t = 0.f;
      cudaEventSynchronize(e.e1);
      if (cudaEventElapsedTime(&t, e.e0, e.e1) == cudaSuccess) {
        ms[e.k][e.shape] += t;
        cnt[e.k][e.shape] += 1;
      }
      cudaEventDestroy(e.e0);
      cudaEventDestroy(e.e1);
    }
    ev.clear();
    bool changed = false;
    for (int k = 0; k < TK_COUNT; ++k) {
      if (!on || unit[k] != kRounds * kNShape || decided[k]) continue;
      decided[k] = true;
      int best = -1;
      double tb = 0.0;
      for (int s = 0; s < kNShape; ++s) {
        if (!cnt[k][s]) continue;
        const double t = ms[k][s] / cnt[k][s];
        if (best < 0 || t < tb) { best = s; tb = t; }
      }
      if (best < 0) continue;   // never timed: keep the default
      changed |= best != pick[k];
      pick[k] = best;
    }
    return changed;
  }
  // fix the shapes and end tuning
  void set(const int *shp) {
    for (int k = 0; k < TK_COUNT; ++k) { pick[k] = shp[k]; unit[k] = kRounds * kNShape; decided[k] = true; }
  }
  void report(cgks_tuning *t) const {
    for (int k = 0; k < TK_COUNT; ++k) {
      t->shape[k] = shape(k);
      t->done[k] = !tuning(k);
      for (int s = 0; s < kNShape; ++s) t->ms[k][s] = cnt[k][s] ? ms[k][s] / cnt[k][s] : 0.0;
    }
  }
  bool decided[TK_COUNT] = { false, false, false, false };
};

// launch kernel tk with a tuner's event pair around it while timed
template <typename Launch>
void tuned_launch(Tuner &tu, int tk, cudaStream_t st, Launch &&go) {
  const bool t = tu.timed(tk);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (t) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  go();
  if (t) {
    cudaEventRecord(e1, st);
    tu.ev.push_back({ tk, tu.shape(tk), e0, e1 });
  }
  tu.used[tk] = true;
}

// call f(std::integral_constant<int, s>) for the runtime shape index s
template <typename F>
void with_shape(int s, F &&f) {
  switch (s) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    default: f(std::integral_constant<int, 0>{}); break;
  }
}
static_assert(kNShape == 5, "with_shape covers every shape");

// ---- the 3-D solver (cgks_device3.cu) ----
struct Solver3;
int s3_create(const HostMesh3 &m, const cgks_params *p, cudaStream_t stream, Timer *timer, Solver3 **out);
void s3_destroy(Solver3 *s);
int s3_set_state(Solver3 *s, const double *W, const double *Wx, bool device);
int s3_get_state(Solver3 *s, double *W, double *Wx, bool device);
// explicit step with dt (<= 0: from CFL); dt_used / status read back (synchronises)
int s3_highorder_step(Solver3 *s, double dt, double *dt_used, int *status);
// n cycles (or explicit steps) without host synchronisation; history of Res
int s3_run(Solver3 *s, int n, bool cycle);
int s3_loworder_smooth(Solver3 *s);
int s3_status(Solver3 *s, int *status);
int s3_history(Solver3 *s, double *res_hist, int n);
int s3_residual(Solver3 *s, double *res, double *r_l2);
int s3_get_rp0(Solver3 *s, double *Rp0);
int s3_wall_loads(Solver3 *s, int32_t tag, int64_t max_faces, int64_t *n_faces, double *x, double *nrm, double *S,
                  double *traction);
long long s3_launches(const Solver3 *s);
int s3_launches_per_call(const Solver3 *s, bool cycle);
size_t s3_footprint(int64_t n_cells, int64_t n_faces, bool mixed);
Tuner *s3_tuner(Solver3 *s);
int s3_set_tuning(Solver3 *s, const int *shape);

}  // namespace cgks
