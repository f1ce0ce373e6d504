// Internal runtime pieces shared by the 2-D and 3-D device runtimes.
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "cgks_internal.h"

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
long long s3_launches(const Solver3 *s);
int s3_launches_per_call(const Solver3 *s, bool cycle);
size_t s3_footprint(int64_t n_cells, int64_t n_faces, bool mixed);

}  // namespace cgks
