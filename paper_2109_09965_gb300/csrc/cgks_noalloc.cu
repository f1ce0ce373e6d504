// Allocation-free variant of the density-residual reduction.
//
// cgks_density_residual_noalloc computes Res = sum|rho_new - rho_old| /
// sum rho_old from two caller-owned device states without allocating any
// device memory.  Its scratch (the per-block partial sums of the two-pass
// reduction) is a file-scope __device__ array of fixed size, so every GPU
// that loads libcgks holds these 64 KiB until the process exits.
//
// In host code the name g_partials is only a host-side stand-in for the
// device array: passing it to a kernel would fault or silently read the
// wrong memory.  The device address is obtained with cudaGetSymbolAddress
// while the calling context is current and cached per CUDA context (a
// device address is valid only in the context it was obtained in, and a
// process may drive one device through several contexts).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/cgks.h"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = 4096;                       // scratch capacity in blocks
constexpr int64_t kMaxCells = int64_t(kMaxBlocks) * kBlock;
constexpr int kMaxContexts = 64;

// [2 * kMaxBlocks] partial sums (numerator, denominator) of one call
__device__ __align__(256) double g_partials[2 * kMaxBlocks];

// cache of the array's address per CUDA context: (context handle, address)
std::mutex g_mu;
void *g_ctx[kMaxContexts] = { nullptr };
double *g_scratch[kMaxContexts] = { nullptr };
int g_n_ctx = 0;

// the driver's cuCtxGetCurrent, looked up through the runtime (no link
// against libcuda); the context handle is the cache key
using CtxGetCurrentFn = int (*)(void **);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  return fn;
}

__device__ __forceinline__ void warp_block_sum2(double a, double b, double *dst) {
  __shared__ double sa[kBlock / 32], sb[kBlock / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (warp == 0) {
    a = lane < kBlock / 32 ? sa[lane] : 0.0;
    b = lane < kBlock / 32 ? sb[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { dst[0] = a; dst[1] = b; }
  }
}

// pass 1: one partial pair per block, every block writes its slot
__global__ void __launch_bounds__(kBlock) k_res_partial(const double *__restrict__ w_new,
                                                        const double *__restrict__ w_old, int64_t n,
                                                        double *__restrict__ scratch) {
  const int64_t c = int64_t(blockIdx.x) * kBlock + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (c < n) {
    const double r_old = w_old[4 * c];
    num = fabs(w_new[4 * c] - r_old);
    den = r_old;
  }
  warp_block_sum2(num, den, &scratch[2 * blockIdx.x]);
}

// pass 2: fixed-order sum of the nblocks partials
__global__ void __launch_bounds__(kBlock) k_res_total(const double *__restrict__ scratch, int nblocks,
                                                      double *__restrict__ res) {
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += kBlock) { a += scratch[2 * k]; b += scratch[2 * k + 1]; }
  __shared__ double tot[2];
  warp_block_sum2(a, b, tot);
  __syncthreads();
  if (threadIdx.x == 0) *res = tot[0] / tot[1];
}

// Device address of g_partials in the calling thread's current context.
// The first call in a context makes the runtime initialise that context
// (if it is not yet) and looks the address up; later calls read the cache.
// Without a context handle, or once the cache is full, the address is
// looked up on every call instead (still no allocation).
int scratch_for_current_context(double **out) {
  void *ctx = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  if (get && get(&ctx) != 0) ctx = nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (ctx) {
    for (int k = 0; k < g_n_ctx; ++k)
      if (g_ctx[k] == ctx) { *out = g_scratch[k]; return CGKS_OK; }
  }
  // with no context current yet this also makes the device's primary
  // context current (the runtime's lazy initialisation)
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return CGKS_ECUDA;
  if (!ctx && get && get(&ctx) != 0) ctx = nullptr;
  if (ctx && g_n_ctx < kMaxContexts) {
    g_ctx[g_n_ctx] = ctx;
    g_scratch[g_n_ctx] = static_cast<double *>(p);
    ++g_n_ctx;
  }
  *out = static_cast<double *>(p);
  return CGKS_OK;
}

}  // namespace

extern "C" int cgks_density_residual_noalloc(const double *W_new_dev, const double *W_old_dev, int64_t n_cells,
                                             double *res_dev, void *stream) {
  if (!W_new_dev || !W_old_dev || !res_dev || n_cells <= 0) return CGKS_EINVAL;
  if (n_cells > kMaxCells) return CGKS_EINVAL;
  double *scratch = nullptr;
  int rc = scratch_for_current_context(&scratch);
  if (rc != CGKS_OK) return rc;
  const int nblocks = static_cast<int>((n_cells + kBlock - 1) / kBlock);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_res_partial<<<nblocks, kBlock, 0, st>>>(W_new_dev, W_old_dev, n_cells, scratch);
  k_res_total<<<1, kBlock, 0, st>>>(scratch, nblocks, res_dev);
  return cudaGetLastError() == cudaSuccess ? CGKS_OK : CGKS_ECUDA;
}
