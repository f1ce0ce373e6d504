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
// wrong memory.  The device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/cgks.h"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = 4096;                       // scratch capacity in blocks
constexpr int64_t kMaxCells = int64_t(kMaxBlocks) * kBlock;
constexpr int kMaxDevices = 64;

// [2 * kMaxBlocks] partial sums (numerator, denominator) of one call
__device__ __align__(256) double g_partials[2 * kMaxBlocks];

std::mutex g_mu;
double *g_scratch[kMaxDevices] = { nullptr };

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

int scratch_for_current_device(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CGKS_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return CGKS_ECUDA;
    g_scratch[dev] = static_cast<double *>(p);
  }
  *out = g_scratch[dev];
  return CGKS_OK;
}

}  // namespace

extern "C" int cgks_density_residual_noalloc(const double *W_new_dev, const double *W_old_dev, int64_t n_cells,
                                             double *res_dev, void *stream) {
  if (!W_new_dev || !W_old_dev || !res_dev || n_cells <= 0) return CGKS_EINVAL;
  if (n_cells > kMaxCells) return CGKS_EINVAL;
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != CGKS_OK) return rc;
  const int nblocks = static_cast<int>((n_cells + kBlock - 1) / kBlock);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_res_partial<<<nblocks, kBlock, 0, st>>>(W_new_dev, W_old_dev, n_cells, scratch);
  k_res_total<<<1, kBlock, 0, st>>>(scratch, nblocks, res_dev);
  return cudaGetLastError() == cudaSuccess ? CGKS_OK : CGKS_ECUDA;
}
