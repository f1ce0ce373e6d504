// Launch shapes of the tunable kernels (shared by the kernels and the
// runtimes).  A shape is (threads per block, items per thread, minimum
// resident blocks per SM).  An item is a cell or a face; for the colour
// sweeps, where a lane group serves one cell, it is a cell per lane group.
// Item k of thread t of block b is (b * ipt + k) * bs + t, so every item is
// computed by the same arithmetic whatever the shape: the shape changes only
// which thread does the work, never the result.
#pragma once

#include "../../include/cgks.h"
#ifdef __CUDACC__
#include "cgks_pdl.cuh"
#endif

namespace cgks {

constexpr int kNShape = CGKS_TUNE_SHAPES;

__host__ __device__ constexpr int shape_bs(int s) {
  return (s == 1 || s == 4) ? 64 : s == 2 ? 256 : 128;
}
__host__ __device__ constexpr int shape_ipt(int s) { return (s == 3 || s == 4) ? 2 : 1; }
// minimum resident blocks per SM (a register cap for the compiler); 1 = none.
// No shape caps registers: under a cap the compiler may fuse multiplies and
// adds differently, and a shape must never change a result.
__host__ __device__ constexpr int shape_minb(int) { return 1; }

// tunable kernels
enum TuneKernel { TK_RECON = 0, TK_FACE, TK_LOFACE, TK_SWEEP, TK_COUNT };
static_assert(TK_COUNT == CGKS_TUNE_KERNELS, "tunable kernel count");
// shapes used without the autotuner: 256-thread cell kernels, 128-thread
// face flux and sweeps
constexpr int kDefaultShape[TK_COUNT] = { 2, 0, 2, 0 };

#ifdef __CUDACC__
// the items of this thread in a launch of shape SH over n items
template <int SH, typename F>
__device__ __forceinline__ void for_items(const int n, F &&f) {
#pragma unroll 1
  for (int k = 0; k < shape_ipt(SH); ++k) {
    const int i = (static_cast<int>(blockIdx.x) * shape_ipt(SH) + k) * shape_bs(SH) + static_cast<int>(threadIdx.x);
    if (i < n) f(i);
  }
}

// The same, for a kernel launched as a programmatic dependent launch: geo(i)
// reads the item's mesh data (which no kernel of a cycle writes), then the
// thread waits for the predecessor kernel before f(i, g) touches anything
// else.  Every thread waits, so the grid completes only after its
// predecessor has.  One copy of the per-item code serves every shape.
template <int SH, typename G, typename F>
__device__ __forceinline__ void for_items_pdl(const int n, G &&geo, F &&f) {
#pragma unroll 1
  for (int k = 0; k < shape_ipt(SH); ++k) {
    const int i = (static_cast<int>(blockIdx.x) * shape_ipt(SH) + k) * shape_bs(SH) + static_cast<int>(threadIdx.x);
    if (i < n) {
      const auto g = geo(i);
      pdl_enter();
      f(i, g);
    }
  }
  pdl_enter();   // threads without items wait too: this grid ends after its predecessor
}
#endif

}  // namespace cgks
