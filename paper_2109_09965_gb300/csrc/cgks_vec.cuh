// Aligned vector loads and stores of runs of a cell's values (float4 in
// FP32, double2 in FP64): the 3-D low level keeps each cell's state and
// primitives in one 16-value record and its increment in one 8-value run,
// so a neighbour's data arrives in one or two cache sectors.
#pragma once

#include <cuda_runtime.h>

namespace cgks {

template <typename T> struct VecOf;
template <> struct VecOf<float> { using V = float4; static constexpr int W = 4; };
template <> struct VecOf<double> { using V = double2; static constexpr int W = 2; };

// N values from a 16-byte aligned address (N a multiple of the vector width)
template <typename T, int N>
__device__ __forceinline__ void vload(const T *__restrict__ p, T out[N]) {
  using V = typename VecOf<T>::V;
  constexpr int W = VecOf<T>::W;
  static_assert(N % W == 0, "whole vectors");
#pragma unroll
  for (int k = 0; k < N / W; ++k) {
    const V x = reinterpret_cast<const V *>(p)[k];
    const T *e = reinterpret_cast<const T *>(&x);
#pragma unroll
    for (int c = 0; c < W; ++c) out[k * W + c] = e[c];
  }
}

template <typename T, int N>
__device__ __forceinline__ void vstore(T *__restrict__ p, const T in[N]) {
  using V = typename VecOf<T>::V;
  constexpr int W = VecOf<T>::W;
  static_assert(N % W == 0, "whole vectors");
#pragma unroll
  for (int k = 0; k < N / W; ++k) {
    V x;
    T *e = reinterpret_cast<T *>(&x);
#pragma unroll
    for (int c = 0; c < W; ++c) e[c] = in[k * W + c];
    reinterpret_cast<V *>(p)[k] = x;
  }
}

}  // namespace cgks
