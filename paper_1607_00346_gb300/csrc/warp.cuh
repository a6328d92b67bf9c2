// Warp-wide column passes shared by the ID kernels: dot products, axpy and
// sums of squares over a row range, with UNR independent loads in flight per
// lane (the column passes are latency-bound otherwise).
#pragma once

#include "common.cuh"

namespace hif {

constexpr int UNR = 8;    // independent loads in flight per lane in the column passes

// sum_{r in [r0, r1)} a[r] b[r] over one warp (result in every lane)
template <typename T>
__device__ __forceinline__ T warp_dot(const T* __restrict__ a, const T* __restrict__ b, int r0,
                                      int r1, int lane) {
  T acc[4] = {T(0), T(0), T(0), T(0)};
  int r = r0 + lane;
  if (r + 32 * (UNR - 1) < r1) {
    // two chunks in flight: the next chunk's loads are issued before this
    // chunk's products wait on theirs
    T x[UNR], y[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      x[u] = a[r + 32 * u];
      y[u] = b[r + 32 * u];
    }
    r += 32 * UNR;
    for (; r + 32 * (UNR - 1) < r1; r += 32 * UNR) {
      T xn[UNR], yn[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        xn[u] = a[r + 32 * u];
        yn[u] = b[r + 32 * u];
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) acc[u & 3] = fma(x[u], y[u], acc[u & 3]);
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        x[u] = xn[u];
        y[u] = yn[u];
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) acc[u & 3] = fma(x[u], y[u], acc[u & 3]);
  }
  for (; r < r1; r += 32) acc[0] = fma(a[r], b[r], acc[0]);
  T s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// sum of squares (double) of a[r0:r1], one warp
template <typename T>
__device__ __forceinline__ double warp_sumsq(const T* __restrict__ a, int r0, int r1, int lane) {
  double acc[2] = {0.0, 0.0};
  int r = r0 + lane;
  for (; r + 32 * (UNR - 1) < r1; r += 32 * UNR) {
    T x[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) x[u] = a[r + 32 * u];
#pragma unroll
    for (int u = 0; u < UNR; ++u) acc[u & 1] += (double)x[u] * (double)x[u];
  }
  for (; r < r1; r += 32) acc[0] += (double)a[r] * (double)a[r];
  double s = acc[0] + acc[1];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}


// b[r] -= t a[r] for r in [r0, r1), one warp
template <typename T>
__device__ __forceinline__ void warp_axpy(T t, const T* __restrict__ a, T* __restrict__ b, int r0,
                                          int r1, int lane) {
  int r = r0 + lane;
  for (; r + 32 * (UNR - 1) < r1; r += 32 * UNR) {
    T x[UNR], y[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      x[u] = a[r + 32 * u];
      y[u] = b[r + 32 * u];
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) b[r + 32 * u] = fma(-t, x[u], y[u]);
  }
  for (; r < r1; r += 32) b[r] = fma(-t, a[r], b[r]);
}

}  // namespace hif
