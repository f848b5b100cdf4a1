// Device helpers shared by the interior-row kernels: per-precision table accessors and the
// banded 1D contraction of a regular support (two WQ points in each of its p+1 elements).
#pragma once
#include "sfa_internal.cuh"

namespace {

template <typename R>
struct Tab;
template <>
struct Tab<double> {
  __device__ static const double* wb00(const Dir1D& D) { return D.WB00; }
  __device__ static const double* wb11(const Dir1D& D) { return D.WB11; }
};
template <>
struct Tab<float> {
  __device__ static const float* wb00(const Dir1D& D) { return D.WB00f; }
  __device__ static const float* wb11(const Dir1D& D) { return D.WB11f; }
};

// y[dj] = sum_q w[dj][q] x[q] over a regular support (band structure at compile time).
template <typename R, int P>
__device__ __forceinline__ void band_apply(const R (&w)[2 * P + 1][2 * P + 2], const R (&x)[2 * P + 2],
                                           R (&y)[2 * P + 1]) {
#pragma unroll
  for (int dj = 0; dj <= 2 * P; ++dj) {
    R s = R(0);
#pragma unroll
    for (int el = (dj - P > 0 ? dj - P : 0); el <= (dj < P ? dj : P); ++el) {
      s += w[dj][2 * el] * x[2 * el];
      s += w[dj][2 * el + 1] * x[2 * el + 1];
    }
    y[dj] = s;
  }
}

template <typename R, int P>
__device__ __forceinline__ void load_table(const R* src, int ld, R (&w)[2 * P + 1][2 * P + 2]) {
#pragma unroll
  for (int dj = 0; dj <= 2 * P; ++dj)
#pragma unroll
    for (int q = 0; q < 2 * P + 2; ++q) w[dj][q] = src[dj * ld + q];
}

}  // namespace
