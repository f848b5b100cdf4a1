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

// The coefficient slab of a pencil: Cs[row * ld + a1] = C[q1lo + a1, q2lo + a2, q3lo + a3]
// with row = a3 nq2 + a2 < nrows and a1 < L1.  A warp takes UR rows and 64 points a1 at a
// time; every lane issues its 2 UR loads before the first store.
template <typename R, int UR>
__device__ __forceinline__ void load_slab(const R* __restrict__ Cwq, int64_t nq1g, int64_t nq2g, int q1lo, int q2lo,
                                          int q3lo, int nq2, int nrows, int L1, R* __restrict__ Cs, int ld) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r0 = warp * UR; r0 < nrows; r0 += nw * UR)
    for (int a0 = 0; a0 < L1; a0 += 64) {
      R v[UR][2];
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int r = r0 + u, a3 = r / nq2, a2 = r - a3 * nq2;
        const R* src = Cwq + (q1lo + a0 + lane) + nq1g * ((q2lo + a2) + nq2g * (int64_t)(q3lo + a3));
#pragma unroll
        for (int h = 0; h < 2; ++h) v[u][h] = (r < nrows && a0 + lane + 32 * h < L1) ? __ldg(src + 32 * h) : R(0);
      }
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int r = r0 + u;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (r < nrows && a0 + lane + 32 * h < L1) Cs[(size_t)r * ld + a0 + lane + 32 * h] = v[u][h];
      }
    }
}

}  // namespace
