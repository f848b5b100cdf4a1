// Helpers shared by the two cut-path translation units (cut_elem.cu: cut-element matrices;
// cut.cu: cut rows).  Not part of the ABI.
#pragma once
#include "sfa_internal.cuh"

namespace {

template <typename R>
struct CTab;
template <>
struct CTab<double> {
  __device__ static const double* wb(const Dir1D& D, int kk) { return kk ? D.WB11 : D.WB00; }
  __device__ static const double* wd(const Dir1D& D, int kk) { return kk ? D.WD11 : D.WD00; }
};
template <>
struct CTab<float> {
  __device__ static const float* wb(const Dir1D& D, int kk) { return kk ? D.WB11f : D.WB00f; }
  __device__ static const float* wd(const Dir1D& D, int kk) { return kk ? D.WD11f : D.WD00f; }
};

struct CoefDesc {
  int kind;
  double c0;
  const double* ck;  // B-spline coefficients (n1 n2 n3)
};

__device__ __forceinline__ int sel3(int d, int a, int b, int c) { return d == 0 ? a : (d == 1 ? b : c); }

constexpr int rup4(int x) { return (x + 3) / 4 * 4; }

// Vector of N consecutive entries from shared memory (16-byte reads; N a multiple of 4).
template <typename R, int N>
__device__ __forceinline__ void lds_vec(const R* __restrict__ src, R (&v)[N]) {
  if (sizeof(R) == 4) {
#pragma unroll
    for (int k = 0; k < N / 4; ++k) {
      const float4 t = reinterpret_cast<const float4*>(src)[k];
      v[4 * k] = t.x, v[4 * k + 1] = t.y, v[4 * k + 2] = t.z, v[4 * k + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const double2 t = reinterpret_cast<const double2*>(src)[k];
      v[2 * k] = t.x, v[2 * k + 1] = t.y;
    }
  }
}

// cp.async of one N-byte word (N = 4 or 8) into shared memory
template <int N>
__device__ __forceinline__ void cp_word(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(N) : "memory");
}
// the same without a memory clobber, for copies whose destination nothing touches before the
// next cp_wait (which has one) and barrier
template <int N>
__device__ __forceinline__ void cp_word_nc(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(N));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// d = a b + c on two float lanes at once (one f32x2 instruction; the pairs are packed and
// unpacked inside the asm, so no value changes type in C++)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

}  // namespace
