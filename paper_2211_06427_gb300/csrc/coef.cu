// "Input for sum factorization" (the I stage of Sec. 3.2 / Fig. 6): the coefficient c at
// every Gauss-superset point of the tensor grid (Sec. 2.2, last paragraph: the WQ and DWQ
// points are all drawn from this superset, so one evaluation serves every rule), and its
// gather onto the compact WQ grid used by the interior-row contraction.
#include "sfa_internal.cuh"

namespace {

template <typename T>
__device__ __forceinline__ const T* basis(const Dir1D& D);
template <>
__device__ __forceinline__ const double* basis<double>(const Dir1D& D) { return D.B; }
template <>
__device__ __forceinline__ const float* basis<float>(const Dir1D& D) { return D.Bf; }

// Row-wise sweeps: one warp per grid row (the slower indices, decoded once), lanes along the
// contiguous first index.
#define SFA_ROWS(nrows)                                                                          \
  const int lane = threadIdx.x & 31;                                                             \
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;                      \
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;                                  \
  for (int64_t row = w0; row < (nrows); row += nwarp)

__global__ void k_coef_1d_analytic(MeshView M, double* f1, double* f2) {
  // separable factors of c = 1 + 0.5 sin(2 pi x) cos(2 pi y) z
  const double twopi = 6.283185307179586476925;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < M.dir[0].nsup) f1[t] = sin(twopi * M.dir[0].t_sup[t]);
  if (t < M.dir[1].nsup) f2[t] = cos(twopi * M.dir[1].t_sup[t]);
}

// rows (s2, s3); c0 or the analytic formula, evaluated in double
__global__ void k_coef_grid_analytic(MeshView M, int kind, double c0, const double* f1, const double* f2, double* C,
                                     float* C32) {
  const int n1 = M.dir[0].nsup, n2 = M.dir[1].nsup, n3 = M.dir[2].nsup;
  SFA_ROWS((int64_t)n2 * n3) {
    const int s2 = (int)(row % n2), s3 = (int)(row / n2);
    const double z = M.dir[2].t_sup[s3], f2v = f2[s2];
    const int64_t o = row * n1;
    for (int s1 = lane; s1 < n1; s1 += 32) {
      const double v = kind == SFA_COEF_CONST ? c0 : 1.0 + 0.5 * f1[s1] * f2v * z;
      if (C) C[o + s1] = v;
      C32[o + s1] = (float)v;
    }
  }
}

// B-spline coefficient field: three sum-factorised passes, one direction each.
// pass 1: T1[k3][k2][s1] = sum_a B1[s1][a] c[k3][k2][e(s1)+a]       rows (k2, k3)
template <typename T, int P>
__global__ void k_coef_pass1(MeshView M, const double* ck, T* T1) {
  constexpr int p = P, q1 = P + 1;
  const Dir1D& D = M.dir[0];
  const T* B = basis<T>(D);
  const int n1 = M.dir[0].n, n2 = M.dir[1].n, n3 = M.dir[2].n, s1n = D.nsup;
  SFA_ROWS((int64_t)n2 * n3) {
    const double* cr = ck + row * n1;
    T* out = T1 + row * s1n;
    for (int s1 = lane; s1 < s1n; s1 += 32) {
      const int e = s1 / q1;
      T acc = T(0);
#pragma unroll
      for (int a = 0; a <= p; ++a) acc += B[s1 * q1 + a] * (T)cr[e + a];
      out[s1] = acc;
    }
  }
}
// pass 2: T2[k3][s2][s1] = sum_a B2[s2][a] T1[k3][e(s2)+a][s1]       rows (s2, k3)
template <typename T, int P>
__global__ void k_coef_pass2(MeshView M, const T* T1, T* T2) {
  constexpr int p = P, q1 = P + 1;
  const Dir1D& D = M.dir[1];
  const T* B = basis<T>(D);
  const int s1n = M.dir[0].nsup, s2n = D.nsup, n2 = M.dir[1].n, n3 = M.dir[2].n;
  SFA_ROWS((int64_t)s2n * n3) {
    const int s2 = (int)(row % s2n);
    const int64_t k3 = row / s2n;
    const int e = s2 / q1;
    const T* in = T1 + (int64_t)s1n * ((int64_t)e + (int64_t)n2 * k3);
    T bw[P + 1];
#pragma unroll
    for (int a = 0; a <= p; ++a) bw[a] = B[s2 * q1 + a];
    T* out = T2 + row * s1n;
    if (sizeof(T) == 4 && (s1n & 3) == 0) {
      // float rows of a multiple of 4 values (16-byte aligned): four values per lane
      const float4* in4 = reinterpret_cast<const float4*>(in);
      float4* out4 = reinterpret_cast<float4*>(out);
      const int n4 = s1n >> 2;
      for (int s4 = lane; s4 < n4; s4 += 32) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int a = 0; a <= p; ++a) {
          const float4 v = in4[(int64_t)a * n4 + s4];
          const float w = (float)bw[a];
          acc.x += w * v.x, acc.y += w * v.y, acc.z += w * v.z, acc.w += w * v.w;
        }
        out4[s4] = acc;
      }
      continue;
    }
#pragma unroll 2
    for (int s1 = lane; s1 < s1n; s1 += 32) {
      T acc = T(0);
#pragma unroll
      for (int a = 0; a <= p; ++a) acc += bw[a] * in[(int64_t)a * s1n + s1];
      out[s1] = acc;
    }
  }
}
// pass 3: C[s3][s2][s1] = sum_a B3[s3][a] T2[e(s3)+a][s2][s1]        rows (s2, s3)
template <typename T, int P>
__global__ void k_coef_pass3(MeshView M, const T* T2, double* C, float* C32) {
  constexpr int p = P, q1 = P + 1;
  const Dir1D& D = M.dir[2];
  const T* B = basis<T>(D);
  const int s1n = M.dir[0].nsup, s2n = M.dir[1].nsup, s3n = D.nsup;
  const int64_t plane = (int64_t)s1n * s2n;
  SFA_ROWS((int64_t)s2n * s3n) {
    const int s2 = (int)(row % s2n), s3 = (int)(row / s2n);
    const int e = s3 / q1;
    const T* in = T2 + (int64_t)e * plane + (int64_t)s2 * s1n;
    T bw[P + 1];
#pragma unroll
    for (int a = 0; a <= p; ++a) bw[a] = B[s3 * q1 + a];
    const int64_t o = row * s1n;
    if (sizeof(T) == 4 && !C && (s1n & 3) == 0) {
      // float only, rows of a multiple of 4 values (16-byte aligned): four values per lane
      const float4* in4 = reinterpret_cast<const float4*>(in);
      float4* out4 = reinterpret_cast<float4*>(C32 + o);
      const int n4 = s1n >> 2;
      const int64_t plane4 = plane >> 2;
      for (int s4 = lane; s4 < n4; s4 += 32) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int a = 0; a <= p; ++a) {
          const float4 v = in4[(int64_t)a * plane4 + s4];
          const float w = (float)bw[a];
          acc.x += w * v.x, acc.y += w * v.y, acc.z += w * v.z, acc.w += w * v.w;
        }
        out4[s4] = acc;
      }
      continue;
    }
#pragma unroll 2
    for (int s1 = lane; s1 < s1n; s1 += 32) {
      T acc = T(0);
#pragma unroll
      for (int a = 0; a <= p; ++a) acc += bw[a] * in[(int64_t)a * plane + s1];
      if (C) C[o + s1] = (double)acc;
      C32[o + s1] = (float)acc;
    }
  }
}

// rows (q2, q3) of the WQ grid
__global__ void k_coef_gather_wq(MeshView M, const double* Csup, const float* Csup32, double* Cwq, float* Cwq32) {
  const Dir1D &A = M.dir[0], &B = M.dir[1], &Cd = M.dir[2];
  SFA_ROWS((int64_t)B.nq * Cd.nq) {
    const int q2 = (int)(row % B.nq), q3 = (int)(row / B.nq);
    const int64_t base = (int64_t)A.nsup * (B.wq_idx[q2] + (int64_t)B.nsup * Cd.wq_idx[q3]);
    const int64_t o = row * A.nq;
    for (int q1 = lane; q1 < A.nq; q1 += 32) {
      const int64_t src = base + A.wq_idx[q1];
      if (Csup) {
        const double v = Csup[src];
        Cwq[o + q1] = v;
        Cwq32[o + q1] = (float)v;
      } else {
        Cwq32[o + q1] = Csup32[src];
      }
    }
  }
}
#undef SFA_ROWS

}  // namespace

// scratch: T1 (nsup1 n2 n3) and T2 (nsup1 nsup2 n3) doubles (or floats), or the two 1D
// factor arrays.  With f64, the double grids Csup/Cwq and their float copies; otherwise only
// the float grids, computed in float (the float paths read nothing else).
cudaError_t launch_coef(const MeshView& M, int coef_kind, double c0, const double* ck, double* scratch1,
                        double* scratch2, double* Csup, float* Csup32, double* Cwq, float* Cwq32, bool f64,
                        cudaStream_t st) {
  if (coef_kind == SFA_COEF_BSPLINE) {
    switch (M.p) {
#define SFA_COEF_CASE(PP)                                                              \
  case PP:                                                                             \
    if (f64) {                                                                         \
      k_coef_pass1<double, PP><<<1216, 256, 0, st>>>(M, ck, scratch1);                 \
      k_coef_pass2<double, PP><<<1216, 256, 0, st>>>(M, scratch1, scratch2);           \
      k_coef_pass3<double, PP><<<1216, 256, 0, st>>>(M, scratch2, Csup, Csup32);       \
    } else {                                                                           \
      float* s1 = reinterpret_cast<float*>(scratch1);                                  \
      float* s2 = reinterpret_cast<float*>(scratch2);                                  \
      k_coef_pass1<float, PP><<<1216, 256, 0, st>>>(M, ck, s1);                        \
      k_coef_pass2<float, PP><<<1216, 256, 0, st>>>(M, s1, s2);                        \
      k_coef_pass3<float, PP><<<1216, 256, 0, st>>>(M, s2, nullptr, Csup32);           \
    }                                                                                  \
    break;
      SFA_COEF_CASE(2)
      SFA_COEF_CASE(3)
      SFA_COEF_CASE(4)
      SFA_COEF_CASE(5)
      SFA_COEF_CASE(6)
#undef SFA_COEF_CASE
      default:
        return cudaErrorInvalidValue;
    }
    SFA_LAUNCHED(3);
  } else {
    int mx = M.dir[0].nsup > M.dir[1].nsup ? M.dir[0].nsup : M.dir[1].nsup;
    k_coef_1d_analytic<<<(mx + 255) / 256, 256, 0, st>>>(M, scratch1, scratch2);
    SFA_LAUNCHED(1);
    k_coef_grid_analytic<<<1216, 256, 0, st>>>(M, coef_kind, c0, scratch1, scratch2, f64 ? Csup : nullptr, Csup32);
    SFA_LAUNCHED(1);
  }
  k_coef_gather_wq<<<1216, 256, 0, st>>>(M, f64 ? Csup : nullptr, Csup32, Cwq, Cwq32);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}
