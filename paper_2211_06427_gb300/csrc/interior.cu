// Interior rows (Sec. 1: weighted quadrature + sum factorization + row assembly; Table 2,
// row loop / sum factorization): for every test function whose support holds only inside
// elements,
//   V[j3][j2][j1] = sum_q3 WB3[j3][q3] sum_q2 WB2[j2][q2] sum_q1 WB1[j1][q1] C[q1,q2,q3]
// with WB_d[dj][q] = w_{i_d}(q) B_{i_d - p + dj}(t_q) (stiffness: the three terms with the
// derivative rule in one direction).  A CTA takes T consecutive rows i1 of one (i2, i3)
// pencil: the contraction over q3 and q2 is shared by all of them, the contraction over q1
// is per row.  Values go straight into the CSR value array (each interior row's band is a
// contiguous, possibly face-clipped, box in [j3][j2][j1] order).
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

template <typename R, int P, bool STIFF>
__global__ void __launch_bounds__(256) k_interior(MeshView M, const R* __restrict__ Cwq, R* __restrict__ values,
                                                  int T, int L1MAX, int RB, int nchunks) {
  constexpr int NB = 2 * P + 1;
  constexpr int NQM = 4 * P;  // bound on WQ points in one support
  constexpr int NT = STIFF ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dir1D &D1 = M.dir[0], &D2 = M.dir[1], &D3 = M.dir[2];
  const int NQL1 = D1.nql, NQL2 = D2.nql, NQL3 = D3.nql;

  const int pencil = M.topo.int_tiles[blockIdx.x / nchunks];
  const int chunk = blockIdx.x % nchunks;
  const int i2 = pencil % D2.n, i3 = pencil / D2.n;
  const int i1a = chunk * T, i1b = min(D1.n, i1a + T);
  if (i1a >= D1.n) return;
  const int64_t rowbase = (int64_t)D1.n * (i2 + (int64_t)D2.n * i3);

  R* Cs = reinterpret_cast<R*>(smem_raw);                    // [a3][a2][a1], later output staging
  R* TB = Cs + (size_t)NQL3 * NQL2 * L1MAX;                   // [term][dj3][dj2][a1]
  R* W3 = TB + (size_t)NT * NB * NB * L1MAX;                  // [kk][dj][q]
  R* W2 = W3 + 2 * NB * NQL3;
  R* W1 = W2 + 2 * NB * NQL2;                                 // [kk][r][dj][q]
  int* rowflag = reinterpret_cast<int*>(W1 + 2 * (size_t)T * NB * NQL1);

  int any = 0;
  for (int r = threadIdx.x; r < T; r += blockDim.x) {
    int f = (i1a + r < i1b) && M.topo.fn_class[rowbase + i1a + r] == F_INT;
    rowflag[r] = f;
  }
  __syncthreads();
  for (int r = 0; r < i1b - i1a; ++r) any |= rowflag[r];
  if (!any) return;

  const int q2lo = D2.qlo[i2], nq2 = D2.nqi[i2];
  const int q3lo = D3.qlo[i3], nq3 = D3.nqi[i3];
  const int Q1lo = D1.qlo[i1a];
  const int L1 = D1.qlo[i1b - 1] + D1.nqi[i1b - 1] - Q1lo;

  // tables
  {
    const R* s3a = Tab<R>::wb00(D3) + (size_t)i3 * NB * NQL3;
    const R* s3b = Tab<R>::wb11(D3) + (size_t)i3 * NB * NQL3;
    const R* s2a = Tab<R>::wb00(D2) + (size_t)i2 * NB * NQL2;
    const R* s2b = Tab<R>::wb11(D2) + (size_t)i2 * NB * NQL2;
    for (int t = threadIdx.x; t < NB * NQL3; t += blockDim.x) {
      W3[t] = s3a[t];
      W3[NB * NQL3 + t] = STIFF ? s3b[t] : R(0);
    }
    for (int t = threadIdx.x; t < NB * NQL2; t += blockDim.x) {
      W2[t] = s2a[t];
      W2[NB * NQL2 + t] = STIFF ? s2b[t] : R(0);
    }
    const R* s1a = Tab<R>::wb00(D1) + (size_t)i1a * NB * NQL1;
    const R* s1b = Tab<R>::wb11(D1) + (size_t)i1a * NB * NQL1;
    const int n1tab = (i1b - i1a) * NB * NQL1;
    for (int t = threadIdx.x; t < n1tab; t += blockDim.x) {
      W1[t] = s1a[t];
      W1[(size_t)T * NB * NQL1 + t] = STIFF ? s1b[t] : R(0);
    }
  }
  // coefficient slab C[q1 in window][q2 in supp i2][q3 in supp i3]
  {
    const int64_t nq1g = D1.nq, nq2g = D2.nq;
    const int total = nq3 * nq2 * L1;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int a1 = t % L1, a2 = (t / L1) % nq2, a3 = t / (L1 * nq2);
      Cs[(a3 * nq2 + a2) * L1 + a1] = Cwq[(Q1lo + a1) + nq1g * ((q2lo + a2) + nq2g * (int64_t)(q3lo + a3))];
    }
  }
  __syncthreads();

  // stages A + B, one (a1, dj3) column per task: contract q3 then q2
  for (int task = threadIdx.x; task < L1 * NB; task += blockDim.x) {
    const int a1 = task % L1, dj3 = task / L1;
    R u00[NQM], u11[NQM];
#pragma unroll
    for (int a2 = 0; a2 < NQM; ++a2) {
      R s0 = R(0), s1 = R(0);
      if (a2 < nq2) {
        for (int a3 = 0; a3 < nq3; ++a3) {
          R c = Cs[(a3 * nq2 + a2) * L1 + a1];
          s0 += W3[dj3 * NQL3 + a3] * c;
          if (STIFF) s1 += W3[NB * NQL3 + dj3 * NQL3 + a3] * c;
        }
      }
      u00[a2] = s0;
      u11[a2] = s1;
    }
    for (int dj2 = 0; dj2 < NB; ++dj2) {
      R ta = R(0), tb = R(0);
#pragma unroll
      for (int a2 = 0; a2 < NQM; ++a2) {
        if (a2 < nq2) {
          R w0 = W2[dj2 * NQL2 + a2];
          if (STIFF) {
            R w1 = W2[NB * NQL2 + dj2 * NQL2 + a2];
            ta += w0 * u11[a2] + w1 * u00[a2];  // pairs with W1_00
            tb += w0 * u00[a2];                 // pairs with W1_11
          } else {
            ta += w0 * u00[a2];
          }
        }
      }
      TB[((0 * NB + dj3) * NB + dj2) * L1MAX + a1] = ta;
      if (STIFF) TB[((1 * NB + dj3) * NB + dj2) * L1MAX + a1] = tb;
    }
  }
  __syncthreads();

  // stage C per row, in batches of RB rows staged in the (now free) slab buffer
  R* Out = Cs;
  const int nrows = i1b - i1a;
  for (int rb0 = 0; rb0 < nrows; rb0 += RB) {
    const int rbn = min(RB, nrows - rb0);
    for (int task = threadIdx.x; task < rbn * NB * NB; task += blockDim.x) {
      const int rl = task / (NB * NB), rem = task % (NB * NB);
      const int dj3 = rem / NB, dj2 = rem % NB;
      const int r = rb0 + rl;
      if (!rowflag[r]) continue;
      const int i1 = i1a + r;
      const int off = D1.qlo[i1] - Q1lo, nq1 = D1.nqi[i1];
      R acc[NB];
#pragma unroll
      for (int k = 0; k < NB; ++k) acc[k] = R(0);
      const R* tba = TB + ((0 * NB + dj3) * NB + dj2) * L1MAX + off;
      const R* tbb = TB + ((1 * NB + dj3) * NB + dj2) * L1MAX + off;
      const R* w1a = W1 + (size_t)r * NB * NQL1;
      const R* w1b = W1 + (size_t)T * NB * NQL1 + (size_t)r * NB * NQL1;
#pragma unroll
      for (int ql = 0; ql < NQM; ++ql) {
        if (ql < nq1) {
          R x = tba[ql];
          R y = STIFF ? tbb[ql] : R(0);
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            acc[k] += w1a[k * NQL1 + ql] * x;
            if (STIFF) acc[k] += w1b[k * NQL1 + ql] * y;
          }
        }
      }
      R* o = Out + (size_t)rl * NB * NB * NB + (dj3 * NB + dj2) * NB;
#pragma unroll
      for (int k = 0; k < NB; ++k) o[k] = acc[k];
    }
    __syncthreads();
    // coalesced write of the (clipped) band of each row
    for (int rl = 0; rl < rbn; ++rl) {
      const int r = rb0 + rl;
      if (!rowflag[r]) continue;
      const int i1 = i1a + r;
      const int lo1 = max(0, P - i1), lo2 = max(0, P - i2), lo3 = max(0, P - i3);
      const int w1 = min(D1.n - 1, i1 + P) - (i1 - P + lo1) + 1;
      const int w2 = min(D2.n - 1, i2 + P) - (i2 - P + lo2) + 1;
      const int w3 = min(D3.n - 1, i3 + P) - (i3 - P + lo3) + 1;
      const int len = w1 * w2 * w3;
      R* dst = values + M.topo.rowptr[rowbase + i1];
      const R* src = Out + (size_t)rl * NB * NB * NB;
      for (int t = threadIdx.x; t < len; t += blockDim.x) {
        int c1 = t % w1, c2 = (t / w1) % w2, c3 = t / (w1 * w2);
        dst[t] = src[((lo3 + c3) * NB + (lo2 + c2)) * NB + (lo1 + c1)];
      }
    }
    __syncthreads();
  }
}

template <typename R, int P, bool STIFF>
cudaError_t launch_interior_t(const MeshView& M, const R* Cwq, R* values, int n_pencils, int T, int L1MAX,
                              cudaStream_t st) {
  constexpr int NB = 2 * P + 1;
  const int NT = STIFF ? 2 : 1;
  const int NQL1 = M.dir[0].nql, NQL2 = M.dir[1].nql, NQL3 = M.dir[2].nql;
  int slab = NQL3 * NQL2 * L1MAX;
  int RB = slab / (NB * NB * NB);
  if (RB < 1) return cudaErrorInvalidValue;
  if (RB > T) RB = T;
  size_t elems = (size_t)slab + (size_t)NT * NB * NB * L1MAX + 2 * NB * (NQL3 + NQL2) + 2 * (size_t)T * NB * NQL1;
  size_t smem = elems * sizeof(R) + T * sizeof(int) + 16;
  cudaError_t e = cudaFuncSetAttribute(k_interior<R, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nchunks = (M.dir[0].n + T - 1) / T;
  int64_t grid = (int64_t)n_pencils * nchunks;
  if (grid == 0) return cudaSuccess;
  k_interior<R, P, STIFF><<<(unsigned)grid, 256, smem, st>>>(M, Cwq, values, T, L1MAX, RB, nchunks);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

// Shared-memory bytes the interior kernel needs for chunk length T (host-side sizing).
size_t interior_smem_bytes(int p, int nql1, int nql2, int nql3, int T, int L1MAX, bool stiff, bool fp64) {
  int NB = 2 * p + 1;
  size_t elems = (size_t)nql3 * nql2 * L1MAX + (size_t)(stiff ? 2 : 1) * NB * NB * L1MAX + 2 * NB * (nql3 + nql2) +
                 2 * (size_t)T * NB * nql1;
  return elems * (fp64 ? 8 : 4) + T * sizeof(int) + 16;
}

cudaError_t launch_interior(const MeshView& M, bool fp64, bool stiff, const void* Cwq, void* values, int n_pencils,
                            int T, int L1MAX, cudaStream_t st) {
#define SFA_INT_CASE(PP)                                                                                   \
  case PP:                                                                                                 \
    if (fp64)                                                                                              \
      return stiff ? launch_interior_t<double, PP, true>(M, (const double*)Cwq, (double*)values, n_pencils, T, L1MAX, st) \
                   : launch_interior_t<double, PP, false>(M, (const double*)Cwq, (double*)values, n_pencils, T, L1MAX, st); \
    return stiff ? launch_interior_t<float, PP, true>(M, (const float*)Cwq, (float*)values, n_pencils, T, L1MAX, st)       \
                 : launch_interior_t<float, PP, false>(M, (const float*)Cwq, (float*)values, n_pencils, T, L1MAX, st);
  switch (M.p) {
    SFA_INT_CASE(2)
    SFA_INT_CASE(3)
    SFA_INT_CASE(4)
    SFA_INT_CASE(5)
    SFA_INT_CASE(6)
  }
#undef SFA_INT_CASE
  return cudaErrorInvalidValue;
}
