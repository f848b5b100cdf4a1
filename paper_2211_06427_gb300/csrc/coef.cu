// "Input for sum factorization" (the I stage of Sec. 3.2 / Fig. 6): the coefficient c at
// every Gauss-superset point of the tensor grid (Sec. 2.2, last paragraph: the WQ and DWQ
// points are all drawn from this superset, so one evaluation serves every rule), and its
// gather onto the compact WQ grid used by the interior-row contraction.
#include "sfa_internal.cuh"

namespace {

__global__ void k_coef_1d_analytic(MeshView M, double* f1, double* f2) {
  // separable factors of c = 1 + 0.5 sin(2 pi x) cos(2 pi y) z
  const double twopi = 6.283185307179586476925;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < M.dir[0].nsup) f1[t] = sin(twopi * M.dir[0].t_sup[t]);
  if (t < M.dir[1].nsup) f2[t] = cos(twopi * M.dir[1].t_sup[t]);
}

__global__ void k_coef_grid_analytic(MeshView M, int kind, double c0, const double* f1, const double* f2, double* C,
                                     float* C32) {
  const int n1 = M.dir[0].nsup, n2 = M.dir[1].nsup, n3 = M.dir[2].nsup;
  int64_t N = (int64_t)n1 * n2 * n3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    int s1 = t % n1, s2 = (t / n1) % n2, s3 = (int)(t / ((int64_t)n1 * n2));
    const double v = kind == SFA_COEF_CONST ? c0 : 1.0 + 0.5 * f1[s1] * f2[s2] * M.dir[2].t_sup[s3];
    C[t] = v;
    C32[t] = (float)v;
  }
}

// B-spline coefficient field: three sum-factorised passes, one direction each.
// pass 1: T1[k3][k2][s1] = sum_a B1[s1][a] c[k3][k2][e(s1)+a]
__global__ void k_coef_pass1(MeshView M, const double* ck, double* T1) {
  const int p = M.p, q1 = p + 1;
  const Dir1D& D = M.dir[0];
  const int n1 = M.dir[0].n, n2 = M.dir[1].n, n3 = M.dir[2].n, s1n = D.nsup;
  int64_t N = (int64_t)s1n * n2 * n3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    int s1 = t % s1n;
    int64_t kk = t / s1n;  // k2 + n2 k3
    int e = s1 / q1;
    double acc = 0.0;
    for (int a = 0; a <= p; ++a) acc += D.B[s1 * q1 + a] * ck[(e + a) + (int64_t)n1 * kk];
    T1[t] = acc;
  }
}
// pass 2: T2[k3][s2][s1] = sum_a B2[s2][a] T1[k3][e(s2)+a][s1]
__global__ void k_coef_pass2(MeshView M, const double* T1, double* T2) {
  const int p = M.p, q1 = p + 1;
  const Dir1D& D = M.dir[1];
  const int s1n = M.dir[0].nsup, s2n = D.nsup, n2 = M.dir[1].n, n3 = M.dir[2].n;
  int64_t N = (int64_t)s1n * s2n * n3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    int s1 = t % s1n, s2 = (t / s1n) % s2n;
    int64_t k3 = t / ((int64_t)s1n * s2n);
    int e = s2 / q1;
    double acc = 0.0;
    for (int a = 0; a <= p; ++a) acc += D.B[s2 * q1 + a] * T1[s1 + (int64_t)s1n * ((e + a) + (int64_t)n2 * k3)];
    T2[t] = acc;
  }
}
// pass 3: C[s3][s2][s1] = sum_a B3[s3][a] T2[e(s3)+a][s2][s1]
__global__ void k_coef_pass3(MeshView M, const double* T2, double* C, float* C32) {
  const int p = M.p, q1 = p + 1;
  const Dir1D& D = M.dir[2];
  const int s1n = M.dir[0].nsup, s2n = M.dir[1].nsup, s3n = D.nsup;
  int64_t plane = (int64_t)s1n * s2n;
  int64_t N = plane * s3n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t s12 = t % plane;
    int s3 = (int)(t / plane);
    int e = s3 / q1;
    double acc = 0.0;
    for (int a = 0; a <= p; ++a) acc += D.B[s3 * q1 + a] * T2[s12 + plane * (e + a)];
    C[t] = acc;
    C32[t] = (float)acc;
  }
}

__global__ void k_coef_gather_wq(MeshView M, const double* Csup, double* Cwq, float* Cwq32) {
  const Dir1D &A = M.dir[0], &B = M.dir[1], &Cd = M.dir[2];
  int64_t N = (int64_t)A.nq * B.nq * Cd.nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    int q1 = t % A.nq, q2 = (t / A.nq) % B.nq, q3 = (int)(t / ((int64_t)A.nq * B.nq));
    double v = Csup[A.wq_idx[q1] + (int64_t)A.nsup * (B.wq_idx[q2] + (int64_t)B.nsup * Cd.wq_idx[q3])];
    Cwq[t] = v;
    Cwq32[t] = (float)v;
  }
}

}  // namespace

// scratch: T1 (nsup1 n2 n3) and T2 (nsup1 nsup2 n3) doubles, or the two 1D factor arrays.
// Csup32 is the float copy read by the float cut-row path.
cudaError_t launch_coef(const MeshView& M, int coef_kind, double c0, const double* ck, double* scratch1,
                        double* scratch2, double* Csup, float* Csup32, double* Cwq, float* Cwq32, cudaStream_t st) {
  if (coef_kind == SFA_COEF_BSPLINE) {
    k_coef_pass1<<<1216, 256, 0, st>>>(M, ck, scratch1);
    SFA_LAUNCHED(1);
    k_coef_pass2<<<1216, 256, 0, st>>>(M, scratch1, scratch2);
    SFA_LAUNCHED(1);
    k_coef_pass3<<<1216, 256, 0, st>>>(M, scratch2, Csup, Csup32);
    SFA_LAUNCHED(1);
  } else {
    int mx = M.dir[0].nsup > M.dir[1].nsup ? M.dir[0].nsup : M.dir[1].nsup;
    k_coef_1d_analytic<<<(mx + 255) / 256, 256, 0, st>>>(M, scratch1, scratch2);
    SFA_LAUNCHED(1);
    k_coef_grid_analytic<<<1216, 256, 0, st>>>(M, coef_kind, c0, scratch1, scratch2, Csup, Csup32);
    SFA_LAUNCHED(1);
  }
  k_coef_gather_wq<<<1216, 256, 0, st>>>(M, Csup, Cwq, Cwq32);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}
