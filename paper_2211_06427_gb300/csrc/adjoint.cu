// Reductions over formed matrices: J = lambda^T A u, and the adjoint dJ/dc with respect to
// the B-spline coefficients of the coefficient field.
//
// Every entry of A is a quadrature sum linear in c: A_ij = sum_x omega_i(x) c(x) Phi_j(x),
// with omega_i the test-function-folded weight of row i at point x.  With U = sum_j u_j B_j
// (every trial function that is nonzero at a quadrature point of row i lies in row i's
// pattern), J = sum_x c(x) Omega(x) U(x) where Omega(x) = sum_i lambda_i omega_i(x), and
//   dJ/dc_k = sum_x N_k(x) Omega(x) U(x)
// (stiffness: sum over d of Omega_d(x) dU/dx_d(x), Omega_d with the derivative rule in d).
// All WQ, DWQ and element Gauss points are Gauss-superset points, so Omega lives on the
// superset grid: interior rows contribute by three transposed passes over their WQ weights,
// DWQ boxes by a scatter, inside elements outside a box element by element; cut-element
// pieces are handled per element with their own Gauss points.
#include <algorithm>

#include "sfa_internal.cuh"

namespace {

// ---------------------------------------------------------------------------------------
// J = lambda^T A u: one warp per row, per-block partials, fixed-order final sum.
template <typename R>
__global__ void k_bilinear(const int64_t* rowptr, const int32_t* colind, int64_t nrows, const R* values,
                           const double* lam, const double* u, double* partial) {
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < nrows; i += (int64_t)gridDim.x * nw) {
    const int64_t a = rowptr[i], b = rowptr[i + 1];
    if (a == b) continue;
    double s = 0.0;
    for (int64_t k = a + lane; k < b; k += 32) s += (double)values[k] * u[colind[k]];
    acc += lam[i] * s;
  }
  acc = warp_sum(acc);
  if (lane == 0) ws[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_sum(const double* partial, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < n; ++k) t += partial[k];
    *out = t;
  }
}

// ---------------------------------------------------------------------------------------
// One-direction linear maps on 3D tensors (x1 fastest).
//   mode 0: coefficients -> superset points, out[s] = sum_a F[s][a] in[e(s)+a]   (F = B or dB)
//   mode 1: superset points -> coefficients, out[k] = sum_{s in supp N_k} B[s][k-e(s)] in[s]
//   mode 2: rows -> superset points with WQ weights, out[s] = sum_i w_i(s) in[i]
__device__ __forceinline__ int wq_of_sup(int s, int n_el, int p) {
  const int q1 = p + 1, e = s / q1, g = s % q1;
  int first = e == 0 ? 0 : (e < n_el - 1 ? q1 + 2 * (e - 1) : q1 + 2 * (n_el - 2));
  if (e == 0 || e == n_el - 1) return first + g;
  if (g == 0) return first;
  if (g == p) return first + 1;
  return -1;
}

__global__ void k_pass(MeshView M, int d, int mode, int kind, const double* __restrict__ in, double* __restrict__ out,
                       int64_t o0, int64_t o1, int64_t o2, int64_t i0, int64_t i1, int64_t i2) {
  const int p = M.p, q1 = p + 1;
  const Dir1D& D = M.dir[d];
  const int64_t N = o0 * o1 * o2;
  const int64_t ostr[3] = {1, o0, o0 * o1};
  const int64_t istr[3] = {1, i0, i0 * i1};
  const int64_t odim[3] = {o0, o1, o2};
  (void)i2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t c[3] = {t % o0, (t / o0) % o1, t / (o0 * o1)};
    const int64_t od = c[d];
    int64_t base = 0;
    for (int k = 0; k < 3; ++k)
      if (k != d) base += c[k] * istr[k];
    (void)ostr;
    (void)odim;
    double acc = 0.0;
    if (mode == 0) {
      const int s = (int)od, e = s / q1;
      const double* F = kind ? D.dB : D.B;
      for (int a = 0; a <= p; ++a) acc += F[s * q1 + a] * in[base + (e + a) * istr[d]];
    } else if (mode == 1) {
      const int k = (int)od;
      for (int e = max(0, k - p); e <= min(D.n_el - 1, k); ++e)
        for (int g = 0; g < q1; ++g) {
          const int s = e * q1 + g;
          acc += D.B[s * q1 + (k - e)] * in[base + s * istr[d]];
        }
    } else {
      const int s = (int)od, e = s / q1;
      const int q = wq_of_sup(s, D.n_el, p);
      if (q >= 0) {
        const double* W = kind ? D.w11 : D.w00;
        for (int a = 0; a <= p; ++a) {
          const int i = e + a;
          if (i >= D.n) break;
          const int ql = q - D.qlo[i];
          if (ql >= 0 && ql < D.nqi[i]) acc += W[(size_t)i * D.nql + ql] * in[base + i * istr[d]];
        }
      }
    }
    out[t] = acc;
  }
}

__global__ void k_mask_interior(const int8_t* fcls, const double* lam, int64_t n, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fcls[i] == F_INT ? lam[i] : 0.0;
}

// DWQ boxes: Omega_t(s) += lambda_i W_i^(t)(s) over the box grid of every box row.
__global__ void k_box_scatter(MeshView M, const double* lam, double* Om0, double* Om1, double* Om2, int stiff) {
  const int p = M.p, q1 = p + 1;
  const int row = M.topo.cut_rows[blockIdx.x];
  const int32_t bcode = M.topo.box[row];
  if (bcode < 0) return;
  const int bd = bcode & 3, bside = (bcode >> 2) & 1, bb = bcode >> 3;
  const int n1 = M.dir[0].n, n2 = M.dir[1].n;
  const int ii[3] = {row % n1, (row / n1) % n2, row / (n1 * n2)};
  int m[3], s0[3], sl0[3], rule = 0;
  for (int d = 0; d < 3; ++d) {
    const Dir1D& D = M.dir[d];
    const int e_lo = max(0, ii[d] - p), e_hi = min(D.n_el - 1, ii[d]);
    if (d == bd) {
      const int ka = bside == 0 ? e_lo : bb, kb = bside == 0 ? bb - 1 : e_hi;
      m[d] = (kb - ka + 1) * q1;
      s0[d] = ka * q1;
      sl0[d] = (ka - e_lo) * q1;
      rule = ((ii[d] * p) + (bb - e_lo - 1)) * 2 + bside;
    } else {
      m[d] = D.nqi[ii[d]];
      s0[d] = D.qlo[ii[d]];
      sl0[d] = 0;
    }
  }
  const double li = lam[row];
  const int64_t ns1 = M.dir[0].nsup, ns2 = M.dir[1].nsup;
  const int total = m[0] * m[1] * m[2];
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int mm[3] = {t % m[0], (t / m[0]) % m[1], t / (m[0] * m[1])};
    int s[3];
    double w0[3], w1[3];
    for (int d = 0; d < 3; ++d) {
      const Dir1D& D = M.dir[d];
      if (d == bd) {
        s[d] = s0[d] + mm[d];
        w0[d] = D.dwq00[(size_t)rule * D.nsl + sl0[d] + mm[d]];
        w1[d] = D.dwq11[(size_t)rule * D.nsl + sl0[d] + mm[d]];
      } else {
        s[d] = D.wq_idx[s0[d] + mm[d]];
        w0[d] = D.w00[(size_t)ii[d] * D.nql + mm[d]];
        w1[d] = D.w11[(size_t)ii[d] * D.nql + mm[d]];
      }
    }
    const int64_t si = s[0] + ns1 * (s[1] + ns2 * s[2]);
    if (!stiff) {
      atomicAdd(&Om0[si], li * w0[0] * w0[1] * w0[2]);
    } else {
      atomicAdd(&Om0[si], li * w1[0] * w0[1] * w0[2]);
      atomicAdd(&Om1[si], li * w0[0] * w1[1] * w0[2]);
      atomicAdd(&Om2[si], li * w0[0] * w0[1] * w1[2]);
    }
  }
}

// Inside elements integrated with element Gauss points by some cut row (outside its box):
// Omega_t(s) += w_s sum_{i in R_e} lambda_i Phi_i^(t)(x_s).  One warp per element; every
// superset point belongs to exactly one element, so plain adds suffice.
__global__ void k_gauss_elems(MeshView M, const double* lam, double* Om0, double* Om1, double* Om2, int stiff) {
  const int p = M.p, q1 = p + 1, Q3 = q1 * q1 * q1;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int ne1 = M.dir[0].n_el, ne2 = M.dir[1].n_el, ne3 = M.dir[2].n_el;
  const int n1 = M.dir[0].n, n2 = M.dir[1].n;
  const int64_t nE = (int64_t)ne1 * ne2 * ne3;
  const int64_t ns1 = M.dir[0].nsup, ns2 = M.dir[1].nsup;
  for (int64_t e = warp; e < nE; e += nw) {
    if (M.topo.elem_state[e] != E_IN) continue;
    const int ev[3] = {(int)(e % ne1), (int)((e / ne1) % ne2), (int)(e / ((int64_t)ne1 * ne2))};
    // rows of this element's local functions that integrate it with Gauss points
    double lt[(SFA_MAXP + 1) * (SFA_MAXP + 1) * (SFA_MAXP + 1)];
    bool any = false;
    for (int a = 0; a < Q3; ++a) {
      const int a1 = a % q1, a2 = (a / q1) % q1, a3 = a / (q1 * q1);
      const int i1 = ev[0] + a1, i2 = ev[1] + a2, i3 = ev[2] + a3;
      const int64_t i = i1 + (int64_t)n1 * (i2 + (int64_t)n2 * i3);
      double v = 0.0;
      if (M.topo.fn_class[i] == F_CUT) {
        const int32_t bc = M.topo.box[i];
        bool in_box = false;
        if (bc >= 0) {
          const int bd = bc & 3, bs = (bc >> 2) & 1, bb = bc >> 3;
          in_box = bs == 0 ? ev[bd] < bb : ev[bd] >= bb;
        }
        if (!in_box) v = lam[i];
      }
      lt[a] = v;
      any = any || v != 0.0;
    }
    if (!any) continue;
    const int nterm = stiff ? 3 : 1;
    for (int g = lane; g < Q3; g += 32) {
      const int g1 = g % q1, g2 = (g / q1) % q1, g3 = g / (q1 * q1);
      const int s[3] = {ev[0] * q1 + g1, ev[1] * q1 + g2, ev[2] * q1 + g3};
      const double w = M.dir[0].w_sup[s[0]] * M.dir[1].w_sup[s[1]] * M.dir[2].w_sup[s[2]];
      const int64_t si = s[0] + ns1 * (s[1] + ns2 * s[2]);
      for (int tm = 0; tm < nterm; ++tm) {
        double acc = 0.0;
        for (int a = 0; a < Q3; ++a) {
          if (lt[a] == 0.0) continue;
          const int a1 = a % q1, a2 = (a / q1) % q1, a3 = a / (q1 * q1);
          const double f1 = (stiff && tm == 0 ? M.dir[0].dB : M.dir[0].B)[s[0] * q1 + a1];
          const double f2 = (stiff && tm == 1 ? M.dir[1].dB : M.dir[1].B)[s[1] * q1 + a2];
          const double f3 = (stiff && tm == 2 ? M.dir[2].dB : M.dir[2].B)[s[2] * q1 + a3];
          acc += lt[a] * f1 * f2 * f3;
        }
        double* Om = tm == 0 ? Om0 : (tm == 1 ? Om1 : Om2);
        Om[si] += w * acc;
      }
    }
  }
}

__global__ void k_combine(int64_t n, const double* Om0, const double* Om1, const double* Om2, const double* U0,
                          const double* U1, const double* U2, int stiff, double* G) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    G[t] = stiff ? Om0[t] * U0[t] + Om1[t] * U1[t] + Om2[t] * U2[t] : Om0[t] * U0[t];
}

// Cut elements: for every piece Gauss point, w_g Lambda(x_g) U(x_g) (stiffness: the dot
// product of the gradients) times N_k(x_g) into the element's (p+1)^3 coefficients, with
// Lambda = sum_a lambda_{e+a} B_{e+a} over the element's local functions.
__global__ void k_cut_adjoint(MeshView M, LevelSet L, const double* lam, const double* u, double* grad, int stiff) {
  const int p = M.p, q1 = p + 1, Q3 = q1 * q1 * q1;
  const int ci = blockIdx.x;
  const int e = M.topo.cut_elems[ci];
  if (M.topo.elem_state[e] != E_CUT) return;
  const int ne1 = M.dir[0].n_el, ne2 = M.dir[1].n_el;
  const int ee[3] = {e % ne1, (e / ne1) % ne2, e / (ne1 * ne2)};
  const int n1 = M.dir[0].n, n2 = M.dir[1].n;
  __shared__ double ll[343], uu[343], gacc[343];
  for (int a = threadIdx.x; a < Q3; a += blockDim.x) {
    const int a1 = a % q1, a2 = (a / q1) % q1, a3 = a / (q1 * q1);
    const int64_t i = (ee[0] + a1) + (int64_t)n1 * ((ee[1] + a2) + (int64_t)n2 * (ee[2] + a3));
    ll[a] = lam[i];
    uu[a] = u[i];
    gacc[a] = 0.0;
  }
  __syncthreads();
  const int pbeg = M.topo.piece_ptr[ci], pend = M.topo.piece_ptr[ci + 1];
  const double* gx = M.gl;
  const double* gw = M.gl + q1;
  // thread per (piece, point); per-thread contributions accumulated in shared memory with
  // atomics (order-dependent rounding only)
  const int64_t total = (int64_t)(pend - pbeg) * Q3;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int pc = pbeg + (int)(t / Q3), g = (int)(t % Q3);
    const uint32_t code = M.topo.pieces[pc];
    const int lev = code & 15;
    const int av[3] = {(int)((code >> 4) & 63), (int)((code >> 10) & 63), (int)((code >> 16) & 63)};
    const int gg[3] = {g % q1, (g / q1) % q1, g / (q1 * q1)};
    double N[3][SFA_MAXP + 1], dN[3][SFA_MAXP + 1], w = 1.0;
    for (int d = 0; d < 3; ++d) {
      const int64_t sx = 1ll << (M.D + 1 - lev);
      const int64_t gi = ((int64_t)ee[d] << lev) + av[d];
      const double a = ls_coord(L, d, gi * sx), b = ls_coord(L, d, (gi + 1) * sx);
      const double x = 0.5 * (a + b) + 0.5 * (b - a) * gx[gg[d]];
      w *= 0.5 * (b - a) * gw[gg[d]];
      struct Kn {
        const double* xb; int p, n_el;
        __device__ double operator()(int k) const { int bb = k - p; bb = bb < 0 ? 0 : (bb > n_el ? n_el : bb); return xb[bb]; }
      } kn{M.dir[d].xb, p, M.dir[d].n_el};
      bspline_eval(kn, p, ee[d] + p, x, N[d], dN[d]);
    }
    double F = 0.0;
    const int nterm = stiff ? 3 : 1;
    for (int tm = 0; tm < nterm; ++tm) {
      double Lv = 0.0, Uv = 0.0;
      for (int a = 0; a < Q3; ++a) {
        const int a1 = a % q1, a2 = (a / q1) % q1, a3 = a / (q1 * q1);
        const double f = (stiff && tm == 0 ? dN[0][a1] : N[0][a1]) * (stiff && tm == 1 ? dN[1][a2] : N[1][a2]) *
                         (stiff && tm == 2 ? dN[2][a3] : N[2][a3]);
        Lv += ll[a] * f;
        Uv += uu[a] * f;
      }
      F += Lv * Uv;
    }
    F *= w;
    for (int a = 0; a < Q3; ++a) {
      const int a1 = a % q1, a2 = (a / q1) % q1, a3 = a / (q1 * q1);
      atomicAdd(&gacc[a], F * N[0][a1] * N[1][a2] * N[2][a3]);
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < Q3; a += blockDim.x) {
    const int a1 = a % q1, a2 = (a / q1) % q1, a3 = a / (q1 * q1);
    const int64_t k = (ee[0] + a1) + (int64_t)n1 * ((ee[1] + a2) + (int64_t)n2 * (ee[2] + a3));
    atomicAdd(&grad[k], gacc[a]);
  }
}

__global__ void k_scale(double* g, int64_t n, const double* scale) {
  const double s = *scale;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) g[t] *= s;
}

cudaError_t pass(const MeshView& M, int d, int mode, int kind, const double* in, double* out, const int64_t* din,
                 int64_t* dout, cudaStream_t st) {
  for (int k = 0; k < 3; ++k) dout[k] = din[k];
  const Dir1D& D = M.dir[d];
  dout[d] = mode == 1 ? D.n : D.nsup;
  k_pass<<<1216, 256, 0, st>>>(M, d, mode, kind, in, out, dout[0], dout[1], dout[2], din[0], din[1], din[2]);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bilinear(const int64_t* rowptr, const int32_t* colind, const int32_t* rows, int64_t nrows,
                            const void* values, bool fp64, const double* lam, const double* u, double* partial,
                            double* J, cudaStream_t st) {
  (void)rows;
  const int nb = 1024;
  if (fp64)
    k_bilinear<double><<<nb, 256, 0, st>>>(rowptr, colind, nrows, (const double*)values, lam, u, partial);
  else
    k_bilinear<float><<<nb, 256, 0, st>>>(rowptr, colind, nrows, (const float*)values, lam, u, partial);
  SFA_LAUNCHED(1);
  k_sum<<<1, 32, 0, st>>>(partial, nb, J);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

// Work buffers (allocated on first use, owned by the mesh): adj[0..2] U / dU fields,
// adj[3..5] Omega fields, adj[6..7] pass scratch.
cudaError_t launch_backward(sfa_mesh* m, bool stiff, const double* lam, const double* u, const double* scale,
                            double* grad, cudaStream_t st) {
  const MeshView& M = m->view;
  const Dir1D &A = M.dir[0], &B = M.dir[1], &C = M.dir[2];
  const int64_t nsup3 = (int64_t)A.nsup * B.nsup * C.nsup;
  const int64_t nscr = std::max<int64_t>(std::max<int64_t>((int64_t)A.nsup * B.n * C.n, (int64_t)A.nsup * B.nsup * C.n),
                                         std::max<int64_t>((int64_t)A.n * B.nsup * C.nsup, (int64_t)A.n * B.n * C.nsup));
  if (!m->adj[0]) {
    for (int k = 0; k < 6; ++k) {
      cudaError_t e = cudaMalloc((void**)&m->adj[k], nsup3 * sizeof(double));
      if (e != cudaSuccess) return e;
      m->allocs.push_back(m->adj[k]);
    }
    for (int k = 6; k < 8; ++k) {
      cudaError_t e = cudaMalloc((void**)&m->adj[k], std::max<int64_t>(nscr, nsup3) * sizeof(double));
      if (e != cudaSuccess) return e;
      m->allocs.push_back(m->adj[k]);
    }
  }
  double *U0 = m->adj[0], *U1 = m->adj[1], *U2 = m->adj[2];
  double *O0 = m->adj[3], *O1 = m->adj[4], *O2 = m->adj[5];
  double *S1 = m->adj[6], *S2 = m->adj[7];
  const int64_t dcoef[3] = {A.n, B.n, C.n};
  int64_t d1[3], d2[3], d3[3];
  cudaError_t err;
  const int nterm = stiff ? 3 : 1;
  // U (mass) or the three partial derivatives of U (stiffness) on the superset grid
  for (int tm = 0; tm < nterm; ++tm) {
    double* Uo = tm == 0 ? U0 : (tm == 1 ? U1 : U2);
    if ((err = pass(M, 0, 0, stiff && tm == 0, u, S1, dcoef, d1, st)) != cudaSuccess) return err;
    if ((err = pass(M, 1, 0, stiff && tm == 1, S1, S2, d1, d2, st)) != cudaSuccess) return err;
    if ((err = pass(M, 2, 0, stiff && tm == 2, S2, Uo, d2, d3, st)) != cudaSuccess) return err;
  }
  // Omega from interior rows: lambda masked to interior rows, three weighted passes
  k_mask_interior<<<608, 256, 0, st>>>(M.topo.fn_class, lam, m->nN, S2);
  SFA_LAUNCHED(1);
  for (int tm = 0; tm < nterm; ++tm) {
    double* Oo = tm == 0 ? O0 : (tm == 1 ? O1 : O2);
    if ((err = pass(M, 0, 2, stiff && tm == 0, S2, S1, dcoef, d1, st)) != cudaSuccess) return err;
    if ((err = pass(M, 1, 2, stiff && tm == 1, S1, Oo, d1, d2, st)) != cudaSuccess) return err;
    // third direction: through S1 again (Oo holds the intermediate)
    if ((err = pass(M, 2, 2, stiff && tm == 2, Oo, S1, d2, d3, st)) != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(Oo, S1, nsup3 * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return err;
  }
  if (m->n_cut_rows > 0) {
    k_box_scatter<<<(unsigned)m->n_cut_rows, 128, 0, st>>>(M, lam, O0, O1, O2, stiff ? 1 : 0);
    SFA_LAUNCHED(1);
    k_gauss_elems<<<1216, 128, 0, st>>>(M, lam, O0, O1, O2, stiff ? 1 : 0);
    SFA_LAUNCHED(1);
  }
  k_combine<<<1216, 256, 0, st>>>(nsup3, O0, O1, O2, U0, U1, U2, stiff ? 1 : 0, S2);
  SFA_LAUNCHED(1);
  // transposed interpolation to the coefficients
  const int64_t dsup[3] = {A.nsup, B.nsup, C.nsup};
  if ((err = pass(M, 0, 1, 0, S2, S1, dsup, d1, st)) != cudaSuccess) return err;
  if ((err = pass(M, 1, 1, 0, S1, S2, d1, d2, st)) != cudaSuccess) return err;
  if ((err = pass(M, 2, 1, 0, S2, grad, d2, d3, st)) != cudaSuccess) return err;
  if (m->n_cut > 0) {
    k_cut_adjoint<<<(unsigned)m->n_cut, 128, 0, st>>>(M, m->ls, lam, u, grad, stiff ? 1 : 0);
    SFA_LAUNCHED(1);
  }
  if (scale) {
    k_scale<<<608, 256, 0, st>>>(grad, m->nN, scale);
    SFA_LAUNCHED(1);
  }
  return cudaGetLastError();
}
