// 1D stage of the method (Sec. 1 "weighted quadrature", Sec. 2.2 steps 1 and 3-6 and the
// Gauss-superset paragraph): Gauss nodes, superset points, B-spline values, the standard
// WQ rules and the one-sided DWQ rules of every 1D test function, and the product tables
// consumed by the row contractions.  All FP64; one warp per weight system.
#include "sfa_internal.cuh"

namespace {

// ------------------------------------------------------------------------------------
// Gauss-Legendre nodes by Newton's method on the Legendre three-term recurrence.
__device__ void legendre_pn(int n, double z, double* pn, double* dpn) {
  double pkm1 = 1.0, pk = z;
  for (int k = 1; k < n; ++k) {
    double pk1 = ((2 * k + 1) * z * pk - k * pkm1) / (k + 1);
    pkm1 = pk;
    pk = pk1;
  }
  if (n == 0) {
    pk = 1.0;
    pkm1 = 0.0;
  }
  *pn = pk;
  *dpn = n * (z * pk - pkm1) / (z * z - 1.0);
}

__global__ void k_gauss(double* gl, int p) {
  int t = threadIdx.x;
  int n1 = p + 1, n2 = 2 * p + 1;
  int n, i;
  double *xo, *wo;
  if (t < n1) {
    n = n1; i = t; xo = gl; wo = gl + n1;
  } else if (t < n1 + n2) {
    n = n2; i = t - n1; xo = gl + 2 * n1; wo = gl + 2 * n1 + n2;
  } else {
    return;
  }
  // node i in ascending order: start from the (n-1-i)-th root of the descending cosine guess
  int id = n - 1 - i;
  double z = cos(3.14159265358979323846 * (id + 0.75) / (n + 0.5));
  double pn, dpn;
  for (int it = 0; it < 100; ++it) {
    legendre_pn(n, z, &pn, &dpn);
    double dz = pn / dpn;
    z -= dz;
    if (fabs(dz) < 1e-15) break;
  }
  legendre_pn(n, z, &pn, &dpn);
  xo[i] = z;
  wo[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
}

// ------------------------------------------------------------------------------------
// Closed-form WQ layout: all p+1 Gauss points in the first and last element, Gauss
// indices {0, p} elsewhere.
__device__ __forceinline__ bool elem_full(int e, int n_el) { return e == 0 || e == n_el - 1; }
__device__ __forceinline__ int elem_qfirst(int e, int n_el, int p) {
  if (e == 0) return 0;
  if (e < n_el - 1) return (p + 1) + 2 * (e - 1);
  return (p + 1) + 2 * (n_el - 2);
}
__device__ __forceinline__ int elem_qcount(int e, int n_el, int p) { return elem_full(e, n_el) ? p + 1 : 2; }

struct OrigKnots {
  const double* xb;
  int p, n_el;
  __device__ double operator()(int k) const {
    int b = k - p;
    b = b < 0 ? 0 : (b > n_el ? n_el : b);
    return xb[b];
  }
};

// Knot vector with x_b inserted `mult` extra times (boundary-index form).
struct RefKnots {
  const double* xb;
  int p, n_el, b, mult;
  __device__ int bidx(int k) const {
    int kk = k <= b + p ? k : (k <= b + p + mult ? -1 : k - mult);
    if (kk < 0) return b;
    int v = kk - p;
    return v < 0 ? 0 : (v > n_el ? n_el : v);
  }
  __device__ double operator()(int k) const { return xb[bidx(k)]; }
};

__global__ void k_points(MeshView M, int d0) {
  const int d = d0 >= 0 ? d0 : (int)blockIdx.y;
  const Dir1D& D = M.dir[d];
  const int p = M.p, q1 = p + 1;
  const double* gx = M.gl;
  const double* gw = M.gl + q1;
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int nthreads = gridDim.x * blockDim.x;
  // element bounds (same formula as the knots)
  for (int e = tid; e <= D.n_el; e += nthreads)
    D.xb[e] = (e == 0) ? D.lo : (e == D.n_el ? D.hi : D.lo + (D.hi - D.lo) * ((double)e / (double)D.n_el));
  __threadfence();
  // the grid is a single block (see launcher), so a block barrier orders the phases
  __syncthreads();
  for (int k = tid; k < D.n_el + 2 * p + 1; k += nthreads) {
    int b = k - p;
    b = b < 0 ? 0 : (b > D.n_el ? D.n_el : b);
    D.U[k] = D.xb[b];
  }
  OrigKnots knot{D.xb, p, D.n_el};
  for (int s = tid; s < D.nsup; s += nthreads) {
    int e = s / q1, g = s % q1;
    double a = D.xb[e], bb = D.xb[e + 1];
    double mid = 0.5 * (a + bb), half = 0.5 * (bb - a);
    double t = mid + half * gx[g];
    D.t_sup[s] = t;
    D.w_sup[s] = half * gw[g];
    double N[SFA_MAXP + 1], dN[SFA_MAXP + 1];
    bspline_eval(knot, p, e + p, t, N, dN);
    for (int r = 0; r <= p; ++r) {
      D.B[s * q1 + r] = N[r];
      D.Bf[s * q1 + r] = (float)N[r];
      D.dB[s * q1 + r] = dN[r];
    }
  }
  for (int q = tid; q < D.nq; q += nthreads) {
    // locate the element of WQ point q
    int e = 0;
    for (int ee = 0; ee < D.n_el; ++ee)
      if (q >= elem_qfirst(ee, D.n_el, p) && q < elem_qfirst(ee, D.n_el, p) + elem_qcount(ee, D.n_el, p)) e = ee;
    int local = q - elem_qfirst(e, D.n_el, p);
    int g = elem_full(e, D.n_el) ? local : (local == 0 ? 0 : p);
    D.wq_idx[q] = e * q1 + g;
  }
  for (int i = tid; i < D.n; i += nthreads) {
    int e_lo = max(0, i - p), e_hi = min(D.n_el - 1, i);
    int a = elem_qfirst(e_lo, D.n_el, p);
    int b = elem_qfirst(e_hi, D.n_el, p) + elem_qcount(e_hi, D.n_el, p);
    D.qlo[i] = a;
    D.nqi[i] = b - a;
  }
}

// ------------------------------------------------------------------------------------
// Warp-cooperative minimum-norm solve  w = argmin ||w||  s.t.  A w = b  (A: m x k, m <= k,
// full row rank).  At holds A^T column by column (column c = trial function c, at At + c*ld,
// rows = points 0..k-1) and is overwritten by Householder QR of A^T = Q R; V receives the
// unit reflectors.  Then z solves R^T z = b and w = Q [z; 0].
__device__ bool warp_min_norm(double* At, double* V, int ld, int k, int m, const double* b, double* w,
                              double* y, double rtol) {
  const int lane = threadIdx.x & 31;
  double rmax = 0.0;
  for (int c = 0; c < m; ++c) {
    double* col = At + c * ld;
    double* vc = V + c * ld;
    double s = 0.0;
    for (int r = c + lane; r < k; r += 32) s += col[r] * col[r];
    s = warp_sum(s);
    double x0 = col[c];
    double nrm = sqrt(s);
    double alpha = (x0 >= 0.0) ? -nrm : nrm;
    double v0 = x0 - alpha;
    double vn2 = s - x0 * x0 + v0 * v0;
    double inv = vn2 > 0.0 ? 1.0 / sqrt(vn2) : 0.0;
    for (int r = c + lane; r < k; r += 32) vc[r] = (r == c ? v0 : col[r]) * inv;
    __syncwarp();
    for (int c2 = c + 1; c2 < m; ++c2) {
      double* col2 = At + c2 * ld;
      double dd = 0.0;
      for (int r = c + lane; r < k; r += 32) dd += vc[r] * col2[r];
      dd = warp_sum(dd);
      for (int r = c + lane; r < k; r += 32) col2[r] -= 2.0 * vc[r] * dd;
      __syncwarp();
    }
    if (lane == 0) col[c] = alpha;
    rmax = fmax(rmax, fabs(alpha));
    __syncwarp();
  }
  bool ok = true;
  for (int c = 0; c < m; ++c)
    if (!(fabs(At[c * ld + c]) > rtol * rmax)) ok = false;
  if (lane == 0) {
    for (int c = 0; c < m; ++c) {
      double acc = b[c];
      for (int r = 0; r < c; ++r) acc -= At[c * ld + r] * y[r];
      y[c] = ok ? acc / At[c * ld + c] : 0.0;
    }
  }
  for (int r = m + lane; r < k; r += 32) y[r] = 0.0;
  __syncwarp();
  for (int c = m - 1; c >= 0; --c) {
    const double* vc = V + c * ld;
    double dd = 0.0;
    for (int r = c + lane; r < k; r += 32) dd += vc[r] * y[r];
    dd = warp_sum(dd);
    for (int r = c + lane; r < k; r += 32) y[r] -= 2.0 * vc[r] * dd;
    __syncwarp();
  }
  for (int r = lane; r < k; r += 32) w[r] = y[r];
  __syncwarp();
  return ok;
}

// Per-warp workspace (doubles): At, V [MM*LD each], b [MM], w, y [LD], acc [NSL], S [p+2],
// plus LD ints of point indices.
struct Work {
  double *At, *V, *b, *w, *y, *acc, *S;
  int* pts;
};
__device__ __forceinline__ int work_doubles(int MM, int LD, int NSL, int p) { return 2 * MM * LD + MM + 2 * LD + NSL + p + 2; }

__device__ Work carve(double* base, int MM, int LD, int NSL, int p) {
  Work W;
  W.At = base;
  W.V = W.At + MM * LD;
  W.b = W.V + MM * LD;
  W.w = W.b + MM;
  W.y = W.w + LD;
  W.acc = W.y + LD;
  W.S = W.acc + NSL;
  W.pts = reinterpret_cast<int*>(W.S + p + 2);
  return W;
}

// ------------------------------------------------------------------------------------
// Standard rules: warp per (function i, kind), kind 0 = w00 (values), 1 = w11 (derivatives).
// Points: the WQ points in supp B_i; trial functions: all j with |j - i| <= p; rhs by
// exact (p+1)-point Gauss per support element; Gauss-folded weights when every support
// element carries its full Gauss set, otherwise the minimum-norm solution (for w11 the
// last trial row is dropped: the derivatives sum to zero, so it is a combination of the
// others and the right-hand side is consistent).
__global__ void k_wq_std(MeshView M, int d0, int LD, int MM, int NSL) {
  const int d = d0 >= 0 ? d0 : (int)blockIdx.y;
  extern __shared__ double smem[];
  const int p = M.p, q1 = p + 1;
  const Dir1D& D = M.dir[d];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int gw = blockIdx.x * (blockDim.x >> 5) + warp;
  int i = gw >> 1, kind = gw & 1;
  if (i >= D.n) return;
  Work W = carve(smem + warp * (work_doubles(MM, LD, NSL, p) + LD), MM, LD, NSL, p);
  const double* F = kind ? D.dB : D.B;
  int e_lo = max(0, i - p), e_hi = min(D.n_el - 1, i);
  int j0 = max(0, i - p), j1 = min(D.n - 1, i + p);
  int m = j1 - j0 + 1;
  int q0 = D.qlo[i], k = D.nqi[i];
  for (int r = lane; r < k; r += 32) {
    int s = D.wq_idx[q0 + r];
    int e = s / q1;
    for (int c = 0; c < m; ++c) {
      int jj = j0 + c - e;
      W.At[c * LD + r] = (jj >= 0 && jj <= p) ? F[s * q1 + jj] : 0.0;
    }
  }
  for (int c = 0; c < m; ++c) {
    double part = 0.0;
    for (int s = e_lo * q1 + lane; s < (e_hi + 1) * q1; s += 32) {
      int e = s / q1;
      int ji = i - e, jc = j0 + c - e;
      double fi = (ji >= 0 && ji <= p) ? F[s * q1 + ji] : 0.0;
      double fc = (jc >= 0 && jc <= p) ? F[s * q1 + jc] : 0.0;
      part += D.w_sup[s] * fi * fc;
    }
    part = warp_sum(part);
    if (lane == 0) W.b[c] = part;
  }
  __syncwarp();
  bool full = true;
  for (int e = e_lo; e <= e_hi; ++e) full = full && elem_full(e, D.n_el);
  double* out = (kind ? D.w11 : D.w00) + (size_t)i * D.nql;
  if (full) {
    for (int r = lane; r < k; r += 32) {
      int s = D.wq_idx[q0 + r];
      int e = s / q1;
      out[r] = D.w_sup[s] * F[s * q1 + (i - e)];
    }
  } else {
    int mm = kind ? m - 1 : m;
    bool ok = warp_min_norm(W.At, W.V, LD, k, mm, W.b, W.w, W.y, 1e-13);
    if (!ok && lane == 0) dev_set_status(M.status, DEV_WQ_SINGULAR);
    for (int r = lane; r < k; r += 32) out[r] = W.w[r];
  }
  for (int r = k + lane; r < D.nql; r += 32) out[r] = 0.0;
}

// ------------------------------------------------------------------------------------
// DWQ rules: warp per (function i, candidate slot, side, kind).  The artificial
// discontinuity sits at x_b, b = e_lo + 1 + slot (an interior knot of supp B_i).
// If every kept element is full in the refined layout (WQ points plus all Gauss points of
// elements b-1 and b) the Gauss-folded weights are used; otherwise x_b is inserted p times
// (Boehm), B_i = sum_k S_k Btilde_k, and every refined function on the kept side gets its
// own WQ rule in the refined basis (same construction as the standard rule); the rule of
// B_i is sum_k S_k wtilde_k.  The far side is zero.
__global__ void k_wq_dwq(MeshView M, int d0, int LD, int MM, int NSL) {
  const int d = d0 >= 0 ? d0 : (int)blockIdx.y;
  extern __shared__ double smem[];
  const int p = M.p, q1 = p + 1;
  const Dir1D& D = M.dir[d];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int gw = blockIdx.x * (blockDim.x >> 5) + warp;
  int kind = gw & 1;
  int rule = gw >> 1;
  int side = rule & 1;
  int slot = (rule >> 1) % p;
  int i = (rule >> 1) / p;
  if (i >= D.n) return;
  Work W = carve(smem + warp * (work_doubles(MM, LD, NSL, p) + LD), MM, LD, NSL, p);
  double* out = (kind ? D.dwq11 : D.dwq00) + (size_t)rule * D.nsl;
  const double* F = kind ? D.dB : D.B;
  int e_lo = max(0, i - p), e_hi = min(D.n_el - 1, i);
  int b = e_lo + 1 + slot;
  for (int r = lane; r < D.nsl; r += 32) W.acc[r] = 0.0;
  __syncwarp();
  if (b > e_hi) {
    for (int r = lane; r < D.nsl; r += 32) out[r] = 0.0;
    return;
  }
  int ka = side == 0 ? e_lo : b, kb = side == 0 ? b - 1 : e_hi;  // kept elements
  auto full_ref = [&](int e) { return elem_full(e, D.n_el) || e == b - 1 || e == b; };
  bool all_full = true;
  for (int e = ka; e <= kb; ++e) all_full = all_full && full_ref(e);
  if (all_full) {
    for (int s = ka * q1 + lane; s < (kb + 1) * q1; s += 32) {
      int e = s / q1;
      W.acc[s - e_lo * q1] = D.w_sup[s] * F[s * q1 + (i - e)];
    }
    __syncwarp();
  } else {
    RefKnots rk{D.xb, p, D.n_el, b, p};
    // Boehm: insert x_b p times into the coefficient vector e_i (window [i, i+r] after r insertions)
    if (lane == 0) {
      double c[SFA_MAXP + 2], dn[SFA_MAXP + 2];
      for (int t = 0; t < p + 2; ++t) c[t] = 0.0;
      c[0] = 1.0;  // index i
      double xi = D.xb[b];
      for (int r = 0; r < p; ++r) {
        RefKnots cur{D.xb, p, D.n_el, b, r};  // knot vector after r insertions
        int s = b + p + r;                      // last index holding x_b
        for (int t = 0; t <= r + 1; ++t) {
          int kidx = i + t;
          double ck = (t <= r) ? c[t] : 0.0;
          double ckm1 = (t >= 1) ? c[t - 1] : 0.0;
          double v;
          if (kidx <= s - p) v = ck;
          else if (kidx <= s) {
            double alpha = (xi - cur(kidx)) / (cur(kidx + p) - cur(kidx));
            v = alpha * ck + (1.0 - alpha) * ckm1;
          } else v = ckm1;
          dn[t] = v;
        }
        for (int t = 0; t <= r + 1; ++t) c[t] = dn[t];
      }
      for (int t = 0; t <= p; ++t) W.S[t] = c[t];
    }
    __syncwarp();
    for (int t = 0; t <= p; ++t) {
      double Sk = W.S[t];
      if (Sk == 0.0) continue;
      int kf = i + t;
      int kb0 = rk.bidx(kf), kb1 = rk.bidx(kf + p + 1);  // refined support: elements kb0..kb1-1
      if (kb0 >= kb1) continue;
      if (side == 0 ? (kb1 > b) : (kb0 < b)) continue;   // not on the kept side
      // points of the refined layout in the support
      int k = 0;
      for (int e = kb0; e < kb1; ++e) {
        if (full_ref(e)) {
          for (int g = 0; g <= p; ++g) W.pts[k++] = e * q1 + g;
        } else {
          W.pts[k++] = e * q1;
          W.pts[k++] = e * q1 + p;
        }
      }
      // trial functions: refined j in [kf - p, kf + p] overlapping supp Btilde_kf
      int jlo = max(0, kf - p), jhi = min(D.n + p - 1, kf + p);
      int jl[2 * SFA_MAXP + 1];
      int m = 0;
      for (int j = jlo; j <= jhi; ++j) {
        int a0 = max(rk.bidx(j), kb0), a1 = min(rk.bidx(j + p + 1), kb1);
        if (a0 < a1) jl[m++] = j;
      }
      __syncwarp();
      for (int r = lane; r < k; r += 32) {
        int s = W.pts[r], e = s / q1;
        int span = e < b ? e + p : e + 2 * p;
        double N[SFA_MAXP + 1], dN[SFA_MAXP + 1];
        bspline_eval(rk, p, span, D.t_sup[s], N, dN);
        for (int c = 0; c < m; ++c) {
          int jj = jl[c] - (span - p);
          W.At[c * LD + r] = (jj >= 0 && jj <= p) ? (kind ? dN[jj] : N[jj]) : 0.0;
        }
      }
      bool full = true;
      for (int e = kb0; e < kb1; ++e) full = full && full_ref(e);
      // right-hand side by exact Gauss over the refined support: one basis evaluation per
      // superset point, partial sums per trial function, then one warp reduction each
      {
        double part[2 * SFA_MAXP + 1];
        for (int c = 0; c < m; ++c) part[c] = 0.0;
        for (int s = kb0 * q1 + lane; s < kb1 * q1; s += 32) {
          int e = s / q1;
          int span = e < b ? e + p : e + 2 * p;
          double N[SFA_MAXP + 1], dN[SFA_MAXP + 1];
          bspline_eval(rk, p, span, D.t_sup[s], N, dN);
          const double* Fv = kind ? dN : N;
          int ji = kf - (span - p);
          double fi = (ji >= 0 && ji <= p) ? Fv[ji] : 0.0;
          const double wf = D.w_sup[s] * fi;
          for (int c = 0; c < m; ++c) {
            int jc = jl[c] - (span - p);
            part[c] += (jc >= 0 && jc <= p) ? wf * Fv[jc] : 0.0;
          }
        }
        for (int c = 0; c < m; ++c) {
          double v = warp_sum(part[c]);
          if (lane == 0) W.b[c] = v;
        }
      }
      __syncwarp();
      if (full) {
        for (int r = lane; r < k; r += 32) {
          int s = W.pts[r], e = s / q1;
          int span = e < b ? e + p : e + 2 * p;
          double N[SFA_MAXP + 1], dN[SFA_MAXP + 1];
          bspline_eval(rk, p, span, D.t_sup[s], N, dN);
          int ji = kf - (span - p);
          W.w[r] = D.w_sup[s] * ((ji >= 0 && ji <= p) ? (kind ? dN[ji] : N[ji]) : 0.0);
        }
        __syncwarp();
      } else {
        int mm = kind ? m - 1 : m;
        bool ok = warp_min_norm(W.At, W.V, LD, k, mm, W.b, W.w, W.y, 1e-13);
        if (!ok && lane == 0) dev_set_status(M.status, DEV_WQ_SINGULAR);
      }
      for (int r = lane; r < k; r += 32) W.acc[W.pts[r] - e_lo * q1] += Sk * W.w[r];
      __syncwarp();
    }
  }
  for (int r = lane; r < D.nsl; r += 32) out[r] = W.acc[r];
}

// ------------------------------------------------------------------------------------
// Bezier coefficients of B_{e+a} on element e: blossom values at (x_e^(p-k), x_{e+1}^(k)),
// by the de Boor triangle with convex weights (one thread per (e, a, k)).
__global__ void k_bezier(MeshView M, int d0) {
  const int d = d0 >= 0 ? d0 : (int)blockIdx.y;
  const Dir1D& D = M.dir[d];
  const int p = M.p, q1 = p + 1;
  OrigKnots knot{D.xb, p, D.n_el};
  const int64_t n = (int64_t)D.n_el * q1 * q1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = t % q1, a = (t / q1) % q1;
    const int e = (int)(t / (q1 * q1));
    const int span = e + p, j = e + a;
    double dd[SFA_MAXP + 1];
    for (int r = 0; r <= p; ++r) dd[r] = (span - p + r == j) ? 1.0 : 0.0;
    for (int r = 1; r <= p; ++r) {
      const double u = (r <= p - k) ? D.xb[e] : D.xb[e + 1];
      for (int i = span; i >= span - p + r; --i) {
        const int li = i - (span - p);
        const double al = (u - knot(i)) / (knot(i + p + 1 - r) - knot(i));
        dd[li] = al * dd[li] + (1.0 - al) * dd[li - 1];
      }
    }
    D.BZ[t] = dd[p];
  }
}

// ------------------------------------------------------------------------------------
// Product tables WB[i][dj][ql] = w_i(q) B_{i-p+dj}(t_q) (values or derivatives), the DWQ
// analogues WD[rule][dj][sl], their float copies, and the Bernstein coefficient tables
// G[e][a][b][k] (degree 2p on element e) of B_{e+a} B_{e+b} (Gd: of the derivative
// products, degree-elevated from 2p-2).
__global__ void k_products(MeshView M, int d0) {
  const int d = d0 >= 0 ? d0 : (int)blockIdx.y;
  const int p = M.p, q1 = p + 1, nb = 2 * p + 1;
  const Dir1D& D = M.dir[d];
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  int nthreads = gridDim.x * blockDim.x;
  // (table sizes stay far below 2^31 entries: 32-bit index arithmetic)
  const int nstd = D.n * nb * D.nql;
  for (int t = tid; t < nstd; t += nthreads) {
    int ql = t % D.nql;
    int dj = (t / D.nql) % nb;
    int i = t / (D.nql * nb);
    int j = i - p + dj;
    double v0 = 0.0, v1 = 0.0;
    if (ql < D.nqi[i] && j >= 0 && j < D.n) {
      int s = D.wq_idx[D.qlo[i] + ql];
      int jj = j - s / q1;
      if (jj >= 0 && jj <= p) {
        v0 = D.w00[(size_t)i * D.nql + ql] * D.B[s * q1 + jj];
        v1 = D.w11[(size_t)i * D.nql + ql] * D.dB[s * q1 + jj];
      }
    }
    D.WB00[t] = v0;
    D.WB11[t] = v1;
    D.WB00f[t] = (float)v0;
    D.WB11f[t] = (float)v1;
  }
  const int nrule = D.n * p * 2;
  const int ndwq = nrule * nb * D.nsl;
  for (int t = tid; t < ndwq; t += nthreads) {
    int sl = t % D.nsl;
    int dj = (t / D.nsl) % nb;
    int rule = t / (D.nsl * nb);
    int i = (int)(rule / (2 * p));
    int j = i - p + dj;
    int e_lo = max(0, i - p);
    int s = e_lo * q1 + sl;
    double v0 = 0.0, v1 = 0.0;
    if (j >= 0 && j < D.n && s < D.nsup) {
      int jj = j - s / q1;
      if (jj >= 0 && jj <= p) {
        v0 = D.dwq00[(size_t)rule * D.nsl + sl] * D.B[s * q1 + jj];
        v1 = D.dwq11[(size_t)rule * D.nsl + sl] * D.dB[s * q1 + jj];
      }
    }
    D.WD00[t] = v0;
    D.WD11[t] = v1;
    D.WD00f[t] = (float)v0;
    D.WD11f[t] = (float)v1;
  }
  // Bernstein coefficients (degree 2p on the element) of the products B_{e+a} B_{e+b} and of
  // the derivative products, from the Bezier coefficients BZ[e][a][k] of B_{e+a} on element e
  // (k_bezier).
  const int nG = D.n_el * q1 * q1;
  for (int t = tid; t < nG; t += nthreads) {
    int bb = t % q1, a = (t / q1) % q1;
    int e = (int)(t / (q1 * q1));
    double Ca[SFA_MAXP + 1], Cb[SFA_MAXP + 1];
    for (int k = 0; k <= p; ++k) {
      Ca[k] = D.BZ[((int64_t)e * q1 + a) * q1 + k];
      Cb[k] = D.BZ[((int64_t)e * q1 + bb) * q1 + k];
    }
    double bin_p[SFA_MAXP + 1], bin_pm1[SFA_MAXP + 1], bin_2p[2 * SFA_MAXP + 1], bin_2pm2[2 * SFA_MAXP + 1];
    // binomial coefficients in integer arithmetic (exact at every step, and no double
    // divisions: the compiler moves this loop-invariant work out of the loop, where double
    // divisions at this GPU's FP64 rate dominated the kernel)
    auto binom = [](int n, int k) {
      int v = 1;
      for (int r = 1; r <= k; ++r) v = v * (n - k + r) / r;
      return (double)v;
    };
    for (int k = 0; k <= p; ++k) bin_p[k] = binom(p, k);
    for (int k = 0; k < p; ++k) bin_pm1[k] = binom(p - 1, k);
    for (int k = 0; k <= 2 * p; ++k) bin_2p[k] = binom(2 * p, k);
    for (int k = 0; k <= 2 * p - 2; ++k) bin_2pm2[k] = binom(2 * p - 2, k);
    double prod[2 * SFA_MAXP + 1], dprod[2 * SFA_MAXP + 1];
    for (int k = 0; k < nb; ++k) prod[k] = dprod[k] = 0.0;
    for (int i = 0; i <= p; ++i)
      for (int j = 0; j <= p; ++j) prod[i + j] += Ca[i] * Cb[j] * bin_p[i] * bin_p[j] / bin_2p[i + j];
    // derivatives: B' = (p / h) sum_i (C_{i+1} - C_i) b^{p-1}_i, product of degree 2p-2, elevated twice
    const double h = D.xb[e + 1] - D.xb[e];
    double Da[SFA_MAXP], Db[SFA_MAXP];
    for (int i = 0; i < p; ++i) {
      Da[i] = p / h * (Ca[i + 1] - Ca[i]);
      Db[i] = p / h * (Cb[i + 1] - Cb[i]);
    }
    double q[2 * SFA_MAXP + 1];
    for (int k = 0; k < nb; ++k) q[k] = 0.0;
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) q[i + j] += Da[i] * Db[j] * bin_pm1[i] * bin_pm1[j] / bin_2pm2[i + j];
    for (int m = 2 * p - 2; m < 2 * p; ++m) {  // degree m -> m + 1
      double r[2 * SFA_MAXP + 1];
      for (int k = 0; k <= m + 1; ++k) {
        double v = 0.0;
        if (k >= 1) v += (double)k / (m + 1) * q[k - 1];
        if (k <= m) v += (1.0 - (double)k / (m + 1)) * q[k];
        r[k] = v;
      }
      for (int k = 0; k <= m + 1; ++k) q[k] = r[k];
    }
    for (int k = 0; k < nb; ++k) {
      D.G[t * nb + k] = prod[k];
      D.Gd[t * nb + k] = q[k];
      D.Gf[t * nb + k] = (float)prod[k];
      D.Gdf[t * nb + k] = (float)q[k];
    }
  }
}

// Per-direction tables for the octree pieces of cut elements and for element Gauss sums.
// Piece geometry follows the sample-grid formula x(k) = lo + (hi - lo) * (k / N),
// N = n_el 2^(D+1), with the same rounded operations as the level-set sampling.
__global__ void k_piece_tables(MeshView M, int d0) {
  const int d = d0 >= 0 ? d0 : (int)blockIdx.y;
  const Dir1D& D = M.dir[d];
  const int p = M.p, q1 = p + 1, nb = 2 * p + 1, PTF = nb + q1 + 2;
  const double* gx = M.gl;
  const double* gw = M.gl + q1;
  const int64_t Nk = (int64_t)D.n_el << (M.D + 1);
  OrigKnots knot{D.xb, p, D.n_el};
  const double twopi = 6.283185307179586476925;
  int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  const int64_t npt = (int64_t)D.n_el * D.npos * q1;
  for (int64_t t = tid; t < npt; t += nth) {
    const int g = t % q1;
    const int pos = (int)((t / q1) % D.npos);
    const int e = (int)(t / ((int64_t)q1 * D.npos));
    int l = 0;
    while ((2 << l) - 1 <= pos) ++l;  // pos in [2^l - 1, 2^(l+1) - 1)
    const int a = pos - ((1 << l) - 1);
    const int64_t sx = 1ll << (M.D + 1 - l);
    const int64_t gi = ((int64_t)e << l) + a;
    auto coord = [&](int64_t k) {
      const double tt = __ddiv_rn((double)k, (double)Nk);
      return __dadd_rn(D.lo, __dmul_rn(__dsub_rn(D.hi, D.lo), tt));
    };
    const double xa = coord(gi * sx), xb2 = coord((gi + 1) * sx);
    const double mid = 0.5 * (xa + xb2), half = 0.5 * (xb2 - xa);
    const double x = mid + half * gx[g];
    double* out = D.PT + t * PTF;
    out[0] = half * gw[g];
    const double x0 = D.xb[e], x1 = D.xb[e + 1];
    const double tl = (x - x0) / (x1 - x0), ul = 1.0 - tl;
    for (int k = 0; k < nb; ++k) {
      int bin = 1;
      for (int r = 1; r <= k; ++r) bin = bin * (nb - 1 - k + r) / r;  // binomial(2p, k), exact
      double v = (double)bin;
      for (int r = 0; r < k; ++r) v *= tl;
      for (int r = k; r < nb - 1; ++r) v *= ul;
      out[1 + k] = v;
    }
    double N[SFA_MAXP + 1], dN[SFA_MAXP + 1];
    bspline_eval(knot, p, e + p, x, N, dN);
    for (int r = 0; r <= p; ++r) out[1 + nb + r] = N[r];
    out[1 + nb + q1] = d == 0 ? sin(twopi * x) : (d == 1 ? cos(twopi * x) : x);
    float* outf = D.PTf + t * PTF;
    for (int f = 0; f < PTF; ++f) outf[f] = (float)out[f];
  }
  const int64_t nge = (int64_t)D.n_el * q1 * q1 * q1;
  for (int64_t t = tid; t < nge; t += nth) {
    const int g = t % q1, b = (t / q1) % q1, ai = (t / (q1 * q1)) % q1;
    const int e = (int)(t / ((int64_t)q1 * q1 * q1));
    const int s = e * q1 + g;
    const double w = D.w_sup[s];
    const double v0 = w * D.B[s * q1 + ai] * D.B[s * q1 + b];
    const double v1 = w * D.dB[s * q1 + ai] * D.dB[s * q1 + b];
    D.GE[t] = v0;
    D.GEd[t] = v1;
    D.GEf[t] = (float)v0;
    D.GEdf[t] = (float)v1;
  }
}

}  // namespace

// Degree-3p monomial moments of every octree position of every element: the piece's Gauss
// points as in k_piece_tables, one thread per (e, pos, m).
__global__ void k_piece_p3(MeshView M, int d0) {
  const int d = d0 >= 0 ? d0 : (int)blockIdx.y;
  const Dir1D& D = M.dir[d];
  const int p = M.p, q1 = p + 1, m3 = 3 * p + 1;
  const double* gx = M.gl;
  const double* gw = M.gl + q1;
  const int64_t Nk = (int64_t)D.n_el << (M.D + 1);
  const int64_t n = (int64_t)D.n_el * D.npos * m3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(t % m3);
    const int pos = (int)((t / m3) % D.npos);
    const int e = (int)(t / ((int64_t)m3 * D.npos));
    int l = 0;
    while ((2 << l) - 1 <= pos) ++l;
    const int a = pos - ((1 << l) - 1);
    const int64_t sx = 1ll << (M.D + 1 - l);
    const int64_t gi = ((int64_t)e << l) + a;
    auto coord = [&](int64_t k) {
      const double tt = __ddiv_rn((double)k, (double)Nk);
      return __dadd_rn(D.lo, __dmul_rn(__dsub_rn(D.hi, D.lo), tt));
    };
    const double xa = coord(gi * sx), xb2 = coord((gi + 1) * sx);
    const double mid = 0.5 * (xa + xb2), half = 0.5 * (xb2 - xa);
    const double x0 = D.xb[e], x1 = D.xb[e + 1];
    double s = 0.0;
    for (int g = 0; g < q1; ++g) {
      const double x = mid + half * gx[g];
      const double tl = (x - x0) / (x1 - x0), ul = 1.0 - tl;
      double v = half * gw[g];
      for (int r = 0; r < m; ++r) v *= tl;
      for (int r = m; r < m3 - 1; ++r) v *= ul;
      s += v;
    }
    D.P3[t] = s;
    D.P3f[t] = (float)s;
  }
}

cudaError_t launch_piece_tables(const MeshView& M, int d, cudaStream_t st) {
  k_piece_tables<<<dim3(152, d < 0 ? 3 : 1), 256, 0, st>>>(M, d);
  SFA_LAUNCHED(1);
  k_piece_p3<<<dim3(64, d < 0 ? 3 : 1), 256, 0, st>>>(M, d);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_gauss(double* gl, int p, cudaStream_t st) {
  k_gauss<<<1, 64, 0, st>>>(gl, p);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

// d >= 0 launches one direction; d < 0 launches all three (grid dimension y = direction).
cudaError_t launch_points(const MeshView& M, int d, cudaStream_t st) {
  // one block per direction: k_points orders its phases with block barriers
  k_points<<<dim3(1, d < 0 ? 3 : 1), 256, 0, st>>>(M, d);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_wq_tables(const MeshView& M, int d, cudaStream_t st) {
  const int p = M.p;
  int nql = 0, nsl = 0, nmax = 0;
  for (int k = 0; k < 3; ++k) {
    if (d >= 0 && k != d) continue;
    nql = nql > M.dir[k].nql ? nql : M.dir[k].nql;
    nsl = nsl > M.dir[k].nsl ? nsl : M.dir[k].nsl;
    nmax = nmax > M.dir[k].n ? nmax : M.dir[k].n;
  }
  int LD = (p + 1) * (p + 1);
  if (nql > LD) LD = nql;
  int MM = 2 * p + 1;
  int NSL = nsl;
  int per_warp = 2 * MM * LD + MM + 2 * LD + NSL + p + 2 + LD;  // doubles (+ LD for the int point list)
  const int warps = 4;
  size_t smem = (size_t)per_warp * warps * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_wq_std, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_wq_dwq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned ny = d < 0 ? 3 : 1;
  int nstd = nmax * 2;
  k_wq_std<<<dim3((nstd + warps - 1) / warps, ny), 32 * warps, smem, st>>>(M, d, LD, MM, NSL);
  SFA_LAUNCHED(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int ndwq = nmax * p * 2 * 2;
  k_wq_dwq<<<dim3((ndwq + warps - 1) / warps, ny), 32 * warps, smem, st>>>(M, d, LD, MM, NSL);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_products(const MeshView& M, int d, cudaStream_t st) {
  k_bezier<<<dim3(64, d < 0 ? 3 : 1), 256, 0, st>>>(M, d);
  SFA_LAUNCHED(1);
  k_products<<<dim3(152, d < 0 ? 3 : 1), 256, 0, st>>>(M, d);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}
