// Load vector b_i ("int f B_i") by the rules of the formation (Sec. 1, the test function folded
// into the weighted-quadrature weights; Sec. 2.2, Eq. 1 for cut test functions), with f the
// mesh's coefficient field or the target function of the paper's experiment,
// f = sin(2xz) cos(3yz) (Sec. 3.1):
//   interior row i:  b_i = sum_q w_i1(q1) w_i2(q2) w_i3(q3) f(x_q) over its WQ tensor grid;
//   cut row i:       the same over its DWQ box (one-sided rule in the box direction), plus
//                    sum_g w_g f(x_g) B_i(x_g) over the Gauss points of the inside support
//                    elements outside the box and of the octree pieces of its cut elements.
// f is tabulated on the Gauss superset grid (the WQ points and the element Gauss points are
// superset points); each cut element's piece sums sum_g w_g f B_a for its (p+1)^3 local
// functions a are formed once (k_load_elem) and read by the rows that touch it.  FP64.
#include "sfa_internal.cuh"

namespace {

__device__ __forceinline__ double paper_source(double x, double y, double z) {
  return sin(2.0 * x * z) * cos(3.0 * y * z);
}

// f = sin(2xz) cos(3yz) on the superset grid, index s1 + nsup1 (s2 + nsup2 s3).
__global__ void k_source_grid(MeshView M, double* __restrict__ F) {
  const Dir1D &A = M.dir[0], &B = M.dir[1], &C = M.dir[2];
  const int64_t n = (int64_t)A.nsup * B.nsup * C.nsup;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int s1 = (int)(t % A.nsup), s2 = (int)((t / A.nsup) % B.nsup), s3 = (int)(t / ((int64_t)A.nsup * B.nsup));
    F[t] = paper_source(A.t_sup[s1], B.t_sup[s2], C.t_sup[s3]);
  }
}

// Coordinate of Gauss point g of the octree cell at position pos of element e in direction d:
// the cell spans sample-grid points [gi sx, (gi + 1) sx] of x(k) = lo + (hi - lo) (k / N).
__device__ __forceinline__ double piece_point(const MeshView& M, int d, int e, int pos, int g) {
  const Dir1D& D = M.dir[d];
  int l = 0;
  while ((2 << l) - 1 <= pos) ++l;
  const int a = pos - ((1 << l) - 1);
  const int64_t Nk = (int64_t)D.n_el << (M.D + 1);
  const int64_t sx = 1ll << (M.D + 1 - l);
  const int64_t gi = ((int64_t)e << l) + a;
  auto coord = [&](int64_t k) {
    const double tt = __ddiv_rn((double)k, (double)Nk);
    return __dadd_rn(D.lo, __dmul_rn(__dsub_rn(D.hi, D.lo), tt));
  };
  const double xa = coord(gi * sx), xb = coord((gi + 1) * sx);
  return 0.5 * (xa + xb) + 0.5 * (xb - xa) * M.gl[g];
}

struct SrcDesc {
  int source;  // 0: the coefficient field, 1: the paper's f
  int coef_kind;
  double c0;
  const double* ck;
};

// Piece sums of one cut element: out[a] = sum_pieces sum_g w_g f(x_g) B_a1 B_a2 B_a3 for its
// local functions a = a1 + Q (a2 + Q a3), by three contractions per piece.  Pieces are dealt
// to the warps in a fixed order, each warp accumulates its own sums, and the warps' sums are
// added in warp order (deterministic).
template <int P>
__global__ void __launch_bounds__(128) k_load_elem(MeshView M, SrcDesc sd, double* __restrict__ out) {
  constexpr int Q = P + 1, Q2 = Q * Q, Q3 = Q2 * Q, NW = 4;
  constexpr int PTF = 2 * P + 1 + Q + 2, NBo = 2 * P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* acc = reinterpret_cast<double*>(smem_raw);  // [NW][Q3]
  double* cblk = acc + NW * Q3;                        // [Q3] coefficient block
  double* wsp = cblk + Q3;                             // per warp: F | T1 | T2 | N[3][Q][Q] | W[3][Q] | A[3][Q] | X[3][Q]
  constexpr int WS = 3 * Q3 + 3 * Q2 + 9 * Q;
  const int ci = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = M.topo.cut_elems[ci];
  const int ne1 = M.dir[0].n_el, ne2 = M.dir[1].n_el;
  const int ee[3] = {e % ne1, (e / ne1) % ne2, e / (ne1 * ne2)};
  for (int t = threadIdx.x; t < NW * Q3; t += blockDim.x) acc[t] = 0.0;
  if (sd.source == 0 && sd.coef_kind == SFA_COEF_BSPLINE) {
    const int n1 = M.dir[0].n, n2 = M.dir[1].n;
    for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
      const int a1 = t % Q, a2 = (t / Q) % Q, a3 = t / Q2;
      cblk[t] = sd.ck[(ee[0] + a1) + (int64_t)n1 * ((ee[1] + a2) + (int64_t)n2 * (ee[2] + a3))];
    }
  }
  __syncthreads();
  const bool live = M.topo.elem_state[e] == E_CUT;
  const int pbeg = M.topo.piece_ptr[ci], pend = live ? M.topo.piece_ptr[ci + 1] : pbeg;
  double* F = wsp + (size_t)warp * WS;
  double* T1 = F + Q3;
  double* T2 = T1 + Q3;
  double* Nv = T2 + Q3;     // [d][a][g]
  double* Wv = Nv + 3 * Q2; // [d][g]
  double* Av = Wv + 3 * Q;  // [d][g] analytic factors
  double* Xv = Av + 3 * Q;  // [d][g] coordinates
  double* my = acc + warp * Q3;
  for (int pc = pbeg + warp; pc < pend; pc += NW) {
    const uint32_t code = M.topo.pieces[pc];
    const int lev = code & 15;
    const int av[3] = {(int)((code >> 4) & 63), (int)((code >> 10) & 63), (int)((code >> 16) & 63)};
    for (int t = lane; t < 3 * Q; t += 32) {
      const int d = t / Q, g = t % Q;
      const Dir1D& D = M.dir[d];
      const int pos = (1 << lev) - 1 + av[d];
      const double* src = D.PT + (((int64_t)ee[d] * D.npos + pos) * Q + g) * PTF;
      Wv[d * Q + g] = src[0];
      for (int a = 0; a < Q; ++a) Nv[(d * Q + a) * Q + g] = src[1 + NBo + a];
      Av[d * Q + g] = src[1 + NBo + Q];
      Xv[d * Q + g] = sd.source == 1 ? piece_point(M, d, ee[d], pos, g) : 0.0;
    }
    __syncwarp();
    for (int g = lane; g < Q3; g += 32) {
      const int g1 = g % Q, g2 = (g / Q) % Q, g3 = g / Q2;
      double f;
      if (sd.source == 1) {
        f = paper_source(Xv[g1], Xv[Q + g2], Xv[2 * Q + g3]);
      } else if (sd.coef_kind == SFA_COEF_BSPLINE) {
        f = 0.0;
        for (int a3 = 0; a3 < Q; ++a3) {
          double s2 = 0.0;
          for (int a2 = 0; a2 < Q; ++a2) {
            double s1 = 0.0;
            for (int a1 = 0; a1 < Q; ++a1) s1 += Nv[a1 * Q + g1] * cblk[a1 + Q * (a2 + Q * a3)];
            s2 += Nv[(Q + a2) * Q + g2] * s1;
          }
          f += Nv[(2 * Q + a3) * Q + g3] * s2;
        }
      } else if (sd.coef_kind == SFA_COEF_ANALYTIC) {
        f = 1.0 + 0.5 * Av[g1] * Av[Q + g2] * Av[2 * Q + g3];
      } else {
        f = sd.c0;
      }
      F[g] = Wv[g1] * Wv[Q + g2] * Wv[2 * Q + g3] * f;
    }
    __syncwarp();
    // T1[a1][g2][g3] = sum_g1 N1[a1][g1] F[g1, g2, g3]
    for (int t = lane; t < Q3; t += 32) {
      const int a1 = t % Q, g23 = t / Q;
      double s = 0.0;
      for (int g1 = 0; g1 < Q; ++g1) s += Nv[a1 * Q + g1] * F[g1 + Q * g23];
      T1[t] = s;
    }
    __syncwarp();
    // T2[a1][a2][g3] = sum_g2 N2[a2][g2] T1[a1][g2][g3]
    for (int t = lane; t < Q3; t += 32) {
      const int a1 = t % Q, a2 = (t / Q) % Q, g3 = t / Q2;
      double s = 0.0;
      for (int g2 = 0; g2 < Q; ++g2) s += Nv[(Q + a2) * Q + g2] * T1[a1 + Q * (g2 + Q * g3)];
      T2[t] = s;
    }
    __syncwarp();
    // acc[a1][a2][a3] += sum_g3 N3[a3][g3] T2[a1][a2][g3]
    for (int t = lane; t < Q3; t += 32) {
      const int a12 = t % Q2, a3 = t / Q2;
      double s = 0.0;
      for (int g3 = 0; g3 < Q; ++g3) s += Nv[(2 * Q + a3) * Q + g3] * T2[a12 + Q2 * g3];
      my[t] += s;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += acc[w * Q3 + t];
    out[(size_t)ci * Q3 + t] = s;
  }
}

// One warp per row (every row of the index space; exterior rows get 0).  F: f on the superset
// grid; Eload: the cut elements' piece sums [n_cut][(p+1)^3].  variant: SFA_VARIANT_DWQ,
// _HYBRID (no box) or _GAUSS (every row by element Gauss points, no weighted quadrature).
template <int P>
__global__ void __launch_bounds__(256) k_load_rows(MeshView M, const double* __restrict__ F,
                                                   const double* __restrict__ Eload, int variant,
                                                   double* __restrict__ b) {
  constexpr int Q = P + 1, Q2 = Q * Q, Q3 = Q2 * Q, MP = Q * Q;  // MP: points of a rule, at most
  __shared__ int sidx[8][3][MP];
  __shared__ double swt[8][3][MP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Dir1D* D = M.dir;
  const int n1 = D[0].n, n2 = D[1].n;
  const int64_t nrows = (int64_t)n1 * n2 * D[2].n;
  const int64_t cs2 = D[0].nsup, cs3 = (int64_t)D[0].nsup * D[1].nsup;
  for (int64_t i = blockIdx.x * 8ll + warp; i < nrows; i += (int64_t)gridDim.x * 8) {
    const int cls = M.topo.fn_class[i];
    if (cls == F_EXT) {
      if (lane == 0) b[i] = 0.0;
      continue;
    }
    const int q12 = fdiv((int)i, M.div_n1);
    const int id[3] = {(int)i - q12 * n1, q12 - fdiv(q12, M.div_n2) * n2, fdiv(q12, M.div_n2)};
    int elo[3], ehi[3];
    for (int d = 0; d < 3; ++d) {
      elo[d] = max(0, id[d] - P);
      ehi[d] = min(D[d].n_el - 1, id[d]);
    }
    const int32_t bcode = (cls == F_CUT && variant == SFA_VARIANT_DWQ) ? M.topo.box[i] : -1;
    const int bd = bcode >= 0 ? (bcode & 3) : -1, bside = (bcode >> 2) & 1, bb = bcode >> 3;
    double part = 0.0;
    if (variant != SFA_VARIANT_GAUSS && (cls == F_INT || bd >= 0)) {
      // weighted-quadrature grid: each direction's rule points (superset index) and weights
      int m[3];
      for (int d = 0; d < 3; ++d) {
        if (d == bd) {
          const int ka = bside == 0 ? elo[d] : bb, kb = bside == 0 ? bb - 1 : ehi[d];
          m[d] = (kb - ka + 1) * Q;
          const int rule = ((id[d] * P) + (bb - elo[d] - 1)) * 2 + bside;
          const int slo = (ka - elo[d]) * Q;
          for (int k = lane; k < m[d]; k += 32) {
            sidx[warp][d][k] = ka * Q + k;
            swt[warp][d][k] = D[d].dwq00[(size_t)rule * D[d].nsl + slo + k];
          }
        } else {
          m[d] = D[d].nqi[id[d]];
          const int q0 = D[d].qlo[id[d]];
          for (int k = lane; k < m[d]; k += 32) {
            sidx[warp][d][k] = D[d].wq_idx[q0 + k];
            swt[warp][d][k] = D[d].w00[(size_t)id[d] * D[d].nql + k];
          }
        }
      }
      __syncwarp();
      // sum_k3 w3 sum_k2 w2 sum_k1 w1 F, lanes over (k2, k3)
      for (int t = lane; t < m[1] * m[2]; t += 32) {
        const int k2 = t % m[1], k3 = t / m[1];
        const double* fb = F + sidx[warp][1][k2] * cs2 + sidx[warp][2][k3] * cs3;
        double s = 0.0;
        for (int k1 = 0; k1 < m[0]; ++k1) s += swt[warp][0][k1] * fb[sidx[warp][0][k1]];
        part += swt[warp][1][k2] * swt[warp][2][k3] * s;
      }
      __syncwarp();
    }
    if (cls == F_CUT || variant == SFA_VARIANT_GAUSS) {
      // Gauss part: every support element, lanes over its Gauss points (inside elements) or
      // lane 0 reading the element's piece sums (cut elements)
      for (int e3 = elo[2]; e3 <= ehi[2]; ++e3)
        for (int e2 = elo[1]; e2 <= ehi[1]; ++e2)
          for (int e1 = elo[0]; e1 <= ehi[0]; ++e1) {
            const int64_t e = e1 + (int64_t)D[0].n_el * (e2 + (int64_t)D[1].n_el * e3);
            const int st = M.topo.elem_state[e];
            const int ee[3] = {e1, e2, e3};
            if (st == E_IN) {
              if (bd >= 0) {
                const int ed = ee[bd];
                if ((bside == 0 && ed < bb) || (bside == 1 && ed >= bb)) continue;  // in the DWQ box
              }
              for (int g = lane; g < Q3; g += 32) {
                const int g1 = g % Q, g2 = (g / Q) % Q, g3 = g / Q2;
                const int s1 = e1 * Q + g1, s2 = e2 * Q + g2, s3 = e3 * Q + g3;
                const double bi = D[0].B[s1 * Q + (id[0] - e1)] * D[1].B[s2 * Q + (id[1] - e2)] *
                                  D[2].B[s3 * Q + (id[2] - e3)];
                part += D[0].w_sup[s1] * D[1].w_sup[s2] * D[2].w_sup[s3] * F[s1 + s2 * cs2 + s3 * cs3] * bi;
              }
            } else if (st == E_CUT && lane == 0) {
              const int ci = M.topo.elem_cut_id[e];
              const int a = (id[0] - e1) + Q * ((id[1] - e2) + Q * (id[2] - e3));
              part += Eload[(size_t)ci * Q3 + a];
            }
          }
    }
    part = warp_sum(part);
    if (lane == 0) b[i] = part;
  }
}

template <int P>
cudaError_t launch_load_t(const MeshView& M, SrcDesc sd, int variant, int n_cut, const double* F, double* Eload,
                          double* b, cudaStream_t st) {
  constexpr int Q = P + 1, Q3 = Q * Q * Q;
  cudaError_t err;
  if (n_cut > 0) {
    const size_t smem = (size_t)(4 * Q3 + Q3 + 4 * (3 * Q3 + 3 * Q * Q + 9 * Q)) * sizeof(double);
    err = cudaFuncSetAttribute(k_load_elem<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_load_elem<P><<<n_cut, 128, smem, st>>>(M, sd, Eload);
    SFA_LAUNCHED(1);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const int64_t nrows = (int64_t)M.dir[0].n * M.dir[1].n * M.dir[2].n;
  const int grid = (int)std::min<int64_t>((nrows + 7) / 8, 152 * 16);
  k_load_rows<P><<<grid, 256, 0, st>>>(M, F, Eload, variant, b);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

// f on the superset grid for the paper's source (the coefficient source uses the coefficient
// grid of the formation, computed by launch_coef).
cudaError_t launch_source_grid(const MeshView& M, double* F, cudaStream_t st) {
  k_source_grid<<<152 * 8, 256, 0, st>>>(M, F);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_load(const MeshView& M, int source, int coef_kind, double c0, const double* ck, int variant,
                        int n_cut, const double* F, double* Eload, double* b, cudaStream_t st) {
  const SrcDesc sd{source, coef_kind, c0, ck};
  switch (M.p) {
    case 2: return launch_load_t<2>(M, sd, variant, n_cut, F, Eload, b, st);
    case 3: return launch_load_t<3>(M, sd, variant, n_cut, F, Eload, b, st);
    case 4: return launch_load_t<4>(M, sd, variant, n_cut, F, Eload, b, st);
    case 5: return launch_load_t<5>(M, sd, variant, n_cut, F, Eload, b, st);
    case 6: return launch_load_t<6>(M, sd, variant, n_cut, F, Eload, b, st);
  }
  return cudaErrorInvalidValue;
}
