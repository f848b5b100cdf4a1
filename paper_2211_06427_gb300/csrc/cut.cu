// Cut rows (Sec. 2.2, Eq. 1: the support of a cut test function is split into a regular
// part and a cut part).  The regular part is the DWQ box (one-sided DWQ rule in the box's
// direction, standard WQ rules in the other two) when one exists; every other inside
// support element is integrated with its (p+1)^3 Gauss points (the points below the
// artificial discontinuity in Fig. 3); every cut element with the Gauss points of its
// octree pieces (Sec. 3.1, sub-elements with standard Gauss rules).
//
// Cut elements are shared by up to (p+1)^3 rows, so each is integrated once:
//   mu_e[k1,k2,k3] = sum_pieces sum_g w_g c(x_g) b_k1(t_1) b_k2(t_2) b_k3(t_3)   (FP64)
// with b_k the degree-2p Bernstein polynomials of the element (t in [0, 1]).  B_a B_b
// restricted to the element is a polynomial of degree <= 2p per direction with Bernstein
// coefficients G[a][b][k] >= 0, so E_e[a][b] = sum_k G1[a1 b1 k1] G2[a2 b2 k2] G3[a3 b3 k3]
// mu_e[k] equals the Gauss sum over the pieces up to rounding, and for the mass matrix with
// c > 0 every term is non-negative (no cancellation, whatever the size of the domain part).
// Each cut row then adds row a(i) of E_e for its cut elements.
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

// ---------------------------------------------------------------------------------------
// Element matrices of cut elements.  One block per cut element; the pieces are spread over
// the warps (fixed assignment), each warp accumulates its own moments, the warps' moments
// are summed in a fixed order, then E = (G1 x G2 x G3) mu by three contractions.
template <typename R, typename MT, int P, bool STIFF>
__global__ void __launch_bounds__(256) k_cut_elemmat(MeshView M, LevelSet L, CoefDesc cf, R* __restrict__ E) {
  constexpr int Q = P + 1, NB = 2 * P + 1, Q3 = Q * Q * Q, NB3 = NB * NB * NB, Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ci = blockIdx.x;
  const int e = M.topo.cut_elems[ci];
  const int ne1 = M.dir[0].n_el, ne2 = M.dir[1].n_el;
  const int ee[3] = {e % ne1, (e / ne1) % ne2, e / (ne1 * ne2)};
  if (M.topo.elem_state[e] != E_CUT) return;
  const int pbeg = M.topo.piece_ptr[ci], pend = M.topo.piece_ptr[ci + 1];
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // shared layout: [mu][Gs][ union( muw | warp scratch | coefficient block , X1 | Y ) ]
  const int WS = Q3 + NB * Q2 + NB * NB * Q + 3 * NB * Q + 3 * Q + 3 * Q * Q;
  MT* mu = reinterpret_cast<MT*>(smem_raw);                           // NB3
  R* Gs = reinterpret_cast<R*>(mu + ((NB3 + 1) / 2) * 2);             // [2][3][Q2*NB]
  MT* uni = reinterpret_cast<MT*>(Gs + ((2 * 3 * Q2 * NB + 1) / 2) * 2);
  MT* muw = uni;                                                      // nwarps * NB3
  MT* wsp = muw + (size_t)nwarps * NB3;                               // nwarps * WS
  MT* cblk = wsp + (size_t)nwarps * WS;                               // Q3 coefficient block
  R* X1 = reinterpret_cast<R*>(uni);                                  // [2][Q2][NB][NB] (after the moments)
  R* Y = X1 + 2 * Q2 * NB * NB;                                       // [2][Q2][NB]

  for (int t = threadIdx.x; t < NB3; t += blockDim.x) mu[t] = MT(0);
  for (int t = threadIdx.x; t < nwarps * NB3; t += blockDim.x) muw[t] = MT(0);
  if (cf.kind == SFA_COEF_BSPLINE) {
    const int n1 = M.dir[0].n, n2 = M.dir[1].n;
    for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
      int a1 = t % Q, a2 = (t / Q) % Q, a3 = t / Q2;
      cblk[t] = (MT)cf.ck[(ee[0] + a1) + (int64_t)n1 * ((ee[1] + a2) + (int64_t)n2 * (ee[2] + a3))];
    }
  }
  for (int t = threadIdx.x; t < 3 * Q2 * NB; t += blockDim.x) {
    int d = t / (Q2 * NB), r = t % (Q2 * NB);
    Gs[t] = (R)M.dir[d].G[(size_t)ee[d] * Q2 * NB + r];
    Gs[3 * Q2 * NB + t] = (R)M.dir[d].Gd[(size_t)ee[d] * Q2 * NB + r];
  }
  __syncthreads();

  // ---- moments, piece by piece, one warp per piece
  {
    MT* F = wsp + (size_t)warp * WS;       // Q3: w c at the piece points [g3][g2][g1]
    MT* S1 = F + Q3;                       // [g3][g2][k1]
    MT* S2 = S1 + NB * Q2;                 // [g3][k2][k1]
    MT* PL = S2 + NB * NB * Q;             // [d][k][g] Bernstein values
    MT* TW = PL + 3 * NB * Q;              // [d][g] weights
    MT* NV = TW + 3 * Q;                   // [d][a][g] basis values (B-spline c)
    MT* mw = muw + (size_t)warp * NB3;
    constexpr int PTF = NB + Q + 2;
    constexpr int MPL = (NB * NB + 31) / 32;  // moment columns k12 per lane
    // register blocking of stage 3, except where it would spill (double moments at p = 6)
    constexpr bool REGB = !(sizeof(MT) == 8 && P >= 6);
    MT macc[REGB ? MPL : 1][NB];
#pragma unroll
    for (int r = 0; r < (REGB ? MPL : 1); ++r)
#pragma unroll
      for (int k = 0; k < NB; ++k) macc[r][k] = MT(0);
    for (int pc = pbeg + warp; pc < pend; pc += nwarps) {
      const uint32_t code = M.topo.pieces[pc];
      const int lev = code & 15;
      const int av[3] = {(int)((code >> 4) & 63), (int)((code >> 10) & 63), (int)((code >> 16) & 63)};
      // per-direction weights, Bernstein values and basis values, from the piece tables
      for (int t = lane; t < 3 * Q; t += 32) {
        const int d = t / Q, g = t % Q;
        const int pos = (1 << lev) - 1 + (d == 0 ? av[0] : (d == 1 ? av[1] : av[2]));
        const int eed = d == 0 ? ee[0] : (d == 1 ? ee[1] : ee[2]);
        const double* PTd = d == 0 ? M.dir[0].PT : (d == 1 ? M.dir[1].PT : M.dir[2].PT);
        const int npos = d == 0 ? M.dir[0].npos : (d == 1 ? M.dir[1].npos : M.dir[2].npos);
        const double* src = PTd + (((int64_t)eed * npos + pos) * Q + g) * PTF;
        TW[d * Q + g] = (MT)src[0];
        for (int k = 0; k < NB; ++k) PL[(d * NB + k) * Q + g] = (MT)src[1 + k];
        if (cf.kind == SFA_COEF_BSPLINE) {
          for (int a2 = 0; a2 < Q; ++a2) NV[(d * Q + a2) * Q + g] = (MT)src[1 + NB + a2];
        } else if (cf.kind == SFA_COEF_ANALYTIC) {
          NV[d * Q * Q + g] = (MT)src[1 + NB + Q];  // d=0 sin(2 pi x), d=1 cos(2 pi y), d=2 z
        }
      }
      __syncwarp();
      if (cf.kind == SFA_COEF_BSPLINE) {
        // c on the piece grid by sum factorisation over the (p+1)^3 coefficient block
        for (int t = lane; t < Q3; t += 32) {  // S1[a3][a2][g1] = sum_a1 c[a1 a2 a3] N1[a1][g1]
          const int g1 = t % Q, a23 = t / Q;
          MT sacc = MT(0);
          for (int a1 = 0; a1 < Q; ++a1) sacc += cblk[a1 + Q * a23] * NV[(0 * Q + a1) * Q + g1];
          S1[t] = sacc;
        }
        __syncwarp();
        for (int t = lane; t < Q3; t += 32) {  // S2[a3][g2][g1] = sum_a2 N2[a2][g2] S1[a3][a2][g1]
          const int g1 = t % Q, g2 = (t / Q) % Q, a3 = t / Q2;
          MT sacc = MT(0);
          for (int a2 = 0; a2 < Q; ++a2) sacc += NV[(1 * Q + a2) * Q + g2] * S1[g1 + Q * (a2 + Q * a3)];
          S2[t] = sacc;
        }
        __syncwarp();
      }
      for (int t = lane; t < Q3; t += 32) {
        const int g1 = t % Q, g2 = (t / Q) % Q, g3 = t / Q2;
        MT c;
        if (cf.kind == SFA_COEF_BSPLINE) {
          c = MT(0);
          for (int a3 = 0; a3 < Q; ++a3) c += NV[(2 * Q + a3) * Q + g3] * S2[g1 + Q * (g2 + Q * a3)];
        } else if (cf.kind == SFA_COEF_ANALYTIC) {
          c = MT(1) + MT(0.5) * NV[0 * Q * Q + g1] * NV[1 * Q * Q + g2] * NV[2 * Q * Q + g3];
        } else {
          c = (MT)cf.c0;
        }
        F[t] = TW[g1] * TW[Q + g2] * TW[2 * Q + g3] * c;
      }
      __syncwarp();
      // stage 1: S1[g23][k1] = sum_g1 PL1[k1][g1] F[g1 + Q g23], lane per (g2, g3)
      for (int g23 = lane; g23 < Q2; g23 += 32) {
        MT f[Q];
#pragma unroll
        for (int g = 0; g < Q; ++g) f[g] = F[g + Q * g23];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          MT v = MT(0);
#pragma unroll
          for (int g = 0; g < Q; ++g) v += PL[(0 * NB + k) * Q + g] * f[g];
          S1[k + NB * g23] = v;
        }
      }
      __syncwarp();
      // stage 2: S2[k1 + NB (k2 + NB g3)] = sum_g2 PL2[k2][g2] S1[k1 + NB (g2 + Q g3)], lane per (k1, g3)
      for (int kg = lane; kg < NB * Q; kg += 32) {
        const int k1 = kg % NB, g3 = kg / NB;
        MT x[Q];
#pragma unroll
        for (int g = 0; g < Q; ++g) x[g] = S1[k1 + NB * (g + Q * g3)];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          MT v = MT(0);
#pragma unroll
          for (int g = 0; g < Q; ++g) v += PL[(1 * NB + k) * Q + g] * x[g];
          S2[k1 + NB * (k + NB * g3)] = v;
        }
      }
      __syncwarp();
      // stage 3: mu[k12][k3] += sum_g3 PL3[k3][g3] S2[k12 + NB^2 g3], lane per k12
      if (REGB) {
        MT pl3[NB][Q];
#pragma unroll
        for (int k = 0; k < NB; ++k)
#pragma unroll
          for (int g = 0; g < Q; ++g) pl3[k][g] = PL[(2 * NB + k) * Q + g];
#pragma unroll
        for (int r = 0; r < (REGB ? MPL : 1); ++r) {
          const int k12 = lane + 32 * r;
          if (k12 < NB * NB) {
            MT x[Q];
#pragma unroll
            for (int g = 0; g < Q; ++g) x[g] = S2[k12 + NB * NB * g];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
              MT v = MT(0);
#pragma unroll
              for (int g = 0; g < Q; ++g) v += pl3[k][g] * x[g];
              macc[r][k] += v;
            }
          }
        }
      } else {
        for (int k12 = lane; k12 < NB * NB; k12 += 32) {
          MT x[Q];
#pragma unroll
          for (int g = 0; g < Q; ++g) x[g] = S2[k12 + NB * NB * g];
          for (int k = 0; k < NB; ++k) {
            MT v = MT(0);
#pragma unroll
            for (int g = 0; g < Q; ++g) v += PL[(2 * NB + k) * Q + g] * x[g];
            mw[k12 + NB * NB * k] += v;
          }
        }
      }
      __syncwarp();
    }
    // the warp's moments into its slot (mu index k12 + NB^2 k3)
#pragma unroll
    for (int r = 0; r < (REGB ? MPL : 0); ++r) {
      const int k12 = lane + 32 * r;
      if (k12 < NB * NB) {
#pragma unroll
        for (int k = 0; k < NB; ++k) mw[k12 + NB * NB * k] = macc[r][k];
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NB3; t += blockDim.x) {
    MT s = MT(0);
    for (int w = 0; w < nwarps; ++w) s += muw[(size_t)w * NB3 + t];
    mu[t] = s;
  }
  __syncthreads();

  // ---- E from the moments.  mu index t = k1 + NB (k2 + NB k3).
  const R* G1 = Gs + 0 * Q2 * NB;
  const R* G2 = Gs + 1 * Q2 * NB;
  const R* G3 = Gs + 2 * Q2 * NB;
  const R* Gd1 = Gs + 3 * Q2 * NB;
  const R* Gd2 = Gs + 4 * Q2 * NB;
  const R* Gd3 = Gs + 5 * Q2 * NB;
  // X1[ab1][k3][k2] = sum_k1 G1[ab1][k1] mu[k1 k2 k3]  (and Gd1)
  for (int t = threadIdx.x; t < Q2 * NB * NB; t += blockDim.x) {
    const int k23 = t % (NB * NB), ab1 = t / (NB * NB);
    R s = R(0), sd = R(0);
    for (int k1 = 0; k1 < NB; ++k1) {
      R m = (R)mu[k1 + NB * k23];
      s += G1[ab1 * NB + k1] * m;
      if (STIFF) sd += Gd1[ab1 * NB + k1] * m;
    }
    X1[t] = s;
    if (STIFF) X1[Q2 * NB * NB + t] = sd;
  }
  __syncthreads();
  R* Eo = E + (size_t)ci * Q3 * Q3;
  for (int ab1 = 0; ab1 < Q2; ++ab1) {
    const int a1 = ab1 / Q, b1 = ab1 % Q;
    // Y[.][ab2][k3] = sum_k2 G2[ab2][k2] X1[ab1][k3][k2]
    for (int t = threadIdx.x; t < Q2 * NB; t += blockDim.x) {
      const int k3 = t % NB, ab2 = t / NB;
      R ya = R(0), yb = R(0), yc = R(0);
      for (int k2 = 0; k2 < NB; ++k2) {
        R x = X1[(ab1 * NB + k3) * NB + k2];
        yc += G2[ab2 * NB + k2] * x;
        if (STIFF) {
          R xd = X1[Q2 * NB * NB + (ab1 * NB + k3) * NB + k2];
          ya += G2[ab2 * NB + k2] * xd;
          yb += Gd2[ab2 * NB + k2] * x;
        }
      }
      Y[t] = STIFF ? ya + yb : yc;
      if (STIFF) Y[Q2 * NB + t] = yc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Q2 * Q2; t += blockDim.x) {
      const int ab3 = t % Q2, ab2 = t / Q2;
      R s = R(0);
      for (int k3 = 0; k3 < NB; ++k3) {
        s += G3[ab3 * NB + k3] * Y[ab2 * NB + k3];
        if (STIFF) s += Gd3[ab3 * NB + k3] * Y[Q2 * NB + ab2 * NB + k3];
      }
      const int a2 = ab2 / Q, b2 = ab2 % Q, a3 = ab3 / Q, b3 = ab3 % Q;
      Eo[(size_t)(a1 + Q * (a2 + Q * a3)) * Q3 + (b1 + Q * (b2 + Q * b3))] = s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Generic 3-stage sum factorisation over a tensor grid of points, accumulated into the
// row's dense band.  Directions are contracted in the order f, s, t (first, second, third);
// for each of them the caller passes the number of points m*, of output functions n*,
// the value and derivative tables T*0/T*1 ([n*][m*]), the superset indices of the points,
// the stride of that direction in the coefficient grid and in the band accumulator.
// Mass:      V = Tt0 (Ts0 (Tf0 C))
// Stiffness: V = Tt0 (Ts0 (Tf1 C) + Ts1 (Tf0 C)) + Tt1 (Ts0 (Tf0 C))
// Everything is passed as scalars (no runtime-indexed local arrays).
template <typename R>
struct SFDir {
  int m, nf;
  const R *t0, *t1;
  const int* sidx;
  int64_t cstride;
  int astride;
};

template <typename R, bool STIFF>
__device__ void sf_accumulate(const R* __restrict__ Csup, const SFDir<R> F, const SFDir<R> Sd, const SFDir<R> Td,
                              int acc0, R* U, R* TBv, R* acc) {
  const int mf = F.m, ms = Sd.m, mt = Td.m;
  const int nff = F.nf, nfs = Sd.nf, nft = Td.nf;
  // U[kk][bf][ms][mt]
  for (int task = threadIdx.x; task < nff * ms * mt; task += blockDim.x) {
    const int it = task % mt, is = (task / mt) % ms, bf = task / (mt * ms);
    const int64_t base = Sd.sidx[is] * Sd.cstride + Td.sidx[it] * Td.cstride;
    R u0 = R(0), u1 = R(0);
    for (int k = 0; k < mf; ++k) {
      const R c = (R)Csup[base + F.sidx[k] * F.cstride];
      u0 += F.t0[bf * mf + k] * c;
      if (STIFF) u1 += F.t1[bf * mf + k] * c;
    }
    U[task] = u0;
    if (STIFF) U[nff * ms * mt + task] = u1;
  }
  __syncthreads();
  // TB[kk'][bf][bs][mt]
  for (int task = threadIdx.x; task < nff * nfs * mt; task += blockDim.x) {
    const int it = task % mt, bs = (task / mt) % nfs, bf = task / (mt * nfs);
    R ta = R(0), tb = R(0);
    for (int k = 0; k < ms; ++k) {
      const R u0 = U[(bf * ms + k) * mt + it];
      const R w0 = Sd.t0[bs * ms + k];
      if (STIFF) {
        const R u1 = U[nff * ms * mt + (bf * ms + k) * mt + it];
        const R w1 = Sd.t1[bs * ms + k];
        ta += w0 * u1 + w1 * u0;
        tb += w0 * u0;
      } else {
        ta += w0 * u0;
      }
    }
    TBv[task] = ta;
    if (STIFF) TBv[nff * nfs * mt + task] = tb;
  }
  __syncthreads();
  // V[bf][bs][bt] -> acc (distinct outputs per thread within this call)
  for (int task = threadIdx.x; task < nff * nfs * nft; task += blockDim.x) {
    const int bt = task % nft, bs = (task / nft) % nfs, bf = task / (nft * nfs);
    R v = R(0);
    for (int k = 0; k < mt; ++k) {
      v += Td.t0[bt * mt + k] * TBv[(bf * nfs + bs) * mt + k];
      if (STIFF) v += Td.t1[bt * mt + k] * TBv[nff * nfs * mt + (bf * nfs + bs) * mt + k];
    }
    acc[acc0 + bf * F.astride + bs * Sd.astride + bt * Td.astride] += v;
  }
  __syncthreads();
}

__device__ __forceinline__ int sel3(int d, int a, int b, int c) { return d == 0 ? a : (d == 1 ? b : c); }

template <typename R>
struct GTab;
template <>
struct GTab<double> {
  __device__ static const double* ge(const Dir1D& D, int kk) { return kk ? D.GEd : D.GE; }
};
template <>
struct GTab<float> {
  __device__ static const float* ge(const Dir1D& D, int kk) { return kk ? D.GEdf : D.GEf; }
};

// One block per cut row.  The DWQ box (regular part) is contracted by the whole block; the
// remaining support elements are spread over the warps (fixed assignment), each warp adding
// its elements' contributions into its own band accumulator: element Gauss sums for inside
// elements outside the box, a row of the element matrix for cut elements.  The warp
// accumulators are summed in a fixed order at the end.
template <typename R, int P, bool STIFF>
__global__ void __launch_bounds__(256) k_cut_rows(MeshView M, const R* __restrict__ Csup, const R* __restrict__ E,
                                                  R* __restrict__ values, int MMAX, int MS, int UNI) {
  constexpr int Q = P + 1, NB = 2 * P + 1, Q3 = Q * Q * Q, NB3 = NB * NB * NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = M.topo.cut_rows[blockIdx.x];
  const int n1 = M.dir[0].n, n2 = M.dir[1].n;
  const int i1 = row % n1, i2 = (row / n1) % n2, i3 = row / (n1 * n2);
  const int32_t bcode = M.topo.box[row];

  R* accw = reinterpret_cast<R*>(smem_raw);              // [nw][NB^3], index dj1 + NB (dj2 + NB dj3)
  R* uni = accw + (size_t)nw * NB3;                      // union: box buffers | per-warp element scratch
  // box buffers
  R* tabs = uni;                                         // [3][2][NB*MMAX]
  R* U = tabs + 3 * 2 * NB * MMAX;                       // [2][NB][MS][MS]
  R* TBv = U + 2 * NB * MS * MS;                         // [2][NB][NB][MS]
  int* sidx_s = reinterpret_cast<int*>(TBv + 2 * NB * NB * MS);  // [3][MMAX]
  // per-warp element scratch: C [Q3], U0/U1 [Q3 each], TA/TB [Q3 each]
  R* ws = uni + (size_t)warp * 5 * Q3;

  for (int t = threadIdx.x; t < nw * NB3; t += blockDim.x) accw[t] = R(0);
  const int64_t cs1 = 1, cs2 = M.dir[0].nsup, cs3 = (int64_t)M.dir[0].nsup * M.dir[1].nsup;
  const int elo1 = max(0, i1 - P), ehi1 = min(M.dir[0].n_el - 1, i1);
  const int elo2 = max(0, i2 - P), ehi2 = min(M.dir[1].n_el - 1, i2);
  const int elo3 = max(0, i3 - P), ehi3 = min(M.dir[2].n_el - 1, i3);
  int bd = -1, bb = 0, bside = 0;
  if (bcode >= 0) {
    bd = bcode & 3;
    bside = (bcode >> 2) & 1;
    bb = bcode >> 3;
  }
  __syncthreads();

  // ---- DWQ box (regular part): direction bd is contracted first; result in accumulator 0
  if (bd >= 0) {
    R* tb00 = tabs + 0 * NB * MMAX;
    R* tb01 = tabs + 1 * NB * MMAX;
    R* tb10 = tabs + 2 * NB * MMAX;
    R* tb11 = tabs + 3 * NB * MMAX;
    R* tb20 = tabs + 4 * NB * MMAX;
    R* tb21 = tabs + 5 * NB * MMAX;
    int* sx0 = sidx_s;
    int* sx1 = sidx_s + MMAX;
    int* sx2 = sidx_s + 2 * MMAX;
    int m0 = 0, m1 = 0, m2 = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const Dir1D& D = M.dir[d];
      const int id = sel3(d, i1, i2, i3), elo = sel3(d, elo1, elo2, elo3), ehi = sel3(d, ehi1, ehi2, ehi3);
      R* t0 = d == 0 ? tb00 : (d == 1 ? tb10 : tb20);
      R* t1 = d == 0 ? tb01 : (d == 1 ? tb11 : tb21);
      int* sx = d == 0 ? sx0 : (d == 1 ? sx1 : sx2);
      int m;
      if (d == bd) {
        const int ka = bside == 0 ? elo : bb, kb = bside == 0 ? bb - 1 : ehi;
        const int s0 = ka * Q;
        m = (kb - ka + 1) * Q;
        const int rule = ((id * P) + (bb - elo - 1)) * 2 + bside;
        const int slo = s0 - elo * Q;
        for (int t = threadIdx.x; t < NB * m; t += blockDim.x) {
          const int dj = t / m, k = t % m;
          t0[t] = CTab<R>::wd(D, 0)[((size_t)rule * NB + dj) * D.nsl + slo + k];
          t1[t] = STIFF ? CTab<R>::wd(D, 1)[((size_t)rule * NB + dj) * D.nsl + slo + k] : R(0);
        }
        for (int t = threadIdx.x; t < m; t += blockDim.x) sx[t] = s0 + t;
      } else {
        m = D.nqi[id];
        const int q0 = D.qlo[id];
        for (int t = threadIdx.x; t < NB * m; t += blockDim.x) {
          const int dj = t / m, k = t % m;
          t0[t] = CTab<R>::wb(D, 0)[((size_t)id * NB + dj) * D.nql + k];
          t1[t] = STIFF ? CTab<R>::wb(D, 1)[((size_t)id * NB + dj) * D.nql + k] : R(0);
        }
        for (int t = threadIdx.x; t < m; t += blockDim.x) sx[t] = D.wq_idx[q0 + t];
      }
      if (d == 0) m0 = m;
      if (d == 1) m1 = m;
      if (d == 2) m2 = m;
    }
    __syncthreads();
    const SFDir<R> D0{m0, NB, tb00, tb01, sx0, cs1, 1};
    const SFDir<R> D1{m1, NB, tb10, tb11, sx1, cs2, NB};
    const SFDir<R> D2{m2, NB, tb20, tb21, sx2, cs3, NB * NB};
    if (bd == 0) sf_accumulate<R, STIFF>(Csup, D0, D1, D2, 0, U, TBv, accw);
    else if (bd == 1) sf_accumulate<R, STIFF>(Csup, D1, D0, D2, 0, U, TBv, accw);
    else sf_accumulate<R, STIFF>(Csup, D2, D0, D1, 0, U, TBv, accw);
  }

  // ---- remaining support elements, one warp per element
  R* acc = accw + (size_t)warp * NB3;
  const int w1 = ehi1 - elo1 + 1, w2 = ehi2 - elo2 + 1, w3 = ehi3 - elo3 + 1;
  const int nsup = w1 * w2 * w3;
  for (int t = warp; t < nsup; t += nw) {
    const int e1 = elo1 + t % w1, e2 = elo2 + (t / w1) % w2, e3 = elo3 + t / (w1 * w2);
    const int64_t e = e1 + (int64_t)M.dir[0].n_el * (e2 + (int64_t)M.dir[1].n_el * e3);
    const int8_t st = M.topo.elem_state[e];
    const int o1 = e1 - i1 + P, o2 = e2 - i2 + P, o3 = e3 - i3 + P;
    if (st == E_IN) {
      if (bd >= 0) {
        const int ed = sel3(bd, e1, e2, e3);
        if ((bside == 0 && ed < bb) || (bside == 1 && ed >= bb)) continue;
      }
      // F_d[b][g] = w(s) B_{i_d}(s) B_{e_d+b}(s) (derivatives for kk = 1), from the tables
      const R* F0 = GTab<R>::ge(M.dir[0], 0) + ((size_t)e1 * Q + (i1 - e1)) * Q * Q;
      const R* F1 = GTab<R>::ge(M.dir[1], 0) + ((size_t)e2 * Q + (i2 - e2)) * Q * Q;
      const R* F2 = GTab<R>::ge(M.dir[2], 0) + ((size_t)e3 * Q + (i3 - e3)) * Q * Q;
      const R* F0d = GTab<R>::ge(M.dir[0], 1) + ((size_t)e1 * Q + (i1 - e1)) * Q * Q;
      const R* F1d = GTab<R>::ge(M.dir[1], 1) + ((size_t)e2 * Q + (i2 - e2)) * Q * Q;
      const R* F2d = GTab<R>::ge(M.dir[2], 1) + ((size_t)e3 * Q + (i3 - e3)) * Q * Q;
      R* C = ws;            // [g3][g2][g1]
      R* U0 = ws + Q3;      // [g3][g2][b1]
      R* U1 = ws + 2 * Q3;
      R* TA = ws + 3 * Q3;  // [g3][b2][b1]
      R* TB = ws + 4 * Q3;
      for (int k = lane; k < Q3; k += 32) {
        const int g1 = k % Q, g2 = (k / Q) % Q, g3 = k / (Q * Q);
        C[k] = (R)Csup[(e1 * Q + g1) * cs1 + (e2 * Q + g2) * cs2 + (e3 * Q + g3) * cs3];
      }
      __syncwarp();
      for (int k = lane; k < Q3; k += 32) {  // contract g1
        const int b1 = k % Q, g23 = k / Q;
        R u0 = R(0), u1 = R(0);
#pragma unroll
        for (int g = 0; g < Q; ++g) {
          const R c = C[g + Q * g23];
          u0 += F0[b1 * Q + g] * c;
          if (STIFF) u1 += F0d[b1 * Q + g] * c;
        }
        U0[k] = u0;
        if (STIFF) U1[k] = u1;
      }
      __syncwarp();
      for (int k = lane; k < Q3; k += 32) {  // contract g2
        const int b1 = k % Q, b2 = (k / Q) % Q, g3 = k / (Q * Q);
        R ta = R(0), tb = R(0);
#pragma unroll
        for (int g = 0; g < Q; ++g) {
          const R x0 = U0[b1 + Q * (g + Q * g3)];
          if (STIFF) {
            const R x1 = U1[b1 + Q * (g + Q * g3)];
            ta += F1[b2 * Q + g] * x1 + F1d[b2 * Q + g] * x0;
            tb += F1[b2 * Q + g] * x0;
          } else {
            ta += F1[b2 * Q + g] * x0;
          }
        }
        TA[k] = ta;
        if (STIFF) TB[k] = tb;
      }
      __syncwarp();
      for (int k = lane; k < Q3; k += 32) {  // contract g3 and add
        const int b1 = k % Q, b2 = (k / Q) % Q, b3 = k / (Q * Q);
        R v = R(0);
#pragma unroll
        for (int g = 0; g < Q; ++g) {
          v += F2[b3 * Q + g] * TA[b1 + Q * (b2 + Q * g)];
          if (STIFF) v += F2d[b3 * Q + g] * TB[b1 + Q * (b2 + Q * g)];
        }
        acc[(o3 + b3) * NB * NB + (o2 + b2) * NB + (o1 + b1)] += v;
      }
      __syncwarp();
    } else if (st == E_CUT) {
      // element matrix row a(i) of this cut element
      const int ci = M.topo.elem_cut_id[e];
      const int a = (i1 - e1) + Q * ((i2 - e2) + Q * (i3 - e3));
      const R* Er = E + ((size_t)ci * Q3 + a) * Q3;
      for (int k = lane; k < Q3; k += 32) {
        const int b1 = k % Q, b2 = (k / Q) % Q, b3 = k / (Q * Q);
        acc[(o3 + b3) * NB * NB + (o2 + b2) * NB + (o1 + b1)] += Er[k];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // ---- fixed-order sum of the warp accumulators, written on the row's pattern
  const int64_t r0 = M.topo.rowptr[row], r1 = M.topo.rowptr[row + 1];
  for (int64_t k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
    const int j = M.topo.colind[k];
    const int j1 = j % n1, j2 = (j / n1) % n2, j3 = j / (n1 * n2);
    const int o = ((j3 - i3 + P) * NB + (j2 - i2 + P)) * NB + (j1 - i1 + P);
    R v = R(0);
    for (int w = 0; w < nw; ++w) v += accw[(size_t)w * NB3 + o];
    values[k] = v;
  }
  (void)UNI;
}

template <typename R, typename MT, int P, bool STIFF>
cudaError_t launch_cut_t(const MeshView& M, const LevelSet& L, int coef_kind, double c0, const double* ck,
                         const R* Csup, R* E, R* values, int n_cut_elems, int n_cut_rows, int part,
                         cudaStream_t st) {
  constexpr int Q = P + 1, NB = 2 * P + 1, Q3 = Q * Q * Q, NB3 = NB * NB * NB, Q2 = Q * Q;
  cudaError_t err = cudaSuccess;
  if (part == 0 && n_cut_elems > 0) {
    const int nwarps = (P >= 5) ? 4 : 8;
    const int WS = Q3 + NB * Q2 + NB * NB * Q + 3 * NB * Q + 3 * Q + 3 * Q * Q;
    size_t partA = (size_t)(nwarps * NB3 + nwarps * WS + Q3) * sizeof(MT);
    size_t partB = (size_t)(2 * Q2 * NB * NB + 2 * Q2 * NB) * sizeof(R);
    size_t smem = (size_t)((NB3 + 1) / 2) * 2 * sizeof(MT) + (size_t)((2 * 3 * Q2 * NB + 1) / 2) * 2 * sizeof(R) +
                  (partA > partB ? partA : partB) + 16;
    err = cudaFuncSetAttribute(k_cut_elemmat<R, MT, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    CoefDesc cf{coef_kind, c0, ck};
    k_cut_elemmat<R, MT, P, STIFF><<<n_cut_elems, 32 * nwarps, smem, st>>>(M, L, cf, E);
    SFA_LAUNCHED(1);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (part == 1 && n_cut_rows > 0) {
    int MS = Q;  // points of a non-DWQ direction: WQ points of a support or an element's Gauss points
    for (int d = 0; d < 3; ++d) MS = MS > M.dir[d].nql ? MS : M.dir[d].nql;
    const int MMAX = MS > P * Q ? MS : P * Q;  // plus the kept side of a DWQ rule
    const int nw = (sizeof(R) == 8 && P >= 5) ? 4 : 8;
    const size_t box = (size_t)(3 * 2 * NB * MMAX + 2 * NB * MS * MS + 2 * NB * NB * MS) * sizeof(R) + 3 * MMAX * sizeof(int);
    const size_t elem = (size_t)nw * 5 * Q3 * sizeof(R);
    const size_t uni = box > elem ? box : elem;
    size_t smem = (size_t)nw * NB3 * sizeof(R) + uni + 16;
    err = cudaFuncSetAttribute(k_cut_rows<R, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_cut_rows<R, P, STIFF><<<n_cut_rows, 32 * nw, smem, st>>>(M, Csup, E, values, MMAX, MS, (int)uni);
    SFA_LAUNCHED(1);
    err = cudaGetLastError();
  }
  return err;
}

}  // namespace

cudaError_t launch_cut(const MeshView& M, const LevelSet& L, bool fp64, bool mom64, bool stiff, int coef_kind,
                       double c0, const double* ck, const void* Csup, void* E, void* values, int n_cut_elems,
                       int n_cut_rows, int part, cudaStream_t st) {
#define SFA_CUT_ARGS(RT) M, L, coef_kind, c0, ck, (const RT*)Csup, (RT*)E, (RT*)values, n_cut_elems, n_cut_rows, part, st
#define SFA_CUT_CASE(PP)                                                                                        \
  case PP:                                                                                                      \
    if (fp64)                                                                                                   \
      return stiff ? launch_cut_t<double, double, PP, true>(SFA_CUT_ARGS(double))                              \
                   : launch_cut_t<double, double, PP, false>(SFA_CUT_ARGS(double));                             \
    if (mom64)                                                                                                  \
      return stiff ? launch_cut_t<float, double, PP, true>(SFA_CUT_ARGS(float))                                 \
                   : launch_cut_t<float, double, PP, false>(SFA_CUT_ARGS(float));                               \
    return stiff ? launch_cut_t<float, float, PP, true>(SFA_CUT_ARGS(float))                                    \
                 : launch_cut_t<float, float, PP, false>(SFA_CUT_ARGS(float));
  switch (M.p) {
    SFA_CUT_CASE(2)
    SFA_CUT_CASE(3)
    SFA_CUT_CASE(4)
    SFA_CUT_CASE(5)
    SFA_CUT_CASE(6)
  }
#undef SFA_CUT_CASE
#undef SFA_CUT_ARGS
  return cudaErrorInvalidValue;
}
