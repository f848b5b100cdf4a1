// Cut-element matrices (Sec. 3.1: cut elements integrated with Gauss points on sub-cells).
// Cut elements are shared by up to (p+1)^3 rows, so each is integrated once:
//   mu_e[k1,k2,k3] = sum_pieces sum_g w_g c(x_g) b_k1(t_1) b_k2(t_2) b_k3(t_3)
// (accumulated in double under SFA_FP64, SFA_FP32_M64 and SFA_TF32X3_M64, in float under the
// other precisions)
// with b_k the degree-2p Bernstein polynomials of the element (t in [0, 1]).  B_a B_b
// restricted to the element is a polynomial of degree <= 2p per direction with Bernstein
// coefficients G[a][b][k] >= 0, so E_e[a][b] = sum_k G1[a1 b1 k1] G2[a2 b2 k2] G3[a3 b3 k3]
// mu_e[k] equals the Gauss sum over the pieces up to rounding, and for the mass matrix with
// c > 0 every term is non-negative (no cancellation, whatever the size of the domain part).
// Each cut row (cut.cu) then adds row a(i) of E_e for its cut elements.
#include "cut_common.cuh"

namespace {

// ---------------------------------------------------------------------------------------
// Bernstein moments of one cut element, grouped by octree position.  The coefficient on
// the element is a sum of separable terms, c(x) = sum_a K[a1][a2][a3] f_a1(x1) f_a2(x2)
// f_a3(x3) (B-spline: A = p+1 basis functions and K the coefficient block; analytic
// 1 + 0.5 sin(2 pi x) cos(2 pi y) z: A = 2; constant: A = 1), and a piece at octree level l,
// position (a1p, a2p, a3p) contributes (T1 x T2 x T3) K with the 1D tables
//   T_d[pos][a][k] = sum_g w_d(g) f_a(t_g) b_k(t_g)          (pos = 2^l - 1 + a_dp)
// over its p+1 Gauss points per direction.  By linearity the pieces of one (l, a2p, a3p)
// slot share stages 2 and 3 (their T1 tables are summed first, in increasing a1p), and the
// slots of one (l, a3p) group share stage 3:
//   X1 = T1sum x_1 K,   X2g += T2 x_2 X1 (slots of the group),   mu += T3 x_3 X2g.
// This is the Gauss sum of the pieces (Sec. 3.1) with the sums reordered.  Each group is
// handled by one warp; groups are dealt to the warps by decreasing size to balance them, a
// warp takes its groups in increasing order, and the per-warp moments are reduced into mu in
// warp order (deterministic).
template <typename MT, int P, int A, int NW>
__device__ void moments_grouped(const MeshView& M, int kind, int ee0, int ee1, int ee2, const uint32_t* __restrict__ pcs,
                                int np, const MT* __restrict__ K, MT* Tpos, uint32_t* smask, int* slist, int* gstart,
                                int* cnt, MT* wscr, int WSG, MT* mu) {
  constexpr int Q = P + 1, NB = 2 * P + 1, PTF = NB + Q + 2;
  constexpr int MPL = (NB * NB + 31) / 32;
  int* gw = cnt + 2;  // warp of each group
  const int D = M.D;
  const int npos = (1 << (D + 1)) - 1, nslot = ((1 << (2 * (D + 1))) - 1) / 3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per-position tables T_d[pos][a][k]
  for (int t = threadIdx.x; t < 3 * npos * A * NB; t += blockDim.x) {
    const int k = t % NB, a = (t / NB) % A, pos = (t / (NB * A)) % npos, d = t / (NB * A * npos);
    const Dir1D& Dd = M.dir[d];
    const int64_t row0 = ((int64_t)sel3(d, ee0, ee1, ee2) * Dd.npos + pos) * Q;
    MT v = MT(0);
#pragma unroll
    for (int g = 0; g < Q; ++g) {
      const MT* src = sizeof(MT) == 4 ? reinterpret_cast<const MT*>(Dd.PTf + (row0 + g) * PTF)
                                      : reinterpret_cast<const MT*>(Dd.PT + (row0 + g) * PTF);
      MT f = MT(1);
      if (kind == SFA_COEF_BSPLINE) f = src[1 + NB + a];
      else if (kind == SFA_COEF_ANALYTIC && a == 1) f = src[1 + NB + Q];
      v += src[0] * f * src[1 + k];
    }
    Tpos[t] = v;
  }
  for (int t = threadIdx.x; t < nslot; t += blockDim.x) smask[t] = 0u;
  __syncthreads();
  // slot of every piece: (l, a2p, a3p), bit a1p
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    const uint32_t code = pcs[t];
    const int l = code & 15, a1p = (code >> 4) & 63, a2p = (code >> 10) & 63, a3p = (code >> 16) & 63;
    const int sb = ((1 << (2 * l)) - 1) / 3;
    atomicOr(&smask[sb + a2p + (a3p << l)], 1u << a1p);
  }
  __syncthreads();
  // nonempty slots in (l, a3p, a2p) order, then the starts of the (l, a3p) groups
  auto group_of = [](int sidx) {
    int l = 0;
    while (((1 << (2 * (l + 1))) - 1) / 3 <= sidx) ++l;
    return ((1 << l) - 1) + ((sidx - ((1 << (2 * l)) - 1) / 3) >> l);
  };
  if (warp == 0) {
    int base = 0;
    for (int c = 0; c < nslot; c += 32) {
      const int sl = c + lane;
      const bool live = sl < nslot && smask[sl] != 0u;
      const unsigned m = __ballot_sync(0xffffffffu, live);
      if (live) slist[base + __popc(m & ((1u << lane) - 1u))] = sl;
      base += __popc(m);
    }
    __syncwarp();
    int ng = 0;
    for (int c = 0; c < base; c += 32) {
      const int i = c + lane;
      bool start = false;
      if (i < base) start = i == 0 || group_of(slist[i]) != group_of(slist[i - 1]);
      const unsigned ms = __ballot_sync(0xffffffffu, start);
      if (start) gstart[ng + __popc(ms & ((1u << lane) - 1u))] = i;
      ng += __popc(ms);
    }
    if (lane == 0) {
      gstart[ng] = base;
      cnt[0] = base;
      cnt[1] = ng;
    }
    __syncwarp();
    // groups to warps: rank by work (slots, then the group's final contraction), largest
    // first, ties by index; ranks dealt to the warps back and forth (0..NW-1, NW-1..0, ...)
    for (int g = lane; g < ng; g += 32) {
      const int cg = 4 * (gstart[g + 1] - gstart[g]) + 5;
      int rank = 0;
      for (int h = 0; h < ng; ++h) {
        const int ch = 4 * (gstart[h + 1] - gstart[h]) + 5;
        rank += (ch > cg) || (ch == cg && h < g);
      }
      const int round = rank / NW, k = rank % NW;
      gw[g] = (round & 1) ? NW - 1 - k : k;
    }
  }
  __syncthreads();
  const int ngroups = cnt[1];
  MT* T1s = wscr + (size_t)warp * WSG;              // [A][NB]
  MT* X1 = T1s + rup4(A * NB);                      // [a2][a3][k1]
  MT* X2 = X1 + rup4(A * A * NB);                   // [a3][k1][k2]
  MT macc[MPL][NB];
#pragma unroll
  for (int r = 0; r < MPL; ++r)
#pragma unroll
    for (int k = 0; k < NB; ++k) macc[r][k] = MT(0);
  for (int g = 0; g < ngroups; ++g) {
    if (gw[g] != warp) continue;
    for (int t = lane; t < A * NB * NB; t += 32) X2[t] = MT(0);
    int l = 0, a3p = 0;
    for (int i = gstart[g]; i < gstart[g + 1]; ++i) {
      const int s = slist[i];
      l = 0;
      while (((1 << (2 * (l + 1))) - 1) / 3 <= s) ++l;
      const int r = s - ((1 << (2 * l)) - 1) / 3;
      const int a2p = r & ((1 << l) - 1);
      a3p = r >> l;
      const uint32_t mask = smask[s];
      // T1 summed over the slot's pieces, increasing a1p
      for (int t = lane; t < A * NB; t += 32) {
        MT v = MT(0);
        uint32_t mm = mask;
        while (mm) {
          const int a1p = __ffs(mm) - 1;
          mm &= mm - 1;
          v += Tpos[(size_t)((0 * npos) + (1 << l) - 1 + a1p) * A * NB + t];
        }
        T1s[t] = v;
      }
      __syncwarp();
      // X1[a2][a3][k1] = sum_a1 K[a1][a2][a3] T1s[a1][k1]
      for (int t = lane; t < A * A * NB; t += 32) {
        const int k1 = t % NB, a23 = t / NB;
        MT v = MT(0);
#pragma unroll
        for (int a1 = 0; a1 < A; ++a1) v += K[a1 + A * a23] * T1s[a1 * NB + k1];
        X1[t] = v;
      }
      __syncwarp();
      // X2[a3][k1][k2] += sum_a2 X1[a2][a3][k1] T2[pos][a2][k2]
      const MT* T2 = Tpos + (size_t)(1 * npos + (1 << l) - 1 + a2p) * A * NB;
      for (int t = lane; t < A * NB * NB; t += 32) {
        const int k2 = t % NB, k1 = (t / NB) % NB, a3 = t / (NB * NB);
        MT v = MT(0);
#pragma unroll
        for (int a2 = 0; a2 < A; ++a2) v += X1[(a2 + A * a3) * NB + k1] * T2[a2 * NB + k2];
        X2[(a3 * NB + k1) * NB + k2] += v;
      }
      __syncwarp();
    }
    // mu[k12 + NB^2 k3] += sum_a3 T3[pos][a3][k3] X2[a3][k12]   (k12 = k1 NB + k2 here)
    const MT* T3 = Tpos + (size_t)(2 * npos + (1 << l) - 1 + a3p) * A * NB;
    MT t3[A][NB];
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int k = 0; k < NB; ++k) t3[a][k] = T3[a * NB + k];
#pragma unroll
    for (int r = 0; r < MPL; ++r) {
      const int k12 = lane + 32 * r;
      if (k12 < NB * NB) {
        MT x[A];
#pragma unroll
        for (int a = 0; a < A; ++a) x[a] = X2[a * NB * NB + k12];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          MT v = MT(0);
#pragma unroll
          for (int a = 0; a < A; ++a) v += t3[a][k] * x[a];
          macc[r][k] += v;
        }
      }
    }
    __syncwarp();
  }
  // warp moments into mu in warp order; the moment index of (k1, k2, k3) is k1 + NB (k2 + NB k3)
  for (int w = 0; w < NW; ++w) {
    if (warp == w) {
#pragma unroll
      for (int r = 0; r < MPL; ++r) {
        const int k12 = lane + 32 * r;
        if (k12 < NB * NB) {
          const int k1 = k12 / NB, k2 = k12 % NB;
#pragma unroll
          for (int k = 0; k < NB; ++k) mu[k1 + NB * (k2 + NB * k)] += macc[r][k];
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Moments through degree-3p piece moments (B-spline or constant coefficient).  On a cut
// element the coefficient is a polynomial of degree p per direction with Bernstein
// coefficients K'[k] = sum_a K[a] BZ1[a1][k1] BZ2[a2][k2] BZ3[a3][k3] (BZ: the Bezier
// coefficients of the B-splines on the element), and b^p_k b^2p_j = C(p,k) C(2p,j)
// t^(k+j) (1-t)^(3p-k-j) per direction, so with the pieces' monomial moments
//   nu[m] = sum_pieces sum_g w_g prod_d t_d^m_d (1 - t_d)^(3p - m_d)
// (a product of the per-direction tables P3 for each piece) the Gauss sums of the method are
//   mu[j] = prod_d C(2p, j_d) sum_k K''[k] nu[k + j],   K''[k] = K'[k] prod_d C(p, k_d).
// This is the same sum over the pieces' Gauss points, reordered: the pieces are accumulated
// once, without the coefficient (slots and groups as in moments_grouped, now on vectors), and
// the coefficient enters through one correlation.  For c > 0 every term is non-negative.
constexpr int binom_i(int n, int k) {
  int v = 1;
  for (int r = 1; r <= k; ++r) v = v * (n - k + r) / r;
  return v;
}

template <typename MT, int P, typename CT = MT>
struct B3Plan {
  static constexpr int Q = P + 1, Q3 = Q * Q * Q, M3 = 3 * P + 1;
  // offsets (elements of MT) for octree depth D: Kb | Kt | Tp[3][npos][M3] | U[npos][M3^2] |
  // T1s[nslot][M3], later nu[M3^3] in the same place (T1s is dead once U is formed), then the
  // slot lists (ints): the slot masks of the three orientations, slist, gstart, per-slot level
  // and middle position, per-group outer position, counts
  __host__ __device__ static int npos(int D) { return (2 << D) - 1; }
  __host__ __device__ static int nslot(int D) { return ((1 << (2 * (D + 1))) - 1) / 3; }
  __host__ __device__ static size_t oTp() { return 2 * (size_t)rup4(Q3); }
  __host__ __device__ static size_t oU(int D) { return oTp() + rup4(3 * npos(D) * M3); }
  __host__ __device__ static size_t oT1(int D) { return oU(D) + (size_t)rup4(npos(D) * M3 * M3); }
  __host__ __device__ static size_t oNu(int D) { return oT1(D); }
  __host__ __device__ static size_t nMT(int D) {
    const size_t t1 = rup4(nslot(D) * M3), nu = (size_t)M3 * M3 * M3;
    return oT1(D) + (t1 > nu ? t1 : nu);
  }
  // the correlation's float copy of nu (double moments, float values): in the U region,
  // dead once nu is formed, where it fits; else after the slot lists
  static constexpr bool CTCOPY = sizeof(CT) != sizeof(MT);
  __host__ __device__ static size_t ct_bytes() { return (size_t)M3 * M3 * M3 * sizeof(CT); }
  __host__ __device__ static bool ct_in_u(int D) { return (size_t)npos(D) * M3 * M3 * sizeof(MT) >= ct_bytes(); }
  __host__ __device__ static size_t oCT(int D) {
    return ct_in_u(D) ? oU(D) * sizeof(MT)
                      : (nMT(D) * sizeof(MT) + (7 * (size_t)nslot(D) + npos(D) + 8) * 4 + 15) / 16 * 16;
  }
  __host__ __device__ static size_t bytes(int D) {
    const size_t base = nMT(D) * sizeof(MT) + (7 * (size_t)nslot(D) + npos(D) + 8) * 4;
    return (CTCOPY && !ct_in_u(D)) ? (base + 15) / 16 * 16 + ct_bytes() : base;
  }
};

// K: the element's (p+1)^3 B-spline coefficient block (index a1 + Q (a2 + Q a3)) already in
// work[0 .. Q3) when bspline, else the constant c0.  Writes mu[j1 + NB (j2 + NB j3)].
// The sums over the pieces (T1s, U, nu) are accumulated in MT; the correlation with the
// coefficient, a fixed map of the accumulated moments like the element-matrix expansion that
// follows it, runs in CT (the value type).  Every stage keeps several independent
// accumulators per thread (register blocking over one direction), so the FP64 pipe is fed by
// independent multiply-adds.
template <typename MT, int P, typename CT>
__device__ void moments_bern3p(const MeshView& M, int ee0, int ee1, int ee2, const uint32_t* __restrict__ pcs,
                               int np, bool bspline, MT c0, MT* work, MT* mu) {
  using B = B3Plan<MT, P, CT>;
  constexpr int Q = P + 1, Q2 = Q * Q, Q3 = Q2 * Q, NB = 2 * P + 1, M3 = B::M3, M3S = M3 * M3;
  constexpr int JB = 3, NJB = (NB + JB - 1) / JB;  // outputs per thread along j3 in the correlation
  const int D = M.D, npos = B::npos(D), nslot = B::nslot(D);
  MT* Kb = work;
  MT* Kt = work + rup4(Q3);
  MT* Tp = work + B::oTp();
  MT* T1s = work + B::oT1(D);
  MT* U = work + B::oU(D);
  MT* nu = work + B::oNu(D);
  uint32_t* smask3 = reinterpret_cast<uint32_t*>(work + B::nMT(D));  // [3][nslot]
  int* slist = reinterpret_cast<int*>(smask3 + 3 * nslot);
  int* gstart = slist + nslot;        // nslot + 1
  int* slev = gstart + nslot + 1;     // level of slot i (list order)
  int* spos2 = slev + nslot;          // middle-direction position of slot i
  int* gpos3 = spos2 + nslot;         // outer-direction position of group g
  int* cnt = gpos3 + npos;
  const int ee[3] = {ee0, ee1, ee2};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per-position tables of this element (asynchronous copies; the caller may have copies of
  // the coefficient block in flight too)
  {
    const uint32_t tps = (uint32_t)__cvta_generic_to_shared(Tp);
    for (int t = threadIdx.x; t < 3 * npos * M3; t += blockDim.x) {
      const int m = t % M3, pos = (t / M3) % npos, d = t / (M3 * npos);
      const Dir1D& Dd = M.dir[d];
      const size_t o = ((size_t)ee[d] * Dd.npos + pos) * M3 + m;
      if constexpr (sizeof(MT) == 4) cp_word_nc<4>(tps + 4u * t, Dd.P3f + o);
      else cp_word_nc<8>(tps + 8u * t, Dd.P3 + o);
    }
    cp_commit();
  }
  for (int t = threadIdx.x; t < 3 * nslot; t += blockDim.x) smask3[t] = 0u;
  cp_wait<0>();
  __syncthreads();
  // Bernstein coefficients of c on the element, scaled by C(p, k_d): a fixed map of the
  // coefficients, in CT (KA, KB2 two CT buffers; with CT narrower than MT both in the Kt
  // region, the MT coefficient block staying in Kb; the three BZ matrices in CT in the U
  // region, which the moment stages fill only later)
  CT* KA;
  CT* KB2;
  if constexpr (sizeof(CT) < sizeof(MT)) {
    KA = reinterpret_cast<CT*>(Kt);
    KB2 = KA + rup4(Q3);
  } else {
    KA = reinterpret_cast<CT*>(Kb);
    KB2 = reinterpret_cast<CT*>(Kt);
  }
  if (bspline) {
    CT* Zc = reinterpret_cast<CT*>(U);  // [d][a][k]
    for (int t = threadIdx.x; t < 3 * Q2; t += blockDim.x) {
      const int d = t / Q2, ak = t - d * Q2;
      Zc[t] = (CT)M.dir[d].BZ[(size_t)sel3(d, ee0, ee1, ee2) * Q2 + ak];
    }
    if constexpr (sizeof(CT) < sizeof(MT))
      for (int t = threadIdx.x; t < Q3; t += blockDim.x) KA[t] = (CT)Kb[t];
    __syncthreads();
    for (int t = threadIdx.x; t < Q3; t += blockDim.x) {  // KB2[k1, a2, a3] = sum_a1 K Z0[a1][k1]
      const int k1 = t % Q, a23 = t / Q;
      CT v = CT(0);
      for (int a1 = 0; a1 < Q; ++a1) v += KA[a1 + Q * a23] * Zc[a1 * Q + k1];
      KB2[t] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Q3; t += blockDim.x) {  // KA[k1, k2, a3] = sum_a2 KB2 Z1[a2][k2]
      const int k1 = t % Q, k2 = (t / Q) % Q, a3 = t / Q2;
      CT v = CT(0);
      for (int a2 = 0; a2 < Q; ++a2) v += KB2[k1 + Q * (a2 + Q * a3)] * Zc[Q2 + a2 * Q + k2];
      KA[t] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Q3; t += blockDim.x) {  // KB2[k] = sum_a3 KA Z2[a3][k3]
      const int k12 = t % Q2, k3 = t / Q2;
      CT v = CT(0);
      for (int a3 = 0; a3 < Q; ++a3) v += KA[k12 + Q2 * a3] * Zc[2 * Q2 + a3 * Q + k3];
      KB2[t] = v;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
    const int k1 = t % Q, k2 = (t / Q) % Q, k3 = t / Q2;
    const CT sc = (CT)(binom_i(P, k1) * binom_i(P, k2) * binom_i(P, k3));
    KA[t] = (bspline ? KB2[t] : (CT)c0) * sc;  // K''
  }
  // The pieces' moments nu[m] = sum_pieces prod_d T_d[pos_d][m_d] are summed direction by
  // direction: over the inner direction within a slot (level, middle position, outer
  // position), over the middle one within a group (level, outer position), then the outer
  // one.  The three cyclic orientations (inner, middle, outer) = (r, r+1, r+2 mod 3) give the
  // same sums; the one with the least FP64 work (slots M3^2 + groups M3^3) is taken.
  // Slot masks of every orientation: slot (l, a_mid, a_out), bit a_in.
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    const uint32_t code = pcs[t];
    const int l = code & 15;
    const int av[3] = {(int)((code >> 4) & 63), (int)((code >> 10) & 63), (int)((code >> 16) & 63)};
    const int sb = ((1 << (2 * l)) - 1) / 3;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int din = r, dmid = r == 2 ? 0 : r + 1, dout = r == 0 ? 2 : r - 1;
      atomicOr(&smask3[r * nslot + sb + av[dmid] + (av[dout] << l)], 1u << av[din]);
    }
  }
  __syncthreads();
  auto level_of = [](int sidx) {
    int l = 0;
    while (((1 << (2 * (l + 1))) - 1) / 3 <= sidx) ++l;
    return l;
  };
  if (warp < 3) {
    // orientation r = warp: count its nonempty slots and groups
    const int r = warp;
    const uint32_t* sm = smask3 + r * nslot;
    int nsl_r = 0, ng_r = 0;
    for (int c = 0; c < nslot; c += 32) nsl_r += __popc(__ballot_sync(0xffffffffu, c + lane < nslot && sm[c + lane] != 0u));
    for (int c = 0; c < npos; c += 32) {
      const int gp = c + lane;  // group position (2^l - 1) + a_out
      bool any = false;
      if (gp < npos) {
        const int l = 31 - __clz(gp + 1), ao = gp + 1 - (1 << l);
        const int sb = ((1 << (2 * l)) - 1) / 3 + (ao << l);
        for (int am = 0; am < (1 << l); ++am) any |= sm[sb + am] != 0u;
      }
      ng_r += __popc(__ballot_sync(0xffffffffu, any));
    }
    if (lane == 0) cnt[3 + r] = nsl_r * M3S + ng_r * M3S * M3;  // below 2^31 for D <= 4, p <= 6
  }
  __syncthreads();
  if (warp == 0) {
    int best = 0;
    for (int r = 1; r < 3; ++r)
      if (cnt[3 + r] < cnt[3 + best]) best = r;
    const uint32_t* smask = smask3 + best * nslot;
    // nonempty slots in (l, a_out, a_mid) order; starts of the (l, a_out) groups
    int base = 0;
    for (int c = 0; c < nslot; c += 32) {
      const int sl = c + lane;
      const bool live = sl < nslot && smask[sl] != 0u;
      const unsigned mk = __ballot_sync(0xffffffffu, live);
      if (live) {
        const int i = base + __popc(mk & ((1u << lane) - 1u));
        const int l = level_of(sl), r = sl - ((1 << (2 * l)) - 1) / 3;
        slist[i] = sl;
        slev[i] = l;
        spos2[i] = (1 << l) - 1 + (r & ((1 << l) - 1));
      }
      base += __popc(mk);
    }
    __syncwarp();
    int ng = 0;
    for (int c = 0; c < base; c += 32) {
      const int i = c + lane;
      bool start = false;
      int g3 = 0;
      if (i < base) {
        const int l0 = slev[i], a30 = (slist[i] - ((1 << (2 * l0)) - 1) / 3) >> l0;
        g3 = (1 << l0) - 1 + a30;
        start = i == 0 || slev[i - 1] != l0 || ((slist[i - 1] - ((1 << (2 * l0)) - 1) / 3) >> l0) != a30;
      }
      const unsigned ms = __ballot_sync(0xffffffffu, start);
      if (start) {
        const int g = ng + __popc(ms & ((1u << lane) - 1u));
        gstart[g] = i;
        gpos3[g] = g3;
      }
      ng += __popc(ms);
    }
    if (lane == 0) {
      gstart[ng] = base;
      cnt[0] = base;
      cnt[1] = ng;
      cnt[2] = best;
    }
  }
  __syncthreads();
  const int nsl = cnt[0], ng = cnt[1], rot = cnt[2];
  const int din = rot, dmid = rot == 2 ? 0 : rot + 1, dout = rot == 0 ? 2 : rot - 1;
  const uint32_t* smask = smask3 + rot * nslot;
  const MT* Tin = Tp + din * npos * M3;
  const MT* Tmid = Tp + dmid * npos * M3;
  const MT* Tout = Tp + dout * npos * M3;
  // T1s[i][m] = sum over the slot's pieces of the inner direction's table (increasing a_in)
  for (int t = threadIdx.x; t < nsl * M3; t += blockDim.x) {
    const int i = t / M3, m = t % M3;
    const int l = slev[i];
    uint32_t mm = smask[slist[i]];
    MT v = MT(0);
    while (mm) {
      const int ain = __ffs(mm) - 1;
      mm &= mm - 1;
      v += Tin[((1 << l) - 1 + ain) * M3 + m];
    }
    T1s[t] = v;
  }
  __syncthreads();
  // U[g][m1 + M3 m2] = sum over the group's slots of T1s[i][m1] T2[pos2(i)][m2], and then
  // nu[m12 + M3S m3] = sum_g U[g][m12] T3[pos3(g)][m3].  The outputs are dealt to the threads
  // round-robin, so that every warp (and so every SM sub-partition's FP64 pipe) gets the same
  // share of the multiply-adds to within one output; two independent chains per thread.
  for (int o = threadIdx.x; o < ng * M3S; o += 2 * blockDim.x) {
    const int o2 = o + blockDim.x;
    const int g = o / M3S, m12 = o - g * M3S, m1 = m12 % M3, m2 = m12 / M3;
    const bool two = o2 < ng * M3S;
    const int gb = two ? o2 / M3S : g, m12b = two ? o2 - gb * M3S : m12, m1b = m12b % M3, m2b = m12b / M3;
    MT acc = MT(0), accb = MT(0);
    for (int i = gstart[g]; i < gstart[g + 1]; ++i) acc += T1s[i * M3 + m1] * Tmid[spos2[i] * M3 + m2];
    if (two)
      for (int i = gstart[gb]; i < gstart[gb + 1]; ++i) accb += T1s[i * M3 + m1b] * Tmid[spos2[i] * M3 + m2b];
    U[(size_t)g * M3S + m12] = acc;
    if (two) U[(size_t)gb * M3S + m12b] = accb;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < M3S * M3; o += 2 * blockDim.x) {
    const int o2 = o + blockDim.x;
    const bool two = o2 < M3S * M3;
    const int m3 = o / M3S, m12 = o - m3 * M3S;
    const int m3b = two ? o2 / M3S : m3, m12b = two ? o2 - m3b * M3S : m12;
    MT acc = MT(0), accb = MT(0);
    for (int g = 0; g < ng; ++g) {
      const MT* t3 = Tout + gpos3[g] * M3;
      acc += U[(size_t)g * M3S + m12] * t3[m3];
      accb += U[(size_t)g * M3S + m12b] * t3[m3b];
    }
    // (m_in, m_mid, m_out) to the canonical index m_0 + M3 m_1 + M3^2 m_2
    auto canon = [&](int m12v, int mo) {
      const int mi = m12v % M3, mm = m12v / M3;
      return rot == 0 ? m12v + M3S * mo : (rot == 1 ? mo + M3 * mi + M3S * mm : mm + M3 * mo + M3S * mi);
    };
    nu[canon(m12, m3)] = acc;
    if (two) nu[canon(m12b, m3b)] = accb;
  }
  __syncthreads();
  {
    // the correlation's operands in CT (K'' is already)
    const CT* nuc = reinterpret_cast<const CT*>(nu);
    if constexpr (B::CTCOPY) {
      CT* nuf = reinterpret_cast<CT*>(reinterpret_cast<unsigned char*>(work) + B::oCT(D));
      for (int t = threadIdx.x; t < M3S * M3; t += blockDim.x) nuf[t] = (CT)nu[t];
      nuc = nuf;
      __syncthreads();
    }
    // mu[j] = prod_d C(2p, j_d) sum_k K''[k] nu[k + j]: thread per (j1, j2, block of JB j3), the
    // nu column m3 = j3b .. j3b + JB - 1 + p of each (k1, k2) in registers
    const CT* Kc = KA;
    for (int t = threadIdx.x; t < NB * NB * NJB; t += blockDim.x) {
      const int j1 = t % NB, j2 = (t / NB) % NB, j3b = (t / (NB * NB)) * JB;
      CT acc[JB];
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) acc[jj] = CT(0);
      for (int k2 = 0; k2 < Q; ++k2)
#pragma unroll
        for (int k1 = 0; k1 < Q; ++k1) {
          CT col[JB + P];
          const CT* nc = nuc + (j1 + k1) + M3 * (j2 + k2);
#pragma unroll
          for (int r = 0; r < JB + P; ++r) col[r] = j3b + r < M3 ? nc[M3S * (j3b + r)] : CT(0);
#pragma unroll
          for (int k3 = 0; k3 < Q; ++k3) {
            const CT kv = Kc[k1 + Q * (k2 + Q * k3)];
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) acc[jj] += kv * col[jj + k3];
          }
        }
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) {
        const int j3 = j3b + jj;
        if (j3 < NB)
          mu[j1 + NB * (j2 + NB * j3)] =
              (MT)(acc[jj] * (CT)(binom_i(2 * P, j1) * binom_i(2 * P, j2) * binom_i(2 * P, j3)));
      }
    }
  }
  __syncthreads();
}

// Shared-memory plan of k_cut_elemmat (offsets in elements, every region 16-byte aligned).
template <typename R, typename MT, int P, bool STIFF>
struct ElemSmem {
  static constexpr int Q = P + 1, NB = 2 * P + 1, Q2 = Q * Q, Q3 = Q2 * Q, NB3 = NB * NB * NB;
  static constexpr int NT = STIFF ? 2 : 1;
  static constexpr int NBP = rup4(NB);         // padded G row
  static constexpr int PLD = rup4(NB * Q);     // Bernstein table of one direction [k][g]
  static constexpr int NW = P >= 5 ? 4 : 8;
  // per-warp moment scratch: F | S1 | S2 | PL[3] | TW | NV
  static constexpr int oS1 = rup4(Q3), oS2 = oS1 + rup4(NB * Q2), oPL = oS2 + rup4(NB * NB * Q);
  static constexpr int oTW = oPL + 3 * PLD, oNV = oTW + rup4(3 * Q), WS = oNV + rup4(3 * Q * Q);
  static constexpr int MU = rup4(NB3);                       // mu (MT)
  static constexpr int GS = 2 * 3 * Q2 * NBP;                // Gs (R): [kind][d][ab][NBP]
  static constexpr int PARTA = NW * NB3 + NW * WS + rup4(Q3);  // muw | scratch | coefficient block (MT)
  // E stage (R), per a1: X1 [kind][b1][k3][k2] | Y [kind][b1][ab2][k3] | staging [a2][Q3]
  static constexpr int oY = rup4(NT * Q * NB * NB), oST = oY + rup4(NT * Q * Q2 * NB), PARTB = oST + Q * Q3;
  static constexpr size_t bytes_a = (size_t)PARTA * sizeof(MT), bytes_b = (size_t)PARTB * sizeof(R);
  static constexpr size_t bytes =
      (size_t)MU * sizeof(MT) + (size_t)GS * sizeof(R) + (bytes_a > bytes_b ? bytes_a : bytes_b);
  // register tables in the first two moment stages where they fit
  static constexpr bool REGT = sizeof(MT) * PLD <= 256;
  // grouped moments (octree depth D): core | position tables | per-warp scratch | slot lists;
  // the coefficient block of the per-piece layout must lie past the core it is copied to
  static constexpr int WSG = rup4(Q * NB) + rup4(Q * Q * NB) + rup4(Q * NB * NB);
  static size_t grouped_a(int D) {
    const int npos = (1 << (D + 1)) - 1, nslot = ((1 << (2 * (D + 1))) - 1) / 3;
    const size_t mt = (size_t)rup4(Q3) + rup4(3 * npos * Q * NB) + (size_t)NW * WSG;
    const size_t ints = 4 * (size_t)nslot + 3;  // smask, slist, gstart, counts, group -> warp
    const size_t cblk_end = (size_t)PARTA;  // the coefficient block sits at the end of PARTA
    const size_t g = mt * sizeof(MT) + ints * 4;
    return g > cblk_end * sizeof(MT) ? g : cblk_end * sizeof(MT);
  }
  static size_t bytes_grouped(int D) {
    const size_t a = grouped_a(D);
    return (size_t)MU * sizeof(MT) + (size_t)GS * sizeof(R) + (a > bytes_b ? a : bytes_b);
  }
};

// E = (G1 x G2 x G3) mu for one cut element (mu index k1 + NB (k2 + NB k3)), one a1 at a
// time, into rows a of E_e (block-wide; scratch: ElemSmem::PARTB elements of R).
template <typename R, typename MT, int P, bool STIFF>
__device__ __forceinline__ void elem_from_moments(const MT* mu, const R* Gs, R* scratch, R* __restrict__ E, int ci) {
  using SM = ElemSmem<R, MT, P, STIFF>;
  constexpr int Q = SM::Q, NB = SM::NB, Q3 = SM::Q3, Q2 = SM::Q2, NBP = SM::NBP;
  // ---- E from the moments (mu index k1 + NB (k2 + NB k3)), one a1 at a time:
  //   X1[kind][b1][k3][k2] = sum_k1 G1,kind[ab1][k1] mu          (ab1 = a1 Q + b1)
  //   mass  Y[b1][ab2][k3] = sum_k2 G2[ab2][k2] X1_0,            E = sum_k3 G3[ab3][k3] Y
  //   stiff Ya = G2 X1_1 + Gd2 X1_0,  Yc = G2 X1_0,              E = G3 Ya + Gd3 Yc
  // rows a = a1 + Q (a2 + Q a3) of E, columns b = b1 + Q (b2 + Q b3).
  const R* G1 = Gs;
  const R* G2 = Gs + 1 * Q2 * NBP;
  const R* G3 = Gs + 2 * Q2 * NBP;
  const R* Gd1 = Gs + 3 * Q2 * NBP;
  const R* Gd2 = Gs + 4 * Q2 * NBP;
  const R* Gd3 = Gs + 5 * Q2 * NBP;
  R* X1 = scratch;
  R* Yb = X1 + SM::oY;
  R* Est = X1 + SM::oST;
  constexpr int Q3P = rup4(Q3);  // row stride of E (16-byte aligned rows)
  R* Eo = E + (size_t)ci * Q3 * Q3P;
  for (int a1 = 0; a1 < Q; ++a1) {
    for (int t = threadIdx.x; t < Q * NB * NB; t += blockDim.x) {
      const int k23 = t % (NB * NB), b1 = t / (NB * NB);
      const int ab1 = a1 * Q + b1;
      R g[NBP], gd[NBP];
      lds_vec<R, NBP>(G1 + ab1 * NBP, g);
      if (STIFF) lds_vec<R, NBP>(Gd1 + ab1 * NBP, gd);
      R s0 = R(0), s1 = R(0);
#pragma unroll
      for (int k1 = 0; k1 < NB; ++k1) {
        const R m = (R)mu[k1 + NB * k23];
        s0 += g[k1] * m;
        if (STIFF) s1 += gd[k1] * m;
      }
      X1[t] = s0;  // [b1][k3][k2]: t = b1 NB^2 + k2 + NB k3 with k23 = k2 + NB k3
      if (STIFF) X1[Q * NB * NB + t] = s1;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Q * Q2; t += blockDim.x) {
      const int ab2 = t % Q2, b1 = t / Q2;
      R g[NBP], gd[NBP];
      lds_vec<R, NBP>(G2 + ab2 * NBP, g);
      if (STIFF) lds_vec<R, NBP>(Gd2 + ab2 * NBP, gd);
      for (int k3 = 0; k3 < NB; ++k3) {
        const R* x0 = X1 + (b1 * NB + k3) * NB;
        const R* x1 = X1 + Q * NB * NB + (b1 * NB + k3) * NB;
        R ya = R(0), yc = R(0);
#pragma unroll
        for (int k2 = 0; k2 < NB; ++k2) {
          const R v0 = x0[k2];
          yc += g[k2] * v0;
          if (STIFF) ya += g[k2] * x1[k2] + gd[k2] * v0;
        }
        Yb[(b1 * Q2 + ab2) * NB + k3] = STIFF ? ya : yc;
        if (STIFF) Yb[((Q + b1) * Q2 + ab2) * NB + k3] = yc;
      }
    }
    __syncthreads();
    for (int a3 = 0; a3 < Q; ++a3) {
      for (int t = threadIdx.x; t < Q * Q2; t += blockDim.x) {
        const int ab2 = t % Q2, b1 = t / Q2;
        const int a2 = ab2 / Q, b2 = ab2 - a2 * Q;
        R ya[NB], yc[NB];
#pragma unroll
        for (int k3 = 0; k3 < NB; ++k3) {
          ya[k3] = Yb[(b1 * Q2 + ab2) * NB + k3];
          if (STIFF) yc[k3] = Yb[((Q + b1) * Q2 + ab2) * NB + k3];
        }
#pragma unroll
        for (int b3 = 0; b3 < Q; ++b3) {
          const int ab3 = a3 * Q + b3;
          R g[NBP], gd[NBP];
          lds_vec<R, NBP>(G3 + ab3 * NBP, g);
          if (STIFF) lds_vec<R, NBP>(Gd3 + ab3 * NBP, gd);
          R v = R(0);
#pragma unroll
          for (int k3 = 0; k3 < NB; ++k3) {
            v += g[k3] * ya[k3];
            if (STIFF) v += gd[k3] * yc[k3];
          }
          Est[a2 * Q3 + b1 + Q * (b2 + Q * b3)] = v;
        }
      }
      __syncthreads();
      // rows a1 + Q (a2 + Q a3), a2 = 0..Q-1: each row Q3 contiguous values
      for (int t = threadIdx.x; t < Q * Q3; t += blockDim.x) {
        const int a2 = t / Q3, b = t - a2 * Q3;
        Eo[(size_t)(a1 + Q * (a2 + Q * a3)) * Q3P + b] = Est[t];
      }
      __syncthreads();
    }
  }
}

// The Bernstein product tables G (and Gd) of the element's three directions into shared
// memory: Gs[kind][d][ab][NBP], rows padded with zeros.
template <typename R, int P>
__device__ __forceinline__ void load_gs(const MeshView& M, int ee0, int ee1, int ee2, R* Gs) {
  constexpr int Q2 = (P + 1) * (P + 1), NB = 2 * P + 1, NBP = rup4(NB);
  for (int t = threadIdx.x; t < 2 * 3 * Q2 * NBP; t += blockDim.x) {
    const int k = t % NBP, ab = (t / NBP) % Q2, d = (t / (NBP * Q2)) % 3, kind = t / (NBP * Q2 * 3);
    const int eed = sel3(d, ee0, ee1, ee2);
    R v = R(0);
    if (k < NB) {
      const size_t o = ((size_t)eed * Q2 + ab) * NB + k;
      if (sizeof(R) == 4) v = (R)(kind ? M.dir[d].Gdf : M.dir[d].Gf)[o];
      else v = (R)(kind ? M.dir[d].Gd : M.dir[d].G)[o];
    }
    Gs[t] = v;
  }
}

// ---------------------------------------------------------------------------------------
// Element matrices of cut elements, any coefficient.  One block per cut element.  The moments
// mu come from one of two equivalent orderings of the pieces' Gauss sums (grouped): 1, the
// position groups of moments_grouped; 0, piece by piece (pieces spread over the warps, the
// warps' moments summed in a fixed order).  Then E = (G1 x G2 x G3) mu by three contractions.
template <typename R, typename MT, int P, bool STIFF>
__global__ void __launch_bounds__(256) k_cut_elemmat(MeshView M, LevelSet L, CoefDesc cf, R* __restrict__ E,
                                                     int grouped, int ci0) {
  using SM = ElemSmem<R, MT, P, STIFF>;
  constexpr int Q = SM::Q, NB = SM::NB, Q3 = SM::Q3, NB3 = SM::NB3, Q2 = SM::Q2, NBP = SM::NBP, PLD = SM::PLD;
  constexpr int NT = SM::NT, WS = SM::WS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ci = ci0 + blockIdx.x;  // cut elements [ci0, ci0 + gridDim.x) of the list
  const int e = M.topo.cut_elems[ci];
  const int ne1 = M.dir[0].n_el, ne2 = M.dir[1].n_el;
  const int ee0 = e % ne1, ee1 = (e / ne1) % ne2, ee2 = e / (ne1 * ne2);
  if (M.topo.elem_state[e] != E_CUT) return;
  const int pbeg = M.topo.piece_ptr[ci], pend = M.topo.piece_ptr[ci + 1];
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  MT* mu = reinterpret_cast<MT*>(smem_raw);  // NB3
  R* Gs = reinterpret_cast<R*>(mu + SM::MU);  // [kind][d][ab][NBP]
  MT* uni = reinterpret_cast<MT*>(Gs + SM::GS);
  MT* muw = uni;                               // nwarps * NB3
  MT* wsp = muw + (size_t)nwarps * NB3;        // nwarps * WS
  MT* cblk = wsp + (size_t)nwarps * WS;        // Q3 coefficient block

  for (int t = threadIdx.x; t < nwarps * NB3; t += blockDim.x) muw[t] = MT(0);
  if (cf.kind == SFA_COEF_BSPLINE) {
    const int n1 = M.dir[0].n, n2 = M.dir[1].n;
    for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
      int a1 = t % Q, a2 = (t / Q) % Q, a3 = t / Q2;
      cblk[t] = (MT)cf.ck[(ee0 + a1) + (int64_t)n1 * ((ee1 + a2) + (int64_t)n2 * (ee2 + a3))];
    }
  }
  load_gs<R, P>(M, ee0, ee1, ee2, Gs);
  __syncthreads();

  if (grouped) {
    // ---- moments by octree position groups
    constexpr int NWc = SM::NW;
    const int D = M.D;
    const int npos = (1 << (D + 1)) - 1, nslot = ((1 << (2 * (D + 1))) - 1) / 3;
    MT* K = uni;                                   // A^3 core of the coefficient
    MT* Tpos = K + rup4(Q3);                       // [3][npos][A][NB]
    MT* wscr = Tpos + rup4(3 * npos * Q * NB);     // [NW][WSG]
    constexpr int WSG = rup4(Q * NB) + rup4(Q * Q * NB) + rup4(Q * NB * NB);
    uint32_t* smask = reinterpret_cast<uint32_t*>(wscr + (size_t)NWc * WSG);
    int* slist = reinterpret_cast<int*>(smask + nslot);
    int* gstart = slist + nslot;
    int* cnt = gstart + nslot + 1;
    for (int t = threadIdx.x; t < NB3; t += blockDim.x) mu[t] = MT(0);
    const uint32_t* pcs = M.topo.pieces + pbeg;
    if (cf.kind == SFA_COEF_BSPLINE) {
      for (int t = threadIdx.x; t < Q3; t += blockDim.x) K[t] = cblk[t];
      __syncthreads();
      moments_grouped<MT, P, Q, NWc>(M, cf.kind, ee0, ee1, ee2, pcs, pend - pbeg, K, Tpos, smask, slist, gstart, cnt,
                                     wscr, WSG, mu);
    } else if (cf.kind == SFA_COEF_ANALYTIC) {
      for (int t = threadIdx.x; t < 8; t += blockDim.x) K[t] = t == 0 ? MT(1) : (t == 7 ? MT(0.5) : MT(0));
      __syncthreads();
      moments_grouped<MT, P, 2, NWc>(M, cf.kind, ee0, ee1, ee2, pcs, pend - pbeg, K, Tpos, smask, slist, gstart, cnt,
                                     wscr, WSG, mu);
    } else {
      if (threadIdx.x == 0) K[0] = (MT)cf.c0;
      __syncthreads();
      moments_grouped<MT, P, 1, NWc>(M, cf.kind, ee0, ee1, ee2, pcs, pend - pbeg, K, Tpos, smask, slist, gstart, cnt,
                                     wscr, WSG, mu);
    }
  } else {
  // ---- moments, piece by piece, one warp per piece
  {
    MT* F = wsp + (size_t)warp * WS;  // Q3: w c at the piece points [g3][g2][g1]
    MT* S1 = F + SM::oS1;             // [g3][g2][k1]
    MT* S2 = F + SM::oS2;             // [g3][k2][k1]
    MT* PL = F + SM::oPL;             // [d][k][g] Bernstein values, PLD per direction
    MT* TW = F + SM::oTW;             // [d][g] weights
    MT* NV = F + SM::oNV;             // [d][a][g] basis values (B-spline c)
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
      const int av0 = (int)((code >> 4) & 63), av1 = (int)((code >> 10) & 63), av2 = (int)((code >> 16) & 63);
      // per-direction weights, Bernstein values and basis values, from the piece tables
      for (int t = lane; t < 3 * Q; t += 32) {
        const int d = t / Q, g = t % Q;
        const int pos = (1 << lev) - 1 + sel3(d, av0, av1, av2);
        const Dir1D& Dd = M.dir[d];
        const int64_t row = (((int64_t)sel3(d, ee0, ee1, ee2) * Dd.npos + pos) * Q + g) * PTF;
        // the table in the moments' own precision (no conversion in the loop)
        const MT* src = sizeof(MT) == 4 ? reinterpret_cast<const MT*>(Dd.PTf + row)
                                        : reinterpret_cast<const MT*>(Dd.PT + row);
        TW[d * Q + g] = src[0];
        for (int k = 0; k < NB; ++k) PL[d * PLD + k * Q + g] = src[1 + k];
        if (cf.kind == SFA_COEF_BSPLINE) {
          for (int a2 = 0; a2 < Q; ++a2) NV[(d * Q + a2) * Q + g] = src[1 + NB + a2];
        } else if (cf.kind == SFA_COEF_ANALYTIC) {
          NV[d * Q * Q + g] = src[1 + NB + Q];  // d=0 sin(2 pi x), d=1 cos(2 pi y), d=2 z
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
      if (SM::REGT) {
        MT pl[PLD];
        lds_vec<MT, PLD>(PL, pl);
        for (int g23 = lane; g23 < Q2; g23 += 32) {
          MT f[Q];
#pragma unroll
          for (int g = 0; g < Q; ++g) f[g] = F[g + Q * g23];
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            MT v = MT(0);
#pragma unroll
            for (int g = 0; g < Q; ++g) v += pl[k * Q + g] * f[g];
            S1[k + NB * g23] = v;
          }
        }
      } else {
        for (int g23 = lane; g23 < Q2; g23 += 32) {
          MT f[Q];
#pragma unroll
          for (int g = 0; g < Q; ++g) f[g] = F[g + Q * g23];
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            MT v = MT(0);
#pragma unroll
            for (int g = 0; g < Q; ++g) v += PL[k * Q + g] * f[g];
            S1[k + NB * g23] = v;
          }
        }
      }
      __syncwarp();
      // stage 2: S2[k1 + NB (k2 + NB g3)] = sum_g2 PL2[k2][g2] S1[k1 + NB (g2 + Q g3)], lane per (k1, g3)
      if (SM::REGT) {
        MT pl[PLD];
        lds_vec<MT, PLD>(PL + PLD, pl);
        for (int kg = lane; kg < NB * Q; kg += 32) {
          const int k1 = kg % NB, g3 = kg / NB;
          MT x[Q];
#pragma unroll
          for (int g = 0; g < Q; ++g) x[g] = S1[k1 + NB * (g + Q * g3)];
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            MT v = MT(0);
#pragma unroll
            for (int g = 0; g < Q; ++g) v += pl[k * Q + g] * x[g];
            S2[k1 + NB * (k + NB * g3)] = v;
          }
        }
      } else {
        for (int kg = lane; kg < NB * Q; kg += 32) {
          const int k1 = kg % NB, g3 = kg / NB;
          MT x[Q];
#pragma unroll
          for (int g = 0; g < Q; ++g) x[g] = S1[k1 + NB * (g + Q * g3)];
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            MT v = MT(0);
#pragma unroll
            for (int g = 0; g < Q; ++g) v += PL[PLD + k * Q + g] * x[g];
            S2[k1 + NB * (k + NB * g3)] = v;
          }
        }
      }
      __syncwarp();
      // stage 3: mu[k12][k3] += sum_g3 PL3[k3][g3] S2[k12 + NB^2 g3], lane per k12
      if (REGB) {
        MT pl3[NB][Q];
#pragma unroll
        for (int k = 0; k < NB; ++k)
#pragma unroll
          for (int g = 0; g < Q; ++g) pl3[k][g] = PL[2 * PLD + k * Q + g];
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
            for (int g = 0; g < Q; ++g) v += PL[2 * PLD + k * Q + g] * x[g];
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
  }  // per-piece moments
  __syncthreads();

  elem_from_moments<R, MT, P, STIFF>(mu, Gs, reinterpret_cast<R*>(uni), E, ci);
}

// Element matrices for a B-spline or constant coefficient: moments by the degree-3p piece
// moments (moments_bern3p), then E = (G1 x G2 x G3) mu.  Shared memory is one work area that
// holds in turn the moment stages and the E stage (the tables Gs, then its scratch), with mu
// at its end, past everything either phase uses (the correlation writes it, the E stage
// reads it).
template <typename R, typename MT, int P, bool STIFF>
struct B3Smem {
  using SM = ElemSmem<R, MT, P, STIFF>;
  static constexpr size_t gs_bytes = (size_t)SM::GS * sizeof(R);  // a multiple of 16
  // float stiffness: the paired expansion (elem_from_moments_f2) and its plan, in floats:
  // Gs2 [d][ab][k < NB + 1][kind] | muf [NB^3] | X1 [b1][k3][k2][2] | Y [b1][ab2][k3][2] |
  // staging [a2 + Q a3][Q3P + 4] (rows of E padded to Q3P = Q3 rounded up to 4; the staging rows
  // 4 longer, so that the lanes of one (b1, ab2) writing rows a3 fall in different banks)
  static constexpr bool F2 = STIFF && sizeof(R) == 4;
  static constexpr int Q = SM::Q, NB = SM::NB, Q2 = SM::Q2, Q3 = SM::Q3;
  static constexpr int oMF = 3 * Q2 * 2 * (NB + 1), oX1 = oMF + rup4(NB * NB * NB), oY = oX1 + rup4(2 * Q * NB * NB),
                       oST = oY + rup4(2 * Q * Q2 * NB), F2W = oST + Q2 * (rup4(Q3) + 4);
  static constexpr size_t e_bytes = F2 ? (size_t)F2W * 4 : gs_bytes + SM::bytes_b;
  __host__ __device__ static size_t omu(int D) {
    const size_t a = B3Plan<MT, P, R>::bytes(D), b = e_bytes;
    return ((a > b ? a : b) + 15) / 16 * 16;
  }
  __host__ __device__ static size_t bytes(int D) { return omu(D) + (size_t)SM::MU * sizeof(MT); }
  // CTAs per SM the registers are budgeted for (shared memory allows four up to p = 4 at
  // octree depth 3)
  static constexpr int MINB = P <= 4 ? 4 : 2;
};

// Gs (as load_gs) by asynchronous copies; zeros in the padding.  The caller waits.
template <typename R, int P>
__device__ __forceinline__ void load_gs_async(const MeshView& M, int ee0, int ee1, int ee2, R* Gs) {
  constexpr int Q2 = (P + 1) * (P + 1), NB = 2 * P + 1, NBP = rup4(NB);
  const uint32_t gs = (uint32_t)__cvta_generic_to_shared(Gs);
  for (int t = threadIdx.x; t < 2 * 3 * Q2 * NBP; t += blockDim.x) {
    const int k = t % NBP, ab = (t / NBP) % Q2, d = (t / (NBP * Q2)) % 3, kind = t / (NBP * Q2 * 3);
    if (k < NB) {
      const size_t o = ((size_t)sel3(d, ee0, ee1, ee2) * Q2 + ab) * NB + k;
      const R* src;
      if constexpr (sizeof(R) == 4) src = reinterpret_cast<const R*>((kind ? M.dir[d].Gdf : M.dir[d].Gf) + o);
      else src = reinterpret_cast<const R*>((kind ? M.dir[d].Gd : M.dir[d].G) + o);
      cp_word_nc<sizeof(R)>(gs + (uint32_t)(t * sizeof(R)), src);
    } else {
      Gs[t] = R(0);
    }
  }
  cp_commit();
}

// E = (G1 x G2 x G3) mu for one cut element, float stiffness: the same three contractions
// as elem_from_moments, with the value and derivative tables of each direction interleaved
// (G, Gd) and the intermediate results kept as pairs, so that every step is a paired
// (f32x2) multiply-add, and every stage spread over all threads:
//   X1[b1][k3][k2] = (sum_k1 Gd1 mu, sum_k1 G1 mu)                          = (x1, x0)
//   Y[b1][ab2][k3] = (sum_k2 G2 x1 + Gd2 x0, sum_k2 G2 x0)                  = (ya, yc)
//   E[a][b]        = sum_k3 G3[ab3] ya + Gd3[ab3] yc
// one a1 at a time; the rows of E_e with that a1 are staged and written while the next a1's
// first stage runs.  W: the work area (B3Smem's F2 plan); mu: NB^3 moments in MT.
template <typename MT, int P>
__device__ __forceinline__ void elem_from_moments_f2(const MeshView& M, int ee0, int ee1, int ee2, const MT* mu,
                                                     float* W, float* __restrict__ E, int ci) {
  using L3 = B3Smem<float, MT, P, true>;
  constexpr int Q = P + 1, NB = 2 * P + 1, Q2 = Q * Q, Q3 = Q2 * Q, NB2 = NB * NB, NBE = NB + 1, ROW = 2 * NBE;
  float* Gs2 = W;
  float* muf = W + L3::oMF;
  float2* X1 = reinterpret_cast<float2*>(W + L3::oX1);
  float2* Y = reinterpret_cast<float2*>(W + L3::oY);
  float* Est = W + L3::oST;
  // tables: Gs2[((d Q2 + ab) NBE + k) 2 + kind]
  {
    const uint32_t gs = (uint32_t)__cvta_generic_to_shared(Gs2);
    for (int t = threadIdx.x; t < 3 * Q2 * NB * 2; t += blockDim.x) {
      const int kind = t & 1, k = (t >> 1) % NB, ab = ((t >> 1) / NB) % Q2, d = (t >> 1) / (NB * Q2);
      const size_t o = ((size_t)sel3(d, ee0, ee1, ee2) * Q2 + ab) * NB + k;
      cp_word_nc<4>(gs + (uint32_t)((((d * Q2 + ab) * NBE + k) * 2 + kind) * 4), (kind ? M.dir[d].Gdf : M.dir[d].Gf) + o);
    }
    cp_commit();
  }
  for (int t = threadIdx.x; t < NB2 * NB; t += blockDim.x) muf[t] = (float)mu[t];
  cp_wait<0>();
  __syncthreads();
  // one table row (NB pairs, NBE of them loaded) of direction d, index ab
  auto row = [&](int d, int ab, float2 (&g)[NBE]) {
    const float4* r4 = reinterpret_cast<const float4*>(Gs2 + (d * Q2 + ab) * ROW);
#pragma unroll
    for (int k = 0; k < NBE / 2; ++k) {
      const float4 v = r4[k];
      g[2 * k] = make_float2(v.x, v.y);
      g[2 * k + 1] = make_float2(v.z, v.w);
    }
  };
  constexpr int Q3P = rup4(Q3), R4 = Q3P / 4, ESTR = Q3P + 4;
  float* Eo = E + (size_t)ci * Q3 * Q3P;
  auto store_rows = [&](int a1) {  // rows a1 + Q (a2 + Q a3) from the staging, 16 bytes at a time
    for (int t = threadIdx.x; t < Q2 * R4; t += blockDim.x) {
      const int r = t / R4, c = t - r * R4;
      reinterpret_cast<float4*>(Eo + (size_t)(a1 + Q * r) * Q3P)[c] = reinterpret_cast<const float4*>(Est + r * ESTR)[c];
    }
  };
  for (int a1 = 0; a1 < Q; ++a1) {
    // X1 for this a1 (and the previous a1's rows go out)
    for (int t = threadIdx.x; t < Q * NB2; t += blockDim.x) {
      const int b1 = t / NB2, k23 = t - b1 * NB2;
      float2 g[NBE];
      row(0, a1 * Q + b1, g);
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int k1 = 0; k1 < NB; ++k1) {
        const float m = muf[k1 + NB * k23];
        s = fma2(g[k1], make_float2(m, m), s);
      }
      X1[t] = make_float2(s.y, s.x);  // [b1][k3][k2] with k23 = k2 + NB k3
    }
    if (a1 > 0) store_rows(a1 - 1);
    __syncthreads();
    // Y: thread per (b1, ab2, k3)
    for (int t = threadIdx.x; t < Q * Q2 * NB; t += blockDim.x) {
      const int k3 = t % NB, q = t / NB, ab2 = q % Q2, b1 = q / Q2;
      float2 g[NBE];
      row(1, ab2, g);
      const float2* x = X1 + (b1 * NB + k3) * NB;
      float2 s = make_float2(0.f, 0.f);
      float yc = 0.f;
#pragma unroll
      for (int k2 = 0; k2 < NB; ++k2) {
        const float2 xv = x[k2];
        s = fma2(g[k2], xv, s);
        yc = fmaf(g[k2].x, xv.y, yc);
      }
      Y[(b1 * Q2 + ab2) * NB + k3] = make_float2(s.x + s.y, yc);
    }
    __syncthreads();
    // E rows of this a1: thread per (b1, ab2, a3), all b3
    for (int t = threadIdx.x; t < Q * Q2 * Q; t += blockDim.x) {
      const int a3 = t % Q, q = t / Q, ab2 = q % Q2, b1 = q / Q2;
      const int a2 = ab2 / Q, b2 = ab2 - a2 * Q;
      float2 y[NB];
#pragma unroll
      for (int k3 = 0; k3 < NB; ++k3) y[k3] = Y[(b1 * Q2 + ab2) * NB + k3];
      float* dst = Est + (a2 + Q * a3) * ESTR + b1 + Q * b2;
#pragma unroll
      for (int b3 = 0; b3 < Q; ++b3) {
        float2 g[NBE];
        row(2, a3 * Q + b3, g);
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int k3 = 0; k3 < NB; ++k3) v = fma2(g[k3], y[k3], v);
        dst[Q2 * b3] = v.x + v.y;
      }
    }
    __syncthreads();
  }
  store_rows(Q - 1);
}

template <typename R, typename MT, int P, bool STIFF>
__global__ void __launch_bounds__(256, B3Smem<R, MT, P, STIFF>::MINB) k_cut_elemmat_b3p(MeshView M, CoefDesc cf, R* __restrict__ E, int ci0) {
  using SM = ElemSmem<R, MT, P, STIFF>;
  using L3 = B3Smem<R, MT, P, STIFF>;
  constexpr int Q = SM::Q, Q2 = SM::Q2, Q3 = SM::Q3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ci = ci0 + blockIdx.x;  // cut elements [ci0, ci0 + gridDim.x) of the list
  const int e = M.topo.cut_elems[ci];
  const int ne1 = M.dir[0].n_el, ne2 = M.dir[1].n_el;
  const int ee0 = e % ne1, ee1 = (e / ne1) % ne2, ee2 = e / (ne1 * ne2);
  if (M.topo.elem_state[e] != E_CUT) return;
  const int pbeg = M.topo.piece_ptr[ci], pend = M.topo.piece_ptr[ci + 1];
  MT* work = reinterpret_cast<MT*>(smem_raw);
  MT* mu = reinterpret_cast<MT*>(smem_raw + L3::omu(M.D));  // NB3
  const bool bspline = cf.kind == SFA_COEF_BSPLINE;
  if (bspline) {
    // the coefficient block; with double moments by asynchronous copies that moments_bern3p
    // waits for together with its own
    const int n1 = M.dir[0].n, n2 = M.dir[1].n;
    const uint32_t ws = (uint32_t)__cvta_generic_to_shared(work);
    for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
      const int a1 = t % Q, a2 = (t / Q) % Q, a3 = t / Q2;
      const double* src = cf.ck + ((ee0 + a1) + (int64_t)n1 * ((ee1 + a2) + (int64_t)n2 * (ee2 + a3)));
      if constexpr (sizeof(MT) == 8) cp_word_nc<8>(ws + 8u * t, src);
      else work[t] = (MT)*src;
    }
  }
  moments_bern3p<MT, P, R>(M, ee0, ee1, ee2, M.topo.pieces + pbeg, pend - pbeg, bspline, (MT)cf.c0, work, mu);
  // the moment stages are done with the work area: the E stage's tables go to its start
  if constexpr (L3::F2) {
    elem_from_moments_f2<MT, P>(M, ee0, ee1, ee2, mu, reinterpret_cast<float*>(smem_raw), reinterpret_cast<float*>(E),
                                ci);
  } else {
    R* Gs = reinterpret_cast<R*>(smem_raw);  // [kind][d][ab][NBP]
    load_gs_async<R, P>(M, ee0, ee1, ee2, Gs);
    cp_wait<0>();
    __syncthreads();
    elem_from_moments<R, MT, P, STIFF>(mu, Gs, reinterpret_cast<R*>(smem_raw + L3::gs_bytes), E, ci);
  }
}

template <typename R, typename MT, int P, bool STIFF>
cudaError_t launch_elem_t(const MeshView& M, const LevelSet& L, int coef_kind, double c0, const double* ck, R* E,
                          int n_cut_elems, int ci0, cudaStream_t st) {
  if (n_cut_elems <= 0) return cudaSuccess;
  using LE = ElemSmem<R, MT, P, STIFF>;
  using L3 = B3Smem<R, MT, P, STIFF>;
  const CoefDesc cf{coef_kind, c0, ck};
  cudaError_t err;
  const bool poly = coef_kind == SFA_COEF_BSPLINE || coef_kind == SFA_COEF_CONST;
  const size_t s3 = L3::bytes(M.D) + 16;
  if (poly && s3 <= 227 * 1024) {
    // degree-3p piece moments for polynomial coefficients
    err = cudaFuncSetAttribute(k_cut_elemmat_b3p<R, MT, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s3);
    if (err != cudaSuccess) return err;
    k_cut_elemmat_b3p<R, MT, P, STIFF><<<n_cut_elems, 256, s3, st>>>(M, cf, E, ci0);
    SFA_LAUNCHED(1);
    return cudaGetLastError();
  }
  // grouped moments where their shared memory fits, else piece by piece
  const size_t sg = LE::bytes_grouped(M.D) + 16;
  const int grouped = sg <= 227 * 1024 ? 1 : 0;
  const size_t smem = grouped ? sg : LE::bytes + 16;
  err = cudaFuncSetAttribute(k_cut_elemmat<R, MT, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_cut_elemmat<R, MT, P, STIFF><<<n_cut_elems, 32 * LE::NW, smem, st>>>(M, L, cf, E, grouped, ci0);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

// Cut-element matrices E (part 0 of the cut path): R the value type, MT the moment type.
cudaError_t launch_cut_elem(const MeshView& M, const LevelSet& L, bool fp64, bool mom64, bool stiff, int coef_kind,
                            double c0, const double* ck, void* E, int n_cut_elems, int ci0, cudaStream_t st) {
#define SFA_ELEM_ARGS(RT) M, L, coef_kind, c0, ck, (RT*)E, n_cut_elems, ci0, st
#define SFA_ELEM_CASE(PP)                                                                                       \
  case PP:                                                                                                      \
    if (fp64)                                                                                                   \
      return stiff ? launch_elem_t<double, double, PP, true>(SFA_ELEM_ARGS(double))                            \
                   : launch_elem_t<double, double, PP, false>(SFA_ELEM_ARGS(double));                           \
    if (mom64)                                                                                                  \
      return stiff ? launch_elem_t<float, double, PP, true>(SFA_ELEM_ARGS(float))                               \
                   : launch_elem_t<float, double, PP, false>(SFA_ELEM_ARGS(float));                             \
    return stiff ? launch_elem_t<float, float, PP, true>(SFA_ELEM_ARGS(float))                                  \
                 : launch_elem_t<float, float, PP, false>(SFA_ELEM_ARGS(float));
  switch (M.p) {
    SFA_ELEM_CASE(2)
    SFA_ELEM_CASE(3)
    SFA_ELEM_CASE(4)
    SFA_ELEM_CASE(5)
    SFA_ELEM_CASE(6)
  }
#undef SFA_ELEM_CASE
#undef SFA_ELEM_ARGS
  return cudaErrorInvalidValue;
}
