// Cut rows (Sec. 2.2, Eq. 1: the support of a cut test function is split into a regular
// part and a cut part).  The regular part is the DWQ box (one-sided DWQ rule in the box's
// direction, standard WQ rules in the other two) when one exists; every other inside
// support element is integrated with its (p+1)^3 Gauss points (the points below the
// artificial discontinuity in Fig. 3); every cut element adds row a(i) of its element matrix
// (cut_elem.cu: the Gauss points of its octree pieces, Sec. 3.1).
#include "cut_common.cuh"

namespace {

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

// Shared-memory plan of k_cut_rows, in elements of R.
template <typename R, int P, bool STIFF>
struct CutRowSmem {
  static constexpr int Q = P + 1, NB = 2 * P + 1, Q2 = Q * Q, Q3 = Q2 * Q, NB3 = NB * NB * NB;
  static constexpr int NT = STIFF ? 2 : 1;
  static constexpr int NBP = (NB + 3) / 4 * 4;  // transposed box table row
  static constexpr int Q2P = (Q2 + 3) / 4 * 4;  // element table
  static constexpr int NW = (sizeof(R) == 8 && P >= 6) ? 2 : (sizeof(R) == 8 && P >= 5) ? 4 : 8;
  // CTAs per SM the registers are budgeted for: three for float rows up to p = 4 (80 registers)
  static constexpr int MINB = (sizeof(R) == 4 && P <= 4) ? 3 : 1;
  // float stiffness: the two derivative placements of an element table interleaved,
  // [b][g < QE][kind] with QE = Q rounded up to even, for paired (f32x2) multiply-adds
  static constexpr bool F2 = STIFF && sizeof(R) == 4;
  static constexpr int QE = (Q + 1) / 2 * 2, TP2 = Q * QE * 2;
  // the paired path's per-warp stage results (float2): U [g2][g3][b1] for odd Q (else
  // [g3][g2][b1]) in 2 Q3P floats, W[b1 + Q b2 + S3 g3] with S3 = Q mod 16 (odd Q) so that
  // every stage reads and writes its pairs without bank conflicts
  static constexpr bool ODDQ = (Q & 1) != 0;
  static constexpr int S3 = ODDQ ? Q2 + ((Q - Q2) % 16 + 16) % 16 : Q2;
  static constexpr int WPF = ((2 * (Q2 + S3 * (Q - 1))) + 3) / 4 * 4;  // W in floats
  static constexpr int ETAB = F2 ? 3 * Q * TP2 : 3 * Q * NT * Q2P;
  static constexpr int Q3P = (Q3 + 3) / 4 * 4;
  // support-element entries in flight per warp (ring of DEPTH buffers of Q3P values)
  static constexpr int DEPTH = sizeof(R) == 4 ? 4 : 2;
  // box buffers for MF points in the DWQ direction, MQ in the others; with stage_c the
  // coefficient block C(k_f, k_s, k_t) of the box is staged in shared memory as well
  __host__ __device__ static size_t box(int MF, int MQ, int stage_c) {
    return (size_t)NT * (MF + 2 * MQ) * NBP + (stage_c ? (size_t)MF * MQ * MQ : 0) + (size_t)NT * MQ * MQ * NB +
           (size_t)NT * MQ * NB * NB + (3 * (size_t)(MF > MQ ? MF : MQ) * sizeof(int) + sizeof(R) - 1) / sizeof(R);
  }
  // per warp: DEPTH ring slots, then U0 | U1 | TA | TB (general path) or U | W (paired path)
  static constexpr size_t wscr = (size_t)DEPTH * Q3P + (F2 && 2 * Q3P + WPF > 4 * Q3P ? 2 * Q3P + WPF : 4 * Q3P);
  static constexpr size_t elem = (size_t)NW * wscr;
  // byte offset of the integer area: per support element its source offset (int64) and
  // class, the compacted element list, the row's column indices
  __host__ __device__ static size_t ioff(int MF, int MQ, int stage_c) {
    const size_t bx = box(MF, MQ, stage_c), uni = bx > elem ? bx : elem;
    return (((size_t)NW * NB3 + ETAB + uni) * sizeof(R) + 15) / 16 * 16;
  }
  __host__ __device__ static size_t bytes(int MF, int MQ, int stage_c) {
    return ioff(MF, MQ, stage_c) + (size_t)Q3P * sizeof(long long) + (2 * Q3P + NB3) * sizeof(int) + 16;
  }
};

// floor(t / d) by one multiply-high, for 0 <= t and t d < 2^32: with mg = ceil(2^32 / d),
// t mg / 2^32 = t / d + t e / (d 2^32) with 0 <= e < d, and the excess stays below 1/d.
struct MDiv {
  unsigned d, mg;
};
__device__ __forceinline__ MDiv mdiv_of(int d) { return {(unsigned)d, d > 1 ? 0xFFFFFFFFu / (unsigned)d + 1u : 0u}; }
__device__ __forceinline__ int qdiv(int t, MDiv m) { return m.d > 1 ? (int)__umulhi((unsigned)t, m.mg) : t; }


// Element Gauss contribution of one inside element to the row (float stiffness), one warp:
// the three contractions of the general path with the two derivative placements carried as
// pairs (f0, f1) of the interleaved tables:
//   stage 1 (g1): (U0, U1)[b1] = sum_g1 (f0, f1)[b1][g1] C        stored as pairs (U1, U0)
//   stage 2 (g2): ta = sum f0 U1 + sum f1 U0,  tb = sum f0 U0       stored as pairs (ta, tb)
//   stage 3 (g3): v = sum f0 ta + sum f1 tb, added to the warp's band at ab
// C: [g3][g2][g1]; T: the row's tables [d][eo][b][g < QE][kind]; U, W: the pair layouts of
// CutRowSmem; ab: the band at the element's offset.
template <typename L>
__device__ __forceinline__ void gauss_elem_f2(const float* __restrict__ C, const float* __restrict__ T, int eo1,
                                              int eo2, int eo3, float2* U, float2* W, float* ab, int lane) {
  constexpr int Q = L::Q, Q2 = L::Q2, QE = L::QE, TP2 = L::TP2, NB = L::NB;
  const float* T0 = T + (0 * Q + eo1) * TP2;
  const float* T1 = T + (1 * Q + eo2) * TP2;
  const float* T2 = T + (2 * Q + eo3) * TP2;
  // one table row b: QE pairs (f0, f1)[b][g]
  auto row = [&](const float* Tt, int b, float2 (&f)[QE]) {
#pragma unroll
    for (int k = 0; k < QE / 2; ++k) {
      const float4 v = reinterpret_cast<const float4*>(Tt + b * QE * 2)[k];
      f[2 * k] = make_float2(v.x, v.y);
      f[2 * k + 1] = make_float2(v.z, v.w);
    }
  };
  constexpr bool ODDQ = L::ODDQ;
  constexpr int S3 = L::S3;
  for (int l = lane; l < Q2; l += 32) {  // stage 1: lane per (g2, g3), g3 fastest for odd Q
    const int g2 = ODDQ ? l / Q : l % Q, g3 = ODDQ ? l % Q : l / Q;
    float2 xx[Q];
#pragma unroll
    for (int g = 0; g < Q; ++g) {
      const float x = C[g + Q * (g2 + Q * g3)];
      xx[g] = make_float2(x, x);
    }
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      float2 f[QE];
      row(T0, b, f);
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int g = 0; g < Q; ++g) a = fma2(f[g], xx[g], a);
      U[b + Q * l] = make_float2(a.y, a.x);
    }
  }
  __syncwarp();
  for (int l = lane; l < Q2; l += 32) {  // stage 2: lane per (b1, g3)
    const int b1 = l % Q, g3 = l / Q;
    float2 xp[Q];
#pragma unroll
    for (int g = 0; g < Q; ++g) xp[g] = ODDQ ? U[l + Q2 * g] : U[b1 + Q * (g + Q * g3)];
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      float2 f[QE];
      row(T1, b, f);
      float2 s = make_float2(0.f, 0.f);
      float tb = 0.f;
#pragma unroll
      for (int g = 0; g < Q; ++g) {
        s = fma2(f[g], xp[g], s);
        tb = fmaf(f[g].x, xp[g].y, tb);
      }
      W[b1 + Q * b + S3 * g3] = make_float2(s.x + s.y, tb);
    }
  }
  __syncwarp();
  for (int l = lane; l < Q2; l += 32) {  // stage 3: lane per (b1, b2)
    const int b1 = l % Q, b2 = l / Q;
    float2 xp[Q];
#pragma unroll
    for (int g = 0; g < Q; ++g) xp[g] = W[l + S3 * g];
    float* ap = ab + b2 * NB + b1;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      float2 f[QE];
      row(T2, b, f);
      float2 v = make_float2(0.f, 0.f);
#pragma unroll
      for (int g = 0; g < Q; ++g) v = fma2(f[g], xp[g], v);
      ap[b * NB * NB] += v.x + v.y;
    }
  }
  __syncwarp();
}

// One block per cut row.  Accumulators: one dense (2p+1)^3 band per warp, summed in a
// fixed order at the end.
//  * DWQ box (regular part, Sec. 2.2): tensor-product rule with the one-sided DWQ rule in
//    the box's direction f and the standard WQ rules in the other two (s, t); contracted by
//    the whole block in the order f, s, t:
//      U = T_f C,  TB = T_s U,  V = T_t TB      (stiffness: the three derivative placements)
//    one thread per output line and derivative placement, the 1D tables transposed
//    ([point][b]) for vector reads; the two placements of the last stage go to the bands
//    of warps 0 and 1.
//  * Inside support elements outside the box: (p+1)^3 Gauss points of the element, three
//    register-blocked stages per warp, tables F_d[b][g] = w B_{i_d} B_{e_d+b} of the row's
//    support elements staged once per row.
//  * Cut elements: row a(i) of the element matrix E_e.
//  Every global read before the arithmetic (tables, the box's coefficient block, the row's
//  column indices, the support elements' coefficients and E rows) is an asynchronous copy
//  into shared memory, issued as early as its address is known.
//  Rows come from `rows` (the cut rows; for the Standard Gauss variant every active row);
//  use_box = 0 ignores the DWQ boxes (Hybrid and Standard Gauss variants, Sec. 3.1), so
//  every inside support element is integrated with its Gauss points.
template <typename R, int P, bool STIFF>
__global__ void __launch_bounds__(256, CutRowSmem<R, P, STIFF>::MINB) k_cut_rows(MeshView M, const R* __restrict__ Csup, const R* __restrict__ E,
                                                  R* __restrict__ values, int MF, int MQ,
                                                  const int32_t* __restrict__ rows, int use_box, int stage_c) {
  using L = CutRowSmem<R, P, STIFF>;
  constexpr int Q = L::Q, NB = L::NB, Q2 = L::Q2, Q3 = L::Q3, NB3 = L::NB3, NT = L::NT, NBP = L::NBP, Q2P = L::Q2P;
  constexpr int NW = L::NW, DEPTH = L::DEPTH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = rows[blockIdx.x];
  const int n1 = M.dir[0].n, n2 = M.dir[1].n;
  const int q12 = fdiv(row, M.div_n1);
  const int i1 = row - q12 * n1, i3 = fdiv(q12, M.div_n2), i2 = q12 - i3 * n2;
  const int32_t bcode = use_box ? M.topo.box[row] : -1;
  const int64_t r0 = M.topo.rowptr[row];
  const int nnz = (int)(M.topo.rowptr[row + 1] - r0);

  R* accw = reinterpret_cast<R*>(smem_raw);  // [NW][NB3], index dj1 + NB (dj2 + NB dj3)
  R* etab = accw + (size_t)NW * NB3;         // [d][eo][kind][Q2P], or [d][eo][TP2] (F2)
  R* uni = etab + L::ETAB;                   // box buffers | per-warp element ring and scratch
  long long* eoff = reinterpret_cast<long long*>(smem_raw + L::ioff(MF, MQ, stage_c));  // [Q3P]
  int* eflag = reinterpret_cast<int*>(eoff + L::Q3P);
  int* elist = eflag + L::Q3P;  // compacted support elements: t | kind << 12
  int* cols = elist + L::Q3P;   // the row's column indices
  __shared__ int s_nel, s_nnz;
  __shared__ long long s_r0;

  const int64_t cs2 = M.dir[0].nsup, cs3 = (int64_t)M.dir[0].nsup * M.dir[1].nsup;
  const int elo1 = max(0, i1 - P), ehi1 = min(M.dir[0].n_el - 1, i1);
  const int elo2 = max(0, i2 - P), ehi2 = min(M.dir[1].n_el - 1, i2);
  const int elo3 = max(0, i3 - P), ehi3 = min(M.dir[2].n_el - 1, i3);
  int bd = -1, bb = 0, bside = 0;
  if (bcode >= 0) {
    bd = bcode & 3;
    bside = (bcode >> 2) & 1;
    bb = bcode >> 3;
  }
  // WQ point ranges of the row's three functions (the standard directions of a DWQ box)
  int nqa = 0, nqb = 0, nqc = 0, qla = 0, qlb = 0, qlc = 0;
  if (use_box) {
    nqa = M.dir[0].nqi[i1], qla = M.dir[0].qlo[i1];
    nqb = M.dir[1].nqi[i2], qlb = M.dir[1].qlo[i2];
    nqc = M.dir[2].nqi[i3], qlc = M.dir[2].qlo[i3];
  }
  // support element classes (1: inside and outside the box, element Gauss points; 2: cut,
  // row of E_e), t = eo1 + Q (eo2 + Q eo3), and where each one's Q^3 values start (the
  // coefficients at its Gauss points in Csup, or row a(i) of E_e)
  const int w1 = ehi1 - elo1 + 1, w2 = ehi2 - elo2 + 1, w3 = ehi3 - elo3 + 1;
  for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
    const int eo1 = t % Q, eo2 = (t / Q) % Q, eo3 = t / Q2;
    int kind = 0;
    long long off = 0;
    if (eo1 < w1 && eo2 < w2 && eo3 < w3) {
      const int e1 = elo1 + eo1, e2 = elo2 + eo2, e3 = elo3 + eo3;
      const int64_t eid = e1 + (int64_t)M.dir[0].n_el * (e2 + (int64_t)M.dir[1].n_el * e3);
      const int8_t st = M.topo.elem_state[eid];
      const int ci = M.topo.elem_cut_id[eid];
      if (st == E_IN) {
        kind = 1;
        if (bd >= 0) {
          const int ed = sel3(bd, e1, e2, e3);
          if ((bside == 0 && ed < bb) || (bside == 1 && ed >= bb)) kind = 0;
        }
        off = (int64_t)e1 * Q + cs2 * ((int64_t)e2 * Q) + cs3 * ((int64_t)e3 * Q);
      } else if (st == E_CUT) {
        kind = 2;
        const int a = (i1 - e1) + Q * ((i2 - e2) + Q * (i3 - e3));
        off = ((int64_t)ci * Q3 + a) * L::Q3P;  // E rows padded to Q3P
      }
    }
    eflag[t] = kind;
    eoff[t] = off;
  }
  {
    // NW * NB3 is a multiple of 4 (NW is 2, 4 or 8 and NB3 is odd only with NW = 8, 4)
    float4* z = reinterpret_cast<float4*>(accw);
    const int nz = (int)((size_t)NW * NB3 * sizeof(R) / 16);
    for (int t = threadIdx.x; t < nz; t += blockDim.x) z[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (threadIdx.x == 0) s_nnz = nnz, s_r0 = r0;
  // the row's column indices
  {
    const uint32_t cs = (uint32_t)__cvta_generic_to_shared(cols);
    for (int k = threadIdx.x; k < nnz; k += blockDim.x) cp_word_nc<4>(cs + 4u * k, M.topo.colind + r0 + k);
  }
  // element Gauss tables of the row's support elements: warp per (d, eo, kind) table, lanes
  // over its Q^2 entries (zeros for positions past the last element)
  for (int c = warp; c < 3 * Q * NT; c += NW) {
    const int kind = c % NT, eo = (c / NT) % Q, d = c / (NT * Q);
    const int e = sel3(d, elo1, elo2, elo3) + eo, id = sel3(d, i1, i2, i3);
    // c = (d Q + eo) NT + kind; entry idx = b Q + g
    R* dst = L::F2 ? etab + (size_t)(d * Q + eo) * L::TP2 + kind : etab + (size_t)c * Q2P;
    auto at = [&](int idx) { return L::F2 ? ((idx / Q) * L::QE + idx % Q) * 2 : idx; };
    if (e <= sel3(d, ehi1, ehi2, ehi3)) {
      const R* src = GTab<R>::ge(M.dir[d], kind) + ((size_t)e * Q + (id - e)) * Q2;
      const uint32_t ds = (uint32_t)__cvta_generic_to_shared(dst);
      for (int idx = lane; idx < Q2; idx += 32) cp_word_nc<sizeof(R)>(ds + (uint32_t)(at(idx) * sizeof(R)), src + idx);
    } else {
      for (int idx = lane; idx < Q2; idx += 32) dst[at(idx)] = R(0);
    }
  }

  // ---- DWQ box
  const int MB = MF > MQ ? MF : MQ;
  R* tabf = uni;                          // [kind][k < MF][NBP]
  R* tabs = tabf + (size_t)NT * MF * NBP; // [kind][k < MQ][NBP]
  R* tabt = tabs + (size_t)NT * MQ * NBP;
  R* Cb = tabt + (size_t)NT * MQ * NBP;   // [kf][kt][ks] (stage_c)
  R* U = Cb + (stage_c ? (size_t)MF * MQ * MQ : 0);  // [kind][kt][ks][bf]
  R* TB = U + (size_t)NT * MQ * MQ * NB;  // [kind][kt][bs][bf]
  int* sx = reinterpret_cast<int*>(TB + (size_t)NT * MQ * NB * NB);  // [3][MB]: f, s, t
  int mf = 0, ms = 0, mt = 0;
  const int df = bd == 0 ? 0 : (bd == 1 ? 1 : 2), ds = bd == 0 ? 1 : 0, dt = bd == 2 ? 1 : 2;
  if (bd >= 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int d = r == 0 ? df : (r == 1 ? ds : dt);
      const Dir1D& D = M.dir[d];
      const int id = sel3(d, i1, i2, i3), elod = sel3(d, elo1, elo2, elo3), ehid = sel3(d, ehi1, ehi2, ehi3);
      const uint32_t tb = (uint32_t)__cvta_generic_to_shared(r == 0 ? tabf : (r == 1 ? tabs : tabt));
      const int cap = r == 0 ? MF : MQ;
      int m;
      if (d == bd) {
        const int ka = bside == 0 ? elod : bb, kb = bside == 0 ? bb - 1 : ehid;
        const int s0 = ka * Q;
        m = (kb - ka + 1) * Q;
        const int rule = ((id * P) + (bb - elod - 1)) * 2 + bside;
        const int slo = s0 - elod * Q;
        const MDiv dm = mdiv_of(m);
        for (int l = threadIdx.x; l < NT * NB * m; l += blockDim.x) {
          const int kb2 = qdiv(l, dm), k = l - kb2 * m, kind = kb2 / NB, b = kb2 - kind * NB;
          cp_word_nc<sizeof(R)>(tb + (uint32_t)((((size_t)kind * cap + k) * NBP + b) * sizeof(R)),
                             CTab<R>::wd(D, kind) + ((size_t)rule * NB + b) * D.nsl + slo + k);
        }
        for (int t = threadIdx.x; t < m; t += blockDim.x) sx[r * MB + t] = s0 + t;
      } else {
        m = sel3(d, nqa, nqb, nqc);
        const int q0 = sel3(d, qla, qlb, qlc);
        const MDiv dm = mdiv_of(m);
        for (int l = threadIdx.x; l < NT * NB * m; l += blockDim.x) {
          const int kb2 = qdiv(l, dm), k = l - kb2 * m, kind = kb2 / NB, b = kb2 - kind * NB;
          cp_word_nc<sizeof(R)>(tb + (uint32_t)((((size_t)kind * cap + k) * NBP + b) * sizeof(R)),
                             CTab<R>::wb(D, kind) + ((size_t)id * NB + b) * D.nql + k);
        }
        const uint32_t sxs = (uint32_t)__cvta_generic_to_shared(sx + r * MB);
        for (int t = threadIdx.x; t < m; t += blockDim.x) cp_word_nc<4>(sxs + 4u * t, D.wq_idx + q0 + t);
      }
      if (r == 0) mf = m;
      if (r == 1) ms = m;
      if (r == 2) mt = m;
    }
  }
  cp_commit();
  cp_wait<0>();
  __syncthreads();
  // compact list of the contributing support elements (warp 0), and the box's coefficient
  // block C(k_f, k_s, k_t) gathered by the whole block
  if (warp == 0) {
    // the element-Gauss entries first, then the E rows, so that dealing the list round-robin
    // gives every warp the same number of each (to within one)
    int base = 0;
#pragma unroll
    for (int want = 1; want <= 2; ++want)
      for (int c = 0; c < Q3; c += 32) {
        const int t = c + lane;
        const bool hit = t < Q3 && eflag[t] == want;
        const unsigned mk = __ballot_sync(0xffffffffu, hit);
        if (hit) elist[base + __popc(mk & ((1u << lane) - 1u))] = t | (want << 12);
        base += __popc(mk);
      }
    if (lane == 0) s_nel = base;
  }
  const int64_t csf = df == 0 ? 1 : (df == 1 ? cs2 : cs3), css = ds == 0 ? 1 : cs2, cst = dt == 1 ? cs2 : cs3;
  const int* sxf = sx;
  const int* sxs = sx + MB;
  const int* sxt = sx + 2 * MB;
  if (bd >= 0) {
    const MDiv dms = mdiv_of(ms), dmt = mdiv_of(mt);
    if (stage_c) {
      const uint32_t cbs = (uint32_t)__cvta_generic_to_shared(Cb);
      // thread per (ks, kt) line, all k_f: Cb[(k mt + kt) ms + ks]
      const uint32_t kstep = (uint32_t)(mt * ms * sizeof(R));
      for (int t = threadIdx.x; t < ms * mt; t += blockDim.x) {
        const int kt = qdiv(t, dms), ks = t - kt * ms;
        const R* src = Csup + sxs[ks] * css + sxt[kt] * cst;
        const uint32_t dst = cbs + (uint32_t)(t * sizeof(R));
        for (int k = 0; k < mf; ++k) cp_word_nc<sizeof(R)>(dst + k * kstep, src + sxf[k] * csf);
      }
      cp_commit();
      cp_wait<0>();
    }
    __syncthreads();
    // U[kind][kt][ks][bf] = sum_k T_f,kind[bf][k] C(k, ks, kt): thread per (ks, kt, kind)
    for (int t = threadIdx.x; t < NT * ms * mt; t += blockDim.x) {
      const int q = qdiv(t, dms), ks = t - q * ms, kind = qdiv(q, dmt), kt = q - kind * mt;
      const R* tk = tabf + (size_t)kind * MF * NBP;
      const R* cb = Csup + sxs[ks] * css + sxt[kt] * cst;
      R u[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) u[b] = R(0);
      for (int k = 0; k < mf; ++k) {
        const R c = stage_c ? Cb[((size_t)k * mt + kt) * ms + ks] : cb[sxf[k] * csf];
        R w[NBP];
        lds_vec<R, NBP>(tk + (size_t)k * NBP, w);
#pragma unroll
        for (int b = 0; b < NB; ++b) u[b] += w[b] * c;
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) U[(((size_t)kind * MQ + kt) * MQ + ks) * NB + b] = u[b];
    }
    __syncthreads();
    // TB[0][kt][bs][bf] = sum_ks T_s,0[bs][ks] U_1 + T_s,1[bs][ks] U_0 (mass: T_s,0 U_0),
    // TB[1][kt][bs][bf] = sum_ks T_s,0[bs][ks] U_0: thread per (bf, kt, placement)
    for (int t = threadIdx.x; t < NT * NB * mt; t += blockDim.x) {
      const int q = t / NB, bf = t - q * NB, part = qdiv(q, dmt), kt = q - part * mt;
      R ta[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) ta[b] = R(0);
      for (int ks = 0; ks < ms; ++ks) {
        const R u0 = U[((size_t)kt * MQ + ks) * NB + bf];
        R w0[NBP];
        lds_vec<R, NBP>(tabs + (size_t)ks * NBP, w0);
        if (STIFF && part == 0) {
          const R u1 = U[(((size_t)MQ + kt) * MQ + ks) * NB + bf];
          R w1[NBP];
          lds_vec<R, NBP>(tabs + ((size_t)MQ + ks) * NBP, w1);
#pragma unroll
          for (int b = 0; b < NB; ++b) ta[b] += w0[b] * u1 + w1[b] * u0;
        } else {
#pragma unroll
          for (int b = 0; b < NB; ++b) ta[b] += w0[b] * u0;
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) TB[(((size_t)part * MQ + kt) * NB + b) * NB + bf] = ta[b];
    }
    __syncthreads();
    // V[bf][bs][bt] = sum_kt T_t,h[bt][kt] TB[h]: thread per (bf, bs, h), into the band of warp h
    const int af = df == 0 ? 1 : (df == 1 ? NB : NB * NB), as_ = ds == 0 ? 1 : NB, at = dt == 1 ? NB : NB * NB;
    for (int t = threadIdx.x; t < NT * NB * NB; t += blockDim.x) {
      const int bf = t % NB, q = t / NB, bs = q % NB, h = q / NB;
      const R* tk = tabt + (size_t)h * MQ * NBP;
      R v[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) v[b] = R(0);
      for (int kt = 0; kt < mt; ++kt) {
        const R x = TB[(((size_t)h * MQ + kt) * NB + bs) * NB + bf];
        R w[NBP];
        lds_vec<R, NBP>(tk + (size_t)kt * NBP, w);
#pragma unroll
        for (int b = 0; b < NB; ++b) v[b] += w[b] * x;
      }
      R* ab = accw + (size_t)h * NB3 + bf * af + bs * as_;
#pragma unroll
      for (int b = 0; b < NB; ++b) ab[b * at] += v[b];
    }
  }
  __syncthreads();  // box buffers share memory with the element ring

  // ---- remaining support elements, in list order; warp w takes entries w, w + NW, ... and
  // keeps DEPTH of them in flight (the coefficients at the element's Gauss points, or the
  // cut element's E row) while it works on the oldest.
  const int nel = s_nel;
  R* acc = accw + (size_t)warp * NB3;
  R* ring = uni + (size_t)warp * L::wscr;
  R* U0 = ring + DEPTH * L::Q3P;  // [g3][g2][b1]
  R* U1 = U0 + L::Q3P;
  R* TA = U1 + L::Q3P;  // [g3][b2][b1]
  R* TBw = TA + L::Q3P;
  // per-lane constants of entry k = lane + 32 j (j < KJ): offset in the coefficient grid
  // of Gauss point (g1, g2, g3) of an element, and band offset b1 + NB (b2 + NB b3)
  constexpr int KJ = (Q3 + 31) / 32;
  // (offsets below (p+1) (1 + nsup1 + nsup1 nsup2) < 2^31 for every mesh the ABI accepts)
  int coff[KJ], boff[KJ];
#pragma unroll
  for (int jj = 0; jj < KJ; ++jj) {
    const int k = lane + 32 * jj;
    const int g1 = k % Q, g2 = (k / Q) % Q, g3 = k / Q2;
    coff[jj] = (int)(g1 + cs2 * g2 + cs3 * g3);
    boff[jj] = (g3 * NB + g2) * NB + g1;
  }
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
  // issue the fetch of list entry j into ring slot `slot` (one commit group per call)
  auto fetch = [&](int j, int slot) {
    if (j < nel) {
      const int code = elist[j], t = code & 4095, kind = code >> 12;
      const long long off = eoff[t];
      const uint32_t dst = ring_s + (uint32_t)(slot * L::Q3P * sizeof(R));
      if (kind == 1) {
        const R* cbase = Csup + off;
#pragma unroll
        for (int jj = 0; jj < KJ; ++jj)
          if (lane + 32 * jj < Q3) cp_word<sizeof(R)>(dst + (uint32_t)((lane + 32 * jj) * sizeof(R)), cbase + coff[jj]);
      } else {
        // the row with its padding, 16 bytes per copy (rows and ring slots 16-byte aligned)
        const R* Er = E + off;
        constexpr int NC = L::Q3P * (int)sizeof(R) / 16;
#pragma unroll
        for (int c = lane; c < NC; c += 32)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * c),
                       "l"(reinterpret_cast<const unsigned char*>(Er) + 16 * c)
                       : "memory");
      }
    }
    cp_commit();
  };
#pragma unroll
  for (int s = 0; s < DEPTH - 1; ++s) fetch(warp + s * NW, s);
  for (int j = warp, it = 0; j < nel; j += NW, ++it) {
    fetch(j + (DEPTH - 1) * NW, (it + DEPTH - 1) % DEPTH);
    cp_wait<DEPTH - 1>();
    __syncwarp();
    const R* cur = ring + (it % DEPTH) * L::Q3P;
    const int code = elist[j], t = code & 4095, kind = code >> 12;
    const int eo1 = t % Q, eo2 = (t / Q) % Q, eo3 = t / Q2;
    const int o1 = elo1 + eo1 - i1 + P, o2 = elo2 + eo2 - i2 + P, o3 = elo3 + eo3 - i3 + P;
    if (L::F2 && kind == 1) {
      gauss_elem_f2<L>(reinterpret_cast<const float*>(cur), reinterpret_cast<const float*>(etab), eo1, eo2, eo3,
                       reinterpret_cast<float2*>(U0), reinterpret_cast<float2*>(U0 + 2 * L::Q3P),
                       reinterpret_cast<float*>(acc + (o3 * NB + o2) * NB + o1), lane);
    } else if (kind == 1) {
      const R* C = cur;  // [g3][g2][g1]
      const R* T0 = etab + ((0 * Q + eo1) * NT) * Q2P;
      const R* T1 = etab + ((1 * Q + eo2) * NT) * Q2P;
      const R* T2 = etab + ((2 * Q + eo3) * NT) * Q2P;
      // contract g1: lane per (g2, g3), all b1
      for (int l = lane; l < Q2; l += 32) {
        R x[Q], f0[Q2P], f1[Q2P];
#pragma unroll
        for (int g = 0; g < Q; ++g) x[g] = C[g + Q * l];
        lds_vec<R, Q2P>(T0, f0);
        if (STIFF) lds_vec<R, Q2P>(T0 + Q2P, f1);
#pragma unroll
        for (int b = 0; b < Q; ++b) {
          R a0 = R(0), a1 = R(0);
#pragma unroll
          for (int g = 0; g < Q; ++g) {
            a0 += f0[b * Q + g] * x[g];
            if (STIFF) a1 += f1[b * Q + g] * x[g];
          }
          U0[b + Q * l] = a0;
          if (STIFF) U1[b + Q * l] = a1;
        }
      }
      __syncwarp();
      // contract g2: lane per (b1, g3), all b2
      for (int l = lane; l < Q2; l += 32) {
        const int b1 = l % Q, g3 = l / Q;
        R x0[Q], x1[Q], f0[Q2P], f1[Q2P];
#pragma unroll
        for (int g = 0; g < Q; ++g) {
          x0[g] = U0[b1 + Q * (g + Q * g3)];
          if (STIFF) x1[g] = U1[b1 + Q * (g + Q * g3)];
        }
        lds_vec<R, Q2P>(T1, f0);
        if (STIFF) lds_vec<R, Q2P>(T1 + Q2P, f1);
#pragma unroll
        for (int b = 0; b < Q; ++b) {
          R ta = R(0), tb = R(0);
#pragma unroll
          for (int g = 0; g < Q; ++g) {
            if (STIFF) {
              ta += f0[b * Q + g] * x1[g] + f1[b * Q + g] * x0[g];
              tb += f0[b * Q + g] * x0[g];
            } else {
              ta += f0[b * Q + g] * x0[g];
            }
          }
          TA[b1 + Q * (b + Q * g3)] = ta;
          if (STIFF) TBw[b1 + Q * (b + Q * g3)] = tb;
        }
      }
      __syncwarp();
      // contract g3 and add: lane per (b1, b2), all b3
      for (int l = lane; l < Q2; l += 32) {
        const int b1 = l % Q, b2 = l / Q;
        R xa[Q], xb[Q], f0[Q2P], f1[Q2P];
#pragma unroll
        for (int g = 0; g < Q; ++g) {
          xa[g] = TA[l + Q2 * g];
          if (STIFF) xb[g] = TBw[l + Q2 * g];
        }
        lds_vec<R, Q2P>(T2, f0);
        if (STIFF) lds_vec<R, Q2P>(T2 + Q2P, f1);
        R* ap = acc + (o3 * NB + (o2 + b2)) * NB + (o1 + b1);
#pragma unroll
        for (int b = 0; b < Q; ++b) {
          R v = R(0);
#pragma unroll
          for (int g = 0; g < Q; ++g) {
            v += f0[b * Q + g] * xa[g];
            if (STIFF) v += f1[b * Q + g] * xb[g];
          }
          ap[b * NB * NB] += v;
        }
      }
      __syncwarp();
    } else {
      R* ab = acc + (o3 * NB + o2) * NB + o1;
#pragma unroll
      for (int jj = 0; jj < KJ; ++jj)
        if (lane + 32 * jj < Q3) ab[boff[jj]] += cur[lane + 32 * jj];
    }
    __syncwarp();  // the next iteration refills cur
  }
  cp_wait<0>();
  __syncthreads();
  // ---- fixed-order sum of the warp accumulators, written on the row's pattern
  const int64_t rb = s_r0;
  const int nz = s_nnz;
  const int jb1 = i1 - P, jb2 = i2 - P, jb3 = i3 - P;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    const int j = cols[k];
    const int qj = fdiv(j, M.div_n1);
    const int j3 = fdiv(qj, M.div_n2);
    const int o = ((j3 - jb3) * NB + (qj - j3 * n2 - jb2)) * NB + (j - qj * n1 - jb1);
    R v = R(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) v += accw[(size_t)w * NB3 + o];
    values[rb + k] = v;
  }
}

template <typename R, int P, bool STIFF>
cudaError_t launch_rows_t(const MeshView& M, const R* Csup, const R* E, R* values, int n_rows, const int32_t* rows,
                          int use_box, cudaStream_t st) {
  if (n_rows <= 0) return cudaSuccess;
  constexpr int Q = P + 1;
  // points of a standard WQ rule (any support) and of the kept side of a DWQ rule
  int MQ = Q;
  for (int d = 0; d < 3; ++d) MQ = MQ > M.dir[d].nql ? MQ : M.dir[d].nql;
  const int MF = MQ > P * Q ? MQ : P * Q;
  using LR = CutRowSmem<R, P, STIFF>;
  // the box's coefficient block is staged in shared memory when the plan still fits
  static int optin = -1;
  if (optin < 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
  }
  const int stage_c = LR::bytes(MF, MQ, 1) + 64 <= (size_t)optin ? 1 : 0;
  const size_t smem = LR::bytes(MF, MQ, stage_c);
  cudaError_t err = cudaFuncSetAttribute(k_cut_rows<R, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_cut_rows<R, P, STIFF><<<n_rows, 32 * LR::NW, smem, st>>>(M, Csup, E, values, MF, MQ, rows, use_box, stage_c);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cut_elem(const MeshView& M, const LevelSet& L, bool fp64, bool mom64, bool stiff, int coef_kind,
                            double c0, const double* ck, void* E, int n_cut_elems, int ci0, cudaStream_t st);

// part 0: cut-element matrices (cut_elem.cu) of the elements [ci0, ci0 + n_cut_elems) of the
// cut-element list; part 1: the rows in `rows` (n_rows of them).
cudaError_t launch_cut(const MeshView& M, const LevelSet& L, bool fp64, bool mom64, bool stiff, int coef_kind,
                       double c0, const double* ck, const void* Csup, void* E, void* values, int n_cut_elems,
                       int n_rows, int part, const int32_t* rows, int use_box, cudaStream_t st, int ci0) {
  if (part == 0) return launch_cut_elem(M, L, fp64, mom64, stiff, coef_kind, c0, ck, E, n_cut_elems, ci0, st);
#define SFA_ROWS_ARGS(RT) M, (const RT*)Csup, (const RT*)E, (RT*)values, n_rows, rows, use_box, st
#define SFA_ROWS_CASE(PP)                                                                                       \
  case PP:                                                                                                      \
    if (fp64)                                                                                                   \
      return stiff ? launch_rows_t<double, PP, true>(SFA_ROWS_ARGS(double))                                    \
                   : launch_rows_t<double, PP, false>(SFA_ROWS_ARGS(double));                                   \
    return stiff ? launch_rows_t<float, PP, true>(SFA_ROWS_ARGS(float))                                         \
                 : launch_rows_t<float, PP, false>(SFA_ROWS_ARGS(float));
  switch (M.p) {
    SFA_ROWS_CASE(2)
    SFA_ROWS_CASE(3)
    SFA_ROWS_CASE(4)
    SFA_ROWS_CASE(5)
    SFA_ROWS_CASE(6)
  }
#undef SFA_ROWS_CASE
#undef SFA_ROWS_ARGS
  return cudaErrorInvalidValue;
}
