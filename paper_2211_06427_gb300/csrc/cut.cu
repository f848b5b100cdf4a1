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
  static constexpr int ETAB = 3 * Q * NT * Q2P;
  // box buffers for MF points in the DWQ direction, MQ in the others
  __host__ __device__ static size_t box(int MF, int MQ) {
    return (size_t)NT * (MF + 2 * MQ) * NBP + (size_t)NT * MQ * MQ * NB + (size_t)NT * MQ * NB * NB +
           (3 * (size_t)(MF > MQ ? MF : MQ) * sizeof(int) + sizeof(R) - 1) / sizeof(R);
  }
  static constexpr int Q3P = (Q3 + 3) / 4 * 4;
  static constexpr size_t elem = (size_t)NW * 6 * Q3P;
  __host__ __device__ static size_t bytes(int MF, int MQ) {
    const size_t bx = box(MF, MQ), uni = bx > elem ? bx : elem;
    return ((size_t)NW * NB3 + ETAB + uni) * sizeof(R) + 2 * Q3P * sizeof(int) + 16;
  }
};

// One block per cut row.  Accumulators: one dense (2p+1)^3 band per warp, summed in a
// fixed order at the end.
//  * DWQ box (regular part, Sec. 2.2): tensor-product rule with the one-sided DWQ rule in
//    the box's direction f and the standard WQ rules in the other two (s, t); contracted by
//    the whole block in the order f, s, t:
//      U = T_f C,  TB = T_s U,  V = T_t TB      (stiffness: the three derivative placements)
//    one thread per output line, the 1D tables transposed ([point][b]) for vector reads.
//  * Inside support elements outside the box: (p+1)^3 Gauss points of the element, three
//    register-blocked stages per warp, tables F_d[b][g] = w B_{i_d} B_{e_d+b} of the row's
//    support elements staged once per row.
//  * Cut elements: row a(i) of the element matrix E_e.
//  Rows come from `rows` (the cut rows; for the Standard Gauss variant every active row);
//  use_box = 0 ignores the DWQ boxes (Hybrid and Standard Gauss variants, Sec. 3.1), so
//  every inside support element is integrated with its Gauss points.
template <typename R, int P, bool STIFF>
__global__ void __launch_bounds__(256, CutRowSmem<R, P, STIFF>::MINB) k_cut_rows(MeshView M, const R* __restrict__ Csup, const R* __restrict__ E,
                                                  R* __restrict__ values, int MF, int MQ,
                                                  const int32_t* __restrict__ rows, int use_box) {
  using L = CutRowSmem<R, P, STIFF>;
  constexpr int Q = L::Q, NB = L::NB, Q2 = L::Q2, Q3 = L::Q3, NB3 = L::NB3, NT = L::NT, NBP = L::NBP, Q2P = L::Q2P;
  constexpr int NW = L::NW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = rows[blockIdx.x];
  const int n1 = M.dir[0].n, n2 = M.dir[1].n;
  const int q12 = fdiv(row, M.div_n1);
  const int i1 = row - q12 * n1, i3 = fdiv(q12, M.div_n2), i2 = q12 - i3 * n2;
  const int32_t bcode = use_box ? M.topo.box[row] : -1;

  R* accw = reinterpret_cast<R*>(smem_raw);  // [NW][NB3], index dj1 + NB (dj2 + NB dj3)
  R* etab = accw + (size_t)NW * NB3;         // [d][eo][kind][Q2P]
  R* uni = etab + L::ETAB;                   // box buffers | per-warp element scratch
  int* eflag = reinterpret_cast<int*>(uni + (L::box(MF, MQ) > L::elem ? L::box(MF, MQ) : L::elem));  // [Q3P]
  int* elist = eflag + L::Q3P;               // compacted support elements: t | kind << 12
  __shared__ int s_nel;

  {
    // NW * NB3 is a multiple of 4 (NW is 2, 4 or 8 and NB3 is odd only with NW = 8, 4)
    float4* z = reinterpret_cast<float4*>(accw);
    const int nz = (int)((size_t)NW * NB3 * sizeof(R) / 16);
    for (int t = threadIdx.x; t < nz; t += blockDim.x) z[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int64_t cs2 = M.dir[0].nsup, cs3 = (int64_t)M.dir[0].nsup * M.dir[1].nsup;
  const int elo1 = max(0, i1 - P), ehi1 = min(M.dir[0].n_el - 1, i1);
  const int elo2 = max(0, i2 - P), ehi2 = min(M.dir[1].n_el - 1, i2);
  const int elo3 = max(0, i3 - P), ehi3 = min(M.dir[2].n_el - 1, i3);
  // element Gauss tables of the row's support elements
  // warp per (d, eo, kind) table, lanes over its Q^2 entries
  for (int c = warp; c < 3 * Q * NT; c += NW) {
    const int kind = c % NT, eo = (c / NT) % Q, d = c / (NT * Q);
    const int e = sel3(d, elo1, elo2, elo3) + eo, id = sel3(d, i1, i2, i3);
    const bool live = e <= sel3(d, ehi1, ehi2, ehi3);
    const R* src = GTab<R>::ge(M.dir[d], kind) + ((size_t)e * Q + (id - e)) * Q2;
    R* dst = etab + (size_t)c * Q2P;  // c = (d Q + eo) NT + kind
    for (int idx = lane; idx < Q2; idx += 32) dst[idx] = live ? src[idx] : R(0);
  }
  int bd = -1, bb = 0, bside = 0;
  if (bcode >= 0) {
    bd = bcode & 3;
    bside = (bcode >> 2) & 1;
    bb = bcode >> 3;
  }

  // ---- DWQ box
  if (bd >= 0) {
    const int df = bd, ds = bd == 0 ? 1 : 0, dt = bd == 2 ? 1 : 2;
    const int MB = MF > MQ ? MF : MQ;
    R* tabf = uni;                          // [kind][k < MF][NBP]
    R* tabs = tabf + (size_t)NT * MF * NBP; // [kind][k < MQ][NBP]
    R* tabt = tabs + (size_t)NT * MQ * NBP;
    R* U = tabt + (size_t)NT * MQ * NBP;    // [kind][kt][ks][bf]
    R* TB = U + (size_t)NT * MQ * MQ * NB;  // [kind][kt][bs][bf]
    int* sx = reinterpret_cast<int*>(TB + (size_t)NT * MQ * NB * NB);  // [3][MB]: f, s, t
    int mf = 0, ms = 0, mt = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int d = r == 0 ? df : (r == 1 ? ds : dt);
      const Dir1D& D = M.dir[d];
      const int id = sel3(d, i1, i2, i3), elod = sel3(d, elo1, elo2, elo3), ehid = sel3(d, ehi1, ehi2, ehi3);
      R* tb = r == 0 ? tabf : (r == 1 ? tabs : tabt);
      const int cap = r == 0 ? MF : MQ;
      int m;
      if (d == bd) {
        const int ka = bside == 0 ? elod : bb, kb = bside == 0 ? bb - 1 : ehid;
        const int s0 = ka * Q;
        m = (kb - ka + 1) * Q;
        const int rule = ((id * P) + (bb - elod - 1)) * 2 + bside;
        const int slo = s0 - elod * Q;
        // warp per point k, lanes over (kind, b)
        for (int k = warp; k < m; k += NW)
          for (int l = lane; l < NT * NB; l += 32) {
            const int kind = l / NB, b = l - kind * NB;
            tb[((size_t)kind * cap + k) * NBP + b] = CTab<R>::wd(D, kind)[((size_t)rule * NB + b) * D.nsl + slo + k];
          }
        for (int t = threadIdx.x; t < m; t += blockDim.x) sx[r * MB + t] = s0 + t;
      } else {
        m = D.nqi[id];
        const int q0 = D.qlo[id];
        for (int k = warp; k < m; k += NW)
          for (int l = lane; l < NT * NB; l += 32) {
            const int kind = l / NB, b = l - kind * NB;
            tb[((size_t)kind * cap + k) * NBP + b] = CTab<R>::wb(D, kind)[((size_t)id * NB + b) * D.nql + k];
          }
        for (int t = threadIdx.x; t < m; t += blockDim.x) sx[r * MB + t] = D.wq_idx[q0 + t];
      }
      if (r == 0) mf = m;
      if (r == 1) ms = m;
      if (r == 2) mt = m;
    }
    __syncthreads();
    const int64_t csf = df == 0 ? 1 : (df == 1 ? cs2 : cs3), css = ds == 0 ? 1 : cs2, cst = dt == 1 ? cs2 : cs3;
    const int* sxf = sx;
    const int* sxs = sx + MB;
    const int* sxt = sx + 2 * MB;
    // U[kind][kt][ks][bf] = sum_k T_f,kind[bf][k] C(k, ks, kt)
    for (int t = threadIdx.x; t < ms * mt; t += blockDim.x) {
      const int ks = t % ms, kt = t / ms;
      const R* cb = Csup + sxs[ks] * css + sxt[kt] * cst;
      R u0[NB], u1[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) u0[b] = u1[b] = R(0);
      for (int k = 0; k < mf; ++k) {
        const R c = cb[sxf[k] * csf];
        R w[NBP];
        lds_vec<R, NBP>(tabf + (size_t)k * NBP, w);
#pragma unroll
        for (int b = 0; b < NB; ++b) u0[b] += w[b] * c;
        if (STIFF) {
          lds_vec<R, NBP>(tabf + ((size_t)MF + k) * NBP, w);
#pragma unroll
          for (int b = 0; b < NB; ++b) u1[b] += w[b] * c;
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        U[((size_t)kt * MQ + ks) * NB + b] = u0[b];
        if (STIFF) U[(((size_t)MQ + kt) * MQ + ks) * NB + b] = u1[b];
      }
    }
    __syncthreads();
    // TA[kt][bs][bf] = sum_ks T_s,0[bs][ks] U_1 + T_s,1[bs][ks] U_0 ; TB = T_s,0 U_0  (mass: TA = T_s,0 U_0)
    for (int t = threadIdx.x; t < NB * mt; t += blockDim.x) {
      const int bf = t % NB, kt = t / NB;
      R ta[NB], tb[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) ta[b] = tb[b] = R(0);
      for (int ks = 0; ks < ms; ++ks) {
        const R u0 = U[((size_t)kt * MQ + ks) * NB + bf];
        R w0[NBP];
        lds_vec<R, NBP>(tabs + (size_t)ks * NBP, w0);
        if (STIFF) {
          const R u1 = U[(((size_t)MQ + kt) * MQ + ks) * NB + bf];
          R w1[NBP];
          lds_vec<R, NBP>(tabs + ((size_t)MQ + ks) * NBP, w1);
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            ta[b] += w0[b] * u1 + w1[b] * u0;
            tb[b] += w0[b] * u0;
          }
        } else {
#pragma unroll
          for (int b = 0; b < NB; ++b) ta[b] += w0[b] * u0;
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        TB[((size_t)kt * NB + b) * NB + bf] = ta[b];
        if (STIFF) TB[(((size_t)MQ + kt) * NB + b) * NB + bf] = tb[b];
      }
    }
    __syncthreads();
    // V[bf][bs][bt] = sum_kt T_t,0[bt][kt] TA + T_t,1[bt][kt] TB, into accumulator 0
    const int af = df == 0 ? 1 : (df == 1 ? NB : NB * NB), as_ = ds == 0 ? 1 : NB, at = dt == 1 ? NB : NB * NB;
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
      const int bf = t % NB, bs = t / NB;
      R v[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) v[b] = R(0);
      for (int kt = 0; kt < mt; ++kt) {
        const R xa = TB[((size_t)kt * NB + bs) * NB + bf];
        R w0[NBP];
        lds_vec<R, NBP>(tabt + (size_t)kt * NBP, w0);
#pragma unroll
        for (int b = 0; b < NB; ++b) v[b] += w0[b] * xa;
        if (STIFF) {
          const R xb = TB[(((size_t)MQ + kt) * NB + bs) * NB + bf];
          R w1[NBP];
          lds_vec<R, NBP>(tabt + ((size_t)MQ + kt) * NBP, w1);
#pragma unroll
          for (int b = 0; b < NB; ++b) v[b] += w1[b] * xb;
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) accw[bf * af + bs * as_ + b * at] += v[b];
    }
  }
  __syncthreads();  // box buffers and element tables are shared with what follows

  // ---- remaining support elements.  Each support element t = eo1 + Q (eo2 + Q eo3) is
  // classified (1: inside and outside the box, element Gauss points; 2: cut, row of E_e) and
  // the contributing ones are listed in order; warp w takes entries w, w + NW, ... and
  // fetches the next entry's 125 values (coefficients at the Gauss points, or the E row)
  // with cp.async while it works on the current one.
  const int w1 = ehi1 - elo1 + 1, w2 = ehi2 - elo2 + 1, w3 = ehi3 - elo3 + 1;
  for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
    const int eo1 = t % Q, eo2 = (t / Q) % Q, eo3 = t / Q2;
    int kind = 0;
    if (eo1 < w1 && eo2 < w2 && eo3 < w3) {
      const int e1 = elo1 + eo1, e2 = elo2 + eo2, e3 = elo3 + eo3;
      const int8_t st = M.topo.elem_state[e1 + (int64_t)M.dir[0].n_el * (e2 + (int64_t)M.dir[1].n_el * e3)];
      if (st == E_IN) {
        kind = 1;
        if (bd >= 0) {
          const int ed = sel3(bd, e1, e2, e3);
          if ((bside == 0 && ed < bb) || (bside == 1 && ed >= bb)) kind = 0;
        }
      } else if (st == E_CUT) {
        kind = 2;
      }
    }
    eflag[t] = kind;
  }
  __syncthreads();
  if (warp == 0) {
    int base = 0;
    for (int c = 0; c < Q3; c += 32) {
      const int t = c + lane;
      const int kind = t < Q3 ? eflag[t] : 0;
      const unsigned mk = __ballot_sync(0xffffffffu, kind != 0);
      if (kind) elist[base + __popc(mk & ((1u << lane) - 1u))] = t | (kind << 12);
      base += __popc(mk);
    }
    if (lane == 0) s_nel = base;
  }
  __syncthreads();
  const int nel = s_nel;
  R* acc = accw + (size_t)warp * NB3;
  R* ws = uni + (size_t)warp * 6 * L::Q3P;
  R* U0 = ws + 2 * L::Q3P;  // [g3][g2][b1]
  R* U1 = ws + 3 * L::Q3P;
  R* TA = ws + 4 * L::Q3P;  // [g3][b2][b1]
  R* TBw = ws + 5 * L::Q3P;
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
  const uint32_t ws_s = (uint32_t)__cvta_generic_to_shared(ws);
  // issue the fetch of list entry j into buffer slot (one commit group per call)
  auto fetch = [&](int j, int slot) {
    if (j < nel) {
      const int code = elist[j], t = code & 4095, kind = code >> 12;
      const int eo1 = t % Q, eo2 = (t / Q) % Q, eo3 = t / Q2;
      const int e1 = elo1 + eo1, e2 = elo2 + eo2, e3 = elo3 + eo3;
      const uint32_t dst = ws_s + (uint32_t)(slot * L::Q3P * sizeof(R));
      if (kind == 1) {
        const R* cbase = Csup + (int64_t)e1 * Q + cs2 * ((int64_t)e2 * Q) + cs3 * ((int64_t)e3 * Q);
#pragma unroll
        for (int jj = 0; jj < KJ; ++jj)
          if (lane + 32 * jj < Q3)
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst + (uint32_t)((lane + 32 * jj) * sizeof(R))),
                         "l"(cbase + coff[jj]), "n"(sizeof(R))
                         : "memory");
      } else {
        const int ci = M.topo.elem_cut_id[e1 + (int64_t)M.dir[0].n_el * (e2 + (int64_t)M.dir[1].n_el * e3)];
        const int a = (i1 - e1) + Q * ((i2 - e2) + Q * (i3 - e3));
        const R* Er = E + ((size_t)ci * Q3 + a) * Q3;
#pragma unroll
        for (int jj = 0; jj < KJ; ++jj)
          if (lane + 32 * jj < Q3)
            asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst + (uint32_t)((lane + 32 * jj) * sizeof(R))),
                         "l"(Er + lane + 32 * jj), "n"(sizeof(R))
                         : "memory");
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  fetch(warp, 0);
  for (int j = warp, it = 0; j < nel; j += NW, ++it) {
    R* cur = ws + (it & 1) * L::Q3P;
    fetch(j + NW, (it + 1) & 1);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp();
    const int code = elist[j], t = code & 4095, kind = code >> 12;
    const int eo1 = t % Q, eo2 = (t / Q) % Q, eo3 = t / Q2;
    const int o1 = elo1 + eo1 - i1 + P, o2 = elo2 + eo2 - i2 + P, o3 = elo3 + eo3 - i3 + P;
    if (kind == 1) {
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
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // ---- fixed-order sum of the warp accumulators, written on the row's pattern
  const int64_t r0 = M.topo.rowptr[row], r1 = M.topo.rowptr[row + 1];
  const int jb1 = i1 - P, jb2 = i2 - P, jb3 = i3 - P;
  for (int64_t k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
    const int j = M.topo.colind[k];
    const int qj = fdiv(j, M.div_n1);
    const int j3 = fdiv(qj, M.div_n2);
    const int o = ((j3 - jb3) * NB + (qj - j3 * n2 - jb2)) * NB + (j - qj * n1 - jb1);
    R v = R(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) v += accw[(size_t)w * NB3 + o];
    values[k] = v;
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
  const size_t smem = LR::bytes(MF, MQ);
  cudaError_t err = cudaFuncSetAttribute(k_cut_rows<R, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_cut_rows<R, P, STIFF><<<n_rows, 32 * LR::NW, smem, st>>>(M, Csup, E, values, MF, MQ, rows, use_box);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cut_elem(const MeshView& M, const LevelSet& L, bool fp64, bool mom64, bool stiff, int coef_kind,
                            double c0, const double* ck, void* E, int n_cut_elems, cudaStream_t st);

// part 0: cut-element matrices (cut_elem.cu); part 1: the rows in `rows` (n_rows of them).
cudaError_t launch_cut(const MeshView& M, const LevelSet& L, bool fp64, bool mom64, bool stiff, int coef_kind,
                       double c0, const double* ck, const void* Csup, void* E, void* values, int n_cut_elems,
                       int n_rows, int part, const int32_t* rows, int use_box, cudaStream_t st) {
  if (part == 0) return launch_cut_elem(M, L, fp64, mom64, stiff, coef_kind, c0, ck, E, n_cut_elems, st);
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
