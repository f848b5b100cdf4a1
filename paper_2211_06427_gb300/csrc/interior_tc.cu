// Interior rows with the q1 contraction on the tensor cores (precisions SFA_TF32 and
// SFA_TF32X3).  Same formula as the SIMT interior kernels (Sec. 1, row assembly by sum
// factorization):
//   V_i[j3][j2][j1] = sum_q1 WB1_i1[j1][q1] TB[(j3, j2)][q1],
//   TB[(j3, j2)][q1] = sum_q2 WB2_i2[j2][q2] sum_q3 WB3_i3[j3][q3] C[q1, q2, q3]
// (stiffness: TB splits into the x-term paired with the derivative rule WB1_11 and the
// y/z-terms paired with WB1_00).  Two kernels share the plan below.  k_interior_tc3 runs all
// three contractions as tcgen05 MMA chains; k_interior_tc (used where the former's shared
// memory does not fit, 3xTF32 stiffness at p = 6) runs the q3 and q2 contractions on the CUDA
// cores in FP32.  The q1 contraction of G consecutive rows i1 of one (i2, i3) pencil is one
// tcgen05 MMA chain
//   D[(r, dj1)][c] = sum_k A_g[(r, dj1)][k] TB[c][k]
// with M = 128 rows (r, dj1) (G (2p+1) <= 128 of them used), N = (2p+1)^2 pairs
// c = (dj3, dj2) padded to a multiple of 16, and K the q1 window of the group.  A_g is the
// banded matrix of the group's WB1 rows, built once per mesh; TB is written by the q2 stage
// directly in the operand layout.  SFA_TF32 rounds both operands to TF32; SFA_TF32X3 splits
// each into a TF32 head and a TF32 tail and accumulates tail*head + head*tail + head*head,
// which restores close to FP32 accuracy.  The accumulator lives in tensor memory; it is read
// back with tcgen05.ld, staged in shared memory and written row by row with coalesced stores.
//
// Every pencil holding interior rows comes here.  In a direction where the pencil's support
// is regular (two WQ points in each of its p+1 elements) the 1D contraction uses the
// compile-time band structure with the table in registers; at the faces of the mesh (a
// support touching the first or last element, up to 3p+1 points) it runs dense over the
// support's points with the table in shared memory.  Rows i1 of any kind are handled, since
// the band matrix carries each row's own q1 window.  The kernel is persistent: CTA b takes
// tasks b, b + grid, ... in (group, pencil) order and reloads A_g only when the group changes.
#include "interior_common.cuh"
#include "tc_sm103.cuh"

namespace {

constexpr long long kWaitLimit = 2000000000ll;  // clock cycles, about one second

constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }

// Compile-time shape of one degree.
template <int P>
struct TcShape {
  static constexpr int NB = 2 * P + 1, NQ = 2 * P + 2, NC = NB * NB, NB3 = NB * NB * NB;
  static constexpr int NPAD = rup(NC, 16);                 // MMA N
  static constexpr int G = P == 6 ? 8 : 128 / NB;          // rows i1 per MMA group
  static constexpr int KG = rup(2 * (G - 1) + NQ + 3, 8);  // q1 window per term, >= any group's
  static constexpr int NQM = 3 * P + 1;                    // points of a face support (n_el >= p+2)
  static constexpr int NQMP = rup(NQM, 4);                 // dense table row length
  static constexpr int USTR = rup(NQM * KG, 8) + 4;        // U row stride per dj3: = 4 mod 8
};

// Shared-memory plan in floats: [U | R1 | A | tables | rowflag], with U + R1 also the
// output staging area once the MMA has completed.
template <int P, bool STIFF, bool X3>
struct TcSmem {
  using S = TcShape<P>;
  static constexpr int NT = STIFF ? 2 : 1, NS = X3 ? 2 : 1;
  static constexpr int KA = NT * S::KG;
  static constexpr int U_ = rup(NT * S::NB * S::USTR, 32);  // 128-byte aligned R1
  static constexpr int R1a = S::NQM * S::NQM * S::KG, R1b = NT * NS * S::NPAD * S::KG;
  static constexpr int R1_ = R1a > R1b ? R1a : R1b;
  static constexpr int RS = rup(S::NB3, 4) + 4;  // staging row stride (row r starts at r RS + shift_r)
  static constexpr int STG = S::G * RS;
  static constexpr int UR = rup((U_ + R1_ > STG) ? U_ + R1_ : STG, 32);  // U + R1, at least the staging
  static constexpr int A_ = NS * 128 * KA;
  static constexpr int TAB = 2 * NT * S::NB * S::NQMP;  // dense tables: [dir 3, dir 2][kind]
  static constexpr size_t bytes = (size_t)(UR + A_ + TAB) * 4 + S::G * sizeof(int);
};

// A_g for every group: band[g][copy][cidx(m, k, KA)], copy 0 the TF32 head, 1 the tail.
// Column k of term t = k / Kg holds q1 = kst_g + k % Kg; row m = r * NB + dj1.
__global__ void k_tc_band(Dir1D D1, int p, int G, int Kg, int KA, int stiff, float* __restrict__ band) {
  const int g = blockIdx.y, NB = 2 * p + 1;
  const int kst = D1.qlo[g * G] & ~3;
  float* base = band + (size_t)g * 2 * 128 * KA;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 128 * KA; t += gridDim.x * blockDim.x) {
    const int m = t / KA, k = t % KA;
    const int r = m / NB, dj = m % NB, i1 = g * G + r;
    double v = 0.0;
    if (r < G && i1 < D1.n) {
      const int term = k / Kg;
      const double* W = (stiff && term == 0) ? D1.WB11 : D1.WB00;
      const int q = kst + (k % Kg) - D1.qlo[i1];
      if (q >= 0 && q < D1.nqi[i1]) v = W[((size_t)i1 * NB + dj) * D1.nql + q];
    }
    const float hi = tc::tf32_round((float)v);
    const float lo = tc::tf32_round((float)(v - (double)hi));
    base[tc::cidx(m, k, KA)] = hi;
    base[128 * KA + tc::cidx(m, k, KA)] = lo;
  }
}

// Dense 1D contraction over a face support: y[dj] = sum_q tab[dj][q] x[q], tab zero-padded.
template <int P>
__device__ __forceinline__ void dense_apply(const float* __restrict__ tab, const float (&x)[TcShape<P>::NQMP],
                                            float (&y)[TcShape<P>::NB]) {
  using S = TcShape<P>;
#pragma unroll
  for (int dj = 0; dj < S::NB; ++dj) {
    float s = 0.f;
    const float4* t4 = reinterpret_cast<const float4*>(tab + dj * S::NQMP);
#pragma unroll
    for (int q4 = 0; q4 < S::NQMP / 4; ++q4) {
      const float4 w = t4[q4];
      s += w.x * x[4 * q4] + w.y * x[4 * q4 + 1] + w.z * x[4 * q4 + 2] + w.w * x[4 * q4 + 3];
    }
    y[dj] = s;
  }
}

template <int P, bool STIFF, bool X3>
__global__ void __launch_bounds__(256, (X3 || P >= 5) ? 1 : 2)
    k_interior_tc(MeshView M, const float* __restrict__ Cwq, float* __restrict__ values, const float* __restrict__ band,
                  int Kg_mesh, int n_pencils, int ntasks, uint32_t tmem_cols, int kRun) {
  using S = TcShape<P>;
  using L = TcSmem<P, STIFF, X3>;
  constexpr int NB = S::NB, NQ = S::NQ, NC = S::NC, NPAD = S::NPAD, G = S::G, KG = S::KG, NQM = S::NQM;
  constexpr int NQMP = S::NQMP, USTR = S::USTR, NB3 = S::NB3;
  constexpr int NT = L::NT, NS = L::NS, KA = L::KA;
  constexpr int TBC = NPAD * KG;  // floats per TB copy
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* U = reinterpret_cast<float*>(smem_raw);  // [kind][dj3][a2 < NQM][a1 < KG], stride USTR per dj3
  float* R1 = U + L::U_;                          // C slab [a3][a2][a1], then TB [term][copy][cidx(c, a1)]
  float* stage = U;                               // output staging [r][NB3] after the MMA
  float* As = U + L::UR;                          // [copy][cidx(m, k, KA)]
  float* tab3 = As + L::A_;                       // [kind][dj][NQMP] (face supports in i3)
  float* tab2 = tab3 + NT * NB * NQMP;            // [kind][dj][NQMP] (face supports in i2)
  int* rowflag = reinterpret_cast<int*>(tab2 + NT * NB * NQMP);
  constexpr int RS = L::RS;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tslot, tmem_cols);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    s_abort = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  constexpr uint32_t idesc = tc::idesc_tf32(128, NPAD);
  if (Kg_mesh > KG) {  // a group's q1 window exceeds the compiled one: refuse the whole launch
    if (tid == 0) dev_set_status(M.status, DEV_BOUNDS);
    ntasks = 0;
  }

  const Dir1D &D1 = M.dir[0], &D2 = M.dir[1], &D3 = M.dir[2];
  const int NQL2 = D2.nql, NQL3 = D3.nql;
  const int64_t nq1g = D1.nq, nq2g = D2.nq;
  int cur_g = -1;
  uint32_t parity = 0;

  // CTA b takes runs of kRun consecutive tasks (one row group, neighbouring pencils that
  // mostly share i3): runs b, b + grid, ...  (kRun >= 1, chosen by the caller)
  for (int t = blockIdx.x * kRun; t < ntasks; t += (t % kRun == kRun - 1) ? (gridDim.x - 1) * kRun + 1 : 1) {
    const int g = t / n_pencils;
    const int pencil = M.topo.int_tiles[t % n_pencils];
    const int i2 = pencil % D2.n, i3 = pencil / D2.n;
    const int i1a = g * G, i1b = min(D1.n, i1a + G);
    const int64_t rowbase = (int64_t)D1.n * (i2 + (int64_t)D2.n * i3);
    __syncthreads();  // the previous task is done with rowflag and the staging area
    for (int r = tid; r < G; r += blockDim.x) rowflag[r] = (i1a + r < i1b) && M.topo.fn_class[rowbase + i1a + r] == F_INT;
    __syncthreads();
    int any = 0;
#pragma unroll
    for (int r = 0; r < G; ++r) any |= rowflag[r];
    if (!any) continue;

    const bool reg2 = i2 - P >= 1 && i2 <= D2.n_el - 2, reg3 = i3 - P >= 1 && i3 <= D3.n_el - 2;
    const int q2lo = D2.qlo[i2], nq2 = D2.nqi[i2];
    const int q3lo = D3.qlo[i3], nq3 = D3.nqi[i3];
    if (nq2 > NQM || nq3 > NQM) {  // excluded on the host (n_el >= p + 2); never taken
      if (tid == 0) dev_set_status(M.status, DEV_BOUNDS);
      continue;
    }
    if (g != cur_g) {  // band matrix of this row group
      const float4* src = reinterpret_cast<const float4*>(band + (size_t)g * 2 * 128 * KA);
      float4* dst = reinterpret_cast<float4*>(As);
      for (int k = tid; k < NS * 128 * KA / 4; k += blockDim.x) dst[k] = src[k];
      cur_g = g;
    }
    // dense tables of face supports, zero past the support's points
    if (!reg3)
      for (int k = tid; k < NT * NB * NQMP; k += blockDim.x) {
        const int q = k % NQMP, dj = (k / NQMP) % NB, kk = k / (NQMP * NB);
        tab3[k] = q < nq3 ? (kk ? D3.WB11f : D3.WB00f)[((size_t)i3 * NB + dj) * NQL3 + q] : 0.f;
      }
    if (!reg2)
      for (int k = tid; k < NT * NB * NQMP; k += blockDim.x) {
        const int q = k % NQMP, dj = (k / NQMP) % NB, kk = k / (NQMP * NB);
        tab2[k] = q < nq2 ? (kk ? D2.WB11f : D2.WB00f)[((size_t)i2 * NB + dj) * NQL2 + q] : 0.f;
      }
    // coefficient slab over the group's q1 window (zero past the last point): a warp per
    // (a3, a2) row, lanes along q1
    {
      const int kst = D1.qlo[i1a] & ~3;
      int a3 = 0, a2 = warp;
      while (a2 >= nq2) a2 -= nq2, ++a3;
      for (; a3 < nq3;) {
        const float* src = Cwq + nq1g * ((q2lo + a2) + nq2g * (int64_t)(q3lo + a3));
        float* dst = R1 + (a3 * NQM + a2) * KG;
#pragma unroll
        for (int a1 = lane; a1 < KG; a1 += 32) dst[a1] = (kst + a1 < nq1g) ? src[kst + a1] : 0.f;
        a2 += 8;  // next row of this warp
        while (a2 >= nq2) a2 -= nq2, ++a3;
      }
    }
    __syncthreads();

    // q3 contraction: kind 0 (WB3_00) for every term, kind 1 (WB3_11) for the z-term;
    // items (a2, a1), threads split by kind
    {
      constexpr int gsize = 256 / NT;
      const int kk = tid / gsize, tg = tid % gsize;
      float* Uo = U + kk * NB * USTR;
      if (reg3) {
        float w[NB][NQ];
        load_table<float, P>((kk ? D3.WB11f : D3.WB00f) + (size_t)i3 * NB * NQL3, NQL3, w);
        for (int it = tg; it < nq2 * KG; it += gsize) {
          const int a2 = it / KG, a1 = it % KG;
          float x[NQ], y[NB];
#pragma unroll
          for (int q = 0; q < NQ; ++q) x[q] = R1[(q * NQM + a2) * KG + a1];
          band_apply<float, P>(w, x, y);
#pragma unroll
          for (int dj = 0; dj < NB; ++dj) Uo[dj * USTR + a2 * KG + a1] = y[dj];
        }
      } else {
        const float* tb = tab3 + kk * NB * NQMP;
        for (int it = tg; it < nq2 * KG; it += gsize) {
          const int a2 = it / KG, a1 = it % KG;
          float x[NQMP], y[NB];
#pragma unroll
          for (int q = 0; q < NQMP; ++q) x[q] = q < nq3 ? R1[(q * NQM + a2) * KG + a1] : 0.f;
          dense_apply<P>(tb, x, y);
#pragma unroll
          for (int dj = 0; dj < NB; ++dj) Uo[dj * USTR + a2 * KG + a1] = y[dj];
        }
      }
    }
    __syncthreads();

    // q2 contraction.  Items (dj3, a1) ordered so that a warp's 32 lanes cover 4 columns a1
    // and 8 rows dj3: the TB stores in the MMA operand layout then fall in distinct banks.
    //   phase 0 (table WB2_00): x-term TB0 = WB2_00 U_0 (final); z-part of TB1 = WB2_00 U_1
    //   phase 1 (table WB2_11): TB1 += WB2_11 U_0 (final)
    for (int phase = 0; phase < (STIFF ? 2 : 1); ++phase) {
      const int gsize = phase == 0 ? 256 / NT : 256;
      const int term = phase == 0 ? tid / gsize : 1;
      const int tg = phase == 0 ? tid % gsize : tid;
      const int kind = phase == 0 ? term : 0;      // U_kind read
      const int tkind = phase == 0 ? 0 : 1;        // table: WB2_00 or WB2_11
      const float* Ui = U + kind * NB * USTR;
      float* TBt = R1 + term * NS * TBC;
      float w[NB][NQ];
      if (reg2) load_table<float, P>((tkind ? D2.WB11f : D2.WB00f) + (size_t)i2 * NB * NQL2, NQL2, w);
      const float* tb = tab2 + tkind * NB * NQMP;
      for (int it = tg; it < NB * KG; it += gsize) {
        const int a1lo = it & 3, s = it >> 2;
        const int dj3 = s % NB, a1 = (s / NB) * 4 + a1lo;
        float y[NB];
        if (reg2) {
          float x[NQ];
#pragma unroll
          for (int q = 0; q < NQ; ++q) x[q] = Ui[dj3 * USTR + q * KG + a1];
          band_apply<float, P>(w, x, y);
        } else {
          float x[NQMP];
#pragma unroll
          for (int q = 0; q < NQMP; ++q) x[q] = q < nq2 ? Ui[dj3 * USTR + q * KG + a1] : 0.f;
          dense_apply<P>(tb, x, y);
        }
#pragma unroll
        for (int dj = 0; dj < NB; ++dj) {
          const int o = tc::cidx(dj3 * NB + dj, a1, KG);
          if (STIFF && phase == 0 && term == 1) {
            TBt[o] = y[dj];  // completed in phase 1
          } else {
            const float v = (STIFF && phase == 1) ? TBt[o] + y[dj] : y[dj];
            const float hi = tc::tf32_round(v);
            TBt[o] = hi;
            if (X3) TBt[TBC + o] = tc::tf32_round(v - hi);
          }
        }
      }
      if (phase == 0)  // padding rows c in [NC, NPAD) of every copy are zero
        for (int k = tid; k < NT * NS * (NPAD - NC) * KG; k += blockDim.x) {
          const int a1 = k % KG, c = NC + (k / KG) % (NPAD - NC), cp = k / (KG * (NPAD - NC));
          R1[cp * TBC + tc::cidx(c, a1, KG)] = 0.f;
        }
      if (STIFF && phase == 0) __syncthreads();
    }
    tc::fence_smem_to_async();
    __syncthreads();

    // q1 contraction on the tensor cores
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(R1);
      constexpr int NPASS = X3 ? 3 : 1;
      bool acc = false;
#pragma unroll
      for (int pass = 0; pass < NPASS; ++pass) {
        const int ac = (X3 && pass == 0) ? 1 : 0;  // tail of A with head of TB
        const int bc = (X3 && pass == 1) ? 1 : 0;  // head of A with tail of TB
#pragma unroll
        for (int term = 0; term < NT; ++term) {
#pragma unroll
          for (int s = 0; s < KG / 8; ++s) {
            const uint64_t ad = tc::sdesc(a0 + (uint32_t)(ac * 128 * KA * 4) + (uint32_t)((term * KG / 4 + 2 * s) * 128),
                                          128, KA * 32);
            const uint64_t bd =
                tc::sdesc(b0 + (uint32_t)((term * NS + bc) * TBC * 4) + (uint32_t)(2 * s * 128), 128, KG * 32);
            tc::mma_tf32(tmem, ad, bd, idesc, acc);
            acc = true;
          }
        }
      }
      tc::commit(&mbar);
    }
    // one thread polls the mbarrier; the others sleep in the barrier
    if (tid == 0 && !tc::mbar_wait(&mbar, parity, kWaitLimit)) {
      s_abort = 1;
      dev_set_status(M.status, DEV_TIMEOUT);
    }
    __syncthreads();
    tc::fence_after_sync();
    if (s_abort) break;
    parity ^= 1u;

    // D -> staging [r][c NB + dj1]: warp w reads lanes 32 (w % 4) .. + 31, column chunks of
    // parity w / 4
    {
      const int quarter = warp & 3, half = warp >> 2;
      const int m = quarter * 32 + lane;
      const int r = m / NB, dj1 = m - (m / NB) * NB;
      const bool live = r < G && rowflag[r];
      // row r's staging starts at r RS + shift, shift = its CSR offset mod 4, so that the
      // copy below moves aligned float4s
      float* sr = stage + r * RS + (live ? (int)(M.topo.rowptr[rowbase + i1a + r] & 3) : 0);
#pragma unroll 1
      for (int ch = half; ch < NPAD / 16; ch += 2) {
        float v[16];
        tc::ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ch * 16), v);
        if (live) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = ch * 16 + j;
            if (c < NC) sr[c * NB + dj1] = v[j];
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    // staging -> CSR values, a warp per row; at the faces of the mesh the band is clipped
    // to the columns j_d in [0, n_d) in each direction
    {
      const int lo2 = max(0, P - i2), w2 = min(D2.n - 1, i2 + P) - (i2 - P + lo2) + 1;
      const int lo3 = max(0, P - i3), w3 = min(D3.n - 1, i3 + P) - (i3 - P + lo3) + 1;
      for (int r = warp; r < G; r += 8) {
        if (!rowflag[r]) continue;
        const int i1 = i1a + r;
        const int lo1 = max(0, P - i1);
        const int w1 = min(D1.n - 1, i1 + P) - (i1 - P + lo1) + 1;
        const int64_t off = M.topo.rowptr[rowbase + i1];
        float* dst = values + off;
        const int sh = (int)(off & 3);
        const float* sr = stage + r * RS + sh;
        if (w1 == NB && w2 == NB && w3 == NB) {
          // head up to a 16-byte boundary, float4 body, tail
          const int head = (4 - sh) & 3;
          if (lane < head) dst[lane] = sr[lane];
          const int nv = (NB3 - head) >> 2;
          const float4* s4 = reinterpret_cast<const float4*>(sr + head);
          float4* d4 = reinterpret_cast<float4*>(dst + head);
          for (int k = lane; k < nv; k += 32) d4[k] = s4[k];
          const int t0 = head + 4 * nv;
          if (t0 + lane < NB3) dst[t0 + lane] = sr[t0 + lane];
        } else {
          // walk the full (dj3, dj2, dj1) box with compile-time strides, keep the in-range part
          const int w12 = w1 * w2;
          for (int k = lane; k < NB3; k += 32) {
            const int d3 = k / (NB * NB), d2 = (k / NB) % NB, d1 = k % NB;
            const int c3 = d3 - lo3, c2 = d2 - lo2, c1 = d1 - lo1;
            if ((unsigned)c3 < (unsigned)w3 && (unsigned)c2 < (unsigned)w2 && (unsigned)c1 < (unsigned)w1)
              dst[c3 * w12 + c2 * w1 + c1] = sr[k];
          }
        }
      }
    }
  }

  __syncthreads();
  if (s_abort) {
    // an MMA chain did not complete in time: give it one more bounded wait before the
    // tensor memory it writes is released
    if (tid == 0) tc::mbar_wait(&mbar, parity, kWaitLimit);
    __syncthreads();
    tc::fence_after_sync();
  }
  if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

// ---------------------------------------------------------------------------------------
// All three contractions on the tensor cores.  Per task (G rows i1 of one pencil):
//   stage A (q3): D_A[(a2, a1)][(kind, dj3)] = sum_a3 C[(a2, a1)][a3] W3_kind[dj3][a3]
//   stage B (q2): D_B[(a1, dj3)][(term, dj2)] = sum_a2 U_kind[(a1, dj3)][a2] W2[dj2][a2]
//                 (stiffness: term 0 = W2_00 U_0; term 1 = W2_11 U_0 + W2_00 U_1)
//   stage C (q1): as k_interior_tc.
// Each accumulator is read back from tensor memory into the next stage's operand layout
// (rounded to TF32, or split into head and tail).  K of stages A and B is the support's
// point count padded to KQ; unused rows and columns carry zeros or are never read.
template <int P>
struct Tc3Shape {
  using S = TcShape<P>;
  static constexpr int KQ = rup(S::NQM, 8);                    // K of stages A, B
  static constexpr int TA = (KQ * S::KG + 127) / 128;          // row tiles of stage A: (a2, a1)
  static constexpr int TBt = (S::NB * S::KG + 127) / 128;      // row tiles of stage B: (a1, dj3)
};

template <int P, bool STIFF, bool X3>
struct Tc3Smem {
  using S = TcShape<P>;
  using H = Tc3Shape<P>;
  static constexpr int NT = STIFF ? 2 : 1, NS = X3 ? 2 : 1;
  static constexpr int KA = NT * S::KG;
  static constexpr int NA = rup(NT * S::NB, 16);  // stage-A N
  static constexpr int NBn = STIFF ? 32 : 16;                                               // stage-B N
  static constexpr int AA = NS * H::TA * 128 * H::KQ;            // stage-A A operand (coefficient slab)
  static constexpr int UU = NT * NS * H::TBt * 128 * H::KQ;       // stage-B A operand
  static constexpr int TBC = S::NPAD * S::KG;                    // stage-C B operand copy
  static constexpr int TBB = NT * NS * TBC;
  static constexpr int RS = rup(S::NB3, 4) + 4;
  static constexpr int STG = S::G * RS;
  static constexpr int R_ = rup(AA > UU ? (AA > TBB ? (AA > STG ? AA : STG) : (TBB > STG ? TBB : STG))
                                        : (UU > TBB ? (UU > STG ? UU : STG) : (TBB > STG ? TBB : STG)), 32);
  static constexpr int BA = NS * NA * H::KQ;                      // W3 operand
  static constexpr int BB = (STIFF ? 2 : 1) * NS * NBn * H::KQ;   // W2 operand(s)
  static constexpr int A_ = NS * 128 * KA;                        // band of stage C
  static constexpr size_t bytes = (size_t)(R_ + rup(BA, 32) + rup(BB, 32) + A_) * 4 + S::G * sizeof(int);
  static constexpr int DCOLS = (H::TA * NA > H::TBt * NBn ? (H::TA * NA > S::NPAD ? H::TA * NA : S::NPAD)
                                                            : (H::TBt * NBn > S::NPAD ? H::TBt * NBn : S::NPAD));
};

// one MMA chain over K steps of 8: D (+)= A B^T, A rows in 128-row tiles of K columns
__device__ __forceinline__ void mma_chain(uint32_t d, uint32_t a, uint32_t b, int K, int ksteps, uint32_t idesc,
                                          bool& acc) {
  for (int s = 0; s < ksteps; ++s) {
    tc::mma_tf32(d, tc::sdesc(a + (uint32_t)(s * 256), 128, (uint32_t)K * 32),
                 tc::sdesc(b + (uint32_t)(s * 256), 128, (uint32_t)K * 32), idesc, acc);
    acc = true;
  }
}

// Row of stage A's operand and accumulator for the point pair (a2, a1): blocks of 8 points
// a1, a2 within a block, a1 innermost.
template <int KQ>
__device__ __forceinline__ int arow_t(int a2, int a1) {
  return ((a1 >> 3) * KQ + a2) * 8 + (a1 & 7);
}

template <int P, bool STIFF, bool X3>
__global__ void __launch_bounds__(256, (X3 || P >= 5) ? 1 : 2)
    k_interior_tc3(MeshView M, const float* __restrict__ Cwq, float* __restrict__ values,
                   const float* __restrict__ band, int Kg_mesh, int n_pencils, int ntasks, uint32_t tmem_cols,
                   int kRun) {
  using S = TcShape<P>;
  using H = Tc3Shape<P>;
  using L = Tc3Smem<P, STIFF, X3>;
  constexpr int NB = S::NB, NC = S::NC, NPAD = S::NPAD, G = S::G, KG = S::KG, NB3 = S::NB3;
  constexpr int KQ = H::KQ, TA = H::TA, TBt = H::TBt;
  constexpr int NT = L::NT, NS = L::NS, KA = L::KA, NA = L::NA, NBn = L::NBn, RS = L::RS, TBC = L::TBC;
  constexpr int NPASS = X3 ? 3 : 1;
  const auto arow = [](int a2, int a1) { return arow_t<KQ>(a2, a1); };
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* Rg = reinterpret_cast<float*>(smem_raw);  // A slab | U | TB | staging (in turn)
  float* Bw3 = Rg + L::R_;                          // [copy][cidx(n, a3, KQ)]
  float* Bw2 = Bw3 + rup(L::BA, 32);                // [chain][copy][cidx(n, a2, KQ)]
  float* As = Bw2 + rup(L::BB, 32);                 // [copy][cidx(m, k, KA)]
  int* rowflag = reinterpret_cast<int*>(As + L::A_);
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // every operand region starts finite (rows and columns no stage writes are multiplied by
  // zeros or land in rows that are never read)
  for (size_t k = tid; k < L::bytes / 4; k += blockDim.x) Rg[k] = 0.f;
  if (warp == 0) tc::tmem_alloc(&tslot, tmem_cols);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    s_abort = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  if (Kg_mesh > KG) {
    if (tid == 0) dev_set_status(M.status, DEV_BOUNDS);
    ntasks = 0;
  }
  const Dir1D &D1 = M.dir[0], &D2 = M.dir[1], &D3 = M.dir[2];
  const int NQL2 = D2.nql, NQL3 = D3.nql;
  const int64_t nq1g = D1.nq, nq2g = D2.nq;
  int cur_g = -1;
  uint32_t parity = 0;
  const uint32_t sR = tc::smem_addr(Rg), sB3 = tc::smem_addr(Bw3), sB2 = tc::smem_addr(Bw2), sA = tc::smem_addr(As);

  // commit the MMAs issued by thread 0 and wait for them (all threads); false on timeout
  auto complete = [&]() -> bool {
    if (tid == 0) tc::commit(&mbar);
    if (tid == 0 && !tc::mbar_wait(&mbar, parity, kWaitLimit)) {
      s_abort = 1;
      dev_set_status(M.status, DEV_TIMEOUT);
    }
    parity ^= 1u;
    __syncthreads();
    tc::fence_after_sync();
    return !s_abort;
  };
  auto split = [&](float v, float* hi_dst, int o, int copy_stride) {
    const float hi = tc::tf32_round(v);
    hi_dst[o] = hi;
    if (X3) hi_dst[copy_stride + o] = tc::tf32_round(v - hi);
  };

  for (int t = blockIdx.x * kRun; t < ntasks; t += (t % kRun == kRun - 1) ? (gridDim.x - 1) * kRun + 1 : 1) {
    const int g = t / n_pencils;
    const int pencil = M.topo.int_tiles[t % n_pencils];
    const int i2 = pencil % D2.n, i3 = pencil / D2.n;
    const int i1a = g * G, i1b = min(D1.n, i1a + G);
    const int64_t rowbase = (int64_t)D1.n * (i2 + (int64_t)D2.n * i3);
    __syncthreads();
    for (int r = tid; r < G; r += blockDim.x) rowflag[r] = (i1a + r < i1b) && M.topo.fn_class[rowbase + i1a + r] == F_INT;
    __syncthreads();
    int any = 0;
#pragma unroll
    for (int r = 0; r < G; ++r) any |= rowflag[r];
    if (!any) continue;
    const int q2lo = D2.qlo[i2], nq2 = D2.nqi[i2];
    const int q3lo = D3.qlo[i3], nq3 = D3.nqi[i3];
    if (nq2 > KQ || nq3 > KQ) {  // excluded on the host; never taken
      if (tid == 0) dev_set_status(M.status, DEV_BOUNDS);
      continue;
    }
    if (g != cur_g) {
      const float4* src = reinterpret_cast<const float4*>(band + (size_t)g * 2 * 128 * KA);
      float4* dst = reinterpret_cast<float4*>(As);
      for (int k = tid; k < NS * 128 * KA / 4; k += blockDim.x) dst[k] = src[k];
      cur_g = g;
    }
    // stage-A operands: the coefficient slab A[arow(a2, a1)][a3] (a3 < KQ, zero past nq3 and
    // past the last q1 point) and W3[(kind NB + dj3)][a3].  A warp item is 8 points a1 x 4
    // points a3 of one a2, which fills the 32 banks.
    {
      const int kst = D1.qlo[i1a] & ~3;
      const int a1l = lane & 7, a3l = lane >> 3;
      for (int item = warp; item < nq2 * (KQ / 4) * (KG / 8); item += 8) {
        const int a1 = (item % (KG / 8)) * 8 + a1l;
        const int rest = item / (KG / 8);
        const int a3 = (rest % (KQ / 4)) * 4 + a3l, a2 = rest / (KQ / 4);
        float v = 0.f;
        if (a3 < nq3 && kst + a1 < nq1g) v = Cwq[nq1g * ((q2lo + a2) + nq2g * (int64_t)(q3lo + a3)) + kst + a1];
        split(v, Rg, tc::cidx(arow(a2, a1), a3, KQ), TA * 128 * KQ);
      }
      for (int k = tid; k < NA * KQ; k += blockDim.x) {
        const int a3 = k % KQ, n = k / KQ, kind = n / NB, dj = n - kind * NB;
        float v = 0.f;
        if (kind < NT && a3 < nq3) v = (kind ? D3.WB11f : D3.WB00f)[((size_t)i3 * NB + dj) * NQL3 + a3];
        split(v, Bw3, tc::cidx(n, a3, KQ), NA * KQ);
      }
      // stage-B operands: chain 0 B = [W2_00 (rows 0..NB) | W2_11 (rows 16..16+NB)],
      // chain 1 B = [0 | W2_00] (stiffness); mass B = W2_00
      for (int k = tid; k < (STIFF ? 2 : 1) * NBn * KQ; k += blockDim.x) {
        const int a2 = k % KQ, n = (k / KQ) % NBn, chain = k / (KQ * NBn);
        float v = 0.f;
        if (a2 < nq2) {
          const int term = n / 16, dj = n % 16;
          if (dj < NB) {
            const float* W = nullptr;
            if (chain == 0) W = term == 0 ? D2.WB00f : (STIFF ? D2.WB11f : nullptr);
            else W = term == 1 ? D2.WB00f : nullptr;
            if (W) v = W[((size_t)i2 * NB + dj) * NQL2 + a2];
          }
        }
        split(v, Bw2 + chain * NS * NBn * KQ, tc::cidx(n, a2, KQ), NBn * KQ);
      }
    }
    tc::fence_smem_to_async();
    __syncthreads();
    // stage A MMAs: row tile ta (rows arow(a2, a1)) into columns ta NA
    if (tid == 0) {
      tc::fence_after_sync();
      constexpr uint32_t id = tc::idesc_tf32(128, NA);
      for (int ta = 0; ta < TA; ++ta) {
        bool acc = false;
        for (int pass = 0; pass < NPASS; ++pass) {
          const int ac = (X3 && pass == 0) ? 1 : 0, bc = (X3 && pass == 1) ? 1 : 0;
          mma_chain(tmem + (uint32_t)(ta * NA), sR + (uint32_t)((ac * TA * 128 * KQ + ta * 128 * KQ) * 4),
                    sB3 + (uint32_t)(bc * NA * KQ * 4), KQ, KQ / 8, id, acc);
        }
      }
    }
    if (!complete()) break;
    // D_A -> U_kind[copy][cidx(a1 NB + dj3, a2, KQ)]; rows with a2 >= nq2 give zeros.  A
    // warp's lanes hold 8 points a1 x 4 points a2: its stores fill the 32 banks.
    {
      const int quarter = warp & 3;
      for (int ta = warp >> 2; ta < TA; ta += 2) {
        const int m = ta * 128 + quarter * 32 + lane;
        const int a2 = (m >> 3) % KQ, a1 = ((m >> 3) / KQ) * 8 + (m & 7);
        const bool live = a1 < KG;
        const bool keep = a2 < nq2;
#pragma unroll
        for (int c0 = 0; c0 < NA; c0 += 16) {
          float v[16];
          tc::ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ta * NA + c0), v);
          if (live) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = c0 + j;
              if (n < NT * NB) {
                const int kind = n / NB, dj3 = n - kind * NB;
                split(keep ? v[j] : 0.f, Rg + kind * NS * TBt * 128 * KQ, tc::cidx(a1 * NB + dj3, a2, KQ),
                      TBt * 128 * KQ);
              }
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    tc::fence_smem_to_async();
    __syncthreads();
    // stage B MMAs: tile tb of rows (a1 NB + dj3) into columns tb NBn
    if (tid == 0) {
      tc::fence_after_sync();
      constexpr uint32_t id = tc::idesc_tf32(128, NBn);
      for (int tb = 0; tb < TBt; ++tb) {
        bool acc = false;
        for (int chain = 0; chain < (STIFF ? 2 : 1); ++chain)
          for (int pass = 0; pass < NPASS; ++pass) {
            const int ac = (X3 && pass == 0) ? 1 : 0, bc = (X3 && pass == 1) ? 1 : 0;
            mma_chain(tmem + (uint32_t)(tb * NBn),
                      sR + (uint32_t)(((chain * NS + ac) * TBt * 128 * KQ + tb * 128 * KQ) * 4),
                      sB2 + (uint32_t)(((chain * NS + bc) * NBn * KQ) * 4), KQ, KQ / 8, id, acc);
          }
      }
    }
    if (!complete()) break;
    // D_B -> TB[term][copy][cidx(dj3 NB + dj2, a1, KG)], padding rows c >= NC zero
    {
      const int quarter = warp & 3;
      float* TB = Rg;
      for (int tb = warp >> 2; tb < TBt; tb += 2) {
        const int r = tb * 128 + quarter * 32 + lane;
        const int a1 = r / NB, dj3 = r - (r / NB) * NB;
        const bool live = a1 < KG;
#pragma unroll
        for (int c0 = 0; c0 < NBn; c0 += 16) {
          float v[16];
          tc::ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tb * NBn + c0), v);
          if (live) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int dj2 = j;  // column c0 + j: term c0 / 16, dj2 = j
              if (dj2 < NB) split(v[j], TB + (c0 / 16) * NS * TBC, tc::cidx(dj3 * NB + dj2, a1, KG), TBC);
            }
          }
        }
      }
      // (D_B is read completely before TB overwrites U: all reads above come from tensor
      // memory, all writes go to the region U occupied, whose MMAs have completed)
      for (int k = tid; k < NT * NS * (NPAD - NC) * KG; k += blockDim.x) {
        const int a1 = k % KG, c = NC + (k / KG) % (NPAD - NC), cp = k / (KG * (NPAD - NC));
        TB[cp * TBC + tc::cidx(c, a1, KG)] = 0.f;
      }
    }
    tc::fence_before_sync();
    tc::fence_smem_to_async();
    __syncthreads();
    // stage C (as k_interior_tc)
    if (tid == 0) {
      tc::fence_after_sync();
      constexpr uint32_t id = tc::idesc_tf32(128, NPAD);
      bool acc = false;
      for (int pass = 0; pass < NPASS; ++pass) {
        const int ac = (X3 && pass == 0) ? 1 : 0, bc = (X3 && pass == 1) ? 1 : 0;
        for (int term = 0; term < NT; ++term)
          for (int s = 0; s < KG / 8; ++s) {
            const uint64_t ad =
                tc::sdesc(sA + (uint32_t)(ac * 128 * KA * 4) + (uint32_t)((term * KG / 4 + 2 * s) * 128), 128, KA * 32);
            const uint64_t bd = tc::sdesc(sR + (uint32_t)((term * NS + bc) * TBC * 4) + (uint32_t)(2 * s * 128), 128, KG * 32);
            tc::mma_tf32(tmem, ad, bd, id, acc);
            acc = true;
          }
      }
    }
    if (!complete()) break;
    // D_C -> staging (row r at r RS + CSR offset mod 4) -> CSR values
    float* stage = Rg;
    {
      const int quarter = warp & 3, half = warp >> 2;
      const int m = quarter * 32 + lane;
      const int r = m / NB, dj1 = m - (m / NB) * NB;
      const bool live = r < G && rowflag[r];
      float* sr = stage + r * RS + (live ? (int)(M.topo.rowptr[rowbase + i1a + r] & 3) : 0);
#pragma unroll 1
      for (int ch = half; ch < NPAD / 16; ch += 2) {
        float v[16];
        tc::ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ch * 16), v);
        if (live) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = ch * 16 + j;
            if (c < NC) sr[c * NB + dj1] = v[j];
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    {
      const int lo2 = max(0, P - i2), w2 = min(D2.n - 1, i2 + P) - (i2 - P + lo2) + 1;
      const int lo3 = max(0, P - i3), w3 = min(D3.n - 1, i3 + P) - (i3 - P + lo3) + 1;
      for (int r = warp; r < G; r += 8) {
        if (!rowflag[r]) continue;
        const int i1 = i1a + r;
        const int lo1 = max(0, P - i1);
        const int w1 = min(D1.n - 1, i1 + P) - (i1 - P + lo1) + 1;
        const int64_t off = M.topo.rowptr[rowbase + i1];
        float* dst = values + off;
        const int sh = (int)(off & 3);
        const float* sr = stage + r * RS + sh;
        if (w1 == NB && w2 == NB && w3 == NB) {
          const int head = (4 - sh) & 3;
          if (lane < head) dst[lane] = sr[lane];
          const int nv = (NB3 - head) >> 2;
          const float4* s4 = reinterpret_cast<const float4*>(sr + head);
          float4* d4 = reinterpret_cast<float4*>(dst + head);
          for (int k = lane; k < nv; k += 32) d4[k] = s4[k];
          const int t0 = head + 4 * nv;
          if (t0 + lane < NB3) dst[t0 + lane] = sr[t0 + lane];
        } else {
          const int w12 = w1 * w2;
          for (int k = lane; k < NB3; k += 32) {
            const int d3 = k / (NB * NB), d2 = (k / NB) % NB, d1 = k % NB;
            const int c3 = d3 - lo3, c2 = d2 - lo2, c1 = d1 - lo1;
            if ((unsigned)c3 < (unsigned)w3 && (unsigned)c2 < (unsigned)w2 && (unsigned)c1 < (unsigned)w1)
              dst[c3 * w12 + c2 * w1 + c1] = sr[k];
          }
        }
      }
    }
  }
  __syncthreads();
  if (s_abort) {
    if (tid == 0) tc::mbar_wait(&mbar, parity ^ 1u, kWaitLimit);
    __syncthreads();
    tc::fence_after_sync();
  }
  if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

template <int P, bool STIFF, bool X3>
cudaError_t launch_tc3_t(const MeshView& M, const float* Cwq, float* values, const float* band, int Kg, int ngroups,
                         int n_pencils, int kRun, cudaStream_t st) {
  using L = Tc3Smem<P, STIFF, X3>;
  const size_t smem = L::bytes;
  auto kern = k_interior_tc3<P, STIFF, X3>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  int dev = 0, nsm = 0, smem_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  uint32_t cols = 32;
  while (cols < (uint32_t)L::DCOLS) cols <<= 1;
  int occ = (int)(smem_sm / (smem + fa.sharedSizeBytes + 1024));
  occ = std::min(occ, 65536 / (256 * std::max(1, (fa.numRegs + 7) / 8 * 8)));
  occ = std::min(occ, (int)(512 / cols));
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int64_t ntasks = (int64_t)ngroups * n_pencils;
  if (ntasks == 0) return cudaSuccess;
  if (kRun < 1) kRun = 1;
  const int grid = (int)std::min<int64_t>((ntasks + kRun - 1) / kRun, (int64_t)nsm * occ);
  kern<<<grid, 256, smem, st>>>(M, Cwq, values, band, Kg, n_pencils, (int)ntasks, cols, kRun);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

template <int P, bool STIFF, bool X3>
cudaError_t launch_tc_t(const MeshView& M, const float* Cwq, float* values, const float* band, int Kg, int ngroups,
                        int n_pencils, int kRun, cudaStream_t st) {
  using L = TcSmem<P, STIFF, X3>;
  const size_t smem = L::bytes;
  auto kern = k_interior_tc<P, STIFF, X3>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  // Resident CTAs per SM from its resources: shared memory (dynamic + static + the 1 KB the
  // runtime reserves per CTA), registers, tensor-memory columns.  The grid is persistent, so
  // an estimate one too high only queues the surplus CTAs behind the first wave.
  int dev = 0, nsm = 0, smem_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  uint32_t cols = 32;
  while (cols < (uint32_t)TcShape<P>::NPAD) cols <<= 1;
  int occ = (int)(smem_sm / (smem + fa.sharedSizeBytes + 1024));
  occ = std::min(occ, 65536 / (256 * std::max(1, (fa.numRegs + 7) / 8 * 8)));
  occ = std::min(occ, (int)(512 / cols));
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int64_t ntasks = (int64_t)ngroups * n_pencils;
  if (ntasks == 0) return cudaSuccess;
  if (kRun < 1) kRun = 1;
  const int grid = (int)std::min<int64_t>((ntasks + kRun - 1) / kRun, (int64_t)nsm * occ);
  kern<<<grid, 256, smem, st>>>(M, Cwq, values, band, Kg, n_pencils, (int)ntasks, cols, kRun);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

// Rows per MMA group and the compiled q1 window for degree p (0 if p is out of range).
void interior_tc_shape(int p, int* G, int* KG) {
  *G = *KG = 0;
  switch (p) {
#define SFA_SHAPE(PP)              \
  case PP:                         \
    *G = TcShape<PP>::G;           \
    *KG = TcShape<PP>::KG;         \
    break;
    SFA_SHAPE(2)
    SFA_SHAPE(3)
    SFA_SHAPE(4)
    SFA_SHAPE(5)
    SFA_SHAPE(6)
#undef SFA_SHAPE
  }
}

cudaError_t launch_tc_band(const MeshView& M, int G, int Kg, int ngroups, float* band_mass, float* band_stiff,
                           cudaStream_t st) {
  if (ngroups <= 0) return cudaSuccess;
  dim3 grid(8, ngroups);
  k_tc_band<<<grid, 256, 0, st>>>(M.dir[0], M.p, G, Kg, Kg, 0, band_mass);
  SFA_LAUNCHED(1);
  k_tc_band<<<grid, 256, 0, st>>>(M.dir[0], M.p, G, Kg, 2 * Kg, 1, band_stiff);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

// The three-stage kernel wherever its shared memory fits one CTA (all but 3xTF32 stiffness at
// p = 6), else the kernel with the q3/q2 stages on the CUDA cores.
template <int P, bool STIFF, bool X3>
cudaError_t launch_tc_any(const MeshView& M, const float* Cwq, float* values, const float* band, int Kg, int ngroups,
                          int n_pencils, int kRun, cudaStream_t st) {
  if constexpr (Tc3Smem<P, STIFF, X3>::bytes <= 227 * 1024)
    return launch_tc3_t<P, STIFF, X3>(M, Cwq, values, band, Kg, ngroups, n_pencils, kRun, st);
  else
    return launch_tc_t<P, STIFF, X3>(M, Cwq, values, band, Kg, ngroups, n_pencils, kRun, st);
}

// Kg is the mesh's widest group window (checked against the compiled one in the kernel);
// the band matrices are laid out with the compiled window.
cudaError_t launch_interior_tc(const MeshView& M, bool stiff, bool x3, const float* Cwq, float* values,
                               const float* band, int Kg, int ngroups, int n_pencils, int run, cudaStream_t st) {
#define SFA_TC_ONE(PP, ST, X) launch_tc_any<PP, ST, X>(M, Cwq, values, band, Kg, ngroups, n_pencils, run, st)
#define SFA_TC_CASE(PP)                                                                              \
  case PP:                                                                                           \
    if (stiff) return x3 ? SFA_TC_ONE(PP, true, true) : SFA_TC_ONE(PP, true, false);                 \
    return x3 ? SFA_TC_ONE(PP, false, true) : SFA_TC_ONE(PP, false, false);
  switch (M.p) {
    SFA_TC_CASE(2)
    SFA_TC_CASE(3)
    SFA_TC_CASE(4)
    SFA_TC_CASE(5)
    SFA_TC_CASE(6)
  }
#undef SFA_TC_CASE
#undef SFA_TC_ONE
  return cudaErrorInvalidValue;
}
