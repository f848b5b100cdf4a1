// Interior rows on the tensor cores (precisions SFA_TF32 and SFA_TF32X3).  Same formula as
// the SIMT interior kernels (Sec. 1, row assembly by sum factorization):
//   V_i[j3][j2][j1] = sum_q1 WB1_i1[j1][q1] TB[(j3, j2)][q1],
//   TB[(j3, j2)][q1] = sum_q2 WB2_i2[j2][q2] sum_q3 WB3_i3[j3][q3] C[q1, q2, q3]
// (stiffness: TB splits into the x-term paired with the derivative rule WB1_11 and the
// y/z-terms paired with WB1_00).  A task is G consecutive rows i1 of one (i2, i3) pencil;
// the three contractions are tcgen05 MMA chains (kind::tf32, FP32 accumulation in tensor
// memory):
//   q3: the coefficient slab against the pencil's WB3 rows,
//   q2: its result against the WB2 rows,
//   q1: D[(r, dj1)][c] = sum_k A_g[(r, dj1)][k] TB[c][k] with M = 128 rows (r, dj1)
//       (G (2p+1) <= 128 used), N the pairs c = (dj2, dj3) and K the group's q1 window; A_g
//       is the banded matrix of the group's WB1 rows, built once per mesh.
// Faces of the mesh need no special case in the contractions: a support touching the first
// or last element has up to 3p+1 points, all within the padded K of the q3 and q2 stages,
// and the tables are zero past each support's points.  SFA_TF32 rounds both operands to
// TF32; SFA_TF32X3 splits each into a TF32 head and a TF32 tail and accumulates
// tail*head + head*tail + head*head, which restores close to FP32 accuracy.  The kernel is
// persistent: CTA b takes runs of tasks b, b + grid, ... in (group, pencil) order.
#include "sfa_internal.cuh"
#include "tc_sm103.cuh"

#include <cuda_bf16.h>

namespace {

constexpr long long kWaitLimit = 2000000000ll;  // clock cycles, about one second

constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }

// Compile-time shape of one degree.  BF: BF16 operands (kind::f16, 16 columns of K per MMA)
// instead of TF32 (kind::tf32, 8 columns).
template <int P, bool BF = false>
struct TcShape {
  static constexpr int NB = 2 * P + 1, NQ = 2 * P + 2, NB3 = NB * NB * NB;
  static constexpr int KR = BF ? 16 : 8;                    // K of one MMA
  static constexpr int EPC = BF ? 8 : 4;                    // elements per 16-byte core-matrix row
  static constexpr int G = P == 6 ? 8 : 128 / NB;           // rows i1 per MMA group
  static constexpr int KG = rup(2 * (G - 1) + NQ + 3, KR);  // q1 window per term, >= any group's
  static constexpr int NQM = 3 * P + 1;                     // points of a face support (n_el >= p+2)
};

template <bool BF>
struct OpT;
template <>
struct OpT<false> {
  using T = float;
  __device__ static T cvt(float x) { return tc::tf32_round(x); }
  __device__ static int cidx(int r, int k, int K) { return tc::cidx(r, k, K); }
};
template <>
struct OpT<true> {
  using T = __nv_bfloat16;
  __device__ static T cvt(float x) { return __float2bfloat16_rn(x); }
  __device__ static int cidx(int r, int k, int K) { return tc::cidx16(r, k, K); }
};

// A_g for every group: band[g][copy][cidx(m, k, KA)], copy 0 the TF32 head, 1 the tail
// (BF16: one copy, rounded to BF16).  Column k of term t = k / Kg holds q1 = kst_g + k % Kg;
// row m = r * NB + dj1.
template <bool BF>
__global__ void k_tc_band(Dir1D D1, int p, int G, int Kg, int KA, int stiff, typename OpT<BF>::T* __restrict__ band) {
  const int g = blockIdx.y, NB = 2 * p + 1;
  const int kst = D1.qlo[g * G] & ~3;
  typename OpT<BF>::T* base = band + (size_t)g * (BF ? 1 : 2) * 128 * KA;
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
    if constexpr (BF) {
      base[OpT<true>::cidx(m, k, KA)] = __double2bfloat16(v);
    } else {
      const float hi = tc::tf32_round((float)v);
      const float lo = tc::tf32_round((float)(v - (double)hi));
      base[tc::cidx(m, k, KA)] = hi;
      base[128 * KA + tc::cidx(m, k, KA)] = lo;
    }
  }
}

// Operand tables of the q3 and q2 stages for every function index i of a direction:
// dirop[i][copy][cidx(kind 16 + dj, a, KQ)] = WB_kind_i[dj][a] (kind 0: WB_00, 1: WB_11), zero
// for dj >= 2p+1 and past the support's nqi points; copy 0 the TF32 head, 1 the tail (BF16:
// one copy).
template <bool BF>
__global__ void k_tc_dirop(Dir1D D, int p, int KQ, typename OpT<BF>::T* __restrict__ out) {
  const int i = blockIdx.x, NB = 2 * p + 1;
  typename OpT<BF>::T* base = out + (size_t)i * (BF ? 1 : 2) * 32 * KQ;
  for (int t = threadIdx.x; t < 32 * KQ; t += blockDim.x) {
    const int n = t / KQ, a = t % KQ, kind = n / 16, dj = n % 16;
    double v = 0.0;
    if (dj < NB && a < D.nqi[i]) v = (kind ? D.WB11 : D.WB00)[((size_t)i * NB + dj) * D.nql + a];
    if constexpr (BF) {
      base[OpT<true>::cidx(n, a, KQ)] = __double2bfloat16(v);
    } else {
      const float hi = tc::tf32_round((float)v);
      const float lo = tc::tf32_round((float)(v - (double)hi));
      base[tc::cidx(n, a, KQ)] = hi;
      base[32 * KQ + tc::cidx(n, a, KQ)] = lo;
    }
  }
}

// ---------------------------------------------------------------------------------------
// All three contractions on the tensor cores.  Per task (G rows i1 of one pencil):
//   stage A (q3): D_A[(slot, a1)][(kind, dj3)] = sum_a3 C[q1, q2, q3] WB3_kind[dj3][a3]
//   stage B (q2): D_B[(a1, dj3)][(term, dj2)] = sum_a2 U_kind[(a1, dj3)][a2] WB2[dj2][a2]
//                 (stiffness: term 0 = WB2_00 U_0; term 1 = WB2_11 U_0 + WB2_00 U_1)
//   stage C (q1): D_C[(r, dj1)][(dj2, dj3)] = sum_(term, a1) A_g[(r, dj1)][(term, a1)] TB_term[(dj2, dj3)][a1]
// with q1 = kst + a1, q2 = q2lo + a2 and q3 = q3lo + a3.  A point q2 of the coefficient slab
// lives in slot q2 mod KQ, so that the slab of the next pencil along i2 (same i3 and row
// group) keeps the points the two share and loads only the new ones.  Each accumulator is
// read back from tensor memory into the next stage's operand layout (rounded to TF32, or
// split into head and tail).  The band A_g sits in tensor memory where the columns allow
// it.  Output rows are staged in shared memory and written by bulk asynchronous copies that
// drain while the next task computes.
template <int P, bool BF = false>
struct Tc3Shape {
  using S = TcShape<P, BF>;
  static constexpr int KQ = rup(S::NQM, S::KR);           // K of stages A, B (slots of the slab)
  static constexpr int TA = (KQ * S::KG + 127) / 128;     // row tiles of stage A
  static constexpr int NBE = S::NB + 1;                   // dj3 slots per block of stage B (even)
  static constexpr int TB = (S::KG * NBE + 127) / 128;    // row tiles of stage B
  static constexpr int NB8 = rup(S::NB, 8);               // dj3 slots per dj2 in the stage-C columns
  static constexpr int NPADC = rup(S::NB * NB8, 16);      // stage-C N
};

constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int pow2cols(int x) { return x <= 32 ? 32 : x <= 64 ? 64 : x <= 128 ? 128 : x <= 256 ? 256 : 512; }

// Shared-memory plan in 4-byte words: [R | slab | W3 | W2 | band | row offsets, flags].  R
// holds in turn the stage-B operand, the stage-C operand and the output staging (and first
// the slab when the slab has no region of its own).  Operand regions are counted in operand
// elements (W converts to words).  Two choices per shape, taken for the most CTAs per SM:
// band in tensor memory (BT; TF32 only) and a slab region of its own (RSL).
template <int P, bool STIFF, bool X3, bool BF = false>
struct Tc3Smem {
  using S = TcShape<P, BF>;
  using H = Tc3Shape<P, BF>;
  static constexpr int ES = BF ? 2 : 4;                     // bytes per operand element
  static constexpr int W(int elems) { return (elems * ES + 3) / 4; }
  static constexpr int NT = STIFF ? 2 : 1, NS = X3 ? 2 : 1;
  static constexpr int KA = NT * S::KG;
  static constexpr int NA = 16 * NT;                         // stage-A N: columns (kind 16 + dj3)
  static constexpr int NBn = 16 * NT;                        // stage-B N: columns (term 16 + dj2)
  static constexpr int AA = NS * H::TA * 128 * H::KQ;        // stage-A operand (coefficient slab)
  static constexpr int UC = H::TB * 128 * H::KQ;             // stage-B operand, one kind and copy
  static constexpr int UU = NT * NS * UC;
  static constexpr int TBC = H::NPADC * S::KG;               // stage-C operand, one term and copy
  static constexpr int TBB = NT * NS * TBC;
  // staging row stride: a multiple of 4 (aligned row bodies) that is 8 mod 32, so that the
  // readback lanes of consecutive rows fall in different banks
  static constexpr int RS = rup(S::NB3, 32) + 8;
  static constexpr int STG = S::G * RS;
  static constexpr int BA = NS * 32 * H::KQ;                 // W3 operand (one direction-table entry)
  static constexpr int BB = NS * 32 * H::KQ;                 // W2 operand
  static constexpr int A_ = NS * 128 * KA;                   // band of stage C
  static constexpr int DCOLS = cmax(cmax(H::TA * NA, H::TB * NBn), H::NPADC);
  static constexpr int BCOL = rup(DCOLS, 16);                // first band column in tensor memory
  static constexpr int r_of(bool rs) {
    return rup(rs ? cmax(W(UU), cmax(W(TBB), STG)) : cmax(cmax(W(AA), W(UU)), cmax(W(TBB), STG)), 32);
  }
  static constexpr size_t bytes_of(bool bt, bool rs) {
    return (size_t)(r_of(rs) + (rs ? W(AA) : 0) + rup(W(BA), 32) + rup(W(BB), 32) + (bt ? 0 : W(A_))) * 4 +
           S::G * (sizeof(long long) + sizeof(int));
  }
  static constexpr int tmem_need(bool bt) { return bt ? BCOL + NS * KA : DCOLS; }
  static constexpr int cols_of(bool bt) { return pow2cols(tmem_need(bt)); }
  // CTAs per SM: shared memory (228 KB per SM, 1 KB reserved per CTA, the static barriers)
  // and tensor-memory columns (512 per SM); 0 if the shape does not fit at all (the band in
  // tensor memory is a TF32 layout only)
  static constexpr int occ_of(bool bt, bool rs) {
    return (bytes_of(bt, rs) > 227 * 1024 || tmem_need(bt) > 512 || (bt && BF))
               ? 0
               : cmin((int)((228 * 1024) / (bytes_of(bt, rs) + 1024 + 64)), 512 / cols_of(bt));
  }
  // the most CTAs per SM; among equals prefer the band in tensor memory, then the slab region
  static constexpr int OCC =
      cmax(cmax(occ_of(true, true), occ_of(true, false)), cmax(occ_of(false, true), occ_of(false, false)));
  static constexpr bool BT = occ_of(true, true) == OCC || occ_of(true, false) == OCC;
  static constexpr bool RSL = occ_of(BT, true) == OCC;
  static constexpr int R_ = r_of(RSL);
  static constexpr size_t bytes = bytes_of(BT, RSL);
  static constexpr int COLS = cols_of(BT);
};

// one MMA chain over K steps of 8 (TF32) or 16 (BF16) columns, 256 bytes each: D (+)= A B^T,
// A rows in 128-row tiles of K columns (8-row groups K * 16 bytes apart)
template <bool BF>
__device__ __forceinline__ void mma_chain(uint32_t d, uint32_t a, uint32_t b, int K, int ksteps, uint32_t idesc,
                                          bool& acc) {
  const uint32_t sbo = (uint32_t)K * 8 * (BF ? 2 : 4);
  for (int s = 0; s < ksteps; ++s) {
    const uint64_t ad = tc::sdesc(a + (uint32_t)(s * 256), 128, sbo), bd = tc::sdesc(b + (uint32_t)(s * 256), 128, sbo);
    if constexpr (BF) tc::mma_f16(d, ad, bd, idesc, acc);
    else tc::mma_tf32(d, ad, bd, idesc, acc);
    acc = true;
  }
}

// Row of stage A's operand and accumulator for slot s and point a1: blocks of 8 points a1,
// slots within a block, a1 innermost.
template <int KQ>
__device__ __forceinline__ int arow_t(int s, int a1) {
  return ((a1 >> 3) * KQ + s) * 8 + (a1 & 7);
}

template <int P, bool STIFF, bool X3, bool BF>
__global__ void __launch_bounds__(256, Tc3Smem<P, STIFF, X3, BF>::OCC >= 2 ? 2 : 1)
    k_interior_tc3(MeshView M, const float* __restrict__ Cwq, float* __restrict__ values,
                   const typename OpT<BF>::T* __restrict__ band, const typename OpT<BF>::T* __restrict__ dirop2,
                   const typename OpT<BF>::T* __restrict__ dirop3, int Kg_mesh, int n_pencils, FastDiv div_np,
                   int ntasks, uint32_t tmem_cols, int kRun, const int32_t* __restrict__ task_list) {
  using S = TcShape<P, BF>;
  using H = Tc3Shape<P, BF>;
  using L = Tc3Smem<P, STIFF, X3, BF>;
  using OT = typename OpT<BF>::T;
  constexpr int ES = L::ES, EPC = S::EPC, KR = S::KR;
  constexpr int DST = (BF ? 1 : 2) * 32 * H::KQ;  // elements per function index of the dirop tables
  constexpr int NB = S::NB, G = S::G, KG = S::KG, NB3 = S::NB3;
  constexpr int KQ = H::KQ, TA = H::TA, TBt = H::TB, NBE = H::NBE, NB8 = H::NB8, NPADC = H::NPADC;
  constexpr int NT = L::NT, NS = L::NS, KA = L::KA, NA = L::NA, NBn = L::NBn, RS = L::RS, TBC = L::TBC, UC = L::UC;
  constexpr bool BT = L::BT, RSL = L::RSL;
  constexpr int NPASS = X3 ? 3 : 1;
  const auto arow = [](int s, int a1) { return arow_t<KQ>(s, a1); };
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* Rg = reinterpret_cast<float*>(smem_raw);  // U | TB | staging (in turn; first the slab if !RSL)
  float* const stage = Rg;                          // output staging [r][RS]
  OT* const Ro = reinterpret_cast<OT*>(Rg);         // the stage-B and stage-C operands in R
  float* const slw = RSL ? Rg + L::R_ : Rg;
  OT* Sl = reinterpret_cast<OT*>(slw);              // [copy][cidx(arow(slot, a1), a3, KQ)]
  float* const w3w = Rg + L::R_ + (RSL ? L::W(L::AA) : 0);
  float* const w2w = w3w + rup(L::W(L::BA), 32);
  float* const asw = w2w + rup(L::W(L::BB), 32);
  OT* Bw3 = reinterpret_cast<OT*>(w3w);             // [copy][cidx(kind 16 + dj3, a3, KQ)]
  OT* Bw2 = reinterpret_cast<OT*>(w2w);             // [copy][cidx(kind 16 + dj2, a2, KQ)]
  OT* As = reinterpret_cast<OT*>(asw);              // [copy][cidx(m, k, KA)] (band in shared memory)
  long long* rowoff = reinterpret_cast<long long*>(asw + (BT ? 0 : L::W(L::A_)));  // CSR offset of each row
  int* rowflag = reinterpret_cast<int*>(rowoff + G);
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
  const int64_t nq1g = D1.nq, nq2g = D2.nq;
  int cur_g = -1, cur_i3 = -1;
  int sl_g = -1, sl_i3 = -1, sl_lo = 0, sl_hi = 0;  // resident slab: row group, i3, q2 window
  uint32_t parity = 0;
  const uint32_t sR = tc::smem_addr(Rg), sS = tc::smem_addr(Sl), sB3 = tc::smem_addr(Bw3), sB2 = tc::smem_addr(Bw2);
  const uint32_t sA = tc::smem_addr(As);

  // commit the MMAs issued by thread 0 and wait for them (all threads); false on timeout.
  // With drain, each warp's lane 0 first waits until its bulk copies have read the staging.
  auto complete = [&](bool drain) -> bool {
    if (tid == 0) tc::commit(&mbar);
    if (drain && lane == 0) tc::bulk_wait_read();
    if (tid == 0 && !tc::mbar_wait(&mbar, parity, kWaitLimit)) {
      s_abort = 1;
      dev_set_status(M.status, DEV_TIMEOUT);
    }
    parity ^= 1u;
    __syncthreads();
    tc::fence_after_sync();
    return !s_abort;
  };
  // operand values: rounded to TF32 (with the tail in the second copy under X3) or to BF16
  auto split = [&](float v, OT* hi_dst, int o, int copy_stride) {
    if constexpr (BF) {
      hi_dst[o] = __float2bfloat16_rn(v);
    } else {
      const float hi = tc::tf32_round(v);
      hi_dst[o] = hi;
      if (X3) hi_dst[copy_stride + o] = tc::tf32_round(v - hi);
    }
  };
  // four consecutive K elements of one core-matrix row (8- or 16-byte aligned)
  auto split4 = [&](float4 v, OT* dst, int copy_stride) {
    if constexpr (BF) {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
      uint2 w;
      w.x = *reinterpret_cast<const uint32_t*>(&lo);
      w.y = *reinterpret_cast<const uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(dst) = w;
    } else {
      const float4 hi = make_float4(tc::tf32_round(v.x), tc::tf32_round(v.y), tc::tf32_round(v.z), tc::tf32_round(v.w));
      *reinterpret_cast<float4*>(dst) = hi;
      if (X3)
        *reinterpret_cast<float4*>(dst + copy_stride) = make_float4(
            tc::tf32_round(v.x - hi.x), tc::tf32_round(v.y - hi.y), tc::tf32_round(v.z - hi.z), tc::tf32_round(v.w - hi.w));
    }
  };

  // Task metadata runs ahead of the work: the pencil index two tasks ahead and the point
  // windows one task ahead are loaded while the current task computes.
  struct Meta {
    int g, i2, i3, q2lo, nq2, q3lo, nq3, kst;
  };
  // task t = run start + position j in the run: CTA b takes runs b, b + grid, ...
  struct TaskPos {
    int t, j;
  };
  auto next_task = [&](TaskPos q) {
    return q.j == kRun - 1 ? TaskPos{q.t + (int)(gridDim.x - 1) * kRun + 1, 0} : TaskPos{q.t + 1, q.j + 1};
  };
  // task t: code g n_pencils + position in the pencil list, from the list of (group, pencil)
  // pairs holding interior rows when there is one (in increasing code order)
  auto split_t = [&](int t, int* g) {
    const int c = task_list ? __ldg(task_list + t) : t;
    *g = n_pencils == 1 ? c : fdiv(c, div_np);
    return c - *g * n_pencils;
  };
  auto meta_of = [&](int t, int pencil) {
    Meta m{};
    if (t < ntasks) {
      int g;
      split_t(t, &g);
      m.g = g;
      m.i3 = fdiv(pencil, M.div_n2);
      m.i2 = pencil - m.i3 * D2.n;
      m.q2lo = D2.qlo[m.i2];
      m.nq2 = D2.nqi[m.i2];
      m.q3lo = D3.qlo[m.i3];
      m.nq3 = D3.nqi[m.i3];
      m.kst = D1.qlo[m.g * G];  // rounded down to 4 where used (no wait on the load here)
    }
    return m;
  };
  auto pencil_of = [&](int t) {
    int g;
    return t < ntasks ? M.topo.int_tiles[split_t(t, &g)] : 0;
  };
  TaskPos tp{(int)blockIdx.x * kRun, 0};
  TaskPos tpn = next_task(tp);
  int t = tp.t, tn = tpn.t;
  Meta cur = meta_of(t, pencil_of(t));
  int pen_n = pencil_of(tn);

  // Operand loads of a task, issued one task ahead (after the current task's slab is in
  // place, while its stage-C MMA, readback and copy-out run) into registers.
  //
  // Stage-A operand: the coefficient slab, point q2 in slot q2 mod KQ (a3 < KQ, zero past
  // nq3 and past the last q1 point).  Points already resident from the previous task (same
  // row group and i3) are kept; the new ones form [wlo, wlo + nl) and [rb, wlo + nq2).
  // Thread (a1, a3 quad) reads 4 rows a3 with loads coalesced along a1 and stores them as one
  // 16-byte word of the operand.
  constexpr int NPR = KG * (KQ / 4), U = 4;
  static_assert(NPR <= 256, "one (a1, a3 quad) pair per thread");
  constexpr int NV = NS * 32 * KQ * ES / 16, NVT = (NV + 255) / 256;  // 16-byte words of one table entry
  struct SlabGeo {
    int wlo, nl, rb, np;
    bool ok0, ok1, ok2, ok3;
    int64_t o0;
  };
  const bool in_slab = tid < NPR;
  const int sa1 = tid % KG, sa3 = (tid / KG) * 4;
  const int64_t s3 = nq1g * nq2g;
  auto slab_geo = [&](const Meta& mt) {
    SlabGeo sg;
    const int kst = mt.kst & ~3;
    const bool reuse = RSL && mt.g == sl_g && mt.i3 == sl_i3;
    const int whi = mt.q2lo + mt.nq2;
    sg.wlo = mt.q2lo;
    sg.nl = mt.nq2;
    sg.rb = whi;
    if (reuse) {
      sg.nl = max(0, min(whi, sl_lo) - sg.wlo);
      sg.rb = max(sg.wlo + sg.nl, max(sg.wlo, sl_hi));
    }
    sg.np = sg.nl + max(0, whi - sg.rb);
    const bool in1 = in_slab && kst + sa1 < nq1g;
    sg.ok0 = in1 && sa3 < mt.nq3;
    sg.ok1 = in1 && sa3 + 1 < mt.nq3;
    sg.ok2 = in1 && sa3 + 2 < mt.nq3;
    sg.ok3 = in1 && sa3 + 3 < mt.nq3;
    sg.o0 = s3 * (int64_t)(mt.q3lo + sa3) + kst + sa1;
    return sg;
  };
  auto slab_batch = [&](const SlabGeo& sg, int k0, float4 (&v)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      const int q2 = k < sg.nl ? sg.wlo + k : sg.rb + (k - sg.nl);
      const int64_t o = sg.o0 + q2 * nq1g;
      const bool live = k < sg.np;
      v[u].x = live && sg.ok0 ? __ldg(Cwq + o) : 0.f;
      v[u].y = live && sg.ok1 ? __ldg(Cwq + o + s3) : 0.f;
      v[u].z = live && sg.ok2 ? __ldg(Cwq + o + 2 * s3) : 0.f;
      v[u].w = live && sg.ok3 ? __ldg(Cwq + o + 3 * s3) : 0.f;
    }
  };
  auto slab_store = [&](const SlabGeo& sg, int k0, const float4 (&v)[U]) {
    if (!in_slab) return;
    OT* dst = Sl + OpT<BF>::cidx(arow(0, sa1), sa3, KQ);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      const int q2 = k < sg.nl ? sg.wlo + k : sg.rb + (k - sg.nl);
      if (k < sg.np) split4(v[u], dst + (q2 % KQ) * KQ * 8, TA * 128 * KQ);
    }
  };
  int pf_fc = 0;
  long long pf_ro = 0;
  bool pf_rin = false, pf_new_i3 = true;
  float4 pf_w2[NVT], pf_w3[NVT], pf_v[U];
  SlabGeo pf_sg{};
  auto prefetch = [&](const Meta& mt) {
    const int i1a_n = mt.g * G;
    const int64_t rowbase_n = (int64_t)D1.n * (mt.i2 + (int64_t)D2.n * mt.i3);
    pf_rin = tid < G && i1a_n + tid < D1.n;
    if (pf_rin) {
      pf_fc = M.topo.fn_class[rowbase_n + i1a_n + tid];
      pf_ro = M.topo.rowptr[rowbase_n + i1a_n + tid];
    }
    pf_new_i3 = mt.i3 != cur_i3;
#pragma unroll
    for (int u = 0; u < NVT; ++u) {
      const int k = tid + 256 * u;
      if (k < NV) {
        pf_w2[u] = __ldg(reinterpret_cast<const float4*>(dirop2 + (size_t)mt.i2 * DST) + k);
        if (pf_new_i3) pf_w3[u] = __ldg(reinterpret_cast<const float4*>(dirop3 + (size_t)mt.i3 * DST) + k);
      }
    }
    pf_sg = slab_geo(mt);
    slab_batch(pf_sg, 0, pf_v);
  };
  if (t < ntasks) prefetch(cur);
  while (t < ntasks) {
    const TaskPos tpn2 = next_task(tpn);
    const int tn2 = tpn2.t;
    const Meta nxt = meta_of(tn, pen_n);
    const int pen_n2 = pencil_of(tn2);
    bool stop = false;
    do {
      const int g = cur.g, i2 = cur.i2, i3 = cur.i3;
      const int i1a = g * G;
      const int nq2 = cur.nq2, nq3 = cur.nq3;
      // clipping of the band at the faces of the mesh: in direction d the row's columns are
      // j_d = i_d - P + lo_d + c, c < w_d
      const int lo2 = max(0, P - i2), w2 = min(D2.n - 1, i2 + P) - (i2 - P + lo2) + 1;
      const int lo3 = max(0, P - i3), w3 = min(D3.n - 1, i3 + P) - (i3 - P + lo3) + 1;
      const bool full = w2 == NB && w3 == NB && i1a >= P && min(D1.n, i1a + G) - 1 + P <= D1.n - 1;
      if (!RSL && lane == 0) tc::bulk_wait_read();  // the slab overwrites the staging
      __syncthreads();  // the previous task is done with the staging area and the row data
      if (nq2 > KQ || nq3 > KQ) {  // excluded on the host; never taken
        if (tid == 0) dev_set_status(M.status, DEV_BOUNDS);
        if (tn < ntasks) prefetch(nxt);
        break;
      }
      // operands of this task: row data, tables and the first batch of slab points were
      // loaded into registers ahead of time (prefetch); further slab batches load here
      const SlabGeo sg = pf_sg;
      if (tid < G) {
        rowflag[tid] = pf_rin && pf_fc == F_INT;
        rowoff[tid] = pf_ro;
      }
#pragma unroll
      for (int u = 0; u < NVT; ++u) {
        const int k = tid + 256 * u;
        if (k < NV) {
          reinterpret_cast<float4*>(Bw2)[k] = pf_w2[u];
          if (pf_new_i3) reinterpret_cast<float4*>(Bw3)[k] = pf_w3[u];
        }
      }
      cur_i3 = i3;
      slab_store(sg, 0, pf_v);
      for (int k0 = U; k0 < sg.np; k0 += U) {
        float4 v[U];
        slab_batch(sg, k0, v);
        slab_store(sg, k0, v);
      }
      sl_g = g;
      sl_i3 = i3;
      sl_lo = sg.wlo;
      sl_hi = sg.wlo + nq2;
      if (g != cur_g) {
        if constexpr (BT) {
          // band rows into tensor memory: lane m holds row m, copy c in columns BCOL + c KA + k
          const int quarter = warp & 3, half = warp >> 2;
          const int m = quarter * 32 + lane;
          const float* src = band + (size_t)g * 2 * 128 * KA;
          for (int c8 = half; c8 < NS * KA / 8; c8 += 2) {
            const int cp = c8 / (KA / 8), k = (c8 % (KA / 8)) * 8;
            const float4 x0 = __ldg(reinterpret_cast<const float4*>(src + cp * 128 * KA + tc::cidx(m, k, KA)));
            const float4 x1 = __ldg(reinterpret_cast<const float4*>(src + cp * 128 * KA + tc::cidx(m, k + 4, KA)));
            const float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            tc::st8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(L::BCOL + c8 * 8), v);
          }
          tc::st_wait();
          tc::fence_before_sync();
        } else {
          const float4* src = reinterpret_cast<const float4*>(band + (size_t)g * (BF ? 1 : 2) * 128 * KA);
          float4* dst = reinterpret_cast<float4*>(As);  // the band as 16-byte words
          for (int k = tid; k < NS * 128 * KA * ES / 16; k += blockDim.x) dst[k] = __ldg(src + k);
        }
        cur_g = g;
      }
      __syncthreads();
      int any = 0;
#pragma unroll
      for (int r = 0; r < G; ++r) any |= rowflag[r];
      if (!any) {
        if (tn < ntasks) prefetch(nxt);
        break;
      }
      tc::fence_smem_to_async();
      __syncthreads();
      // stage A MMAs: row tile ta (rows arow(slot, a1)) into columns ta NA
      if (tid == 0) {
        tc::fence_after_sync();
        constexpr uint32_t id = BF ? tc::idesc_bf16(128, NA) : tc::idesc_tf32(128, NA);
        for (int ta = 0; ta < TA; ++ta) {
          bool acc = false;
          for (int pass = 0; pass < NPASS; ++pass) {
            const int ac = (X3 && pass == 0) ? 1 : 0, bc = (X3 && pass == 1) ? 1 : 0;
            mma_chain<BF>(tmem + (uint32_t)(ta * NA), sS + (uint32_t)((ac * TA * 128 * KQ + ta * 128 * KQ) * ES),
                          sB3 + (uint32_t)(bc * 32 * KQ * ES), KQ, KQ / KR, id, acc);
          }
        }
      }
      if (!complete(RSL)) {
        stop = true;
        break;
      }
      // D_A -> U_kind[copy][cidx(brow(a1, dj3), a2, KQ)] with brow(a1, dj3) = ((a1 >> 2) NBE +
      // dj3) 4 + (a1 & 3); slots outside the pencil's q2 window give zeros.  With NBE even the
      // address is a per-lane base plus a constant per dj3.
      {
        const int quarter = warp & 3;
        const int s0 = cur.q2lo % KQ;
        // work units (tile, kind) split over the two warp halves
        for (int u = warp >> 2; u < TA * NT; u += 2) {
          const int ta = u / NT, kind = u - (u / NT) * NT;
          const int m = ta * 128 + quarter * 32 + lane;
          const int slot = (m >> 3) % KQ, a1 = ((m >> 3) / KQ) * 8 + (m & 7);
          const int a2 = slot >= s0 ? slot - s0 : slot - s0 + KQ;
          const bool live = a1 < KG;
          const bool keep = a2 < nq2;
          const int ub = (a1 >> 2) * (NBE / 2) * KQ * 8 + (a1 & 3) * EPC + (a2 / EPC) * 8 * EPC + (a2 % EPC);
          float v[16];
          tc::ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ta * NA + 16 * kind), v);
          if (live) {
            OT* ud = Ro + kind * NS * UC + ub;
#pragma unroll
            for (int dj3 = 0; dj3 < NB; ++dj3)
              split(keep ? v[dj3] : 0.f, ud, (dj3 >> 1) * KQ * 8 + (dj3 & 1) * 4 * EPC, UC);
          }
        }
      }
      tc::fence_before_sync();
      tc::fence_smem_to_async();
      __syncthreads();
      // stage B MMAs: row tile tb (rows brow(a1, dj3)) into columns tb NBn.  Chain 0 multiplies
      // U_0 by [WB2_00 | WB2_11] (all NBn columns); for stiffness chain 1 adds U_1 WB2_00 into
      // the term-1 columns (N = 16 from column 16).
      if (tid == 0) {
        tc::fence_after_sync();
        constexpr uint32_t id0 = BF ? tc::idesc_bf16(128, NBn) : tc::idesc_tf32(128, NBn);
        constexpr uint32_t id1 = BF ? tc::idesc_bf16(128, 16) : tc::idesc_tf32(128, 16);
        for (int tb = 0; tb < TBt; ++tb) {
          bool acc = false;
          for (int chain = 0; chain < NT; ++chain)
            for (int pass = 0; pass < NPASS; ++pass) {
              const int ac = (X3 && pass == 0) ? 1 : 0, bc = (X3 && pass == 1) ? 1 : 0;
              mma_chain<BF>(tmem + (uint32_t)(tb * NBn + 16 * chain),
                            sR + (uint32_t)(((chain * NS + ac) * UC + tb * 128 * KQ) * ES),
                            sB2 + (uint32_t)(bc * 32 * KQ * ES), KQ, KQ / KR, chain ? id1 : id0, acc);
            }
        }
      }
      if (!complete(false)) {
        stop = true;
        break;
      }
      // D_B -> TB[term][copy][cidx(dj2 NB8 + dj3, a1, KG)]: a per-lane base plus a constant per
      // dj2.  Rows of padding slots dj3 >= NB are never written; they only feed stage-C
      // columns that are never read.
      {
        const int quarter = warp & 3;
        for (int tb = warp >> 2; tb < TBt; tb += 2) {
          const int r = tb * 128 + quarter * 32 + lane;
          const int X = r >> 2, a1 = (X / NBE) * 4 + (r & 3), dj3 = X % NBE;
          const bool live = a1 < KG && dj3 < NB;
          const int tbb = (dj3 >> 3) * KG * 8 + (dj3 & 7) * EPC + (a1 / EPC) * 8 * EPC + (a1 % EPC);
#pragma unroll
          for (int term = 0; term < NT; ++term) {
            float v[16];
            tc::ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tb * NBn + 16 * term), v);
            if (live) {
              OT* td = Ro + term * NS * TBC + tbb;
#pragma unroll
              for (int dj2 = 0; dj2 < NB; ++dj2) split(v[dj2], td, dj2 * (NB8 / 8) * KG * 8, TBC);
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::fence_smem_to_async();
      __syncthreads();
      // stage C: D_C[(r, dj1)][dj2 NB8 + dj3] over the band and TB
      if (tid == 0) {
        tc::fence_after_sync();
        constexpr uint32_t id = BF ? tc::idesc_bf16(128, NPADC) : tc::idesc_tf32(128, NPADC);
        bool acc = false;
        for (int pass = 0; pass < NPASS; ++pass) {
          const int ac = (X3 && pass == 0) ? 1 : 0, bc = (X3 && pass == 1) ? 1 : 0;
          for (int term = 0; term < NT; ++term)
            for (int s = 0; s < KG / KR; ++s) {
              const uint64_t bd =
                  tc::sdesc(sR + (uint32_t)((term * NS + bc) * TBC * ES) + (uint32_t)(2 * s * 128), 128, KG * 8 * ES);
              if constexpr (BT) {
                tc::mma_tf32_ta(tmem, tmem + (uint32_t)(L::BCOL + ac * KA + term * KG + 8 * s), bd, id, acc);
              } else {
                const uint64_t ad =
                    tc::sdesc(sA + (uint32_t)(ac * 128 * KA * ES) + (uint32_t)((term * KG / EPC + 2 * s) * 128), 128,
                              KA * 8 * ES);
                if constexpr (BF) tc::mma_f16(tmem, ad, bd, id, acc);
                else tc::mma_tf32(tmem, ad, bd, id, acc);
              }
              acc = true;
            }
        }
      }
      if (tn < ntasks) prefetch(nxt);  // lands while stage C, its readback and the copy-out run
      if (!complete(false)) {
        stop = true;
        break;
      }
      // D_C -> staging.  Row r starts at r RS + (its CSR offset mod 4).  Column dj2 NB8 + dj3 of
      // lane (r, dj1) goes to (dj3 NB + dj2) NB + dj1 in a task away from the faces of the mesh;
      // otherwise to its place in the row's clipped box, so that every row is contiguous.
      {
        const int quarter = warp & 3, half = warp >> 2;
        const int m = quarter * 32 + lane;
        const int r = m / NB, dj1 = m - (m / NB) * NB;
        const bool live = r < G && rowflag[r];
        float* sr = stage + r * RS + (live ? (int)(rowoff[r] & 3) : 0);
        constexpr int CPC = 16 / NB8;  // dj2 values per column chunk
        if (full) {
          float* sd = sr + dj1;
#pragma unroll 1
          for (int ch = half; ch < NPADC / 16; ch += 2) {
            float v[16];
            tc::ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ch * 16), v);
            if (live) {
              float* sc = sd + ch * CPC * NB;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int dj3 = j % NB8, dj2 = ch * CPC + j / NB8;
                if (dj3 < NB && dj2 < NB) sc[dj3 * NB * NB + (j / NB8) * NB] = v[j];
              }
            }
          }
        } else {
          const int i1 = i1a + r;
          const int lo1 = max(0, P - i1), w1 = min(D1.n - 1, i1 + P) - (i1 - P + lo1) + 1;
          const int c1 = dj1 - lo1;
          const bool ok1 = live && (unsigned)c1 < (unsigned)w1;
#pragma unroll 1
          for (int ch = half; ch < NPADC / 16; ch += 2) {
            float v[16];
            tc::ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ch * 16), v);
            if (ok1) {
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int dj3 = j % NB8, dj2 = ch * CPC + j / NB8;
                const int c2 = dj2 - lo2, c3 = dj3 - lo3;
                if (dj3 < NB && (unsigned)c2 < (unsigned)w2 && (unsigned)c3 < (unsigned)w3)
                  sr[(c3 * w2 + c2) * w1 + c1] = v[j];
              }
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::fence_smem_to_async();
      __syncthreads();
      // staging -> CSR values, a warp per row: head up to a 16-byte boundary and tail by the
      // lanes, the aligned body by one bulk asynchronous copy (drained before the staging
      // area is written again)
      for (int r = warp; r < G; r += 8) {
        if (!rowflag[r]) continue;
        int len = NB3;
        if (!full) {
          const int i1 = i1a + r;
          const int lo1 = max(0, P - i1), w1 = min(D1.n - 1, i1 + P) - (i1 - P + lo1) + 1;
          len = w1 * w2 * w3;
        }
        const int64_t off = rowoff[r];
        float* dst = values + off;
        const int sh = (int)(off & 3);
        const float* sr = stage + r * RS + sh;
        const int head = (4 - sh) & 3;
        const int nv = (len - head) >> 2;
        const int t0 = head + 4 * nv;
        if (lane < head) dst[lane] = sr[lane];
        if (t0 + lane < len) dst[t0 + lane] = sr[t0 + lane];
        if (lane == 0 && nv > 0) tc::bulk_s2g(dst + head, sr + head, (uint32_t)nv * 16u);
      }
      if (lane == 0) tc::bulk_commit();
    } while (false);
    if (stop) break;
    t = tn;
    tn = tn2;
    tpn = tpn2;
    cur = nxt;
    pen_n = pen_n2;
  }

  if (lane == 0) tc::bulk_wait();
  __syncthreads();
  if (s_abort) {
    if (tid == 0) tc::mbar_wait(&mbar, parity ^ 1u, kWaitLimit);
    __syncthreads();
    tc::fence_after_sync();
  }
  if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

template <int P, bool STIFF, bool X3, bool BF>
cudaError_t launch_tc3_t(const MeshView& M, const float* Cwq, float* values, const void* band, const void* dirop2,
                         const void* dirop3, int Kg, int ngroups, int n_pencils, int kRun, const int32_t* tasks,
                         int n_tasks, cudaStream_t st) {
  using L = Tc3Smem<P, STIFF, X3, BF>;
  using OT = typename OpT<BF>::T;
  const size_t smem = L::bytes;
  auto kern = k_interior_tc3<P, STIFF, X3, BF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  int dev = 0, nsm = 0, smem_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  const uint32_t cols = (uint32_t)L::COLS;
  int occ = (int)(smem_sm / (smem + fa.sharedSizeBytes + 1024));
  occ = std::min(occ, 65536 / (256 * std::max(1, (fa.numRegs + 7) / 8 * 8)));
  occ = std::min(occ, (int)(512 / cols));
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int64_t ntasks = tasks ? (int64_t)n_tasks : (int64_t)ngroups * n_pencils;
  if (ntasks == 0) return cudaSuccess;
  if (kRun < 1) kRun = 1;
  const int grid = (int)std::min<int64_t>((ntasks + kRun - 1) / kRun, (int64_t)nsm * occ);
  const FastDiv div_np = make_fastdiv(std::max(2, n_pencils));
  kern<<<grid, 256, smem, st>>>(M, Cwq, values, static_cast<const OT*>(band), static_cast<const OT*>(dirop2),
                                static_cast<const OT*>(dirop3), Kg, n_pencils, div_np, (int)ntasks, cols, kRun, tasks);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

template <bool BF>
void shape_of(int p, int* G, int* KG, int* KQ) {
  *G = *KG = *KQ = 0;
  switch (p) {
#define SFA_SHAPE(PP)                \
  case PP:                           \
    *G = TcShape<PP, BF>::G;         \
    *KG = TcShape<PP, BF>::KG;       \
    *KQ = Tc3Shape<PP, BF>::KQ;      \
    break;
    SFA_SHAPE(2)
    SFA_SHAPE(3)
    SFA_SHAPE(4)
    SFA_SHAPE(5)
    SFA_SHAPE(6)
#undef SFA_SHAPE
  }
}

template <bool BF>
cudaError_t tables_of(const MeshView& M, int G, int Kg, int KQ, int ngroups, void* band_mass, void* band_stiff,
                      void* dirop2, void* dirop3, cudaStream_t st) {
  using OT = typename OpT<BF>::T;
  dim3 grid(8, ngroups);
  k_tc_band<BF><<<grid, 256, 0, st>>>(M.dir[0], M.p, G, Kg, Kg, 0, static_cast<OT*>(band_mass));
  SFA_LAUNCHED(1);
  k_tc_band<BF><<<grid, 256, 0, st>>>(M.dir[0], M.p, G, Kg, 2 * Kg, 1, static_cast<OT*>(band_stiff));
  SFA_LAUNCHED(1);
  k_tc_dirop<BF><<<M.dir[1].n, 256, 0, st>>>(M.dir[1], M.p, KQ, static_cast<OT*>(dirop2));
  SFA_LAUNCHED(1);
  k_tc_dirop<BF><<<M.dir[2].n, 256, 0, st>>>(M.dir[2], M.p, KQ, static_cast<OT*>(dirop3));
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

// Rows per MMA group, the compiled q1 window and the slab K for degree p and operand type
// (0 if p is out of range).
void interior_tc_shape(int p, bool bf, int* G, int* KG, int* KQ) {
  if (bf) shape_of<true>(p, G, KG, KQ);
  else shape_of<false>(p, G, KG, KQ);
}

// Operand tables of the tensor-core interior rows (band matrices and q2/q3 tables), TF32
// head/tail copies (bf = false) or BF16 (bf = true), for the compiled windows Kg and KQ.
cudaError_t launch_tc_band(const MeshView& M, bool bf, int G, int Kg, int KQ, int ngroups, void* band_mass,
                           void* band_stiff, void* dirop2, void* dirop3, cudaStream_t st) {
  if (ngroups <= 0) return cudaSuccess;
  return bf ? tables_of<true>(M, G, Kg, KQ, ngroups, band_mass, band_stiff, dirop2, dirop3, st)
            : tables_of<false>(M, G, Kg, KQ, ngroups, band_mass, band_stiff, dirop2, dirop3, st);
}

// Every shape fits one CTA (checked at compile time).
template <int P, bool STIFF, bool X3, bool BF>
cudaError_t launch_tc_any(const MeshView& M, const float* Cwq, float* values, const void* band, const void* dirop2,
                          const void* dirop3, int Kg, int ngroups, int n_pencils, int kRun, const int32_t* tasks,
                          int n_tasks, cudaStream_t st) {
  static_assert(Tc3Smem<P, STIFF, X3, BF>::OCC >= 1, "tensor-core interior shape does not fit one SM");
  return launch_tc3_t<P, STIFF, X3, BF>(M, Cwq, values, band, dirop2, dirop3, Kg, ngroups, n_pencils, kRun, tasks,
                                        n_tasks, st);
}

// Kg is the mesh's widest group window (checked against the compiled one in the kernel);
// the band matrices are laid out with the compiled window.  bf: BF16 operands (one pass).
// tasks: the (group, pencil) codes that hold interior rows (n_tasks of them), or null for
// every pair.
cudaError_t launch_interior_tc(const MeshView& M, bool stiff, bool x3, bool bf, const float* Cwq, float* values,
                               const void* band, const void* dirop2, const void* dirop3, int Kg, int ngroups,
                               int n_pencils, int run, const int32_t* tasks, int n_tasks, cudaStream_t st) {
#define SFA_TC_ONE(PP, ST, X, B) \
  launch_tc_any<PP, ST, X, B>(M, Cwq, values, band, dirop2, dirop3, Kg, ngroups, n_pencils, run, tasks, n_tasks, st)
#define SFA_TC_CASE(PP)                                                                                  \
  case PP:                                                                                               \
    if (bf) return stiff ? SFA_TC_ONE(PP, true, false, true) : SFA_TC_ONE(PP, false, false, true);     \
    if (stiff) return x3 ? SFA_TC_ONE(PP, true, true, false) : SFA_TC_ONE(PP, true, false, false);     \
    return x3 ? SFA_TC_ONE(PP, false, true, false) : SFA_TC_ONE(PP, false, false, false);
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
