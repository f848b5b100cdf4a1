// Interior rows (Sec. 1: weighted quadrature + sum factorization + row assembly; Table 2,
// row loop / sum factorization): for every test function whose support holds only inside
// elements,
//   V[j3][j2][j1] = sum_q3 WB3[j3][q3] sum_q2 WB2[j2][q2] sum_q1 WB1[j1][q1] C[q1,q2,q3]
// with WB_d[dj][q] = w_{i_d}(q) B_{i_d - p + dj}(t_q) (stiffness: the three terms with the
// derivative rule in one direction).  A CTA takes T consecutive rows i1 of one (i2, i3)
// pencil; the contractions over q3 (stage A) and q2 (stage B) are shared by those rows,
// the contraction over q1 (stage C) is per row.  Each row's band is a contiguous (possibly
// face-clipped) box in [j3][j2][j1] order of the CSR value array.
//
// Work split: stage A tasks are (kind, q2, 32 q1 columns), stage B tasks (j3, 32 q1
// columns) and stage C gives one warp per row with lanes over the (j3, j2) pairs; each task
// keeps its 1D table in registers, so shared memory only feeds the contracted data.  For a
// regular support (two WQ points in each of its p+1 elements) the tables are banded with a
// compile-time structure: dj only meets the points of elements max(0, dj-p)..min(p, dj),
// and only those products are formed.  Supports touching the first or last element use
// the generic dense path.
#include "interior_common.cuh"

size_t interior_smem_bytes(int p, int nql1, int nql2, int nql3, int T, int L1MAX, bool stiff, bool fp64);

namespace {

template <typename R, int P, bool STIFF>
__global__ void __launch_bounds__(256) k_interior(MeshView M, const R* __restrict__ Cwq, R* __restrict__ values,
                                                  int T, int L1MAX, int nchunks, int skip_regular) {
  constexpr int NB = 2 * P + 1, NQR = 2 * P + 2;  // band width, points of a regular support
  constexpr int NQM = 4 * P;                      // bound on WQ points in any support
  constexpr int NC = NB * NB;                     // (j3, j2) pairs
  constexpr bool REGT = sizeof(R) == 4 || P <= 4;  // banded register tables fit
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dir1D &D1 = M.dir[0], &D2 = M.dir[1], &D3 = M.dir[2];
  const int NQL2 = D2.nql, NQL3 = D3.nql, NQL1 = D1.nql;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;

  const int pencil = M.topo.int_tiles[blockIdx.x / nchunks];
  const int chunk = blockIdx.x % nchunks;
  const int i2 = pencil % D2.n, i3 = pencil / D2.n;
  if (skip_regular && i2 - P >= 1 && i2 <= D2.n_el - 2 && i3 - P >= 1 && i3 <= D3.n_el - 2) return;
  const int i1a = chunk * T, i1b = min(D1.n, i1a + T);
  if (i1a >= D1.n) return;
  const int64_t rowbase = (int64_t)D1.n * (i2 + (int64_t)D2.n * i3);

  const int L1P = L1MAX | 1;  // odd row stride of the TB arrays (bank spread)
  // same region sizes as interior_smem_bytes: slab region (C, then the two TB arrays) and
  // U region (U, then per-warp output staging)
  size_t slab = (size_t)NQL3 * NQL2 * L1MAX;
  if ((size_t)2 * NC * L1P > slab) slab = (size_t)2 * NC * L1P;
  size_t ureg = (size_t)2 * NB * NQL2 * L1MAX;
  if ((size_t)8 * NB * NB * NB > ureg) ureg = (size_t)8 * NB * NB * NB;
  R* Cs = reinterpret_cast<R*>(smem_raw);               // [a3][a2][a1]; later TB [term][pair][a1]
  R* U = Cs + slab;                                      // [kind][dj3][a2][a1]; later output staging
  R* TBx = Cs;
  R* TByz = Cs + (size_t)NC * L1P;
  long long* rowoff = reinterpret_cast<long long*>((reinterpret_cast<uintptr_t>(U + ureg) + 7) & ~uintptr_t(7));
  // (rowoff: CSR offset of each row, 8-byte aligned; qoff: first q1 point of each row)
  int* qoff = reinterpret_cast<int*>(rowoff + T);
  int* rowflag = qoff + T;

  int any = 0;
  for (int r = threadIdx.x; r < T; r += blockDim.x) {
    const bool in = i1a + r < i1b;
    const int fc = in ? M.topo.fn_class[rowbase + i1a + r] : 0;
    const long long ro = in ? M.topo.rowptr[rowbase + i1a + r] : 0;
    const int qo = in ? D1.qlo[i1a + r] : 0;
    rowflag[r] = in && fc == F_INT;
    rowoff[r] = ro;
    qoff[r] = qo;
  }
  __syncthreads();
  for (int r = 0; r < i1b - i1a; ++r) any |= rowflag[r];
  if (!any) return;

  const int q2lo = D2.qlo[i2], nq2 = D2.nqi[i2];
  const int q3lo = D3.qlo[i3], nq3 = D3.nqi[i3];
  const int Q1lo = D1.qlo[i1a];
  const int L1 = D1.qlo[i1b - 1] + D1.nqi[i1b - 1] - Q1lo;
  // regular support: p+1 elements, none of them the first or last (two WQ points each)
  const bool reg2 = i2 - P >= 1 && i2 <= D2.n_el - 2, reg3 = i3 - P >= 1 && i3 <= D3.n_el - 2;

  // coefficient slab C[a3][a2][a1]
  load_slab<R, 4>(Cwq, D1.nq, D2.nq, Q1lo, q2lo, q3lo, nq2, nq3 * nq2, L1, Cs, L1);
  __syncthreads();

  // ---- stage A: U_kk[dj3][a2][a1] = sum_a3 W3_kk[dj3][a3] C[a3][a2][a1]
  {
    const int nblk = (L1 + 31) >> 5;
    const int ntask = (STIFF ? 2 : 1) * nq2 * nblk;
    const R* W3base = Tab<R>::wb00(D3) + (size_t)i3 * NB * NQL3;
    const R* W3base1 = Tab<R>::wb11(D3) + (size_t)i3 * NB * NQL3;
    for (int task = warp; task < ntask; task += nw) {
      const int kk = task / (nq2 * nblk), rem = task % (nq2 * nblk);
      const int a2 = rem / nblk, a1 = (rem % nblk) * 32 + lane;
      const R* W3 = kk ? W3base1 : W3base;
      R* Uo = U + (size_t)kk * NB * NQL2 * L1MAX;
      if (REGT && reg3) {
        R w[NB][NQR], x[NQR], y[NB];
        load_table<R, P>(W3, NQL3, w);
        if (a1 < L1) {
#pragma unroll
          for (int q = 0; q < NQR; ++q) x[q] = Cs[(q * nq2 + a2) * L1 + a1];
          band_apply<R, P>(w, x, y);
#pragma unroll
          for (int dj = 0; dj < NB; ++dj) Uo[(dj * NQL2 + a2) * L1MAX + a1] = y[dj];
        }
      } else if (a1 < L1) {
        for (int dj = 0; dj < NB; ++dj) {
          R s = R(0);
          for (int q = 0; q < nq3; ++q) s += W3[dj * NQL3 + q] * Cs[(q * nq2 + a2) * L1 + a1];
          Uo[(dj * NQL2 + a2) * L1MAX + a1] = s;
        }
      }
    }
  }
  __syncthreads();

  // ---- stage B: TBx[dj3 NB + dj2][a1] = sum_a2 W2_00[dj2][a2] U_00[dj3][a2][a1]
  //               TByz (stiffness)       = sum_a2 W2_00 U_11 + W2_11 U_00   (two phases)
  {
    const int nblk = (L1 + 31) >> 5;
    const R* W2a = Tab<R>::wb00(D2) + (size_t)i2 * NB * NQL2;
    const R* W2b = Tab<R>::wb11(D2) + (size_t)i2 * NB * NQL2;
    const R* U0 = U;
    const R* U1 = U + (size_t)NB * NQL2 * L1MAX;
    for (int phase = 0; phase < (STIFF ? 2 : 1); ++phase) {
      const int ntask = NB * nblk;
      for (int task = warp; task < ntask; task += nw) {
        const int dj3 = task / nblk, a1 = (task % nblk) * 32 + lane;
        if (REGT && reg2) {
          R w[NB][NQR], x[NQR], y[NB];
          load_table<R, P>(phase == 0 ? W2a : W2b, NQL2, w);
          if (a1 < L1) {
            // phase 0: x-term from U_00 and, for stiffness, the z-term from U_11 (same table)
#pragma unroll
            for (int q = 0; q < NQR; ++q) x[q] = U0[(dj3 * NQL2 + q) * L1MAX + a1];
            band_apply<R, P>(w, x, y);
            if (phase == 0) {
#pragma unroll
              for (int dj = 0; dj < NB; ++dj) TBx[(dj3 * NB + dj) * L1P + a1] = y[dj];
              if (STIFF) {
#pragma unroll
                for (int q = 0; q < NQR; ++q) x[q] = U1[(dj3 * NQL2 + q) * L1MAX + a1];
                band_apply<R, P>(w, x, y);
#pragma unroll
                for (int dj = 0; dj < NB; ++dj) TByz[(dj3 * NB + dj) * L1P + a1] = y[dj];
              }
            } else {
#pragma unroll
              for (int dj = 0; dj < NB; ++dj) TByz[(dj3 * NB + dj) * L1P + a1] += y[dj];
            }
          }
        } else if (a1 < L1) {
          const R* W2 = phase == 0 ? W2a : W2b;
          for (int dj = 0; dj < NB; ++dj) {
            R s0 = R(0), s1 = R(0);
            for (int q = 0; q < nq2; ++q) {
              s0 += W2[dj * NQL2 + q] * U0[(dj3 * NQL2 + q) * L1MAX + a1];
              if (STIFF && phase == 0) s1 += W2[dj * NQL2 + q] * U1[(dj3 * NQL2 + q) * L1MAX + a1];
            }
            if (phase == 0) {
              TBx[(dj3 * NB + dj) * L1P + a1] = s0;
              if (STIFF) TByz[(dj3 * NB + dj) * L1P + a1] = s1;
            } else {
              TByz[(dj3 * NB + dj) * L1P + a1] += s0;
            }
          }
        }
      }
      __syncthreads();
    }
  }

  // ---- stage C: one warp per row, lanes over (dj3, dj2) pairs; band staged per warp
  R* stage = U + (size_t)warp * NB * NB * NB;
  const int nrows = i1b - i1a;
  for (int r = warp; r < nrows; r += nw) {
    if (!rowflag[r]) continue;
    const int i1 = i1a + r;
    const int off = qoff[r] - Q1lo;
    const R* W1a = Tab<R>::wb00(D1) + (size_t)i1 * NB * NQL1;
    const R* W1b = Tab<R>::wb11(D1) + (size_t)i1 * NB * NQL1;
    if (REGT && i1 - P >= 1 && i1 <= D1.n_el - 2) {
      R wa[NB][NQR], wb[NB][NQR];
      load_table<R, P>(W1a, NQL1, wa);
      if (STIFF) load_table<R, P>(W1b, NQL1, wb);
      for (int c = lane; c < NC; c += 32) {
        R x[NQR], y[NB];
        if (STIFF) {
          // V = W1_11 TBx + W1_00 TByz
#pragma unroll
          for (int q = 0; q < NQR; ++q) x[q] = TBx[c * L1P + off + q];
          band_apply<R, P>(wb, x, y);
          R z[NB];
#pragma unroll
          for (int q = 0; q < NQR; ++q) x[q] = TByz[c * L1P + off + q];
          band_apply<R, P>(wa, x, z);
#pragma unroll
          for (int dj = 0; dj < NB; ++dj) stage[c * NB + dj] = y[dj] + z[dj];
        } else {
#pragma unroll
          for (int q = 0; q < NQR; ++q) x[q] = TBx[c * L1P + off + q];
          band_apply<R, P>(wa, x, y);
#pragma unroll
          for (int dj = 0; dj < NB; ++dj) stage[c * NB + dj] = y[dj];
        }
      }
    } else {
      const int nq1 = D1.nqi[i1];
      for (int c = lane; c < NC; c += 32) {
        for (int dj = 0; dj < NB; ++dj) {
          R s = R(0);
          for (int q = 0; q < nq1; ++q) {
            if (STIFF)
              s += W1b[dj * NQL1 + q] * TBx[c * L1P + off + q] + W1a[dj * NQL1 + q] * TByz[c * L1P + off + q];
            else
              s += W1a[dj * NQL1 + q] * TBx[c * L1P + off + q];
          }
          stage[c * NB + dj] = s;
        }
      }
    }
    __syncwarp();
    // coalesced write of the (clipped) band; staging order [dj3][dj2][dj1] is the row order
    const int lo1 = max(0, P - i1), lo2 = max(0, P - i2), lo3 = max(0, P - i3);
    const int w1 = min(D1.n - 1, i1 + P) - (i1 - P + lo1) + 1;
    const int w2 = min(D2.n - 1, i2 + P) - (i2 - P + lo2) + 1;
    const int w3 = min(D3.n - 1, i3 + P) - (i3 - P + lo3) + 1;
    R* dst = values + rowoff[r];
    if (w1 == NB && w2 == NB && w3 == NB) {
      for (int t = lane; t < NB * NB * NB; t += 32) dst[t] = stage[t];
    } else {
      const int len = w1 * w2 * w3;
      for (int t = lane; t < len; t += 32) {
        const int c1 = t % w1, c2 = (t / w1) % w2, c3 = t / (w1 * w2);
        dst[t] = stage[((lo3 + c3) * NB + (lo2 + c2)) * NB + (lo1 + c1)];
      }
    }
    __syncwarp();
  }
  (void)NQM;
}

// ---------------------------------------------------------------------------------------
// Regular pencils: i2 and i3 both regular (two WQ points in each of their p+1 support
// elements), so q2 and q3 windows have exactly 2p+2 points and all three contractions have
// compile-time band structure.  Threads are split by table (kind or term) so each keeps one
// banded table in registers; stage C runs two register passes per row (stiffness).
template <typename R, int P, bool STIFF>
__global__ void __launch_bounds__(256, (sizeof(R) == 8 && P >= 4) ? 1 : 2) k_interior_reg(MeshView M, const R* __restrict__ Cwq, R* __restrict__ values,
                                                         int T, int L1MAX, int nchunks) {
  constexpr int NB = 2 * P + 1, NQ = 2 * P + 2, NC = NB * NB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dir1D &D1 = M.dir[0], &D2 = M.dir[1], &D3 = M.dir[2];
  const int NQL1 = D1.nql, NQL2 = D2.nql, NQL3 = D3.nql;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pencil = M.topo.int_tiles[blockIdx.x / nchunks];
  const int chunk = blockIdx.x % nchunks;
  const int i2 = pencil % D2.n, i3 = pencil / D2.n;
  if (!(i2 - P >= 1 && i2 <= D2.n_el - 2 && i3 - P >= 1 && i3 <= D3.n_el - 2)) return;  // boundary pencil
  const int i1a = chunk * T, i1b = min(D1.n, i1a + T);
  if (i1a >= D1.n) return;
  const int64_t rowbase = (int64_t)D1.n * (i2 + (int64_t)D2.n * i3);

  const int L1P = (L1MAX & ~3) + 6;  // TB row stride: even (8-byte pairs), = 2 mod 4 (banks)
  size_t slab = (size_t)NQ * NQ * L1MAX;
  if ((size_t)2 * NC * L1P > slab) slab = (size_t)2 * NC * L1P;
  R* Cs = reinterpret_cast<R*>(smem_raw);  // C [a3][a2][a1], later TBx | TByz [pair][a1]
  R* U = Cs + slab;                        // U [kind][dj3][a2][a1], later per-warp staging
  size_t ureg = (size_t)2 * NB * NQ * L1MAX;
  if ((size_t)8 * NB * NB * NB > ureg) ureg = (size_t)8 * NB * NB * NB;
  long long* rowoff = reinterpret_cast<long long*>((reinterpret_cast<uintptr_t>(U + ureg) + 7) & ~uintptr_t(7));
  // (rowoff: CSR offset of each row, 8-byte aligned; qoff: first q1 point of each row)
  int* qoff = reinterpret_cast<int*>(rowoff + T);
  int* rowflag = qoff + T;
  R* TBx = Cs;
  R* TByz = Cs + (size_t)NC * L1P;

  for (int r = threadIdx.x; r < T; r += blockDim.x) {
    const bool in = i1a + r < i1b;
    const int fc = in ? M.topo.fn_class[rowbase + i1a + r] : 0;
    const long long ro = in ? M.topo.rowptr[rowbase + i1a + r] : 0;
    const int qo = in ? D1.qlo[i1a + r] : 0;
    rowflag[r] = in && fc == F_INT;
    rowoff[r] = ro;
    qoff[r] = qo;
  }
  __syncthreads();
  int any = 0;
  for (int r = 0; r < i1b - i1a; ++r) any |= rowflag[r];
  if (!any) return;

  const int q2lo = D2.qlo[i2], q3lo = D3.qlo[i3];
  const int Q1lo = D1.qlo[i1a];
  const int L1 = D1.qlo[i1b - 1] + D1.nqi[i1b - 1] - Q1lo;
  load_slab<R, 4>(Cwq, D1.nq, D2.nq, Q1lo, q2lo, q3lo, NQ, NQ * NQ, L1, Cs, L1MAX);
  __syncthreads();

  // stage A: threads [0, half) kind 00, [half, 2 half) kind 11 (stiffness); item = (a2, a1)
  {
    const int groups = STIFF ? 2 : 1;
    const int gsize = blockDim.x / groups;
    const int kk = threadIdx.x / gsize, tg = threadIdx.x % gsize;
    R w[NB][NQ];
    load_table<R, P>((kk ? Tab<R>::wb11(D3) : Tab<R>::wb00(D3)) + (size_t)i3 * NB * NQL3, NQL3, w);
    R* Uo = U + (size_t)kk * NB * NQ * L1MAX;
    for (int it = tg; it < NQ * L1; it += gsize) {
      const int a2 = it / L1, a1 = it % L1;
      R x[NQ], y[NB];
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[q] = Cs[(q * NQ + a2) * L1MAX + a1];
      band_apply<R, P>(w, x, y);
#pragma unroll
      for (int dj = 0; dj < NB; ++dj) Uo[(dj * NQ + a2) * L1MAX + a1] = y[dj];
    }
  }
  __syncthreads();
  // stage B phase 0 (table W2_00): x-term TBx = W2_00 U00; z-term TByz = W2_00 U11
  {
    const int groups = STIFF ? 2 : 1;
    const int gsize = blockDim.x / groups;
    const int term = threadIdx.x / gsize, tg = threadIdx.x % gsize;
    R w[NB][NQ];
    load_table<R, P>(Tab<R>::wb00(D2) + (size_t)i2 * NB * NQL2, NQL2, w);
    const R* Ui = U + (size_t)term * NB * NQ * L1MAX;
    R* To = term ? TByz : TBx;
    for (int it = tg; it < NB * L1; it += gsize) {
      const int dj3 = it / L1, a1 = it % L1;
      R x[NQ], y[NB];
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[q] = Ui[(dj3 * NQ + q) * L1MAX + a1];
      band_apply<R, P>(w, x, y);
#pragma unroll
      for (int dj = 0; dj < NB; ++dj) To[(dj3 * NB + dj) * L1P + a1] = y[dj];
    }
  }
  if (STIFF) {
    __syncthreads();
    // stage B phase 1 (table W2_11): y-term TByz += W2_11 U00
    R w[NB][NQ];
    load_table<R, P>(Tab<R>::wb11(D2) + (size_t)i2 * NB * NQL2, NQL2, w);
    for (int it = threadIdx.x; it < NB * L1; it += blockDim.x) {
      const int dj3 = it / L1, a1 = it % L1;
      R x[NQ], y[NB];
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[q] = U[(dj3 * NQ + q) * L1MAX + a1];
      band_apply<R, P>(w, x, y);
#pragma unroll
      for (int dj = 0; dj < NB; ++dj) TByz[(dj3 * NB + dj) * L1P + a1] += y[dj];
    }
  }
  __syncthreads();

  // stage C: warp per row, lanes over (dj3, dj2) pairs, one register table per pass
  R* stage = U + (size_t)warp * NB * NB * NB;
  const int nrows = i1b - i1a;
  for (int r = warp; r < nrows; r += (blockDim.x >> 5)) {
    if (!rowflag[r]) continue;
    const int i1 = i1a + r;
    const int off = qoff[r] - Q1lo;
    const R* W1a = Tab<R>::wb00(D1) + (size_t)i1 * NB * NQL1;
    const R* W1b = Tab<R>::wb11(D1) + (size_t)i1 * NB * NQL1;
    if (i1 - P >= 1 && i1 <= D1.n_el - 2) {
      for (int pass = 0; pass < (STIFF ? 2 : 1); ++pass) {
        // stiffness: pass 0 W1_11 TBx, pass 1 += W1_00 TByz; mass: W1_00 TBx
        R w[NB][NQ];
        load_table<R, P>((STIFF && pass == 0) ? W1b : W1a, NQL1, w);
        const R* src = pass == 0 ? TBx : TByz;
        for (int c = lane; c < NC; c += 32) {
          R x[NQ], y[NB];
          const R* xs = src + c * L1P + off;
#pragma unroll
          for (int q = 0; q < NQ; ++q) x[q] = xs[q];
          band_apply<R, P>(w, x, y);
          R* o = stage + c * NB;
          if (pass == 0) {
#pragma unroll
            for (int dj = 0; dj < NB; ++dj) o[dj] = y[dj];
          } else {
#pragma unroll
            for (int dj = 0; dj < NB; ++dj) o[dj] += y[dj];
          }
        }
      }
    } else {
      const int nq1 = D1.nqi[i1];
      for (int c = lane; c < NC; c += 32) {
        for (int dj = 0; dj < NB; ++dj) {
          R sacc = R(0);
          for (int q = 0; q < nq1; ++q) {
            if (STIFF)
              sacc += W1b[dj * NQL1 + q] * TBx[c * L1P + off + q] + W1a[dj * NQL1 + q] * TByz[c * L1P + off + q];
            else
              sacc += W1a[dj * NQL1 + q] * TBx[c * L1P + off + q];
          }
          stage[c * NB + dj] = sacc;
        }
      }
    }
    __syncwarp();
    const int lo1 = max(0, P - i1);
    const int w1 = min(D1.n - 1, i1 + P) - (i1 - P + lo1) + 1;
    R* dst = values + rowoff[r];
    if (w1 == NB) {
      for (int t = lane; t < NB * NB * NB; t += 32) dst[t] = stage[t];
    } else {
      const int len = w1 * NB * NB;
      for (int t = lane; t < len; t += 32) {
        const int c1 = t % w1, c23 = t / w1;
        dst[t] = stage[c23 * NB + lo1 + c1];
      }
    }
    __syncwarp();
  }
}

}  // namespace

size_t interior_reg_smem_bytes(int p, int T, int L1MAX, bool fp64) {
  const int NB = 2 * p + 1, NQ = 2 * p + 2;
  const size_t L1P = (size_t)((L1MAX & ~3) + 6);
  size_t slab = (size_t)NQ * NQ * L1MAX;
  if (2 * (size_t)NB * NB * L1P > slab) slab = 2 * (size_t)NB * NB * L1P;
  size_t u = 2 * (size_t)NB * NQ * L1MAX;
  if (8 * (size_t)NB * NB * NB > u) u = 8 * (size_t)NB * NB * NB;
  return (slab + u) * (fp64 ? 8 : 4) + 8 + T * (sizeof(long long) + 2 * sizeof(int)) + 16;
}

namespace {

template <typename R, int P, bool STIFF>
cudaError_t launch_interior_reg_t(const MeshView& M, const R* Cwq, R* values, int n_pencils, int T, int L1MAX,
                                  cudaStream_t st) {
  const size_t smem = interior_reg_smem_bytes(P, T, L1MAX, sizeof(R) == 8);
  cudaError_t e = cudaFuncSetAttribute(k_interior_reg<R, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nchunks = (M.dir[0].n + T - 1) / T;
  const int64_t grid = (int64_t)n_pencils * nchunks;
  if (grid == 0) return cudaSuccess;
  k_interior_reg<R, P, STIFF><<<(unsigned)grid, 256, smem, st>>>(M, Cwq, values, T, L1MAX, nchunks);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

template <typename R, int P, bool STIFF>
cudaError_t launch_interior_t(const MeshView& M, const R* Cwq, R* values, int n_pencils, int T, int L1MAX,
                              int skip_regular, cudaStream_t st) {
  const size_t smem = interior_smem_bytes(P, M.dir[0].nql, M.dir[1].nql, M.dir[2].nql, T, L1MAX, STIFF, sizeof(R) == 8);
  cudaError_t e = cudaFuncSetAttribute(k_interior<R, P, STIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nchunks = (M.dir[0].n + T - 1) / T;
  int64_t grid = (int64_t)n_pencils * nchunks;
  if (grid == 0) return cudaSuccess;
  k_interior<R, P, STIFF><<<(unsigned)grid, 256, smem, st>>>(M, Cwq, values, T, L1MAX, nchunks, skip_regular);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

}  // namespace

// Shared-memory bytes of the interior kernel for chunk length T (host-side sizing):
// the coefficient slab (reused for the two TB arrays), the U arrays (reused as per-warp
// output staging) and the row flags.
size_t interior_smem_bytes(int p, int nql1, int nql2, int nql3, int T, int L1MAX, bool stiff, bool fp64) {
  (void)nql1;
  (void)stiff;
  const int NB = 2 * p + 1;
  const size_t L1P = (size_t)(L1MAX | 1);
  size_t slab = (size_t)nql3 * nql2 * L1MAX;
  const size_t tb = 2 * (size_t)NB * NB * L1P;
  if (tb > slab) slab = tb;
  size_t u = 2 * (size_t)NB * nql2 * L1MAX;
  const size_t staging = 8 * (size_t)NB * NB * NB;  // 8 warps
  if (staging > u) u = staging;
  return (slab + u) * (fp64 ? 8 : 4) + 8 + T * (sizeof(long long) + 2 * sizeof(int)) + 16;
}

// Regular pencils go to k_interior_reg with chunk length Treg (L1 window Lreg), the others
// to the generic k_interior (chunk T, window L1MAX).
cudaError_t launch_interior(const MeshView& M, bool fp64, bool stiff, const void* Cwq, void* values, int n_pencils,
                            int T, int L1MAX, int Treg, int Lreg, cudaStream_t st) {
  // Treg > 0: regular pencils on k_interior_reg, the rest on k_interior; Treg == 0: all
  // pencils on k_interior; Treg < 0: only the non-regular pencils (k_interior)
  const int use_reg = Treg > 0;
  const int skip_reg = Treg != 0;
  cudaError_t e = cudaSuccess;
#define SFA_INT_CASE(PP)                                                                                         \
  case PP:                                                                                                       \
    if (fp64) {                                                                                                  \
      if (stiff) {                                                                                               \
        if (use_reg) e = launch_interior_reg_t<double, PP, true>(M, (const double*)Cwq, (double*)values, n_pencils, Treg, Lreg, st); \
        if (e == cudaSuccess) e = launch_interior_t<double, PP, true>(M, (const double*)Cwq, (double*)values, n_pencils, T, L1MAX, skip_reg, st); \
      } else {                                                                                                   \
        if (use_reg) e = launch_interior_reg_t<double, PP, false>(M, (const double*)Cwq, (double*)values, n_pencils, Treg, Lreg, st); \
        if (e == cudaSuccess) e = launch_interior_t<double, PP, false>(M, (const double*)Cwq, (double*)values, n_pencils, T, L1MAX, skip_reg, st); \
      }                                                                                                          \
    } else {                                                                                                     \
      if (stiff) {                                                                                               \
        if (use_reg) e = launch_interior_reg_t<float, PP, true>(M, (const float*)Cwq, (float*)values, n_pencils, Treg, Lreg, st); \
        if (e == cudaSuccess) e = launch_interior_t<float, PP, true>(M, (const float*)Cwq, (float*)values, n_pencils, T, L1MAX, skip_reg, st); \
      } else {                                                                                                   \
        if (use_reg) e = launch_interior_reg_t<float, PP, false>(M, (const float*)Cwq, (float*)values, n_pencils, Treg, Lreg, st); \
        if (e == cudaSuccess) e = launch_interior_t<float, PP, false>(M, (const float*)Cwq, (float*)values, n_pencils, T, L1MAX, skip_reg, st); \
      }                                                                                                          \
    }                                                                                                            \
    return e;
  switch (M.p) {
    SFA_INT_CASE(2)
    SFA_INT_CASE(3)
    SFA_INT_CASE(4)
    SFA_INT_CASE(5)
    SFA_INT_CASE(6)
  }
#undef SFA_INT_CASE
  return cudaErrorInvalidValue;
}
