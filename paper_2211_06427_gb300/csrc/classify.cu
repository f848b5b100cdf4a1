// Geometry stage (Sec. 2.1 function types, Sec. 2.2 step 2 choice of the artificial
// discontinuity, Sec. 3.1 cut-element sub-cells): element states by 9 level-set samples,
// octree pieces of cut elements, function classes, the DWQ box of every cut function and
// the CSR pattern of the active rows.  Integer work; the level set is evaluated in FP64
// with a fixed, uncontracted operation order.
#include "sfa_internal.cuh"

namespace {

// Level-set signs that need double arithmetic, out of line: the FP64 sign behind the float
// filter (a handful of samples per launch) and the sign of level sets without a cached
// table.  Inlined, the compiler hoisted the loop-invariant part of their double arithmetic
// (the setup of the exact divisions in ls_coord) into the octree's cell loop, where it ran
// for every cell although the path is not taken for a cached gyroid; on this GPU's FP64
// rate that made the kernel FP64-bound.
__device__ __noinline__ bool ls_neg_fp64(const LevelSet& L, int64_t k1, int64_t k2, int64_t k3) {
  return ls_phi_k(L, k1, k2, k3) < 0.0;
}
__device__ __noinline__ bool ls_neg_any(const LevelSet& L, int64_t k1, int64_t k2, int64_t k3) {
  return ls_neg_k(L, k1, k2, k3);
}

// Element states: corners k = e * 2^(D+1) and (e+1) * 2^(D+1), centre e * 2^(D+1) + 2^D.
__global__ void k_elem_state(LevelSet L, int D, int ne1, int ne2, int ne3, int8_t* state, int32_t* cut_flag) {
  int64_t nE = (int64_t)ne1 * ne2 * ne3;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nE; e += (int64_t)gridDim.x * blockDim.x) {
    int e1 = e % ne1, e2 = (e / ne1) % ne2, e3 = (int)(e / ((int64_t)ne1 * ne2));
    int64_t s = 1ll << (D + 1);
    int64_t k0[3] = {e1 * s, e2 * s, e3 * s};
    int nneg = 0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 2; ++c) nneg += ls_neg_any(L, k0[0] + a * s, k0[1] + b * s, k0[2] + c * s);
    nneg += ls_neg_any(L, k0[0] + s / 2, k0[1] + s / 2, k0[2] + s / 2);
    // inside iff phi < 0 at all nine samples, outside iff phi >= 0 at all nine
    int c = nneg == 9 ? 1 : (nneg == 0 ? 0 : 2);
    state[e] = c == 1 ? E_IN : (c == 0 ? E_OUT : E_CUT);
    cut_flag[e] = c == 2 ? 1 : 0;
  }
}

// Block-wide exclusive scan of one int per thread (blockDim <= 1024).  Returns the block total.
__device__ int block_scan_excl(int v, int* out, int* warp_tot) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_tot[lane] = w;  // inclusive per warp
  }
  __syncthreads();
  int before = warp ? warp_tot[warp - 1] : 0;
  *out = before + x - v;
  int total = warp_tot[nw - 1];
  __syncthreads();
  return total;
}

// Octree of one cut element per block.  phi is sampled once on the (2^D + 1)^3 corner grid
// of the finest cells; every finest cell walks its ancestors from level 1 to D: the first
// inside ancestor is its piece, an outside ancestor means none, and a still-cut cell at
// level D is kept iff phi(centre) < 0.  A piece is emitted by the first finest cell it
// covers, so pieces come out in finest-cell order; each element's pieces go to its slab
// (capacity 8^D) and their count to counts[].

__global__ void __launch_bounds__(256, 4) k_octree(LevelSet L, int D, int ne1, int ne2, const int32_t* cut_elems, int n_cut,
                         int32_t* counts, uint32_t* slab, int8_t* state) {
  // neg[idx] = (phi < 0) on the (2^D + 1)^3 corner grid: one comparison per sample
  extern __shared__ unsigned char neg[];
  __shared__ int warp_tot[32];
  int ci = blockIdx.x;
  if (ci >= n_cut) return;
  int e = cut_elems[ci];
  int e1 = e % ne1, e2 = (e / ne1) % ne2, e3 = e / (ne1 * ne2);
  const int G = (1 << D) + 1;
  const int64_t b1 = (int64_t)e1 << (D + 1), b2 = (int64_t)e2 << (D + 1), b3 = (int64_t)e3 << (D + 1);
  // gyroid: the element's sample indices b_d + r, r <= 2^(D+1), have their float sin/cos
  // cached here for the filtered sign test (ls_neg_k with the table reads from shared memory)
  __shared__ float trs[3][2][2 * (1 << SFA_MAX_OCTREE_DEPTH) + 1];
  const bool cached = L.kind == SFA_LS_GYROID && L.trigf != nullptr;
  const int R = 2 << D;
  if (cached) {
    const int64_t S = L.trig_stride;
    for (int t = threadIdx.x; t < 3 * (R + 1); t += blockDim.x) {
      const int d = t / (R + 1), r = t % (R + 1);
      const int64_t k = (d == 0 ? b1 : (d == 1 ? b2 : b3)) + r;
      trs[d][0][r] = L.trigf[(2 * d + 0) * S + k];
      trs[d][1][r] = L.trigf[(2 * d + 1) * S + k];
    }
  }
  __syncthreads();
  auto neg_at = [&](int r1, int r2, int r3) -> bool {
    if (cached) {
      const float a = __fmul_rn(trs[0][0][r1], trs[1][1][r2]);
      const float b = __fmul_rn(trs[1][0][r2], trs[2][1][r3]);
      const float c = __fmul_rn(trs[2][0][r3], trs[0][1][r1]);
      const float v = __fsub_rn(__fadd_rn(__fadd_rn(a, b), c), L.isof);
      if (fabsf(v) > L.filt) return v < 0.f;
      return ls_neg_fp64(L, b1 + r1, b2 + r2, b3 + r3);  // rare: about 0.1 samples per element
    }
    return ls_neg_any(L, b1 + r1, b2 + r2, b3 + r3);
  };
  for (int idx = threadIdx.x; idx < G * G * G; idx += blockDim.x) {
    int a1 = idx % G, a2 = (idx / G) % G, a3 = idx / (G * G);
    neg[idx] = neg_at(2 * a1, 2 * a2, 2 * a3) ? 1 : 0;
  }
  __syncthreads();
  const int ncell = 1 << (3 * D), mask = (1 << D) - 1;
  int running = 0;
  for (int base = 0; base < ncell; base += blockDim.x) {
    int c = base + threadIdx.x;
    int emit = 0;
    uint32_t code = 0;
    if (c < ncell) {
      int c1 = c & mask, c2 = (c >> D) & mask, c3 = c >> (2 * D);
      int owner = -1;  // level of the piece, -1 none
      int oa1 = 0, oa2 = 0, oa3 = 0;
      for (int l = (D == 0 ? 0 : 1); l <= D; ++l) {
        int sh = D - l, size = 1 << sh;
        int a1 = c1 >> sh, a2 = c2 >> sh, a3 = c3 >> sh;
        int cl;
        int centre_neg = 0;
        if (l == D) centre_neg = neg_at(2 * c1 + 1, 2 * c2 + 1, 2 * c3 + 1);
        if (l == 0) {
          cl = 2;  // the element itself is cut
        } else {
          int lo1 = a1 << sh, lo2 = a2 << sh, lo3 = a3 << sh;
          int nneg = 0;
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y)
              for (int z = 0; z < 2; ++z) nneg += neg[(lo1 + x * size) + G * ((lo2 + y * size) + G * (lo3 + z * size))];
          if (l < D) {
            int h = size >> 1;
            nneg += neg[(lo1 + h) + G * ((lo2 + h) + G * (lo3 + h))];
          } else {
            nneg += centre_neg;
          }
          cl = nneg == 9 ? 1 : (nneg == 0 ? 0 : 2);
        }
        if (cl == 1) {
          owner = l; oa1 = a1; oa2 = a2; oa3 = a3;
          break;
        }
        if (cl == 0) break;
        if (l == D) {
          if (centre_neg) {
            owner = l; oa1 = a1; oa2 = a2; oa3 = a3;
          }
          break;
        }
      }
      if (owner >= 0) {
        int osz = 1 << (D - owner);
        emit = ((c1 & (osz - 1)) == 0 && (c2 & (osz - 1)) == 0 && (c3 & (osz - 1)) == 0) ? 1 : 0;
        code = (uint32_t)owner | ((uint32_t)oa1 << 4) | ((uint32_t)oa2 << 10) | ((uint32_t)oa3 << 16);
      }
    }
    int pos;
    int tot = block_scan_excl(emit, &pos, warp_tot);
    if (emit) slab[(size_t)ci * ncell + running + pos] = code;
    running += tot;
  }
  if (threadIdx.x == 0) {
    counts[ci] = running;
    if (running == 0) state[e] = E_CUT_EMPTY;
  }
}

// Pieces of cut element ci: its slab prefix, moved to the compacted piece array.
__global__ void k_copy_pieces(const uint32_t* slab, int ncell, const int32_t* piece_ptr, uint32_t* pieces) {
  const int ci = blockIdx.x;
  const int a = piece_ptr[ci], n = piece_ptr[ci + 1] - a;
  for (int t = threadIdx.x; t < n; t += blockDim.x) pieces[a + t] = slab[(size_t)ci * ncell + t];
}

__global__ void k_fn_class(int p, int ne1, int ne2, int ne3, const int8_t* state, int8_t* fcls) {
  int n1 = ne1 + p, n2 = ne2 + p, n3 = ne3 + p;
  int64_t N = (int64_t)n1 * n2 * n3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int i1 = i % n1, i2 = (i / n1) % n2, i3 = (int)(i / ((int64_t)n1 * n2));
    bool all_in = true, any_dom = false;
    for (int e3 = max(0, i3 - p); e3 <= min(ne3 - 1, i3); ++e3)
      for (int e2 = max(0, i2 - p); e2 <= min(ne2 - 1, i2); ++e2)
        for (int e1 = max(0, i1 - p); e1 <= min(ne1 - 1, i1); ++e1) {
          int8_t s = state[e1 + (int64_t)ne1 * (e2 + (int64_t)ne2 * e3)];
          all_in = all_in && (s == E_IN);
          any_dom = any_dom || (s == E_IN) || (s == E_CUT);
        }
    fcls[i] = all_in ? F_INT : (any_dom ? F_CUT : F_EXT);
  }
}

// DWQ box choice and row lengths.  Box: direction d, boundary b strictly inside the support
// in d, side low/high; kept = full support in the other directions x the side's elements in
// d; valid iff every kept element is inside; most elements wins, ties to smallest d, low
// side, smallest b.  Row length: active columns with |j_d - i_d| <= p.
__global__ void k_box_rowlen(int p, int ne1, int ne2, int ne3, const int8_t* state, const int8_t* fcls,
                             int32_t* box, int64_t* rowlen, unsigned long long* counters) {
  int n1 = ne1 + p, n2 = ne2 + p, n3 = ne3 + p;
  int ne[3] = {ne1, ne2, ne3}, nn[3] = {n1, n2, n3};
  int64_t N = (int64_t)n1 * n2 * n3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int idx[3] = {(int)(i % n1), (int)((i / n1) % n2), (int)(i / ((int64_t)n1 * n2))};
    int8_t fc = fcls[i];
    int32_t bcode = -1;
    int64_t len = 0;
    if (fc == F_CUT) {
      int lo[3], hi[3];
      for (int d = 0; d < 3; ++d) {
        lo[d] = max(0, idx[d] - p);
        hi[d] = min(ne[d] - 1, idx[d]);
      }
      int best_score = 0;
      for (int d = 0; d < 3; ++d) {
        bool ok[SFA_MAXP + 1];
        int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
        for (int k = lo[d]; k <= hi[d]; ++k) {
          bool all = true;
          for (int a = lo[o1]; a <= hi[o1] && all; ++a)
            for (int c = lo[o2]; c <= hi[o2] && all; ++c) {
              int e[3];
              e[d] = k; e[o1] = a; e[o2] = c;
              all = state[e[0] + (int64_t)ne1 * (e[1] + (int64_t)ne2 * e[2])] == E_IN;
            }
          ok[k - lo[d]] = all;
        }
        int other = (hi[o1] - lo[o1] + 1) * (hi[o2] - lo[o2] + 1);
        for (int side = 0; side < 2; ++side)
          for (int b = lo[d] + 1; b <= hi[d]; ++b) {
            int ka = side == 0 ? lo[d] : b, kb = side == 0 ? b - 1 : hi[d];
            bool valid = true;
            for (int k = ka; k <= kb; ++k) valid = valid && ok[k - lo[d]];
            int score = (kb - ka + 1) * other;
            if (valid && score > best_score) {
              best_score = score;
              bcode = d | (side << 2) | (b << 3);
            }
          }
      }
      atomicAdd(&counters[1], 1ull);
      if (bcode >= 0) atomicAdd(&counters[2], 1ull);
      // work of the cut-row kernel: inside support elements outside the box (element Gauss),
      // cut support elements (rows of E), and the point counts of the box (m_f in the box
      // direction, m_s and m_t in the other two, ascending)
      {
        const int bd = bcode >= 0 ? (bcode & 3) : -1, bside = (bcode >> 2) & 1, bb = bcode >> 3;
        unsigned long long ng = 0, nc = 0;
        for (int e3 = lo[2]; e3 <= hi[2]; ++e3)
          for (int e2 = lo[1]; e2 <= hi[1]; ++e2)
            for (int e1 = lo[0]; e1 <= hi[0]; ++e1) {
              const int8_t st = state[e1 + (int64_t)ne1 * (e2 + (int64_t)ne2 * e3)];
              if (st == E_CUT) {
                ++nc;
              } else if (st == E_IN) {
                const int ed = bd == 0 ? e1 : (bd == 1 ? e2 : e3);
                const bool in_box = bd >= 0 && ((bside == 0 && ed < bb) || (bside == 1 && ed >= bb));
                if (!in_box) ++ng;
              }
            }
        atomicAdd(&counters[4], ng);
        atomicAdd(&counters[5], nc);
        if (bd >= 0) {
          int mq[3];
          for (int d = 0; d < 3; ++d) {
            int m = 0;
            for (int e = lo[d]; e <= hi[d]; ++e) m += (e == 0 || e == ne[d] - 1) ? p + 1 : 2;
            mq[d] = m;
          }
          const int kept = bside == 0 ? bb - lo[bd] : hi[bd] - bb + 1;
          const unsigned long long mf = (unsigned long long)kept * (p + 1);
          const int ds = bd == 0 ? 1 : 0, dt = bd == 2 ? 1 : 2;
          const unsigned long long ms = mq[ds], mt = mq[dt];
          atomicAdd(&counters[6], mf * ms * mt);
          atomicAdd(&counters[7], ms * mt);
          atomicAdd(&counters[8], mt);
        }
      }
    }
    if (fc != F_EXT) {
      int w[3], jl[3];
      for (int d = 0; d < 3; ++d) {
        jl[d] = max(0, idx[d] - p);
        w[d] = min(nn[d] - 1, idx[d] + p) - jl[d] + 1;
      }
      if (fc == F_INT) {
        len = (int64_t)w[0] * w[1] * w[2];
        atomicAdd(&counters[0], 1ull);
        atomicAdd(&counters[3], (unsigned long long)len);
      } else {
        for (int c3 = 0; c3 < w[2]; ++c3)
          for (int c2 = 0; c2 < w[1]; ++c2)
            for (int c1 = 0; c1 < w[0]; ++c1) {
              int64_t j = (jl[0] + c1) + (int64_t)n1 * ((jl[1] + c2) + (int64_t)n2 * (jl[2] + c3));
              len += fcls[j] != F_EXT;
            }
      }
    }
    box[i] = bcode;
    rowlen[i] = len;
  }
}

// Column indices: one warp per row, band entries in ascending j, compacted by ballot.  A row
// whose band is not clipped by a face uses the table of full-band offsets
// dj1 + n1 (dj2 + n2 dj3) staged in shared memory; interior rows take every entry.
__global__ void k_colind(int p, int n1, int n2, int n3, FastDiv dv1, FastDiv dv2, const int8_t* fcls,
                         const int64_t* rowptr, int32_t* colind) {
  extern __shared__ int offt[];
  const int nb = 2 * p + 1, nb3 = nb * nb * nb;
  for (int t = threadIdx.x; t < nb3; t += blockDim.x) {
    const int c1 = t % nb, c2 = (t / nb) % nb, c3 = t / (nb * nb);
    offt[t] = c1 + n1 * (c2 + n2 * c3);
  }
  __syncthreads();
  int lane = threadIdx.x & 31;
  int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t N = (int64_t)n1 * n2 * n3;
  for (int64_t i = warp; i < N; i += nwarps) {
    int8_t fc = fcls[i];
    if (fc == F_EXT) continue;
    const int q12 = fdiv((int)i, dv1);
    const int i1 = (int)i - q12 * n1, i3 = fdiv(q12, dv2), i2 = q12 - i3 * n2;
    int jl1 = max(0, i1 - p), jl2 = max(0, i2 - p), jl3 = max(0, i3 - p);
    int w1 = min(n1 - 1, i1 + p) - jl1 + 1, w2 = min(n2 - 1, i2 + p) - jl2 + 1, w3 = min(n3 - 1, i3 + p) - jl3 + 1;
    int64_t out = rowptr[i];
    const int jb = jl1 + n1 * (jl2 + n2 * jl3);
    if (w1 == nb && w2 == nb && w3 == nb) {
      if (fc == F_INT) {
        for (int t = lane; t < nb3; t += 32) colind[out + t] = jb + offt[t];
      } else {
        for (int base = 0; base < nb3; base += 32) {
          const int t = base + lane;
          int j = 0;
          bool act = false;
          if (t < nb3) {
            j = jb + offt[t];
            act = fcls[j] != F_EXT;
          }
          unsigned m = __ballot_sync(0xffffffffu, act);
          if (act) colind[out + __popc(m & ((1u << lane) - 1u))] = j;
          out += __popc(m);
        }
      }
      continue;
    }
    // clipped band: (c1, c2, c3) of entry t = base + lane advanced by 32 per step
    const int total = w1 * w2 * w3;
    int c1 = lane, c2 = 0, c3 = 0;
    while (c1 >= w1) {
      c1 -= w1;
      if (++c2 == w2) c2 = 0, ++c3;
    }
    for (int base = 0; base < total; base += 32) {
      int t = base + lane;
      bool act = false;
      int j = 0;
      if (t < total) {
        j = jb + c1 + n1 * (c2 + n2 * c3);
        act = fc == F_INT || fcls[j] != F_EXT;
      }
      unsigned m = __ballot_sync(0xffffffffu, act);
      if (act) colind[out + __popc(m & ((1u << lane) - 1u))] = (int32_t)j;
      out += __popc(m);
      c1 += 32;
      while (c1 >= w1) {
        c1 -= w1;
        if (++c2 == w2) c2 = 0, ++c3;
      }
    }
  }
}

// ---- device-wide exclusive scan (int64), three phases ----------------------------------
constexpr int SCAN_T = 1024, SCAN_PER = 4, SCAN_BLK = SCAN_T * SCAN_PER;

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_blocks(const T* in, int64_t n, int64_t* out, int64_t* block_sums) {
  __shared__ int64_t wt[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_BLK + threadIdx.x * SCAN_PER;
  int64_t v[SCAN_PER], s = 0;
  for (int k = 0; k < SCAN_PER; ++k) {
    v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = wt[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wt[lane] = w;
  }
  __syncthreads();
  int64_t run = (warp ? wt[warp - 1] : 0) + x - s;
  for (int k = 0; k < SCAN_PER; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == SCAN_T - 1) block_sums[blockIdx.x] = wt[31];
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* block_sums, int64_t nb, int64_t* out, int64_t n) {
  // single block, sequential over chunks of 1024
  __shared__ int64_t wt[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += 1024) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? block_sums[i] : 0;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t w = wt[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wt[lane] = w;
    }
    __syncthreads();
    int64_t excl = carry + (warp ? wt[warp - 1] : 0) + x - v;
    if (i < nb) block_sums[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) carry += wt[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* block_sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_BLK;
  int64_t add = block_sums[blockIdx.x];
  for (int k = threadIdx.x; k < SCAN_BLK; k += SCAN_T)
    if (base + k < n) out[base + k] += add;
}

template <typename T>
cudaError_t scan_excl(const T* in, int64_t n, int64_t* out, int64_t* scratch, cudaStream_t st) {
  int64_t nb = (n + SCAN_BLK - 1) / SCAN_BLK;
  if (nb == 0) nb = 1;
  k_scan_blocks<T><<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, out, scratch);
  SFA_LAUNCHED(1);
  k_scan_sums<<<1, 1024, 0, st>>>(scratch, nb, out, n);
  SFA_LAUNCHED(1);
  k_scan_add<<<(unsigned)nb, SCAN_T, 0, st>>>(out, n, scratch);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

// scatter-compaction: out[scan[i]] = i where flag[i] (and map[i] = rank or -1)
template <typename T>
__global__ void k_compact(const T* flag, const int64_t* scan, int64_t n, int32_t* out, int32_t* map) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bool f = flag[i] != 0;
    if (f) out[scan[i]] = (int32_t)i;
    if (map) map[i] = f ? (int32_t)scan[i] : -1;
  }
}

__global__ void k_flag_class(const int8_t* fcls, int64_t n, int8_t want, int32_t* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = fcls[i] == want;
}

// (row group g, pencil k) pairs of the tensor-core interior kernel that hold an interior row:
// flag[g npen + k] for rows i1 in [g G, g G + G) of pencil int_tiles[k]
__global__ void k_flag_tc_tasks(const int8_t* fcls, const int32_t* pencils, int npen, int n1, int G, int ngroups,
                                int32_t* flag) {
  const int64_t n = (int64_t)ngroups * npen;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(t / npen), k = (int)(t % npen);
    const int64_t base = (int64_t)n1 * pencils[k];
    const int hi = min(n1, g * G + G);
    int any = 0;
    for (int i1 = g * G; i1 < hi && !any; ++i1) any = fcls[base + i1] == F_INT;
    flag[t] = any;
  }
}

// Work counts of the cut-element moments: per cut element the nonempty octree slots (level,
// a2, a3) and groups (level, a3) of its pieces, summed into counters[0] and counters[1].
// One block per cut element.
__global__ void k_slot_counts(const uint32_t* pieces, const int32_t* piece_ptr, int D, int p,
                              unsigned long long* counters) {
  // nonempty slots (l, a_mid, a_out) and groups (l, a_out) of the cut element's pieces in the
  // cyclic orientation (inner, middle, outer) = (r, r+1, r+2 mod 3) with the least FP64 work
  // slots (3p+1)^2 + groups (3p+1)^3, the one the moment kernel takes
  extern __shared__ uint32_t smask3[];
  const int nslot = ((1 << (2 * (D + 1))) - 1) / 3, npos = (2 << D) - 1;
  for (int t = threadIdx.x; t < 3 * nslot; t += blockDim.x) smask3[t] = 0u;
  __syncthreads();
  const int pb = piece_ptr[blockIdx.x], pe = piece_ptr[blockIdx.x + 1];
  for (int t = pb + threadIdx.x; t < pe; t += blockDim.x) {
    const uint32_t code = pieces[t];
    const int l = code & 15;
    const int av[3] = {(int)((code >> 4) & 63), (int)((code >> 10) & 63), (int)((code >> 16) & 63)};
    const int sb = ((1 << (2 * l)) - 1) / 3;
    for (int r = 0; r < 3; ++r) {
      const int dmid = r == 2 ? 0 : r + 1, dout = r == 0 ? 2 : r - 1;
      smask3[r * nslot + sb + av[dmid] + (av[dout] << l)] = 1u;
    }
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const long long m3 = 3 * p + 1;
  long long best_cost = -1;
  int best_s = 0, best_g = 0;
  for (int r = 0; r < 3; ++r) {
    const uint32_t* sm = smask3 + r * nslot;
    int ns = 0, ng = 0;
    for (int c = 0; c < nslot; c += 32) ns += __popc(__ballot_sync(0xffffffffu, c + lane < nslot && sm[c + lane] != 0u));
    for (int c = 0; c < npos; c += 32) {
      const int gp = c + lane;
      bool any = false;
      if (gp < npos) {
        const int l = 31 - __clz(gp + 1), ao = gp + 1 - (1 << l);
        const int sb = ((1 << (2 * l)) - 1) / 3 + (ao << l);
        for (int am = 0; am < (1 << l); ++am) any |= sm[sb + am] != 0u;
      }
      ng += __popc(__ballot_sync(0xffffffffu, any));
    }
    const long long cost = ns * m3 * m3 + ng * m3 * m3 * m3;
    if (best_cost < 0 || cost < best_cost) best_cost = cost, best_s = ns, best_g = ng;
  }
  if (lane == 0 && (best_s || best_g)) {
    atomicAdd(&counters[0], (unsigned long long)best_s);
    atomicAdd(&counters[1], (unsigned long long)best_g);
  }
}

// active rows (not exterior)
__global__ void k_flag_active(const int8_t* fcls, int64_t n, int32_t* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = fcls[i] != F_EXT;
}

// pencils (i2, i3) holding at least one interior row
__global__ void k_flag_pencils(const int8_t* fcls, int n1, int n2, int n3, int32_t* flag) {
  int64_t np = (int64_t)n2 * n3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < np; t += (int64_t)gridDim.x * blockDim.x) {
    int any = 0;
    for (int i1 = 0; i1 < n1 && !any; ++i1) any = fcls[i1 + (int64_t)n1 * t] == F_INT;
    flag[t] = any;
  }
}

__global__ void k_trig(LevelSet L, double* trig, float* trigf) {
  const int64_t S = L.trig_stride;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * S; t += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(t / S);
    const int64_t k = t % S;
    if (k > L.Nk[d]) continue;
    const double X = __dmul_rn(L.freq, ls_coord(L, d, k));
    const double sv = sin(X), cv = cos(X);
    trig[(2 * d + 0) * S + k] = sv;
    trig[(2 * d + 1) * S + k] = cv;
    trigf[(2 * d + 0) * S + k] = (float)sv;
    trigf[(2 * d + 1) * S + k] = (float)cv;
  }
}

__global__ void k_i64_to_i32(const int64_t* in, int64_t n, int32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)in[i];
}

}  // namespace

// ----------------------------------------------------------------------------------------
// Host launchers used by the API translation unit.
cudaError_t launch_trig(LevelSet L, double* trig, float* trigf, cudaStream_t st) {
  L.trig = nullptr;
  L.trigf = nullptr;
  k_trig<<<152, 256, 0, st>>>(L, trig, trigf);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_i64_to_i32(const int64_t* in, int64_t n, int32_t* out, cudaStream_t st) {
  k_i64_to_i32<<<152, 256, 0, st>>>(in, n, out);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_elem_state(const LevelSet& L, int D, const int* ne, int8_t* state, int32_t* cut_flag, cudaStream_t st) {
  k_elem_state<<<608, 256, 0, st>>>(L, D, ne[0], ne[1], ne[2], state, cut_flag);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_scan_i32(const int32_t* in, int64_t n, int64_t* out, int64_t* scratch, cudaStream_t st) {
  return scan_excl<int32_t>(in, n, out, scratch, st);
}
cudaError_t launch_scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* scratch, cudaStream_t st) {
  return scan_excl<int64_t>(in, n, out, scratch, st);
}

cudaError_t launch_compact_i32(const int32_t* flag, const int64_t* scan, int64_t n, int32_t* out, int32_t* map,
                               cudaStream_t st) {
  k_compact<int32_t><<<608, 256, 0, st>>>(flag, scan, n, out, map);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_octree(const LevelSet& L, int D, const int* ne, const int32_t* cut_elems, int n_cut, int32_t* counts,
                          uint32_t* slab, int8_t* state, cudaStream_t st) {
  if (n_cut == 0) return cudaSuccess;
  int G = (1 << D) + 1;
  size_t smem = (size_t)G * G * G;
  cudaError_t e = cudaFuncSetAttribute(k_octree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_octree<<<n_cut, 256, smem, st>>>(L, D, ne[0], ne[1], cut_elems, n_cut, counts, slab, state);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_pieces(const uint32_t* slab, int D, int n_cut, const int32_t* piece_ptr, uint32_t* pieces,
                               cudaStream_t st) {
  if (n_cut == 0) return cudaSuccess;
  k_copy_pieces<<<n_cut, 128, 0, st>>>(slab, 1 << (3 * D), piece_ptr, pieces);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_fn_class(int p, const int* ne, const int8_t* state, int8_t* fcls, cudaStream_t st) {
  k_fn_class<<<608, 256, 0, st>>>(p, ne[0], ne[1], ne[2], state, fcls);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_box_rowlen(int p, const int* ne, const int8_t* state, const int8_t* fcls, int32_t* box,
                              int64_t* rowlen, unsigned long long* counters, cudaStream_t st) {
  k_box_rowlen<<<608, 256, 0, st>>>(p, ne[0], ne[1], ne[2], state, fcls, box, rowlen, counters);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_colind(int p, const int* n, const int8_t* fcls, const int64_t* rowptr, int32_t* colind,
                          cudaStream_t st) {
  const size_t smem = (size_t)(2 * p + 1) * (2 * p + 1) * (2 * p + 1) * sizeof(int);
  k_colind<<<1216, 256, smem, st>>>(p, n[0], n[1], n[2], make_fastdiv(n[0]), make_fastdiv(n[1]), fcls, rowptr, colind);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_flag_class(const int8_t* fcls, int64_t n, int8_t want, int32_t* flag, cudaStream_t st) {
  k_flag_class<<<608, 256, 0, st>>>(fcls, n, want, flag);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_flag_tc_tasks(const int8_t* fcls, const int32_t* pencils, int npen, int n1, int G, int ngroups,
                                 int32_t* flag, cudaStream_t st) {
  k_flag_tc_tasks<<<608, 256, 0, st>>>(fcls, pencils, npen, n1, G, ngroups, flag);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_slot_counts(const uint32_t* pieces, const int32_t* piece_ptr, int n_cut, int D, int p,
                               unsigned long long* counters, cudaStream_t st) {
  if (n_cut <= 0) return cudaSuccess;
  const int nslot = ((1 << (2 * (D + 1))) - 1) / 3;
  k_slot_counts<<<n_cut, 128, 3 * nslot * sizeof(uint32_t), st>>>(pieces, piece_ptr, D, p, counters);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_flag_active(const int8_t* fcls, int64_t n, int32_t* flag, cudaStream_t st) {
  k_flag_active<<<608, 256, 0, st>>>(fcls, n, flag);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}

cudaError_t launch_flag_pencils(const int8_t* fcls, const int* n, int32_t* flag, cudaStream_t st) {
  k_flag_pencils<<<608, 256, 0, st>>>(fcls, n[0], n[1], n[2], flag);
  SFA_LAUNCHED(1);
  return cudaGetLastError();
}
