// Internal declarations shared by the libsfa translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/sfa.h"

#define SFA_MAXP SFA_MAX_DEGREE
#define SFA_WARP 32

// Device status codes written into the mesh status word (first nonzero wins).
enum : int {
  DEV_OK = 0,
  DEV_WQ_SINGULAR = 1,
  DEV_BOUNDS = 2,
  DEV_TIMEOUT = 3,
};

// Precision classes (include/sfa.h, sfa_precision).
inline bool prec_valid(int p) { return p >= SFA_FP64 && p <= SFA_BF16; }
// interior rows on the tensor cores
inline bool prec_tc(int p) { return p == SFA_TF32 || p == SFA_TF32X3 || p == SFA_TF32X3_M64 || p == SFA_BF16; }
// head/tail split products on the tensor cores
inline bool prec_x3(int p) { return p == SFA_TF32X3 || p == SFA_TF32X3_M64; }
// cut-cell moments accumulated in double
inline bool prec_mom64(int p) { return p == SFA_FP64 || p == SFA_FP32_M64 || p == SFA_TF32X3_M64; }

// Element states, function classes.
enum : int8_t { E_OUT = 0, E_IN = 1, E_CUT = 2, E_CUT_EMPTY = 3 };
enum : int8_t { F_EXT = 0, F_INT = 1, F_CUT = 2 };

// ---------------------------------------------------------------------------------------
// One direction of the tensor-product space, as seen by kernels.
// Superset point s lies in element s / (p+1), Gauss index s % (p+1).
// WQ point q (0..nq-1) is superset point wq_idx[q].  Function i has its WQ points at
// q in [qlo[i], qlo[i] + nqi[i]) (local index ql = q - qlo[i] < nql).
// Standard tables: w00/w11 [n][nql]; WB00/WB11 [n][2p+1][nql] = w(q) * B_{i-p+dj}(t_q)
// (resp. w11 * B').  DWQ tables: rule r = ((i * p) + slot) * 2 + side, slot = b - e_lo - 1;
// dwq00/dwq11 [nrule][nsl] over local superset index sl = s - e_lo(i) (p+1);
// WD00/WD11 [nrule][2p+1][nsl].  Bernstein product tables G/Gd [n_el][p+1][p+1][2p+1].
struct Dir1D {
  int n_el, n, nsup, nq, nql, nsl;
  double lo, hi;
  double* xb;     // n_el + 1
  double* U;      // n_el + 2p + 1 knots
  double* t_sup;  // nsup
  double* w_sup;  // nsup
  double* B;      // nsup * (p+1)
  double* dB;     // nsup * (p+1)
  int* wq_idx;    // nq
  int* qlo;       // n
  int* nqi;       // n
  double *w00, *w11;
  float* Bf;  // float copy of B (float coefficient passes)
  double *WB00, *WB11;
  float *WB00f, *WB11f;
  double *dwq00, *dwq11;
  double *WD00, *WD11;
  float *WD00f, *WD11f;
  double *G, *Gd;
  float *Gf, *Gdf;  // float copies for the float element-matrix kernel
  double* BZ;  // [n_el][p+1][p+1] Bezier coefficients of B_{e+a} on element e
  // Octree-piece tables: for element e, piece position pos = (2^l - 1) + a (level l, local
  // cell a < 2^l) and Gauss index g: PT[((e * npos + pos) * (p+1) + g) * PTF + f] with
  // f = 0 weight, 1..2p+1 Bernstein values (degree 2p, element coordinate), then p+1
  // B-spline values of functions e..e+p, then the analytic-coefficient factor.
  double* PT;
  float* PTf;  // float copy (float moments)
  int npos;
  // Degree-3p monomial moments of the pieces: P3[(e * npos + pos) * (3p+1) + m] =
  // sum_g w_g t_g^m (1 - t_g)^(3p - m) over the piece's Gauss points (t in element coordinates),
  // double and float.
  double* P3;
  float* P3f;
  // Element Gauss products GE[e][ai][b][g] = w(s) B_{e+ai}(s) B_{e+b}(s), s = e (p+1) + g
  // (GEd: derivatives), double and float.
  double *GE, *GEd;
  float *GEf, *GEdf;
};

struct LevelSet {
  int kind;
  int n_balls;
  double balls[4 * SFA_MAX_BALLS];
  double freq, iso;
  double pt[3], nn[3];
  double lo[3], hi[3];
  int64_t Nk[3];  // n_el * 2^(D+1): sample grid resolution
  // gyroid: sin/cos of freq * x(k) on the sample grid, [2 d + {0 sin, 1 cos}][trig_stride]
  const double* trig;
  int64_t trig_stride;
  // float copy of the trig table and the sign filter: |phi32| > filt implies that the
  // FP64 evaluation below has the same sign (gyroid only)
  const float* trigf;
  float isof, filt;
};

struct Gauss {
  double x[2 * SFA_MAXP + 1], w[2 * SFA_MAXP + 1];   // (p+1)-point rule
  double x2[2 * SFA_MAXP + 1], w2[2 * SFA_MAXP + 1]; // (2p+1)-point rule
};

// Classification results (device pointers).
struct Topo {
  int8_t* elem_state;   // n_el^3
  int32_t* elem_cut_id; // n_el^3, -1 if not cut
  int32_t* cut_elems;   // n_cut
  int32_t* piece_ptr;   // n_cut + 1
  uint32_t* pieces;     // n_pieces
  int8_t* fn_class;     // n^3
  int32_t* box;         // n^3
  int64_t* rowptr;      // n^3 + 1
  int32_t* colind;      // nnz
  int32_t* cut_rows;    // n_cut_rows
  int32_t* active_rows; // every active row (Standard Gauss variant)
  int32_t* tc_tasks;    // (row group, pencil) codes of the tensor-core interior kernel with interior rows
  int32_t* int_tiles;   // n_tiles: packed (i2, i3, chunk)
};

// Exact division of a non-negative 31-bit numerator by a fixed divisor d >= 2:
// floor(x / d) = umulhi(x, m) >> sh with s = ceil(log2 d), m = ceil(2^(31+s) / d) < 2^32 and
// sh = s - 1 (the rounding error x (m d - 2^(31+s)) / 2^(31+s) stays below 1/d).
struct FastDiv {
  uint32_t m;
  int sh;
};
inline FastDiv make_fastdiv(int d) {
  int s = 0;
  while ((1 << s) < d) ++s;
  const unsigned long long num = 1ull << (31 + s);
  return FastDiv{(uint32_t)((num + (unsigned long long)d - 1) / (unsigned long long)d), s - 1};
}
__device__ __forceinline__ int fdiv(int x, FastDiv f) { return (int)(__umulhi((uint32_t)x, f.m) >> f.sh); }

// Everything a kernel needs about one mesh, passed by value.
struct MeshView {
  int p, D;
  Dir1D dir[3];
  const double* gl;  // Gauss: x[p+1], w[p+1], x2[2p+1], w2[2p+1]
  Topo topo;
  int* status;
  FastDiv div_n1, div_n2;  // by the function counts n1, n2 (global index decoding)
};

// ---------------------------------------------------------------------------------------
// The mesh object behind the opaque ABI handle (host side).
struct sfa_mesh {
  sfa_mesh_desc desc{};
  int p = 0, D = 0;
  int ne[3] = {0, 0, 0}, n[3] = {0, 0, 0};
  int64_t nE = 0, nN = 0;
  MeshView view{};
  LevelSet ls{};
  double* gl = nullptr;
  int* status = nullptr;
  // classification results
  int64_t nnz = 0, n_cut = 0, n_pieces = 0, n_cut_rows = 0, n_pencils = 0;
  int64_t n_int_rows = 0, n_box_rows = 0, nnz_int = 0, n_cut_nonempty = 0, n_active = 0, n_tc_tasks = 0;
  int64_t cut_work[5] = {0, 0, 0, 0, 0};  // see sfa_mesh_info
  int64_t moment_slots = 0, moment_groups = 0;
  int64_t* scan_scratch = nullptr;
  int32_t* flags = nullptr;
  int64_t* rowlen = nullptr;
  int64_t* scan_out = nullptr;
  unsigned long long* counters = nullptr;
  // coefficient at points
  double *Csup = nullptr, *Cwq = nullptr, *cs1 = nullptr, *cs2 = nullptr, *coef_copy = nullptr;
  float *Cwq32 = nullptr, *Csup32 = nullptr;
  void* E = nullptr;
  void* host_values = nullptr;
  int64_t host_values_bytes = 0;
  double* bil_partial = nullptr;
  bool tables_ready = false, classified = false;
  std::string err;
  std::vector<void*> allocs;
  cudaEvent_t ev[12]{};
  // side stream of a formation (the cut-element matrices run there, concurrently with the
  // coefficient and interior stages) and its fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool ev_ok = false;
  bool ev_used[12]{};
  // classification buffers reused across classifications when large enough
  std::vector<std::pair<void*, size_t>> cls_pool;
  // adjoint work buffers (allocated on first use)
  double* adj[8]{};
  // tensor-core interior rows: G rows per MMA group, compiled q1 window KG per term (the
  // mesh needs Kg_mesh <= KG), band matrices of the WB1 rows (mass [WB00], stiffness
  // [WB11 | WB00]), TF32 head and tail
  int tc_G = 0, tc_KG = 0, tc_KQ = 0, tc_ngroups = 0, tc_Kg_mesh = 0;
  bool tc_ok = false;
  // bumped by every call that changes tables or pattern (invalidates captured batches)
  uint64_t gen = 0;
  // end-to-end calls (sfa_form_host): the cut rows run in kHostChunks chunks of the cut-row
  // list, and the values of every row up to a chunk's end go to the host on copy_st while the
  // next chunk computes.  chunk_rows / chunk_vals: first row and first value of each chunk's
  // copy (kHostChunks + 1 entries, host), valid for classification generation chunk_gen.
  static constexpr int kHostChunks = 8;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t chunk_ev[kHostChunks + 1]{};
  int64_t* chunk_dev = nullptr;
  std::vector<int64_t> chunk_rows, chunk_vals;
  uint64_t chunk_gen = ~0ull;
  float* tc_band[2] = {nullptr, nullptr};
  float* tc_dirop[2] = {nullptr, nullptr};  // q2 / q3 operand tables (directions 2, 3)
  // the same tables in BF16 (one copy), for the BF16 windows KG_bf, KQ_bf
  int tc_KG_bf = 0, tc_KQ_bf = 0;
  uint16_t* tc_band_bf[2] = {nullptr, nullptr};
  uint16_t* tc_dirop_bf[2] = {nullptr, nullptr};
};

// ---------------------------------------------------------------------------------------
// Host-side error helpers.
struct ErrCtx {
  std::string msg;
};

#define SFA_CUDA_TRY(ctx, call)                                                         \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess) {                                                            \
      (ctx).msg = std::string(#call) + ": " + cudaGetErrorString(_e);                   \
      return SFA_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

// ---------------------------------------------------------------------------------------
// Device helpers.
__device__ __forceinline__ void dev_set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// B-spline values and first derivatives of the p+1 functions span-p..span at x, for a
// knot vector given by an accessor knot(k).  Triangular Cox-de Boor scheme; derivatives
// from the degree p-1 values.  Requires knot(span) <= x < knot(span+1) (non-empty span).
template <typename KnotFn>
__device__ __forceinline__ void bspline_eval(const KnotFn& knot, int p, int span, double x, double* N,
                                             double* dN) {
  double left[SFA_MAXP + 1], right[SFA_MAXP + 1], Np[SFA_MAXP + 1];
  N[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = x - knot(span + 1 - j);
    right[j] = knot(span + j) - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double tmp = N[r] / (right[r + 1] + left[j - r]);
      N[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    N[j] = saved;
    if (j == p - 1) {
      for (int r = 0; r < p; ++r) Np[r] = N[r];
    }
  }
  if (p == 1) Np[0] = 1.0;
  for (int r = 0; r <= p; ++r) {
    int k = span - p + r;
    double v = 0.0;
    if (r >= 1) v += p * Np[r - 1] / (knot(k + p) - knot(k));
    if (r <= p - 1) v -= p * Np[r] / (knot(k + p + 1) - knot(k + 1));
    dN[r] = v;
  }
}

// Level set with a fixed evaluation order and no contraction (the classification is a
// discrete decision; the same sequence of correctly rounded operations is used by the
// CPU reference of the same rule).
__device__ __forceinline__ double ls_coord(const LevelSet& L, int d, int64_t k) {
  double t = __ddiv_rn((double)k, (double)L.Nk[d]);
  return __dadd_rn(L.lo[d], __dmul_rn(__dsub_rn(L.hi[d], L.lo[d]), t));
}

__device__ __forceinline__ double ls_phi(const LevelSet& L, double x, double y, double z) {
  switch (L.kind) {
    case SFA_LS_FULL:
      return -1.0;
    case SFA_LS_BALLS: {
      double out = 0.0;
      for (int b = 0; b < L.n_balls; ++b) {
        double dx = __dsub_rn(x, L.balls[4 * b + 0]);
        double dy = __dsub_rn(y, L.balls[4 * b + 1]);
        double dz = __dsub_rn(z, L.balls[4 * b + 2]);
        double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        double v = __dsub_rn(__dsqrt_rn(r2), L.balls[4 * b + 3]);
        out = (b == 0) ? v : fmin(out, v);
      }
      return out;
    }
    case SFA_LS_GYROID: {
      double X = __dmul_rn(L.freq, x), Y = __dmul_rn(L.freq, y), Z = __dmul_rn(L.freq, z);
      double a = __dmul_rn(sin(X), cos(Y));
      double b = __dmul_rn(sin(Y), cos(Z));
      double c = __dmul_rn(sin(Z), cos(X));
      return __dsub_rn(__dadd_rn(__dadd_rn(a, b), c), L.iso);
    }
    case SFA_LS_PLANE: {
      double a = __dmul_rn(L.nn[0], __dsub_rn(x, L.pt[0]));
      double b = __dmul_rn(L.nn[1], __dsub_rn(y, L.pt[1]));
      double c = __dmul_rn(L.nn[2], __dsub_rn(z, L.pt[2]));
      return __dadd_rn(__dadd_rn(a, b), c);
    }
  }
  return 1.0;
}

__device__ __forceinline__ double ls_phi_k(const LevelSet& L, int64_t k1, int64_t k2, int64_t k3) {
  if (L.kind == SFA_LS_GYROID && L.trig) {
    // same rounded arguments and operation order as ls_phi, with sin/cos looked up per axis
    const double* T = L.trig;
    const int64_t S = L.trig_stride;
    double a = __dmul_rn(T[0 * S + k1], T[3 * S + k2]);
    double b = __dmul_rn(T[2 * S + k2], T[5 * S + k3]);
    double c = __dmul_rn(T[4 * S + k3], T[1 * S + k1]);
    return __dsub_rn(__dadd_rn(__dadd_rn(a, b), c), L.iso);
  }
  return ls_phi(L, ls_coord(L, 0, k1), ls_coord(L, 1, k2), ls_coord(L, 2, k3));
}

// phi(x(k)) < 0, decided exactly as by the FP64 evaluation of ls_phi_k.  For the gyroid the
// float evaluation from the rounded tables decides whenever |phi32| > filt: each table value
// carries a relative error <= u = 2^-24, so the three products are within 3.01 u of the FP64
// products (|sin cos| <= 1) and the two additions and the subtraction add <= u (3 + |iso|)
// each; the total stays below 22 u (1 + |iso|) < 1.4e-6 (1 + |iso|), far under
// filt = 1e-5 (1 + |iso|), and the FP64 value is within 1e-15 of the exact one, so both
// signs agree.  Only samples with |phi32| <= filt are evaluated in FP64.
__device__ __forceinline__ bool ls_neg_k(const LevelSet& L, int64_t k1, int64_t k2, int64_t k3) {
  if (L.kind == SFA_LS_GYROID && L.trigf) {
    const float* T = L.trigf;
    const int64_t S = L.trig_stride;
    const float a = __fmul_rn(T[0 * S + k1], T[3 * S + k2]);
    const float b = __fmul_rn(T[2 * S + k2], T[5 * S + k3]);
    const float c = __fmul_rn(T[4 * S + k3], T[1 * S + k1]);
    const float v = __fsub_rn(__fadd_rn(__fadd_rn(a, b), c), L.isof);
    if (fabsf(v) > L.filt) return v < 0.f;
  }
  return ls_phi_k(L, k1, k2, k3) < 0.0;
}

// Records the process-wide last-error message (defined in api.cu).
void sfa_record_error(const std::string& msg);

// Count of kernels this library has launched (for reports).
extern std::atomic<long long> g_sfa_launches;
#define SFA_LAUNCHED(n) (g_sfa_launches += (n))

// ---------------------------------------------------------------------------------------
// Host-side launchers (defined in the translation unit of each stage).
cudaError_t launch_gauss(double* gl, int p, cudaStream_t st);
cudaError_t launch_trig(LevelSet L, double* trig, float* trigf, cudaStream_t st);
cudaError_t launch_points(const MeshView& M, int d, cudaStream_t st);
cudaError_t launch_wq_tables(const MeshView& M, int d, cudaStream_t st);
cudaError_t launch_products(const MeshView& M, int d, cudaStream_t st);
cudaError_t launch_piece_tables(const MeshView& M, int d, cudaStream_t st);
