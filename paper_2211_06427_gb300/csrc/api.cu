// C ABI of libsfa (declared in include/sfa.h): mesh lifetime, orchestration of the
// stages on the caller's stream, and host-side sizing.  No arithmetic of the method runs
// here; every step is a kernel in one of the stage translation units.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sfa_internal.cuh"

// launchers from the stage translation units
cudaError_t launch_elem_state(const LevelSet& L, int D, const int* ne, int8_t* state, int32_t* cut_flag, cudaStream_t st);
cudaError_t launch_scan_i32(const int32_t* in, int64_t n, int64_t* out, int64_t* scratch, cudaStream_t st);
cudaError_t launch_scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* scratch, cudaStream_t st);
cudaError_t launch_compact_i32(const int32_t* flag, const int64_t* scan, int64_t n, int32_t* out, int32_t* map,
                               cudaStream_t st);
cudaError_t launch_octree(const LevelSet& L, int D, const int* ne, const int32_t* cut_elems, int n_cut, int32_t* counts,
                          uint32_t* slab, int8_t* state, cudaStream_t st);
cudaError_t launch_copy_pieces(const uint32_t* slab, int D, int n_cut, const int32_t* piece_ptr, uint32_t* pieces,
                               cudaStream_t st);
cudaError_t launch_fn_class(int p, const int* ne, const int8_t* state, int8_t* fcls, cudaStream_t st);
cudaError_t launch_box_rowlen(int p, const int* ne, const int8_t* state, const int8_t* fcls, int32_t* box,
                              int64_t* rowlen, unsigned long long* counters, cudaStream_t st);
cudaError_t launch_colind(int p, const int* n, const int8_t* fcls, const int64_t* rowptr, int32_t* colind, cudaStream_t st);
cudaError_t launch_flag_class(const int8_t* fcls, int64_t n, int8_t want, int32_t* flag, cudaStream_t st);
cudaError_t launch_flag_pencils(const int8_t* fcls, const int* n, int32_t* flag, cudaStream_t st);
cudaError_t launch_flag_active(const int8_t* fcls, int64_t n, int32_t* flag, cudaStream_t st);
cudaError_t launch_slot_counts(const uint32_t* pieces, const int32_t* piece_ptr, int n_cut, int D, int p,
                               unsigned long long* counters, cudaStream_t st);
cudaError_t launch_flag_tc_tasks(const int8_t* fcls, const int32_t* pencils, int npen, int n1, int G, int ngroups,
                                 int32_t* flag, cudaStream_t st);
cudaError_t launch_coef(const MeshView& M, int coef_kind, double c0, const double* ck, double* scratch1,
                        double* scratch2, double* Csup, float* Csup32, double* Cwq, float* Cwq32, bool f64,
                        cudaStream_t st);
size_t interior_smem_bytes(int p, int nql1, int nql2, int nql3, int T, int L1MAX, bool stiff, bool fp64);
cudaError_t launch_interior(const MeshView& M, bool fp64, bool stiff, const void* Cwq, void* values, int n_pencils,
                            int T, int L1MAX, int Treg, int Lreg, cudaStream_t st);
void interior_tc_shape(int p, bool bf, int* G, int* KG, int* KQ);
cudaError_t launch_tc_band(const MeshView& M, bool bf, int G, int Kg, int KQ, int ngroups, void* band_mass,
                           void* band_stiff, void* dirop2, void* dirop3, cudaStream_t st);
cudaError_t launch_interior_tc(const MeshView& M, bool stiff, bool x3, bool bf, const float* Cwq, float* values,
                               const void* band, const void* dirop2, const void* dirop3, int Kg, int ngroups,
                               int n_pencils, int run, const int32_t* tasks, int n_tasks, cudaStream_t st);
size_t interior_reg_smem_bytes(int p, int T, int L1MAX, bool fp64);
cudaError_t launch_cut(const MeshView& M, const LevelSet& L, bool fp64, bool mom64, bool stiff, int coef_kind,
                       double c0, const double* ck, const void* Csup, void* E, void* values, int n_cut_elems,
                       int n_rows, int part, const int32_t* rows, int use_box, cudaStream_t st, int ci0 = 0);
cudaError_t launch_source_grid(const MeshView& M, double* F, cudaStream_t st);
cudaError_t launch_load(const MeshView& M, int source, int coef_kind, double c0, const double* ck, int variant,
                        int n_cut, const double* F, double* Eload, double* b, cudaStream_t st);
cudaError_t launch_i64_to_i32(const int64_t* in, int64_t n, int32_t* out, cudaStream_t st);
cudaError_t launch_bilinear(const int64_t* rowptr, const int32_t* colind, const int32_t* rows, int64_t nrows,
                            const void* values, bool fp64, const double* lam, const double* u, double* partial,
                            double* J, cudaStream_t st);
cudaError_t launch_backward(sfa_mesh* m, bool stiff, const double* lam, const double* u, const double* scale,
                            double* grad, cudaStream_t st);

std::atomic<long long> g_sfa_launches{0};

namespace {
std::mutex g_err_mu;
std::string g_err;
void set_global_err(const std::string& s) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = s;
}
}  // namespace

// The process-wide last-error message (sfa_get_last_error with a NULL mesh), for the
// translation units without a mesh.
void sfa_record_error(const std::string& msg) { set_global_err(msg); }

namespace {
inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// closed-form WQ layout bookkeeping (host copy of the integer rules used by the kernels)
inline bool h_full(int e, int ne) { return e == 0 || e == ne - 1; }
inline int h_qfirst(int e, int ne, int p) { return e == 0 ? 0 : (e < ne - 1 ? (p + 1) + 2 * (e - 1) : (p + 1) + 2 * (ne - 2)); }
inline int h_qcount(int e, int ne, int p) { return h_full(e, ne) ? p + 1 : 2; }
inline int h_qlo(int i, int ne, int p) { return h_qfirst(std::max(0, i - p), ne, p); }
inline int h_qhi(int i, int ne, int p) {
  int eh = std::min(ne - 1, i);
  return h_qfirst(eh, ne, p) + h_qcount(eh, ne, p);
}
}  // namespace

namespace {
sfa_status fail(sfa_mesh* m, sfa_status s, const std::string& msg) {
  if (m) m->err = msg;
  set_global_err(msg);
  return s;
}

template <typename T>
sfa_status dalloc(sfa_mesh* m, T** p, size_t count, std::vector<void*>* list = nullptr) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(m, SFA_ERR_OOM, std::string("cudaMalloc ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  (list ? list : &m->allocs)->push_back((void*)*p);
  return SFA_OK;
}

// Classification-sized buffers: slot k keeps its allocation across classifications and
// grows only when a larger size is needed (so re-classifying a mesh does not allocate).
template <typename T>
sfa_status cls_alloc(sfa_mesh* m, int slot, T** p, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if ((int)m->cls_pool.size() <= slot) m->cls_pool.resize(slot + 1, {nullptr, 0});
  auto& e = m->cls_pool[slot];
  if (e.second < bytes) {
    if (e.first) cudaFree(e.first);
    e = {nullptr, 0};
    cudaError_t err = cudaMalloc(&e.first, bytes);
    if (err != cudaSuccess) {
      cudaGetLastError();
      e.first = nullptr;
      return fail(m, SFA_ERR_OOM, std::string("cudaMalloc ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(err));
    }
    e.second = bytes;
  }
  *p = reinterpret_cast<T*>(e.first);
  return SFA_OK;
}

#define TRY(x)                   \
  do {                           \
    sfa_status _s = (x);         \
    if (_s != SFA_OK) return _s; \
  } while (0)
#define CU(m, call)                                                                    \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      cudaGetLastError();                                                              \
      return fail(m, SFA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    }                                                                                  \
  } while (0)

// Chunk length of the regular-pencil kernel: the largest T whose shared memory allows two
// CTAs per SM (or one), with the window length over all chunks.
int pick_Treg(const sfa_mesh* m, bool fp64, int* L1out) {
  const int cands[6] = {40, 34, 24, 16, 8, 4};
  for (int limit_kb : {110, 220}) {
    for (int T : cands) {
      int L1 = 0;
      for (int a = 0; a < m->n[0]; a += T) {
        int b = std::min(m->n[0], a + T);
        L1 = std::max(L1, h_qhi(b - 1, m->ne[0], m->p) - h_qlo(a, m->ne[0], m->p));
      }
      if (interior_reg_smem_bytes(m->p, T, L1, fp64) <= (size_t)limit_kb * 1024) {
        *L1out = L1;
        return T;
      }
    }
  }
  return -1;
}

int pick_T(const sfa_mesh* m, bool fp64, bool stiff, int* L1out) {
  const int cands[5] = {16, 8, 4, 2, 1};
  for (int limit_kb : {100, 220}) {
    for (int T : cands) {
      int L1 = 0;
      for (int a = 0; a < m->n[0]; a += T) {
        int b = std::min(m->n[0], a + T);
        L1 = std::max(L1, h_qhi(b - 1, m->ne[0], m->p) - h_qlo(a, m->ne[0], m->p));
      }
      size_t sm = interior_smem_bytes(m->p, m->view.dir[0].nql, m->view.dir[1].nql, m->view.dir[2].nql, T, L1, stiff, fp64);
      if (sm <= (size_t)limit_kb * 1024) {
        *L1out = L1;
        return T;
      }
    }
  }
  return -1;
}

// Window length over all chunks of T rows i1 (q1 points from the chunk's first row to the
// end of its last row).
int chunk_window(const sfa_mesh* m, int T) {
  int L1 = 0;
  for (int a = 0; a < m->n[0]; a += T) {
    const int b = std::min(m->n[0], a + T);
    L1 = std::max(L1, h_qhi(b - 1, m->ne[0], m->p) - h_qlo(a, m->ne[0], m->p));
  }
  return L1;
}

// Tile choices of the interior-row kernels per (degree, precision, operator), set by
// sfa_autotune; 0 keeps the built-in choice.
struct TuneChoice {
  int Treg = 0, Tgen = 0, tc_run = 0;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TuneChoice> g_tune;
TuneChoice tune_get(int p, int prec, int op) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(p, prec, op));
  return it == g_tune.end() ? TuneChoice{} : it->second;
}

// Instantiated graphs of sfa_form_batched, keyed by the exact argument list and the meshes'
// generations at capture time.
struct BatchEntry {
  int op = 0, prec = 0, device = 0;
  std::vector<sfa_mesh*> meshes;
  std::vector<void*> values;
  std::vector<uint64_t> gens;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_batch_mu;
std::vector<BatchEntry> g_batch;  // at most kBatchCache entries, oldest first
constexpr size_t kBatchCache = 8;

void batch_forget(sfa_mesh* m) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t k = 0; k < g_batch.size();) {
    if (std::find(g_batch[k].meshes.begin(), g_batch[k].meshes.end(), m) != g_batch[k].meshes.end()) {
      cudaGraphExecDestroy(g_batch[k].exec);
      g_batch.erase(g_batch.begin() + k);
    } else {
      ++k;
    }
  }
}

void rec(sfa_mesh* m, int k, cudaStream_t st) {
  if (m->ev_ok) {
    cudaEventRecord(m->ev[k], st);
    m->ev_used[k] = true;
  }
}
}  // namespace

extern "C" {

const char* sfa_status_string(sfa_status s) {
  switch (s) {
    case SFA_OK: return "ok";
    case SFA_ERR_INVALID_ARG: return "invalid argument";
    case SFA_ERR_CUDA: return "CUDA error";
    case SFA_ERR_OOM: return "out of device memory";
    case SFA_ERR_NOT_READY: return "tables or pattern not built";
    case SFA_ERR_WQ_SINGULAR: return "singular weighted-quadrature system";
    case SFA_ERR_TIMEOUT: return "device wait timed out";
    case SFA_ERR_DEVICE_BOUNDS: return "device index out of bounds";
    case SFA_ERR_UNSUPPORTED: return "unsupported in this build";
  }
  return "unknown status";
}

sfa_status sfa_get_last_error(const sfa_mesh* mesh, char* buf, size_t n) {
  if (!buf || n == 0) return SFA_ERR_INVALID_ARG;
  std::string s;
  if (mesh) s = mesh->err;
  else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    s = g_err;
  }
  std::snprintf(buf, n, "%s", s.c_str());
  return SFA_OK;
}

sfa_status sfa_create_mesh(const sfa_mesh_desc* desc, void* stream, sfa_mesh** out) {
  if (!desc || !out) return fail(nullptr, SFA_ERR_INVALID_ARG, "null desc or out");
  *out = nullptr;
  const sfa_mesh_desc& d = *desc;
  if (d.p < 2 || d.p > SFA_MAX_DEGREE) return fail(nullptr, SFA_ERR_INVALID_ARG, "degree p must be in [2, 6]");
  for (int k = 0; k < 3; ++k) {
    if (d.n_el[k] < 1 || d.n_el[k] > 1024) return fail(nullptr, SFA_ERR_INVALID_ARG, "n_el must be in [1, 1024]");
    if (!(d.hi[k] > d.lo[k])) return fail(nullptr, SFA_ERR_INVALID_ARG, "need lo < hi");
  }
  if (d.octree_depth < 0 || d.octree_depth > SFA_MAX_OCTREE_DEPTH)
    return fail(nullptr, SFA_ERR_INVALID_ARG, "octree_depth must be in [0, 4]");
  if (d.ls < SFA_LS_FULL || d.ls > SFA_LS_PLANE) return fail(nullptr, SFA_ERR_INVALID_ARG, "unknown level set");
  if (d.ls == SFA_LS_BALLS && (d.n_balls < 1 || d.n_balls > SFA_MAX_BALLS))
    return fail(nullptr, SFA_ERR_INVALID_ARG, "n_balls must be in [1, 64]");
  if (d.coef < SFA_COEF_CONST || d.coef > SFA_COEF_BSPLINE) return fail(nullptr, SFA_ERR_INVALID_ARG, "unknown coefficient kind");
  if (d.coef == SFA_COEF_BSPLINE && !d.coef_bspline)
    return fail(nullptr, SFA_ERR_INVALID_ARG, "B-spline coefficient pointer is null");
  int64_t nn = 1;
  for (int k = 0; k < 3; ++k) nn *= (d.n_el[k] + d.p);
  if (nn >= (int64_t)1 << 31) return fail(nullptr, SFA_ERR_INVALID_ARG, "too many functions for int32 column indices");

  sfa_mesh* m = new sfa_mesh();
  m->desc = d;
  m->p = d.p;
  m->D = d.octree_depth;
  cudaStream_t st = S(stream);
  m->nE = 1;
  m->nN = 1;
  for (int k = 0; k < 3; ++k) {
    m->ne[k] = d.n_el[k];
    m->n[k] = d.n_el[k] + d.p;
    m->nE *= m->ne[k];
    m->nN *= m->n[k];
  }
  const int p = m->p, q1 = p + 1, nb = 2 * p + 1;
  MeshView& V = m->view;
  V.p = p;
  V.div_n1 = make_fastdiv(m->n[0]);
  V.div_n2 = make_fastdiv(m->n[1]);
  V.D = m->D;
  sfa_status s = SFA_OK;
  auto cleanup = [&](sfa_status r) {
    sfa_destroy_mesh(m);
    return r;
  };
#define CTRY(x)                                   \
  do {                                            \
    sfa_status _s = (x);                          \
    if (_s != SFA_OK) return cleanup(_s);         \
  } while (0)
  for (int k = 0; k < 3; ++k) {
    Dir1D& D = V.dir[k];
    D.n_el = m->ne[k];
    D.n = m->n[k];
    D.nsup = m->ne[k] * q1;
    D.nq = h_qfirst(D.n_el - 1, D.n_el, p) + h_qcount(D.n_el - 1, D.n_el, p);
    int nql = 0;
    for (int i = 0; i < D.n; ++i) nql = std::max(nql, h_qhi(i, D.n_el, p) - h_qlo(i, D.n_el, p));
    D.nql = nql;
    D.nsl = q1 * q1;
    D.lo = d.lo[k];
    D.hi = d.hi[k];
    int64_t nrule = (int64_t)D.n * p * 2;
    CTRY(dalloc(m, &D.xb, D.n_el + 1));
    CTRY(dalloc(m, &D.U, D.n_el + 2 * p + 1));
    CTRY(dalloc(m, &D.t_sup, D.nsup));
    CTRY(dalloc(m, &D.w_sup, D.nsup));
    CTRY(dalloc(m, &D.B, (size_t)D.nsup * q1));
    CTRY(dalloc(m, &D.dB, (size_t)D.nsup * q1));
    CTRY(dalloc(m, &D.Bf, (size_t)D.nsup * q1));
    CTRY(dalloc(m, &D.wq_idx, D.nq));
    CTRY(dalloc(m, &D.qlo, D.n));
    CTRY(dalloc(m, &D.nqi, D.n));
    CTRY(dalloc(m, &D.w00, (size_t)D.n * D.nql));
    CTRY(dalloc(m, &D.w11, (size_t)D.n * D.nql));
    CTRY(dalloc(m, &D.WB00, (size_t)D.n * nb * D.nql));
    CTRY(dalloc(m, &D.WB11, (size_t)D.n * nb * D.nql));
    CTRY(dalloc(m, &D.WB00f, (size_t)D.n * nb * D.nql));
    CTRY(dalloc(m, &D.WB11f, (size_t)D.n * nb * D.nql));
    CTRY(dalloc(m, &D.dwq00, (size_t)nrule * D.nsl));
    CTRY(dalloc(m, &D.dwq11, (size_t)nrule * D.nsl));
    CTRY(dalloc(m, &D.WD00, (size_t)nrule * nb * D.nsl));
    CTRY(dalloc(m, &D.WD11, (size_t)nrule * nb * D.nsl));
    CTRY(dalloc(m, &D.WD00f, (size_t)nrule * nb * D.nsl));
    CTRY(dalloc(m, &D.WD11f, (size_t)nrule * nb * D.nsl));
    CTRY(dalloc(m, &D.G, (size_t)D.n_el * q1 * q1 * nb));
    CTRY(dalloc(m, &D.Gd, (size_t)D.n_el * q1 * q1 * nb));
    CTRY(dalloc(m, &D.Gf, (size_t)D.n_el * q1 * q1 * nb));
    CTRY(dalloc(m, &D.Gdf, (size_t)D.n_el * q1 * q1 * nb));
    CTRY(dalloc(m, &D.BZ, (size_t)D.n_el * q1 * q1));
    D.npos = (2 << m->D) - 1;
    CTRY(dalloc(m, &D.PT, (size_t)D.n_el * D.npos * q1 * (nb + q1 + 2)));
    CTRY(dalloc(m, &D.PTf, (size_t)D.n_el * D.npos * q1 * (nb + q1 + 2)));
    CTRY(dalloc(m, &D.P3, (size_t)D.n_el * D.npos * (3 * p + 1)));
    CTRY(dalloc(m, &D.P3f, (size_t)D.n_el * D.npos * (3 * p + 1)));
    CTRY(dalloc(m, &D.GE, (size_t)D.n_el * q1 * q1 * q1));
    CTRY(dalloc(m, &D.GEd, (size_t)D.n_el * q1 * q1 * q1));
    CTRY(dalloc(m, &D.GEf, (size_t)D.n_el * q1 * q1 * q1));
    CTRY(dalloc(m, &D.GEdf, (size_t)D.n_el * q1 * q1 * q1));
  }
  CTRY(dalloc(m, &m->gl, 2 * (q1 + nb)));
  V.gl = m->gl;
  CTRY(dalloc(m, &m->status, 1));
  V.status = m->status;
  // tensor-core interior rows: G rows i1 fill the 128 MMA rows (r, dj1); the q1 window of
  // a group starts at its first row's first point rounded down to 4 and covers the last
  // row's points.  The kernel is compiled for a window KG that covers every group's
  // (checked here, and again on the device) and for face supports of at most 3p+1 points,
  // which needs n_el >= p + 2 in directions 2 and 3.
  {
    const int n1 = m->n[0], ne1 = m->ne[0];
    int G = 0, KG = 0, KQ = 0, Gb = 0, KGb = 0, KQb = 0;
    interior_tc_shape(p, false, &G, &KG, &KQ);
    interior_tc_shape(p, true, &Gb, &KGb, &KQb);
    int Kg = 0;
    for (int a = 0; G > 0 && a < n1; a += G) {
      const int b = std::min(n1, a + G) - 1;
      const int kst = h_qlo(a, ne1, p) & ~3;
      Kg = std::max(Kg, h_qhi(b, ne1, p) - kst);
    }
    m->tc_G = G;
    m->tc_KG = KG;
    m->tc_KQ = KQ;
    m->tc_KG_bf = KGb;
    m->tc_KQ_bf = KQb;
    m->tc_ngroups = G > 0 ? (n1 + G - 1) / G : 0;
    m->tc_Kg_mesh = Kg;
    m->tc_ok = G > 0 && Kg <= KG && m->ne[1] >= p + 2 && m->ne[2] >= p + 2;
    CTRY(dalloc(m, &m->tc_band[0], (size_t)std::max(1, m->tc_ngroups) * 2 * 128 * KG));
    CTRY(dalloc(m, &m->tc_band[1], (size_t)std::max(1, m->tc_ngroups) * 2 * 128 * 2 * KG));
    // q2 / q3 operand tables: [i][copy][32 rows (kind, dj)][KQ points]
    for (int d = 1; d < 3; ++d) CTRY(dalloc(m, &m->tc_dirop[d - 1], (size_t)m->n[d] * 2 * 32 * std::max(8, KQ)));
    // BF16 copies (one rounding, no tail), laid out for the BF16 windows
    CTRY(dalloc(m, &m->tc_band_bf[0], (size_t)std::max(1, m->tc_ngroups) * 128 * KGb));
    CTRY(dalloc(m, &m->tc_band_bf[1], (size_t)std::max(1, m->tc_ngroups) * 128 * 2 * KGb));
    for (int d = 1; d < 3; ++d) CTRY(dalloc(m, &m->tc_dirop_bf[d - 1], (size_t)m->n[d] * 32 * std::max(16, KQb)));
  }
  // level set
  LevelSet& L = m->ls;
  L.kind = d.ls;
  L.n_balls = d.ls == SFA_LS_BALLS ? d.n_balls : 0;
  for (int b = 0; b < 4 * L.n_balls; ++b) L.balls[b] = d.balls[b];
  L.freq = d.gyroid_freq;
  L.iso = d.gyroid_iso;
  for (int k = 0; k < 3; ++k) {
    L.pt[k] = d.plane_pt[k];
    L.nn[k] = d.plane_n[k];
    L.lo[k] = d.lo[k];
    L.hi[k] = d.hi[k];
    L.Nk[k] = (int64_t)m->ne[k] << (m->D + 1);
  }
  L.trig = nullptr;
  L.trigf = nullptr;
  L.trig_stride = std::max(L.Nk[0], std::max(L.Nk[1], L.Nk[2])) + 1;
  if (L.kind == SFA_LS_GYROID) {
    double* trig = nullptr;
    float* trigf = nullptr;
    CTRY(dalloc(m, &trig, 6 * L.trig_stride));
    CTRY(dalloc(m, &trigf, 6 * L.trig_stride));
    if (launch_trig(L, trig, trigf, st) != cudaSuccess) return cleanup(fail(m, SFA_ERR_CUDA, "trig table kernel launch"));
    L.trig = trig;
    L.trigf = trigf;
    L.isof = (float)L.iso;
    L.filt = (float)(1e-5 * (1.0 + std::fabs(L.iso)));
  }
  // classification buffers of fixed size
  Topo& T = V.topo;
  CTRY(dalloc(m, &T.elem_state, m->nE));
  CTRY(dalloc(m, &T.elem_cut_id, m->nE));
  CTRY(dalloc(m, &T.fn_class, m->nN));
  CTRY(dalloc(m, &T.box, m->nN));
  CTRY(dalloc(m, &T.rowptr, m->nN + 1));
  CTRY(dalloc(m, &m->rowlen, m->nN));
  CTRY(dalloc(m, &m->flags, std::max(m->nE, m->nN)));
  CTRY(dalloc(m, &m->scan_out, std::max(m->nE, m->nN) + 1));
  CTRY(dalloc(m, &m->scan_scratch, std::max(m->nE, m->nN) / 4096 + 2));
  CTRY(dalloc(m, &m->counters, 16));
  // coefficient grids
  const Dir1D &A = V.dir[0], &B = V.dir[1], &C = V.dir[2];
  int64_t nsup3 = (int64_t)A.nsup * B.nsup * C.nsup;
  int64_t nq3 = (int64_t)A.nq * B.nq * C.nq;
  CTRY(dalloc(m, &m->Csup, nsup3));
  CTRY(dalloc(m, &m->Csup32, nsup3));
  CTRY(dalloc(m, &m->Cwq, nq3));
  CTRY(dalloc(m, &m->Cwq32, nq3));
  CTRY(dalloc(m, &m->cs1, std::max<int64_t>((int64_t)A.nsup * B.n * C.n, std::max(A.nsup, B.nsup))));
  CTRY(dalloc(m, &m->cs2, std::max<int64_t>((int64_t)A.nsup * B.nsup * C.n, std::max(A.nsup, B.nsup))));
  CTRY(dalloc(m, &m->bil_partial, 1024));
  if (cudaMemsetAsync(m->status, 0, sizeof(int), st) != cudaSuccess) return cleanup(fail(m, SFA_ERR_CUDA, "memset"));
  if (launch_gauss(m->gl, p, st) != cudaSuccess) return cleanup(fail(m, SFA_ERR_CUDA, "gauss kernel launch"));
  m->ev_ok = true;
  for (int k = 0; k < 12; ++k)
    if (cudaEventCreate(&m->ev[k]) != cudaSuccess) m->ev_ok = false;
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&m->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->join, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(fail(m, SFA_ERR_CUDA, "side stream"));
#undef CTRY
  (void)s;
  *out = m;
  return SFA_OK;
}

int64_t sfa_launch_count(void) { return (int64_t)g_sfa_launches.load(); }

sfa_status sfa_destroy_mesh(sfa_mesh* m) {
  if (!m) return SFA_OK;
  batch_forget(m);
  for (auto& e : m->cls_pool)
    if (e.first) cudaFree(e.first);
  for (void* p : m->allocs) cudaFree(p);
  for (int k = 0; k < 12; ++k)
    if (m->ev[k]) cudaEventDestroy(m->ev[k]);
  if (m->fork) cudaEventDestroy(m->fork);
  if (m->join) cudaEventDestroy(m->join);
  if (m->side) cudaStreamDestroy(m->side);
  for (int k = 0; k <= sfa_mesh::kHostChunks; ++k)
    if (m->chunk_ev[k]) cudaEventDestroy(m->chunk_ev[k]);
  if (m->copy_st) cudaStreamDestroy(m->copy_st);
  delete m;
  return SFA_OK;
}

sfa_status sfa_build_wq_tables(sfa_mesh* m, void* stream) {
  if (!m) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh");
  cudaStream_t st = S(stream);
  ++m->gen;
  rec(m, 0, st);
  CU(m, launch_points(m->view, -1, st));
  CU(m, launch_wq_tables(m->view, -1, st));
  CU(m, launch_products(m->view, -1, st));
  CU(m, launch_piece_tables(m->view, -1, st));
  CU(m, launch_tc_band(m->view, false, m->tc_G, m->tc_KG, m->tc_KQ, m->tc_ngroups, m->tc_band[0],
                       m->tc_band[1], m->tc_dirop[0], m->tc_dirop[1], st));
  CU(m, launch_tc_band(m->view, true, m->tc_G, m->tc_KG_bf, m->tc_KQ_bf, m->tc_ngroups, m->tc_band_bf[0],
                       m->tc_band_bf[1], m->tc_dirop_bf[0], m->tc_dirop_bf[1], st));
  rec(m, 1, st);
  m->tables_ready = true;
  return SFA_OK;
}

sfa_status sfa_classify_cells(sfa_mesh* m, void* stream) {
  if (!m) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh");
  cudaStream_t st = S(stream);
  m->classified = false;
  ++m->gen;
  Topo& T = m->view.topo;
  rec(m, 2, st);
  // elements
  CU(m, launch_elem_state(m->ls, m->D, m->ne, T.elem_state, m->flags, st));
  CU(m, launch_scan_i32(m->flags, m->nE, m->scan_out, m->scan_scratch, st));
  int64_t ncut = 0;
  CU(m, cudaMemcpyAsync(&ncut, m->scan_out + m->nE, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU(m, cudaStreamSynchronize(st));
  m->n_cut = ncut;
  TRY(cls_alloc(m, 0, &T.cut_elems, ncut));
  CU(m, launch_compact_i32(m->flags, m->scan_out, m->nE, T.cut_elems, T.elem_cut_id, st));
  // octree pieces
  int32_t* counts = nullptr;
  TRY(cls_alloc(m, 1, &counts, ncut + 1));
  TRY(cls_alloc(m, 2, &T.piece_ptr, ncut + 1));
  uint32_t* slab = nullptr;
  TRY(cls_alloc(m, 10, &slab, (size_t)std::max<int64_t>(ncut, 1) << (3 * m->D)));
  CU(m, launch_octree(m->ls, m->D, m->ne, T.cut_elems, (int)ncut, counts, slab, T.elem_state, st));
  int64_t* pscan = nullptr;
  TRY(cls_alloc(m, 3, &pscan, ncut + 1));
  int64_t* pscratch = nullptr;
  TRY(cls_alloc(m, 4, &pscratch, ncut / 4096 + 2));
  CU(m, launch_scan_i32(counts, ncut, pscan, pscratch, st));
  int64_t npieces = 0;
  CU(m, cudaMemcpyAsync(&npieces, pscan + ncut, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU(m, cudaStreamSynchronize(st));
  if (npieces >= ((int64_t)1 << 31)) return fail(m, SFA_ERR_INVALID_ARG, "too many octree pieces");
  m->n_pieces = npieces;
  CU(m, launch_i64_to_i32(pscan, ncut + 1, T.piece_ptr, st));
  TRY(cls_alloc(m, 5, &T.pieces, npieces));
  CU(m, launch_copy_pieces(slab, m->D, (int)ncut, T.piece_ptr, T.pieces, st));
  // functions, boxes, pattern
  CU(m, launch_fn_class(m->p, m->ne, T.elem_state, T.fn_class, st));
  CU(m, cudaMemsetAsync(m->counters, 0, 16 * sizeof(unsigned long long), st));
  CU(m, launch_box_rowlen(m->p, m->ne, T.elem_state, T.fn_class, T.box, m->rowlen, m->counters, st));
  CU(m, launch_slot_counts(T.pieces, T.piece_ptr, (int)ncut, m->D, m->p, m->counters + 9, st));
  CU(m, launch_scan_i64(m->rowlen, m->nN, T.rowptr, m->scan_scratch, st));
  int64_t nnz = 0;
  CU(m, cudaMemcpyAsync(&nnz, T.rowptr + m->nN, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU(m, cudaStreamSynchronize(st));
  m->nnz = nnz;
  TRY(cls_alloc(m, 6, &T.colind, nnz));
  CU(m, launch_colind(m->p, m->n, T.fn_class, T.rowptr, T.colind, st));
  // cut-row list
  CU(m, launch_flag_class(T.fn_class, m->nN, F_CUT, m->flags, st));
  CU(m, launch_scan_i32(m->flags, m->nN, m->scan_out, m->scan_scratch, st));
  int64_t ncr = 0;
  CU(m, cudaMemcpyAsync(&ncr, m->scan_out + m->nN, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU(m, cudaStreamSynchronize(st));
  m->n_cut_rows = ncr;
  TRY(cls_alloc(m, 7, &T.cut_rows, ncr));
  CU(m, launch_compact_i32(m->flags, m->scan_out, m->nN, T.cut_rows, nullptr, st));
  // every active row (the Standard Gauss variant forms them all as Gauss rows); the count is
  // the interior plus cut rows, known from the counters below
  TRY(cls_alloc(m, 11, &T.active_rows, m->nN));
  CU(m, launch_flag_active(T.fn_class, m->nN, m->flags, st));
  CU(m, launch_scan_i32(m->flags, m->nN, m->scan_out, m->scan_scratch, st));
  CU(m, launch_compact_i32(m->flags, m->scan_out, m->nN, T.active_rows, nullptr, st));
  // pencils with interior rows
  int64_t npen_all = (int64_t)m->n[1] * m->n[2];
  CU(m, launch_flag_pencils(T.fn_class, m->n, m->flags, st));
  CU(m, launch_scan_i32(m->flags, npen_all, m->scan_out, m->scan_scratch, st));
  int64_t npen = 0;
  CU(m, cudaMemcpyAsync(&npen, m->scan_out + npen_all, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU(m, cudaStreamSynchronize(st));
  m->n_pencils = npen;
  TRY(cls_alloc(m, 8, &T.int_tiles, npen));
  CU(m, launch_compact_i32(m->flags, m->scan_out, npen_all, T.int_tiles, nullptr, st));
  // tasks of the tensor-core interior kernel: (row group, pencil) pairs with interior rows
  m->n_tc_tasks = 0;
  if (m->tc_G > 0 && npen > 0) {
    const int64_t npair = (int64_t)m->tc_ngroups * npen;
    CU(m, launch_flag_tc_tasks(T.fn_class, T.int_tiles, (int)npen, m->n[0], m->tc_G, m->tc_ngroups, m->flags, st));
    CU(m, launch_scan_i32(m->flags, npair, m->scan_out, m->scan_scratch, st));
    int64_t ntk = 0;
    CU(m, cudaMemcpyAsync(&ntk, m->scan_out + npair, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CU(m, cudaStreamSynchronize(st));
    m->n_tc_tasks = ntk;
    TRY(cls_alloc(m, 12, &T.tc_tasks, ntk));
    CU(m, launch_compact_i32(m->flags, m->scan_out, npair, T.tc_tasks, nullptr, st));
  }
  // element matrices of cut elements (double-sized; the float path uses the same buffer);
  // each row padded to a multiple of 4 values (16-byte aligned rows)
  const int64_t q3 = (int64_t)(m->p + 1) * (m->p + 1) * (m->p + 1);
  double* Eb = nullptr;
  TRY(cls_alloc(m, 9, &Eb, (size_t)std::max<int64_t>(ncut, 1) * q3 * ((q3 + 3) / 4 * 4)));  // rows padded to 4
  m->E = Eb;
  unsigned long long cnt[16];
  CU(m, cudaMemcpyAsync(cnt, m->counters, sizeof(cnt), cudaMemcpyDeviceToHost, st));
  int status = 0;
  CU(m, cudaMemcpyAsync(&status, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  rec(m, 3, st);
  CU(m, cudaStreamSynchronize(st));
  m->n_int_rows = (int64_t)cnt[0];
  m->n_box_rows = (int64_t)cnt[2];
  m->nnz_int = (int64_t)cnt[3];
  m->n_active = m->n_int_rows + m->n_cut_rows;
  for (int k = 0; k < 5; ++k) m->cut_work[k] = (int64_t)cnt[4 + k];
  m->moment_slots = (int64_t)cnt[9];
  m->moment_groups = (int64_t)cnt[10];
  if (status == DEV_WQ_SINGULAR) return fail(m, SFA_ERR_WQ_SINGULAR, "a weighted-quadrature system was singular");
  if (status != 0) return fail(m, SFA_ERR_DEVICE_BOUNDS, "device status " + std::to_string(status));
  m->classified = true;
  return SFA_OK;
}

sfa_status sfa_get_pattern(const sfa_mesh* m, int64_t* n_rows, int64_t* nnz, const int64_t** rowptr,
                           const int32_t** colind) {
  if (!m) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh");
  if (!m->classified) return SFA_ERR_NOT_READY;
  if (n_rows) *n_rows = m->nN;
  if (nnz) *nnz = m->nnz;
  if (rowptr) *rowptr = m->view.topo.rowptr;
  if (colind) *colind = m->view.topo.colind;
  return SFA_OK;
}

sfa_status sfa_get_info(const sfa_mesh* m, sfa_mesh_info* info) {
  if (!m || !info) return fail(nullptr, SFA_ERR_INVALID_ARG, "null argument");
  if (!m->classified) return SFA_ERR_NOT_READY;
  info->n_rows = m->nN;
  info->nnz = m->nnz;
  info->n_interior_rows = m->n_int_rows;
  info->n_cut_rows = m->n_cut_rows;
  info->n_box_rows = m->n_box_rows;
  info->n_cut_elements = m->n_cut;
  info->n_pieces = m->n_pieces;
  info->nnz_interior = m->nnz_int;
  info->cut_gauss_pairs = m->cut_work[0];
  info->cut_elem_pairs = m->cut_work[1];
  info->box_points_fst = m->cut_work[2];
  info->box_points_st = m->cut_work[3];
  info->box_points_t = m->cut_work[4];
  info->moment_slots = m->moment_slots;
  info->moment_groups = m->moment_groups;
  return SFA_OK;
}

// One formation.  variant: SFA_VARIANT_DWQ (the method), SFA_VARIANT_HYBRID (cut rows take no
// DWQ box) or SFA_VARIANT_GAUSS (every active row through the Gauss row kernel, no WQ).
// serial: every stage on `st`, one after another (for per-stage device times).
// Device-to-host copy of the values overlapped with the cut rows (sfa_form_host).
struct HostCopy {
  void* dst;
  int esize;
};

static sfa_status form_impl(sfa_mesh* m, sfa_operator op, sfa_precision prec, void* values, cudaStream_t st,
                            const double* ck, bool record = true, int variant = SFA_VARIANT_DWQ,
                            bool serial = false, const HostCopy* hc = nullptr) {
  if (!m->tables_ready || !m->classified) return fail(m, SFA_ERR_NOT_READY, "build tables and classify first");
  if (!prec_valid(prec)) return fail(m, SFA_ERR_INVALID_ARG, "unknown precision");
  if (op != SFA_MASS && op != SFA_STIFFNESS) return fail(m, SFA_ERR_INVALID_ARG, "unknown operator");
  if (variant < SFA_VARIANT_DWQ || variant > SFA_VARIANT_GAUSS) return fail(m, SFA_ERR_INVALID_ARG, "unknown variant");
  if (!values && m->nnz > 0) return fail(m, SFA_ERR_INVALID_ARG, "null values");
  if (prec_tc(prec) && (reinterpret_cast<uintptr_t>(values) & 15) != 0)
    return fail(m, SFA_ERR_INVALID_ARG, "tensor-core precisions need a 16-byte aligned values buffer");
  const bool fp64 = prec == SFA_FP64, stiff = op == SFA_STIFFNESS;
  const bool tcm = prec_tc(prec);
  const bool mom64 = prec_mom64(prec);  // cut-cell moments in double
  const bool gauss = variant == SFA_VARIANT_GAUSS;
  // The cut-element matrices need only the coefficient's B-spline coefficients and the piece
  // tables, so they overlap the coefficient grid and the interior rows, which run on the
  // mesh's high-priority side stream (their blocks are scheduled first as the matrices'
  // blocks retire); the cut rows need both and follow the join.
  if (record) rec(m, 4, st);
  cudaStream_t hs = st;
  if (!serial) {
    CU(m, cudaEventRecord(m->fork, st));
    CU(m, cudaStreamWaitEvent(m->side, m->fork, 0));
    hs = m->side;
  }
  CU(m, launch_coef(m->view, m->desc.coef, m->desc.coef_const, ck, m->cs1, m->cs2, m->Csup, m->Csup32, m->Cwq,
                    m->Cwq32, fp64, hs));
  if (record) rec(m, 5, hs);
  if (m->n_pencils > 0 && !gauss) {
    int L1 = 0, Lreg = 0;
    int T = pick_T(m, fp64, stiff, &L1);
    int Treg = pick_Treg(m, fp64, &Lreg);
    if (T < 0) return fail(m, SFA_ERR_UNSUPPORTED, "interior tile does not fit in shared memory");
    const TuneChoice tch = tune_get(m->p, (int)prec, (int)op);
    if (tch.Treg > 0 && Treg > 0) {  // a tuned chunk, if it fits this mesh's window
      const int L = chunk_window(m, tch.Treg);
      if (interior_reg_smem_bytes(m->p, tch.Treg, L, fp64) <= 220 * 1024) Treg = tch.Treg, Lreg = L;
    }
    const int tc_run = tch.tc_run > 0 ? tch.tc_run : 4;
    if (tcm && m->tc_ok) {
      const bool bf = prec == SFA_BF16;
      CU(m, launch_interior_tc(m->view, stiff, prec_x3(prec), bf, m->Cwq32, (float*)values,
                               bf ? (const void*)m->tc_band_bf[stiff ? 1 : 0] : (const void*)m->tc_band[stiff ? 1 : 0],
                               bf ? (const void*)m->tc_dirop_bf[0] : (const void*)m->tc_dirop[0],
                               bf ? (const void*)m->tc_dirop_bf[1] : (const void*)m->tc_dirop[1], m->tc_Kg_mesh,
                               m->tc_ngroups, (int)m->n_pencils, tc_run, m->view.topo.tc_tasks, (int)m->n_tc_tasks,
                               hs));
    } else if (tcm) {
      // meshes below p + 2 elements in direction 2 or 3: every pencil on the CUDA cores
      CU(m, launch_interior(m->view, false, stiff, m->Cwq32, values, (int)m->n_pencils, T, L1, 0, 0, hs));
    } else {
      CU(m, launch_interior(m->view, fp64, stiff, fp64 ? (const void*)m->Cwq : (const void*)m->Cwq32, values,
                            (int)m->n_pencils, T, L1, Treg > 0 ? Treg : 0, Lreg, hs));
    }
  }
  if (record) rec(m, 6, hs);
  if (!serial) CU(m, cudaEventRecord(m->join, hs));
  const void* csup = fp64 ? (const void*)m->Csup : (const void*)m->Csup32;
  CU(m, launch_cut(m->view, m->ls, fp64, mom64, stiff, m->desc.coef, m->desc.coef_const, ck, csup, m->E, values,
                   (int)m->n_cut, 0, 0, nullptr, 0, st));
  if (record) rec(m, 7, st);
  if (!serial) CU(m, cudaStreamWaitEvent(st, m->join, 0));
  if (record) rec(m, 11, st);
  const int32_t* rows = gauss ? m->view.topo.active_rows : m->view.topo.cut_rows;
  const int nrows = (int)(gauss ? m->n_active : m->n_cut_rows);
  if (!hc) {
    CU(m, launch_cut(m->view, m->ls, fp64, mom64, stiff, m->desc.coef, m->desc.coef_const, ck, csup, m->E, values,
                     (int)m->n_cut, nrows, 1, rows, variant == SFA_VARIANT_DWQ ? 1 : 0, st));
    if (record) rec(m, 8, st);
    return SFA_OK;
  }
  // chunk c of the cut-row list, then the values of rows [chunk_rows[c], chunk_rows[c + 1])
  // (all final: interior rows joined above, cut rows of chunks <= c) to the host
  constexpr int K = sfa_mesh::kHostChunks;
  unsigned char* dv = static_cast<unsigned char*>(values);
  unsigned char* hv = static_cast<unsigned char*>(hc->dst);
  for (int c = 0; c < K; ++c) {
    const int a = (int)((int64_t)c * nrows / K), b = (int)((int64_t)(c + 1) * nrows / K);
    CU(m, launch_cut(m->view, m->ls, fp64, mom64, stiff, m->desc.coef, m->desc.coef_const, ck, csup, m->E, values,
                     (int)m->n_cut, b - a, 1, rows + a, 1, st));
    const int64_t v0 = m->chunk_vals[c], v1 = m->chunk_vals[c + 1];
    CU(m, cudaEventRecord(m->chunk_ev[c], st));
    CU(m, cudaStreamWaitEvent(m->copy_st, m->chunk_ev[c], 0));
    if (v1 > v0)
      CU(m, cudaMemcpyAsync(hv + v0 * hc->esize, dv + v0 * hc->esize, (size_t)(v1 - v0) * hc->esize,
                            cudaMemcpyDeviceToHost, m->copy_st));
  }
  CU(m, cudaEventRecord(m->chunk_ev[K], m->copy_st));
  CU(m, cudaStreamWaitEvent(st, m->chunk_ev[K], 0));
  if (record) rec(m, 8, st);
  return SFA_OK;
}

namespace {
// first row of each host-copy chunk (the first cut row of the chunk; 0 and nN at the ends)
// and its first value
__global__ void k_chunk_offsets(const int32_t* rows, int64_t n, const int64_t* rowptr, int64_t nN, int K,
                                int64_t* out) {
  const int c = threadIdx.x;
  if (c > K) return;
  const int64_t r = c == 0 ? 0 : (c == K ? nN : (int64_t)rows[(int64_t)c * n / K]);
  out[c] = r;
  out[K + 1 + c] = rowptr[r];
}
}  // namespace

// chunk offsets of the mesh's current classification (synchronous, once per classification)
static sfa_status host_chunks(sfa_mesh* m, cudaStream_t st) {
  constexpr int K = sfa_mesh::kHostChunks;
  if (m->chunk_gen == m->gen) return SFA_OK;
  if (!m->copy_st) {
    if (cudaStreamCreateWithFlags(&m->copy_st, cudaStreamNonBlocking) != cudaSuccess)
      return fail(m, SFA_ERR_CUDA, "copy stream");
    for (int k = 0; k <= K; ++k)
      if (cudaEventCreateWithFlags(&m->chunk_ev[k], cudaEventDisableTiming) != cudaSuccess)
        return fail(m, SFA_ERR_CUDA, "copy events");
  }
  if (!m->chunk_dev) TRY(dalloc(m, &m->chunk_dev, 2 * (K + 1)));
  k_chunk_offsets<<<1, 32, 0, st>>>(m->view.topo.cut_rows, m->n_cut_rows, m->view.topo.rowptr, m->nN, K,
                                    m->chunk_dev);
  SFA_LAUNCHED(1);
  CU(m, cudaGetLastError());
  std::vector<int64_t> h(2 * (K + 1));
  CU(m, cudaMemcpyAsync(h.data(), m->chunk_dev, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CU(m, cudaStreamSynchronize(st));
  m->chunk_rows.assign(h.begin(), h.begin() + K + 1);
  m->chunk_vals.assign(h.begin() + K + 1, h.end());
  m->chunk_gen = m->gen;
  return SFA_OK;
}

sfa_status sfa_form(sfa_mesh* m, sfa_operator op, sfa_precision prec, void* values, void* stream) {
  if (!m) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh");
  return form_impl(m, op, prec, values, S(stream), m->desc.coef_bspline);
}
sfa_status sfa_form_variant(sfa_mesh* m, sfa_operator op, sfa_precision prec, sfa_variant variant, void* values,
                            void* stream) {
  if (!m) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh");
  return form_impl(m, op, prec, values, S(stream), m->desc.coef_bspline, true, (int)variant);
}

sfa_status sfa_form_profile(sfa_mesh* m, sfa_operator op, sfa_precision prec, sfa_variant variant, void* values,
                            void* stream, float* ms4) {
  if (!m || !ms4) return fail(m, SFA_ERR_INVALID_ARG, "null argument");
  if (!m->ev_ok) return fail(m, SFA_ERR_CUDA, "stage events unavailable");
  cudaStream_t st = S(stream);
  TRY(form_impl(m, op, prec, values, st, m->desc.coef_bspline, true, (int)variant, true));
  auto el = [&](int a, int b) {
    float v = -1.0f;
    if (cudaEventSynchronize(m->ev[b]) != cudaSuccess || cudaEventElapsedTime(&v, m->ev[a], m->ev[b]) != cudaSuccess) {
      cudaGetLastError();
      return -1.0f;
    }
    return v;
  };
  ms4[0] = el(4, 5);
  ms4[1] = el(5, 6);
  ms4[2] = el(6, 7);
  ms4[3] = el(11, 8);
  for (int k = 0; k < 4; ++k)
    if (ms4[k] < 0.0f) return fail(m, SFA_ERR_CUDA, "stage timing failed");
  return SFA_OK;
}

sfa_status sfa_form_load(sfa_mesh* m, sfa_source source, sfa_variant variant, double* b, void* stream) {
  if (!m) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh");
  if (!m->tables_ready || !m->classified) return fail(m, SFA_ERR_NOT_READY, "build tables and classify first");
  if (!b) return fail(m, SFA_ERR_INVALID_ARG, "null load buffer");
  if (source != SFA_SRC_COEF && source != SFA_SRC_PAPER) return fail(m, SFA_ERR_INVALID_ARG, "unknown source");
  if (variant < SFA_VARIANT_DWQ || variant > SFA_VARIANT_GAUSS) return fail(m, SFA_ERR_INVALID_ARG, "unknown variant");
  cudaStream_t st = S(stream);
  const double* ck = m->desc.coef_bspline;
  if (source == SFA_SRC_COEF)
    CU(m, launch_coef(m->view, m->desc.coef, m->desc.coef_const, ck, m->cs1, m->cs2, m->Csup, m->Csup32, m->Cwq,
                      m->Cwq32, true, st));
  else
    CU(m, launch_source_grid(m->view, m->Csup, st));
  CU(m, launch_load(m->view, (int)source, m->desc.coef, m->desc.coef_const, ck, (int)variant, (int)m->n_cut, m->Csup,
                    static_cast<double*>(m->E), b, st));
  return SFA_OK;
}

sfa_status sfa_form_mass(sfa_mesh* m, sfa_precision prec, void* values, void* stream) {
  return sfa_form(m, SFA_MASS, prec, values, stream);
}
sfa_status sfa_form_stiffness(sfa_mesh* m, sfa_precision prec, void* values, void* stream) {
  return sfa_form(m, SFA_STIFFNESS, prec, values, stream);
}

sfa_status sfa_form_host(sfa_mesh* m, sfa_operator op, sfa_precision prec, const double* coef_host, void* values_host,
                         void* stream) {
  if (!m || !values_host) return fail(m, SFA_ERR_INVALID_ARG, "null argument");
  if (!m->classified) return fail(m, SFA_ERR_NOT_READY, "classify first");
  cudaStream_t st = S(stream);
  const double* ck = m->desc.coef_bspline;
  if (m->desc.coef == SFA_COEF_BSPLINE) {
    if (!coef_host) return fail(m, SFA_ERR_INVALID_ARG, "B-spline coefficients required");
    if (!m->coef_copy) TRY(dalloc(m, &m->coef_copy, m->nN));
    CU(m, cudaMemcpyAsync(m->coef_copy, coef_host, m->nN * sizeof(double), cudaMemcpyHostToDevice, st));
    ck = m->coef_copy;
  }
  int64_t bytes = m->nnz * (prec == SFA_FP64 ? 8 : 4);
  if (m->host_values_bytes < bytes) {
    if (m->host_values) {
      cudaFree(m->host_values);
      m->allocs.erase(std::remove(m->allocs.begin(), m->allocs.end(), m->host_values), m->allocs.end());
    }
    unsigned char* hv = nullptr;
    TRY(dalloc(m, &hv, (size_t)bytes));
    m->host_values = hv;
    m->host_values_bytes = bytes;
  }
  if (m->n_cut_rows > 0) {
    // the values go to the host in chunks, each while the next chunk of cut rows computes
    TRY(host_chunks(m, st));
    const HostCopy hc{values_host, prec == SFA_FP64 ? 8 : 4};
    TRY(form_impl(m, op, prec, m->host_values, st, ck, true, SFA_VARIANT_DWQ, false, &hc));
  } else {
    TRY(form_impl(m, op, prec, m->host_values, st, ck));
    CU(m, cudaMemcpyAsync(values_host, m->host_values, bytes, cudaMemcpyDeviceToHost, st));
  }
  CU(m, cudaStreamSynchronize(st));
  return SFA_OK;
}

sfa_status sfa_bilinear(const sfa_mesh* mc, sfa_precision prec, const void* values, const double* lam, const double* u,
                        double* J, void* stream) {
  sfa_mesh* m = const_cast<sfa_mesh*>(mc);
  if (!m || !values || !lam || !u || !J) return fail(m, SFA_ERR_INVALID_ARG, "null argument");
  if (!m->classified) return fail(m, SFA_ERR_NOT_READY, "classify first");
  CU(m, launch_bilinear(m->view.topo.rowptr, m->view.topo.colind, nullptr, m->nN, values, prec == SFA_FP64, lam, u,
                        m->bil_partial, J, S(stream)));
  return SFA_OK;
}

sfa_status sfa_form_backward(sfa_mesh* m, sfa_operator op, const double* lam, const double* u, const double* scale,
                             double* grad, void* stream) {
  if (!m || !lam || !u || !grad) return fail(m, SFA_ERR_INVALID_ARG, "null argument");
  if (!m->tables_ready || !m->classified) return fail(m, SFA_ERR_NOT_READY, "build tables and classify first");
  if (m->desc.coef != SFA_COEF_BSPLINE) return fail(m, SFA_ERR_INVALID_ARG, "backward needs a B-spline coefficient field");
  rec(m, 9, S(stream));
  cudaError_t e = launch_backward(m, op == SFA_STIFFNESS, lam, u, scale, grad, S(stream));
  rec(m, 10, S(stream));
  if (e == cudaErrorNotSupported) return fail(m, SFA_ERR_UNSUPPORTED, "backward not available");
  if (e != cudaSuccess) return fail(m, SFA_ERR_CUDA, std::string("backward: ") + cudaGetErrorString(e));
  return SFA_OK;
}

sfa_status sfa_table_size(const sfa_mesh* m, int dir, int which, int64_t* count, int32_t* stride) {
  if (!m || dir < 0 || dir > 2 || which < 0 || which > 3 || !count) return fail(nullptr, SFA_ERR_INVALID_ARG, "bad table query");
  const Dir1D& D = m->view.dir[dir];
  if (which < 2) {
    *count = (int64_t)D.n * D.nql;
    if (stride) *stride = D.nql;
  } else {
    *count = (int64_t)D.n * m->p * 2 * D.nsl;
    if (stride) *stride = D.nsl;
  }
  return SFA_OK;
}

static double* table_ptr(const sfa_mesh* m, int dir, int which) {
  const Dir1D& D = m->view.dir[dir];
  switch (which) {
    case 0: return D.w00;
    case 1: return D.w11;
    case 2: return D.dwq00;
    case 3: return D.dwq11;
  }
  return nullptr;
}

sfa_status sfa_export_table(const sfa_mesh* mc, int dir, int which, double* host_out, int64_t count, void* stream) {
  sfa_mesh* m = const_cast<sfa_mesh*>(mc);
  int64_t n = 0;
  TRY(sfa_table_size(m, dir, which, &n, nullptr));
  if (!host_out || count != n) return fail(m, SFA_ERR_INVALID_ARG, "table size mismatch");
  CU(m, cudaMemcpyAsync(host_out, table_ptr(m, dir, which), n * sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
  CU(m, cudaStreamSynchronize(S(stream)));
  return SFA_OK;
}

sfa_status sfa_import_table(sfa_mesh* m, int dir, int which, const double* host_in, int64_t count, void* stream) {
  int64_t n = 0;
  TRY(sfa_table_size(m, dir, which, &n, nullptr));
  if (!host_in || count != n) return fail(m, SFA_ERR_INVALID_ARG, "table size mismatch");
  if (!m->tables_ready) return fail(m, SFA_ERR_NOT_READY, "build tables first");
  ++m->gen;
  CU(m, cudaMemcpyAsync(table_ptr(m, dir, which), host_in, n * sizeof(double), cudaMemcpyHostToDevice, S(stream)));
  CU(m, launch_products(m->view, dir, S(stream)));
  CU(m, launch_tc_band(m->view, false, m->tc_G, m->tc_KG, m->tc_KQ, m->tc_ngroups, m->tc_band[0],
                       m->tc_band[1], m->tc_dirop[0], m->tc_dirop[1], S(stream)));
  CU(m, launch_tc_band(m->view, true, m->tc_G, m->tc_KG_bf, m->tc_KQ_bf, m->tc_ngroups, m->tc_band_bf[0],
                       m->tc_band_bf[1], m->tc_dirop_bf[0], m->tc_dirop_bf[1], S(stream)));
  CU(m, cudaStreamSynchronize(S(stream)));
  return SFA_OK;
}

sfa_status sfa_get_array(const sfa_mesh* m, const char* name, const void** ptr, int64_t* count, int32_t* dtype) {
  if (!m || !name || !ptr || !count || !dtype) return fail(nullptr, SFA_ERR_INVALID_ARG, "null argument");
  const Topo& T = m->view.topo;
  std::string s(name);
  if (s == "elem_state") { *ptr = T.elem_state; *count = m->nE; *dtype = 0; }
  else if (s == "fn_class") { *ptr = T.fn_class; *count = m->nN; *dtype = 0; }
  else if (s == "box") { *ptr = T.box; *count = m->nN; *dtype = 1; }
  else if (s == "cut_elems") { *ptr = T.cut_elems; *count = m->n_cut; *dtype = 1; }
  else if (s == "piece_ptr") { *ptr = T.piece_ptr; *count = m->n_cut + 1; *dtype = 1; }
  else if (s == "pieces") { *ptr = T.pieces; *count = m->n_pieces; *dtype = 2; }
  else if (s == "cut_rows") { *ptr = T.cut_rows; *count = m->n_cut_rows; *dtype = 1; }
  else if (s == "coef_sup") { *ptr = m->Csup; *count = (int64_t)m->view.dir[0].nsup * m->view.dir[1].nsup * m->view.dir[2].nsup; *dtype = 4; }
  else if (s == "gauss") { *ptr = m->gl; *count = 2 * (3 * m->p + 2); *dtype = 4; }
  else return fail(const_cast<sfa_mesh*>(m), SFA_ERR_INVALID_ARG, "unknown array " + s);
  if (!m->classified && s != "gauss" && s != "coef_sup") return SFA_ERR_NOT_READY;
  return SFA_OK;
}

sfa_status sfa_check_device_status(sfa_mesh* m, void* stream) {
  if (!m) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh");
  cudaStream_t st = S(stream);
  int status = 0;
  CU(m, cudaMemcpyAsync(&status, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(m, cudaStreamSynchronize(st));
  CU(m, cudaMemsetAsync(m->status, 0, sizeof(int), st));
  if (status == DEV_WQ_SINGULAR) return fail(m, SFA_ERR_WQ_SINGULAR, "a weighted-quadrature system was singular");
  if (status == DEV_TIMEOUT) return fail(m, SFA_ERR_TIMEOUT, "device wait timed out");
  if (status != 0) return fail(m, SFA_ERR_DEVICE_BOUNDS, "device bounds check failed");
  return SFA_OK;
}

sfa_status sfa_get_stage_ms(sfa_mesh* m, float* ms) {
  if (!m || !ms) return fail(nullptr, SFA_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < 7; ++k) ms[k] = -1.0f;
  if (!m->ev_ok) return SFA_OK;
  auto el = [&](int a, int b) {
    float v = -1.0f;
    if (m->ev_used[a] && m->ev_used[b] && cudaEventSynchronize(m->ev[b]) == cudaSuccess &&
        cudaEventElapsedTime(&v, m->ev[a], m->ev[b]) == cudaSuccess)
      return v;
    cudaGetLastError();
    return -1.0f;
  };
  ms[0] = el(0, 1);
  ms[1] = el(2, 3);
  ms[2] = el(4, 5);
  ms[3] = el(5, 6);
  ms[4] = el(4, 7);   // from the start of the formation (overlaps the two before)
  ms[5] = el(11, 8);  // after the join
  ms[6] = el(9, 10);
  return SFA_OK;
}

sfa_status sfa_autotune(sfa_mesh* m, sfa_operator op, sfa_precision prec, void* values, void* stream) {
  if (!m) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh");
  cudaStream_t st = S(stream);
  // one full formation first: coefficient grids, and the values are valid on return
  TRY(form_impl(m, op, prec, values, st, m->desc.coef_bspline, false));
  if (m->n_pencils == 0) return SFA_OK;
  const bool fp64 = prec == SFA_FP64, stiff = op == SFA_STIFFNESS;
  const bool tcm = prec_tc(prec);
  cudaEvent_t a = nullptr, b = nullptr;
  CU(m, cudaEventCreate(&a));
  CU(m, cudaEventCreate(&b));
  auto timed = [&](auto&& launch) -> float {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(a, st);
      if (launch() != cudaSuccess) return 1e30f;
      cudaEventRecord(b, st);
      float ms = 0.f;
      if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 1e30f;
      best = std::min(best, ms);
    }
    return best;
  };
  TuneChoice tc = tune_get(m->p, (int)prec, (int)op);
  float tbest = 1e30f;
  if (tcm && m->tc_ok) {
    for (int run : {1, 2, 4, 8}) {
      const float t = timed([&] {
        const bool bf = prec == SFA_BF16;
        return launch_interior_tc(
            m->view, stiff, prec_x3(prec), bf, m->Cwq32, (float*)values,
            bf ? (const void*)m->tc_band_bf[stiff ? 1 : 0] : (const void*)m->tc_band[stiff ? 1 : 0],
            bf ? (const void*)m->tc_dirop_bf[0] : (const void*)m->tc_dirop[0],
            bf ? (const void*)m->tc_dirop_bf[1] : (const void*)m->tc_dirop[1], m->tc_Kg_mesh, m->tc_ngroups,
            (int)m->n_pencils, run, m->view.topo.tc_tasks, (int)m->n_tc_tasks, st);
      });
      if (t < tbest) tbest = t, tc.tc_run = run;
    }
  } else if (!tcm) {
    int L1 = 0;
    const int T = pick_T(m, fp64, stiff, &L1);
    if (T < 0) return fail(m, SFA_ERR_UNSUPPORTED, "interior tile does not fit in shared memory");
    for (int Tr : {8, 16, 24, 34, 40}) {
      const int L = chunk_window(m, Tr);
      if (interior_reg_smem_bytes(m->p, Tr, L, fp64) > 220 * 1024) continue;
      const float t = timed([&] {
        return launch_interior(m->view, fp64, stiff, fp64 ? (const void*)m->Cwq : (const void*)m->Cwq32, values,
                               (int)m->n_pencils, T, L1, Tr, L, st);
      });
      if (t < tbest) tbest = t, tc.Treg = Tr;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaGetLastError();
  if (tbest >= 1e30f) return fail(m, SFA_ERR_CUDA, "autotune: no candidate ran");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[std::make_tuple(m->p, (int)prec, (int)op)] = tc;
  }
  // leave the values of the tuned configuration in the buffer
  TRY(form_impl(m, op, prec, values, st, m->desc.coef_bspline, false));
  CU(m, cudaStreamSynchronize(st));
  return SFA_OK;
}

sfa_status sfa_get_tuning(int p, sfa_operator op, sfa_precision prec, int32_t* out3) {
  if (!out3) return fail(nullptr, SFA_ERR_INVALID_ARG, "null argument");
  const TuneChoice tc = tune_get(p, (int)prec, (int)op);
  out3[0] = tc.Treg;
  out3[1] = tc.Tgen;
  out3[2] = tc.tc_run;
  return SFA_OK;
}

sfa_status sfa_form_batched(sfa_mesh* const* meshes, int count, sfa_operator op, sfa_precision prec,
                            void* const* values, void* stream) {
  if (!meshes || !values || count <= 0) return fail(nullptr, SFA_ERR_INVALID_ARG, "empty or null batch");
  for (int k = 0; k < count; ++k) {
    if (!meshes[k]) return fail(nullptr, SFA_ERR_INVALID_ARG, "null mesh in batch");
    if (!meshes[k]->tables_ready || !meshes[k]->classified)
      return fail(meshes[k], SFA_ERR_NOT_READY, "build tables and classify every mesh of the batch first");
    for (int j = 0; j < k; ++j)
      if (meshes[j] == meshes[k]) return fail(meshes[k], SFA_ERR_INVALID_ARG, "a mesh appears twice in the batch");
  }
  cudaStream_t st = S(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, SFA_ERR_CUDA, "cudaGetDevice failed");
  }
  std::vector<sfa_mesh*> ms(meshes, meshes + count);
  std::vector<void*> vs(values, values + count);
  std::vector<uint64_t> gens(count);
  for (int k = 0; k < count; ++k) gens[k] = meshes[k]->gen;
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto& e : g_batch)
      if (e.op == (int)op && e.prec == (int)prec && e.device == dev && e.meshes == ms && e.values == vs &&
          e.gens == gens) {
        exec = e.exec;
        break;
      }
  }
  if (!exec) {
    // capture: every mesh's formation on its own branch (up to 16 concurrent branches)
    const int ns = std::min(count, 16);
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> side(ns, nullptr);
    std::vector<cudaEvent_t> join(ns, nullptr);
    cudaEvent_t fork = nullptr;
    auto release = [&] {
      for (auto& x : side)
        if (x) cudaStreamDestroy(x);
      for (auto& x : join)
        if (x) cudaEventDestroy(x);
      if (fork) cudaEventDestroy(fork);
      if (origin) cudaStreamDestroy(origin);
    };
    bool ok = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (int s = 0; ok && s < ns; ++s)
      ok = cudaStreamCreateWithFlags(&side[s], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&join[s], cudaEventDisableTiming) == cudaSuccess;
    if (!ok || cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      release();
      return fail(nullptr, SFA_ERR_CUDA, "batch capture setup failed");
    }
    sfa_status r = SFA_OK;
    ok = cudaEventRecord(fork, origin) == cudaSuccess;
    for (int s = 0; ok && s < ns; ++s) ok = cudaStreamWaitEvent(side[s], fork, 0) == cudaSuccess;
    for (int k = 0; ok && r == SFA_OK && k < count; ++k)
      r = form_impl(meshes[k], op, prec, values[k], side[k % ns], meshes[k]->desc.coef_bspline, false);
    for (int s = 0; ok && s < ns; ++s)
      ok = cudaEventRecord(join[s], side[s]) == cudaSuccess && cudaStreamWaitEvent(origin, join[s], 0) == cudaSuccess;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
    if (r == SFA_OK && (!ok || ec != cudaSuccess || !graph)) r = fail(nullptr, SFA_ERR_CUDA, "batch capture failed");
    if (r == SFA_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      exec = nullptr;
      r = fail(nullptr, SFA_ERR_CUDA, "batch graph instantiation failed");
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    release();
    if (r != SFA_OK) return r;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (g_batch.size() >= kBatchCache) {
      cudaGraphExecDestroy(g_batch.front().exec);
      g_batch.erase(g_batch.begin());
    }
    BatchEntry e;
    e.op = (int)op;
    e.prec = (int)prec;
    e.device = dev;
    e.meshes = ms;
    e.values = vs;
    e.gens = gens;
    e.exec = exec;
    g_batch.push_back(e);
  }
  if (cudaGraphLaunch(exec, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, SFA_ERR_CUDA, "batch graph launch failed");
  }
  return SFA_OK;
}

}  // extern "C"

