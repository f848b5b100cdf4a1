/*
 * sfa.h — C ABI of libsfa: fast formation of mass and Laplace-stiffness matrices for
 * C^{p-1} tensor-product B-spline background meshes on a box cut by an implicit boundary
 * (Marussig, "Fast formation and assembly for spline-based 3D fictitious domain methods",
 * arXiv 2211.06427).  Rows are formed one test function at a time (Sec. 1, "row
 * assembly") by contracting per-test-function 1D weighted-quadrature tables with the
 * coefficient field, one direction at a time ("sum factorization"); cut test functions
 * use discontinuous weighted quadrature on their regular support (Sec. 2.2, Eq. 1) and
 * cut elements are integrated with Gauss points on octree sub-cells.
 *
 * Conventions shared by every entry point
 *  - Plain pointers only.  "device" pointers must be addressable by the current CUDA
 *    device (cudaMalloc / torch CUDA tensors); "host" pointers are ordinary memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Every
 *    call enqueues its kernels on `stream` and returns without waiting, except where a
 *    function says it synchronises.
 *  - Indexing: element e = e1 + n_el1 (e2 + n_el2 e3); function/row/column index
 *    i = i1 + n1 (i2 + n2 i3) with n_d = n_el_d + p; i1 is fastest.
 *  - Errors are returned, never raised or aborted.  A kernel that detects a bad state
 *    (singular weight system, out-of-range index) writes a per-mesh device status word;
 *    the next call that synchronises (sfa_classify_cells, sfa_check_device_status)
 *    reports it.  No kernel traps.
 *  - Ownership: the mesh owns every buffer it allocates (tables, pattern, scratch) and
 *    frees them in sfa_destroy_mesh.  Output buffers (`values`, `grad`, `J`) are
 *    caller-owned device memory.
 */
#ifndef SFA_H
#define SFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SFA_OK = 0,
  SFA_ERR_INVALID_ARG = 1,   /* a null pointer, a size out of range, an unknown enum */
  SFA_ERR_CUDA = 2,          /* a CUDA runtime call failed (message in sfa_get_last_error) */
  SFA_ERR_OOM = 3,           /* device allocation failed */
  SFA_ERR_NOT_READY = 4,     /* tables or pattern not built yet */
  SFA_ERR_WQ_SINGULAR = 5,   /* a weighted-quadrature exactness system was singular */
  SFA_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  SFA_ERR_DEVICE_BOUNDS = 7, /* a kernel found an index outside its buffer and skipped it */
  SFA_ERR_UNSUPPORTED = 8    /* a valid request this build does not implement */
} sfa_status;

typedef enum { SFA_LS_FULL = 0, SFA_LS_BALLS = 1, SFA_LS_GYROID = 2, SFA_LS_PLANE = 3 } sfa_levelset_kind;
typedef enum { SFA_COEF_CONST = 0, SFA_COEF_ANALYTIC = 1, SFA_COEF_BSPLINE = 2 } sfa_coef_kind;
/* Arithmetic of the row contractions.  SFA_FP64 writes double values; the others float.
 * The weight systems are always solved in double.
 *  SFA_FP32      every contraction in float with float accumulation, including the
 *                cut-cell moments;
 *  SFA_FP32_M64  as SFA_FP32 but the cut-cell moments are accumulated in double;
 *  SFA_TF32      as SFA_FP32, but the three directional contractions of the interior
 *                rows run on the tensor cores (tcgen05 kind::tf32) with both operands of
 *                each rounded to TF32 (10-bit mantissa) and FP32 accumulation;
 *  SFA_TF32X3    as SFA_TF32 with each operand split into a TF32 head and tail and the
 *                three leading products accumulated (close to FP32 accuracy);
 *  SFA_TF32X3_M64  the mixed form: interior rows as SFA_TF32X3 (tensor cores), cut-cell
 *                moments accumulated in double, the other cut-row work in float;
 *  SFA_BF16      as SFA_TF32, but the operands of the interior rows' three contractions are
 *                rounded to BF16 (8-bit mantissa) and multiplied on the tensor cores
 *                (tcgen05 kind::f16) with FP32 accumulation.
 *  The tensor-core precisions need values_dev 16-byte aligned (SFA_ERR_INVALID_ARG
 *  otherwise) and form every interior row on the CUDA cores on meshes with fewer than p + 2
 *  elements in direction 2 or 3.
 *  The measured error of each mode against the FP64 path is stated in the tests. */
typedef enum {
  SFA_FP64 = 0,
  SFA_FP32 = 1,
  SFA_TF32 = 2,
  SFA_TF32X3 = 3,
  SFA_FP32_M64 = 4,
  SFA_TF32X3_M64 = 5,
  SFA_BF16 = 6
} sfa_precision;
typedef enum { SFA_MASS = 0, SFA_STIFFNESS = 1 } sfa_operator;
/* The three formation methods the paper compares (Sec. 3.1):
 *  SFA_VARIANT_DWQ     the method: interior rows by weighted quadrature, the regular part of
 *                      each cut row by its DWQ box (Sec. 2.2), the rest by Gauss points;
 *  SFA_VARIANT_HYBRID  "Hybrid Gauss": interior rows by weighted quadrature, cut rows wholly
 *                      by Gauss points (no DWQ box);
 *  SFA_VARIANT_GAUSS   "Standard Gauss": every row by the (p+1)^3 Gauss points of each inside
 *                      support element and the octree pieces of each cut one; its matrix is
 *                      the element-loop Gauss matrix, formed row by row. */
typedef enum { SFA_VARIANT_DWQ = 0, SFA_VARIANT_HYBRID = 1, SFA_VARIANT_GAUSS = 2 } sfa_variant;

#define SFA_MAX_BALLS 64
#define SFA_MAX_DEGREE 6
#define SFA_MAX_OCTREE_DEPTH 4

/* Mesh description (copied by sfa_create_mesh; only coef_bspline is kept by reference).
 *  n_el[3]      elements per direction, 1 <= n_el <= 1024
 *  p            degree, 2 <= p <= SFA_MAX_DEGREE; knots are open and uniform on [lo, hi]
 *  ls           level set phi, domain = {phi < 0} (Sec. 2.1):
 *                 FULL   phi = -1
 *                 BALLS  phi = min_b (|x - c_b| - r_b), balls[4 b .. 4 b + 3] = (cx, cy, cz, r)
 *                 GYROID phi = sin(f x) cos(f y) + sin(f y) cos(f z) + sin(f z) cos(f x) - iso
 *                 PLANE  phi = n . (x - plane_pt)
 *  octree_depth D, 0 <= D <= SFA_MAX_OCTREE_DEPTH: cut cells are split into 8 children down
 *               to depth D; a still-cut leaf is kept iff phi(centre) < 0.
 *  coef         c(x): CONST coef_const; ANALYTIC 1 + 0.5 sin(2 pi x) cos(2 pi y) z;
 *               BSPLINE sum_k c_k N_k(x) on the mesh's own knots and degree, with
 *               coef_bspline a DEVICE pointer to n1*n2*n3 doubles (index k1 + n1 (k2 + n2 k3)),
 *               borrowed: it is read at every form / backward call and must outlive them. */
typedef struct {
  int32_t n_el[3];
  int32_t p;
  double lo[3], hi[3];
  int32_t ls;
  int32_t n_balls;
  double balls[4 * SFA_MAX_BALLS];
  double gyroid_freq, gyroid_iso;
  double plane_pt[3], plane_n[3];
  int32_t octree_depth;
  int32_t coef;
  double coef_const;
  const double* coef_bspline;
} sfa_mesh_desc;

typedef struct sfa_mesh sfa_mesh; /* opaque, library-owned */

/* Counts known after sfa_classify_cells (host values). */
typedef struct {
  int64_t n_rows;          /* n1*n2*n3, the full row index space */
  int64_t nnz;             /* structural entries of the active rows */
  int64_t n_interior_rows; /* rows formed purely by weighted quadrature */
  int64_t n_cut_rows;      /* active rows with a cut or empty element in their support */
  int64_t n_box_rows;      /* cut rows with a DWQ box (regular part by DWQ) */
  int64_t n_cut_elements;  /* cut elements that carry at least one octree piece */
  int64_t n_pieces;        /* octree pieces (inside sub-cells and kept leaves) */
  int64_t nnz_interior;    /* entries in interior rows */
  /* work of the cut rows, summed over them: */
  int64_t cut_gauss_pairs; /* inside support elements outside the row's box (element Gauss) */
  int64_t cut_elem_pairs;  /* cut support elements (a row of the element matrix each) */
  int64_t box_points_fst;  /* DWQ boxes: points m_f m_s m_t (f the box direction, s < t the others) */
  int64_t box_points_st;   /*            m_s m_t */
  int64_t box_points_t;    /*            m_t */
  /* octree pieces of the cut elements, summed over them: nonempty slots (level, a_mid,
   * a_out) and groups (level, a_out) of the pieces, in each element's cyclic direction order
   * (inner, middle, outer) with the least moment work (the work of the cut-element moments): */
  int64_t moment_slots;
  int64_t moment_groups;
} sfa_mesh_info;

/* Validate `desc`, allocate the mesh and its 1D point data.  No kernel runs yet. */
sfa_status sfa_create_mesh(const sfa_mesh_desc* desc, void* stream, sfa_mesh** out);

/* Sec. 1 / Sec. 2.2 steps 1, 3-6: Gauss superset, WQ point subset, B-spline values, and
 * for every 1D test function the standard WQ weights (mass w00 and derivative w11) and
 * every one-sided DWQ rule (all interior knots of its support, both sides).  FP64. */
sfa_status sfa_build_wq_tables(sfa_mesh* mesh, void* stream);

/* Sec. 2.1 / Sec. 2.2 step 2 and the cut-cell rule: element states, octree pieces of cut
 * elements, function types, the DWQ box of every cut function, and the CSR pattern
 * (row i active iff not exterior; columns = active j with |j_d - i_d| <= p, ascending).
 * SYNCHRONISES `stream` once to learn nnz and sizes; also reports any device status. */
sfa_status sfa_classify_cells(sfa_mesh* mesh, void* stream);

/* Mesh-owned device pattern: rowptr (n_rows + 1 int64), colind (nnz int32). */
sfa_status sfa_get_pattern(const sfa_mesh* mesh, int64_t* n_rows, int64_t* nnz,
                           const int64_t** rowptr_dev, const int32_t** colind_dev);
sfa_status sfa_get_info(const sfa_mesh* mesh, sfa_mesh_info* info);

/* Form the matrix values on the pattern (Sec. 1 row assembly, Sec. 2.2 Eq. 1):
 * coefficient at the quadrature points, interior rows by WQ + sum factorisation, cut rows
 * by the DWQ box plus Gauss points on the remaining inside elements and on the octree
 * pieces of cut elements.  `values_dev`: caller-owned device buffer of nnz doubles
 * (SFA_FP64) or floats (other precisions), every entry written.  Never allocates or
 * synchronises. */
sfa_status sfa_form(sfa_mesh* mesh, sfa_operator op, sfa_precision prec, void* values_dev, void* stream);
sfa_status sfa_form_mass(sfa_mesh* mesh, sfa_precision prec, void* values_dev, void* stream);
/* As sfa_form with the formation method chosen (sfa_form is SFA_VARIANT_DWQ).  Same pattern,
 * same buffer contract; SFA_ERR_INVALID_ARG for an unknown variant. */
sfa_status sfa_form_variant(sfa_mesh* mesh, sfa_operator op, sfa_precision prec, sfa_variant variant,
                            void* values_dev, void* stream);
/* As sfa_form_variant, but every stage runs on `stream` one after another, and the device time
 * of each (CUDA events) is written to ms4 (host floats): [0] coefficient at the points,
 * [1] interior rows, [2] cut-element matrices, [3] cut rows.  Synchronises `stream`.  For
 * per-kernel rooflines; the stages of sfa_form overlap. */
sfa_status sfa_form_profile(sfa_mesh* mesh, sfa_operator op, sfa_precision prec, sfa_variant variant,
                            void* values_dev, void* stream, float* ms4);
sfa_status sfa_form_stiffness(sfa_mesh* mesh, sfa_precision prec, void* values_dev, void* stream);

/* Load-vector source f: the mesh's coefficient field c, or the target function of the
 * paper's experiment f = sin(2xz) cos(3yz) (Sec. 3.1). */
typedef enum { SFA_SRC_COEF = 0, SFA_SRC_PAPER = 1 } sfa_source;

/* Load vector b_i = "int f B_i" by the rules of the formation (Sec. 1: the test function is
 * folded into the weighted-quadrature weights; Sec. 2.2, Eq. 1 for cut rows): interior rows
 * sum_q w_i1 w_i2 w_i3 f(x_q) over their WQ grid, cut rows the same over their DWQ box plus
 * f B_i at the Gauss points of the remaining inside support elements and of the octree pieces
 * of the cut ones.  `variant` as in sfa_form_variant.  b_dev: caller-owned device buffer of
 * n_rows doubles, every entry written (exterior rows 0).  FP64.  Uses the mesh's coefficient
 * grid and cut-element buffers as scratch (the next formation recomputes them), so it never
 * allocates; it does not synchronise. */
sfa_status sfa_form_load(sfa_mesh* mesh, sfa_source source, sfa_variant variant, double* b_dev, void* stream);

/* Adjoint with respect to the B-spline coefficient field (coef = SFA_COEF_BSPLINE):
 * grad_dev[k] = dJ/dc_k for J = lambda^T A(c) u, lambda/u/grad: n_rows doubles on the
 * device.  J is linear in c, so this is exact.  If scale_dev is not NULL the gradient is
 * multiplied by *scale_dev (a device double).  grad_dev is overwritten.  FP64. */
sfa_status sfa_form_backward(sfa_mesh* mesh, sfa_operator op, const double* lambda_dev, const double* u_dev,
                             const double* scale_dev, double* grad_dev, void* stream);

/* J = lambda^T A u for formed values (double for SFA_FP64, float otherwise); *J_dev is a
 * device double, overwritten. */
sfa_status sfa_bilinear(const sfa_mesh* mesh, sfa_precision prec, const void* values_dev,
                        const double* lambda_dev, const double* u_dev, double* J_dev, void* stream);

/* End-to-end call with host buffers: copies coef_host (n_rows doubles, or NULL for
 * non-B-spline coefficients) to the mesh's device copy, forms, and copies the values to
 * values_host (nnz doubles or floats; pinned memory lets the copies run asynchronously).  With
 * cut rows, the cut rows run in chunks and each finished row range is copied while the next
 * chunk computes, on a copy stream the mesh owns; the first call after a classification
 * synchronises once to learn the chunk boundaries.  Synchronises `stream` before returning. */
sfa_status sfa_form_host(sfa_mesh* mesh, sfa_operator op, sfa_precision prec, const double* coef_host,
                         void* values_host, void* stream);

/* Many meshes, one launch.  Forms mesh k's matrix (operator op, precision prec) into
 * values_dev[k] for k < count, as sfa_form would, with every mesh's formation on its own
 * branch of one CUDA graph (up to 16 branches run concurrently) launched on `stream`.  The
 * paper forms one mesh at a time; batching serves many small independent meshes, whose
 * single launches would leave the GPU mostly idle.
 *  - Every mesh must have its tables built and be classified; a mesh may appear once.
 *  - The first call with a given argument list captures the graph; later calls with the
 *    same meshes, value pointers, op and precision replay it (a small cache of the 8 most
 *    recent lists).  Rebuilding a mesh's tables, reclassifying it, importing a table or
 *    destroying it invalidates the batches that contain it.
 *  - The first call for an argument list is not itself capturable; replays only enqueue.
 *  - Errors: SFA_ERR_INVALID_ARG (null or repeated meshes, count <= 0), SFA_ERR_NOT_READY,
 *    SFA_ERR_CUDA (capture or launch failed; nothing was enqueued). */
sfa_status sfa_form_batched(sfa_mesh* const* meshes, int count, sfa_operator op, sfa_precision prec,
                            void* const* values_dev, void* stream);

/* Autotuner for the interior-row tiles: times the candidate chunk lengths of the regular-
 * pencil kernel (FP64 / FP32) or the task run lengths of the tensor-core kernel (TF32 /
 * TF32X3) on this mesh and keeps the fastest for (p, op, prec), process-wide; later forms of
 * every mesh with that degree use it where it fits.  values_dev receives this mesh's matrix
 * (it is formed before and after the trials).  Synchronises `stream`.  The paper has no
 * counterpart (its kernels are serial). */
sfa_status sfa_autotune(sfa_mesh* mesh, sfa_operator op, sfa_precision prec, void* values_dev, void* stream);

/* The tuned choice for (p, op, prec): out3 = {regular-pencil chunk, generic chunk,
 * tensor-core run length}, 0 where nothing was tuned. */
sfa_status sfa_get_tuning(int p, sfa_operator op, sfa_precision prec, int32_t* out3);

/* Weight tables for the parity decomposition (export: device -> host; import: host ->
 * device, then the product tables are rebuilt).  which: 0 = w00, 1 = w11 (standard rules,
 * layout [n_d][nql], local WQ point index), 2 = dwq00, 3 = dwq11 (one-sided rules, layout
 * [n_d][p][2][nsl], candidate b = e_lo + 1 + slot, side 0 low / 1 high, local superset
 * index within the support).  Sizes in doubles via sfa_table_size.  Export/import
 * synchronise `stream`. */
sfa_status sfa_table_size(const sfa_mesh* mesh, int dir, int which, int64_t* count, int32_t* stride);
sfa_status sfa_export_table(const sfa_mesh* mesh, int dir, int which, double* host_out, int64_t count, void* stream);
sfa_status sfa_import_table(sfa_mesh* mesh, int dir, int which, const double* host_in, int64_t count, void* stream);

/* Introspection of mesh-owned device arrays by name (for tests and tools): "elem_state"
 * (int8 per element: 0 out, 1 in, 2 cut with pieces, 3 cut without), "fn_class" (int8 per
 * function: 0 exterior, 1 interior, 2 cut), "box" (int32 per function: -1 or
 * d | side << 2 | b << 3), "cut_elems" (int32 element ids), "piece_ptr" (int32, per cut
 * element + 1), "pieces" (uint32: level | a1 << 4 | a2 << 10 | a3 << 16, local cell
 * coordinates at that level).  dtype: 0 int8, 1 int32, 2 uint32, 3 int64, 4 double. */
sfa_status sfa_get_array(const sfa_mesh* mesh, const char* name, const void** dev_ptr, int64_t* count,
                         int32_t* dtype);

/* Synchronise `stream` and report (and clear) the mesh's device status word. */
sfa_status sfa_check_device_status(sfa_mesh* mesh, void* stream);

/* Milliseconds of the last call's stages (CUDA events on its stream), for reports:
 * [0] tables, [1] classification+pattern, [2] coefficient at points, [3] interior rows,
 * [4] cut-element matrices, [5] cut rows, [6] backward.  Synchronises on the events. */
sfa_status sfa_get_stage_ms(sfa_mesh* mesh, float* ms7);

/* J = lambda^T A u for a CSR matrix, allocating nothing (no mesh needed).  The paper has
 * no counterpart: this is a service for callers that may not call cudaMalloc where they
 * need the reduction (a solver inside a memory pool it does not own, a host callback
 * that must not touch the allocator).  rowptr (n_rows + 1 int64), colind (nnz int32),
 * values (double for SFA_FP64, float otherwise), lambda and u (n_rows doubles) are device
 * arrays; *J_dev (a device double) is overwritten.  Scratch is one double per row in a
 * fixed array compiled into the library, so n_rows must not exceed 1048576 (8 MiB, held
 * on every GPU that loads the library until the process exits); larger inputs return
 * SFA_ERR_INVALID_ARG before any work.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is cached per device for the life of the process,
 * so it assumes the device's primary context is never reset (no cudaDeviceReset between
 * calls).  All calls share the array: calls that overlap on the GPU race.  Nothing needs
 * clearing between calls (each call writes every entry it reads).  An error left pending by
 * earlier work on the calling thread is returned as SFA_ERR_CUDA before any launch, with its
 * message in sfa_get_last_error(NULL, ...). */
sfa_status sfa_bilinear_static(const int64_t* rowptr_dev, const int32_t* colind_dev, int64_t n_rows, sfa_precision prec,
                               const void* values_dev, const double* lambda_dev, const double* u_dev, double* J_dev,
                               void* stream);

/* Number of kernels this library has launched since it was loaded (all meshes). */
int64_t sfa_launch_count(void);

sfa_status sfa_destroy_mesh(sfa_mesh* mesh);
const char* sfa_status_string(sfa_status s);
/* Last error message recorded on this mesh (or the global one if mesh is NULL). */
sfa_status sfa_get_last_error(const sfa_mesh* mesh, char* buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* SFA_H */
