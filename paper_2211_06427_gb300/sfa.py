"""Python binding of libsfa's C ABI (include/sfa.h): argument marshalling only.

Every computation happens in the CUDA library; this module turns workload descriptions
(``paper_2211_06427_gb300.synthetic``) into ``sfa_mesh_desc`` structs, passes device
pointers of torch tensors and the current torch stream, and wraps mesh-owned device
arrays as zero-copy torch views.  There is no CPU fallback: importing this module fails
if libsfa.so has not been built.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsfa.so")

SFA_MASS, SFA_STIFFNESS = 0, 1
SFA_FP64, SFA_FP32, SFA_TF32, SFA_TF32X3, SFA_FP32_M64, SFA_TF32X3_M64, SFA_BF16 = 0, 1, 2, 3, 4, 5, 6
LS = {"full": 0, "ball": 1, "balls": 1, "gyroid": 2, "plane": 3}
COEF = {"const": 0, "analytic": 1, "bspline": 2}
OPS = {"mass": SFA_MASS, "stiffness": SFA_STIFFNESS}
PRECS = {"fp64": SFA_FP64, "fp32": SFA_FP32, "tf32": SFA_TF32, "tf32x3": SFA_TF32X3, "fp32_m64": SFA_FP32_M64,
         "tf32x3_m64": SFA_TF32X3_M64, "bf16": SFA_BF16}
MAX_BALLS = 64

EXPORTED = [
    "sfa_create_mesh", "sfa_build_wq_tables", "sfa_classify_cells", "sfa_get_pattern", "sfa_get_info",
    "sfa_form", "sfa_form_mass", "sfa_form_stiffness", "sfa_form_backward", "sfa_bilinear", "sfa_form_host",
    "sfa_table_size", "sfa_export_table", "sfa_import_table", "sfa_get_array", "sfa_check_device_status",
    "sfa_get_stage_ms", "sfa_destroy_mesh", "sfa_status_string", "sfa_get_last_error", "sfa_launch_count",
    "sfa_bilinear_static", "sfa_form_batched", "sfa_autotune", "sfa_get_tuning", "sfa_form_variant",
    "sfa_form_profile", "sfa_form_load",
]
SOURCES = {"coef": 0, "paper": 1}
VARIANTS = {"dwq": 0, "hybrid": 1, "gauss": 2}


class MeshDesc(ctypes.Structure):
    _fields_ = [
        ("n_el", ctypes.c_int32 * 3), ("p", ctypes.c_int32), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("ls", ctypes.c_int32), ("n_balls", ctypes.c_int32), ("balls", ctypes.c_double * (4 * MAX_BALLS)),
        ("gyroid_freq", ctypes.c_double), ("gyroid_iso", ctypes.c_double),
        ("plane_pt", ctypes.c_double * 3), ("plane_n", ctypes.c_double * 3),
        ("octree_depth", ctypes.c_int32), ("coef", ctypes.c_int32), ("coef_const", ctypes.c_double),
        ("coef_bspline", ctypes.c_void_p),
    ]


class MeshInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "n_rows", "nnz", "n_interior_rows", "n_cut_rows", "n_box_rows", "n_cut_elements", "n_pieces", "nnz_interior",
        "cut_gauss_pairs", "cut_elem_pairs", "box_points_fst", "box_points_st", "box_points_t",
        "moment_slots", "moment_groups")]


class SfaError(RuntimeError):
    pass


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libsfa.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "sfa_create_mesh": [ctypes.POINTER(MeshDesc), vp, ctypes.POINTER(vp)],
        "sfa_build_wq_tables": [vp, vp],
        "sfa_classify_cells": [vp, vp],
        "sfa_get_pattern": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(vp)],
        "sfa_get_info": [vp, ctypes.POINTER(MeshInfo)],
        "sfa_form": [vp, ctypes.c_int, ctypes.c_int, vp, vp],
        "sfa_form_mass": [vp, ctypes.c_int, vp, vp],
        "sfa_form_stiffness": [vp, ctypes.c_int, vp, vp],
        "sfa_form_backward": [vp, ctypes.c_int, vp, vp, vp, vp, vp],
        "sfa_bilinear": [vp, ctypes.c_int, vp, vp, vp, vp, vp],
        "sfa_form_host": [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp],
        "sfa_table_size": [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(i64), ctypes.POINTER(i32)],
        "sfa_export_table": [vp, ctypes.c_int, ctypes.c_int, vp, i64, vp],
        "sfa_import_table": [vp, ctypes.c_int, ctypes.c_int, vp, i64, vp],
        "sfa_get_array": [vp, ctypes.c_char_p, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i32)],
        "sfa_check_device_status": [vp, vp],
        "sfa_get_stage_ms": [vp, ctypes.POINTER(ctypes.c_float)],
        "sfa_destroy_mesh": [vp],
        "sfa_status_string": [ctypes.c_int],
        "sfa_get_last_error": [vp, ctypes.c_char_p, ctypes.c_size_t],
        "sfa_launch_count": [],
        "sfa_bilinear_static": [vp, vp, i64, ctypes.c_int, vp, vp, vp, vp, vp],
        "sfa_form_batched": [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp), vp],
        "sfa_autotune": [vp, ctypes.c_int, ctypes.c_int, vp, vp],
        "sfa_get_tuning": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(i32)],
        "sfa_form_variant": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp],
        "sfa_form_load": [vp, ctypes.c_int, ctypes.c_int, vp, vp],
        "sfa_form_profile": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.POINTER(ctypes.c_float)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "sfa_status_string" else ctypes.c_int
    lib.sfa_launch_count.restype = ctypes.c_int64
    return lib


def bilinear_static(rowptr, colind, values, lam, u, prec="fp64", out=None, stream=None):
    """J = lambda^T A u from raw CSR device tensors through the allocation-free entry point
    (for callers that may not allocate device memory at that point)."""
    import torch
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device="cuda")
    _check(lib().sfa_bilinear_static(ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(colind.data_ptr()),
                                     rowptr.numel() - 1, PRECS[prec], ctypes.c_void_p(values.data_ptr()),
                                     ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def form_batched(meshes, op="stiffness", prec="fp32", outs=None, stream=None):
    """Form every mesh of the list in one graph launch (captured on the first call with these
    meshes and buffers, replayed afterwards); returns the value tensors."""
    import torch
    dtype = torch.float64 if PRECS[prec] == SFA_FP64 else torch.float32
    if outs is None:
        outs = [torch.empty(max(m.nnz, 1), dtype=dtype, device="cuda") for m in meshes]
    n = len(meshes)
    hs = (ctypes.c_void_p * n)(*[m.h for m in meshes])
    vs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check(lib().sfa_form_batched(hs, n, OPS[op], PRECS[prec], vs, _stream_handle(stream)))
    return [o[:m.nnz] for o, m in zip(outs, meshes)]


def get_tuning(p, op="stiffness", prec="fp32"):
    """(regular-pencil chunk, generic chunk, tensor-core run length) tuned for degree p; 0 = built-in."""
    out = (ctypes.c_int32 * 3)()
    _check(lib().sfa_get_tuning(int(p), OPS[op], PRECS[prec], out))
    return tuple(int(v) for v in out)


def launch_count():
    """Kernels launched by the library since it was loaded."""
    return int(lib().sfa_launch_count())


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(status, mesh_handle=None):
    if status != 0:
        buf = ctypes.create_string_buffer(512)
        lib().sfa_get_last_error(mesh_handle, buf, 512)
        raise SfaError(f"{lib().sfa_status_string(status).decode()}: {buf.value.decode()}")


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class _DevArray:
    """__cuda_array_interface__ wrapper of a mesh-owned device array."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}


_DTYPES = {0: "|i1", 1: "<i4", 2: "<u4", 3: "<i8", 4: "<f8"}


def make_desc(d, coef_ptr=None):
    """Fill an sfa_mesh_desc from a workload description dict."""
    c = MeshDesc()
    for k in range(3):
        c.n_el[k] = int(d["n_el"][k])
        c.lo[k] = float(d.get("lo", (0, 0, 0))[k])
        c.hi[k] = float(d.get("hi", (1, 1, 1))[k])
        c.plane_pt[k] = float(d.get("plane_pt", (0, 0, 0))[k])
        c.plane_n[k] = float(d.get("plane_n", (0, 0, 1))[k])
    c.p = int(d["p"])
    c.ls = LS[d["ls"]]
    balls = np.asarray(d.get("balls") or [], dtype=np.float64).reshape(-1)
    if balls.size > 4 * MAX_BALLS:
        raise ValueError("too many balls")
    c.n_balls = balls.size // 4
    for k, v in enumerate(balls):
        c.balls[k] = float(v)
    c.gyroid_freq = float(d.get("gyroid_freq", 6.0))
    c.gyroid_iso = float(d.get("gyroid_iso", 0.3))
    c.octree_depth = int(d.get("octree_depth", 3))
    c.coef = COEF[d.get("coef", "const")]
    c.coef_const = float(d.get("coef_const", 1.0))
    c.coef_bspline = coef_ptr
    return c


class Mesh:
    """A mesh in the library: tables and pattern are built on construction (``setup``)."""

    def __init__(self, desc, device="cuda", setup=True, stream=None):
        import torch
        self.desc = desc
        self.torch = torch
        self.n = tuple(int(v) + int(desc["p"]) for v in desc["n_el"])
        self.n_rows = self.n[0] * self.n[1] * self.n[2]
        self.coef = None
        coef_ptr = None
        if desc.get("coef") == "bspline":
            self.coef = torch.as_tensor(np.asarray(desc["coef_bspline"], dtype=np.float64), device=device).contiguous()
            if self.coef.numel() != self.n_rows:
                raise ValueError("coef_bspline must have n1*n2*n3 entries")
            coef_ptr = ctypes.c_void_p(self.coef.data_ptr())
        self._desc_c = make_desc(desc, coef_ptr)
        h = ctypes.c_void_p()
        _check(lib().sfa_create_mesh(ctypes.byref(self._desc_c), _stream_handle(stream), ctypes.byref(h)))
        self.h = h
        if setup:
            self.build_tables(stream)
            self.classify(stream)

    def close(self):
        if getattr(self, "h", None):
            lib().sfa_destroy_mesh(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_tables(self, stream=None):
        _check(lib().sfa_build_wq_tables(self.h, _stream_handle(stream)), self.h)

    def classify(self, stream=None):
        _check(lib().sfa_classify_cells(self.h, _stream_handle(stream)), self.h)
        self.info = self.get_info()
        self.nnz = self.info["nnz"]

    def get_info(self):
        inf = MeshInfo()
        _check(lib().sfa_get_info(self.h, ctypes.byref(inf)), self.h)
        return {k: int(getattr(inf, k)) for k, _ in MeshInfo._fields_}

    def pattern(self):
        """(rowptr, colind) as zero-copy torch views of the mesh-owned device arrays."""
        nr, nnz = ctypes.c_int64(), ctypes.c_int64()
        rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().sfa_get_pattern(self.h, ctypes.byref(nr), ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci)),
               self.h)
        t = self.torch
        rowptr = t.as_tensor(_DevArray(rp.value, (nr.value + 1,), "<i8"), device="cuda")
        colind = t.as_tensor(_DevArray(ci.value or 0, (nnz.value,), "<i4"), device="cuda") if nnz.value else \
            t.zeros(0, dtype=t.int32, device="cuda")
        return rowptr, colind

    def array(self, name):
        ptr, cnt, dt = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().sfa_get_array(self.h, name.encode(), ctypes.byref(ptr), ctypes.byref(cnt), ctypes.byref(dt)),
               self.h)
        if cnt.value == 0:
            return self.torch.zeros(0, dtype=self.torch.float64, device="cuda")
        return self.torch.as_tensor(_DevArray(ptr.value, (cnt.value,), _DTYPES[dt.value]), device="cuda")

    def form(self, op="mass", prec="fp64", out=None, stream=None, variant="dwq"):
        t = self.torch
        dtype = t.float64 if PRECS[prec] == SFA_FP64 else t.float32
        if out is None:
            out = t.empty(max(self.nnz, 1), dtype=dtype, device="cuda")
        if variant == "dwq":
            _check(lib().sfa_form(self.h, OPS[op], PRECS[prec], ctypes.c_void_p(out.data_ptr()),
                                  _stream_handle(stream)), self.h)
        else:
            _check(lib().sfa_form_variant(self.h, OPS[op], PRECS[prec], VARIANTS[variant],
                                          ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), self.h)
        return out[:self.nnz]

    def form_load(self, source="coef", variant="dwq", out=None, stream=None):
        """Load vector b_i (n_rows doubles on the device, exterior rows 0)."""
        t = self.torch
        if out is None:
            out = t.empty(self.n_rows, dtype=t.float64, device="cuda")
        _check(lib().sfa_form_load(self.h, SOURCES[source], VARIANTS[variant], ctypes.c_void_p(out.data_ptr()),
                                   _stream_handle(stream)), self.h)
        return out

    def form_profile(self, op="mass", prec="fp64", out=None, stream=None, variant="dwq"):
        """Form with the stages serialised; returns the values and the device ms of
        (coefficient, interior rows, cut-element matrices, cut rows)."""
        t = self.torch
        dtype = t.float64 if PRECS[prec] == SFA_FP64 else t.float32
        if out is None:
            out = t.empty(max(self.nnz, 1), dtype=dtype, device="cuda")
        ms = (ctypes.c_float * 4)()
        _check(lib().sfa_form_profile(self.h, OPS[op], PRECS[prec], VARIANTS[variant], ctypes.c_void_p(out.data_ptr()),
                                      _stream_handle(stream), ms), self.h)
        return out[:self.nnz], list(ms)

    def autotune(self, op="stiffness", prec="fp32", out=None, stream=None):
        """Tune the interior-row tiles for this degree on this mesh; returns the values."""
        t = self.torch
        dtype = t.float64 if PRECS[prec] == SFA_FP64 else t.float32
        if out is None:
            out = t.empty(max(self.nnz, 1), dtype=dtype, device="cuda")
        _check(lib().sfa_autotune(self.h, OPS[op], PRECS[prec], ctypes.c_void_p(out.data_ptr()),
                                  _stream_handle(stream)), self.h)
        return out[:self.nnz]

    def form_host(self, op, prec, coef_host, values_host, stream=None):
        """End-to-end call with host buffers (numpy or pinned torch CPU tensors)."""
        cptr = None
        if coef_host is not None:
            cptr = ctypes.c_void_p(coef_host.data_ptr() if hasattr(coef_host, "data_ptr") else coef_host.ctypes.data)
        vptr = ctypes.c_void_p(values_host.data_ptr() if hasattr(values_host, "data_ptr") else values_host.ctypes.data)
        _check(lib().sfa_form_host(self.h, OPS[op], PRECS[prec], cptr, vptr, _stream_handle(stream)), self.h)

    def bilinear(self, values, lam, u, prec="fp64", out=None, stream=None):
        t = self.torch
        if out is None:
            out = t.empty(1, dtype=t.float64, device="cuda")
        _check(lib().sfa_bilinear(self.h, PRECS[prec], ctypes.c_void_p(values.data_ptr()),
                                  ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), self.h)
        return out

    def backward(self, op, lam, u, scale=None, out=None, stream=None):
        t = self.torch
        if out is None:
            out = t.empty(self.n_rows, dtype=t.float64, device="cuda")
        sptr = ctypes.c_void_p(scale.data_ptr()) if scale is not None else None
        _check(lib().sfa_form_backward(self.h, OPS[op], ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                       sptr, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), self.h)
        return out

    def table_size(self, d, which):
        cnt, stride = ctypes.c_int64(), ctypes.c_int32()
        _check(lib().sfa_table_size(self.h, d, which, ctypes.byref(cnt), ctypes.byref(stride)), self.h)
        return cnt.value, stride.value

    def export_table(self, d, which, stream=None):
        cnt, stride = self.table_size(d, which)
        buf = np.zeros(cnt, dtype=np.float64)
        _check(lib().sfa_export_table(self.h, d, which, buf.ctypes.data_as(ctypes.c_void_p), cnt,
                                      _stream_handle(stream)), self.h)
        return buf.reshape(-1, stride)

    def import_table(self, d, which, arr, stream=None):
        cnt, stride = self.table_size(d, which)
        buf = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
        _check(lib().sfa_import_table(self.h, d, which, buf.ctypes.data_as(ctypes.c_void_p), cnt,
                                      _stream_handle(stream)), self.h)

    def check_device_status(self, stream=None):
        _check(lib().sfa_check_device_status(self.h, _stream_handle(stream)), self.h)

    def stage_ms(self):
        arr = (ctypes.c_float * 7)()
        _check(lib().sfa_get_stage_ms(self.h, arr), self.h)
        return list(arr)


class SfaFormBilinear:
    """J = lambda^T A(c) u as a torch.autograd.Function of the B-spline coefficients c.

    Forward forms A(c) with the library and reduces it; backward calls the library's
    adjoint (dJ/dc is exact: J is linear in c)."""

    @staticmethod
    def build():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, coef, mesh, op, lam, u):
                if coef.data_ptr() != mesh.coef.data_ptr():
                    mesh.coef.copy_(coef)
                vals = mesh.form(op, "fp64")
                J = mesh.bilinear(vals, lam, u)
                ctx.mesh, ctx.op = mesh, op
                ctx.save_for_backward(lam, u)
                return J[0]

            @staticmethod
            def backward(ctx, gJ):
                lam, u = ctx.saved_tensors
                scale = gJ.reshape(1).to(torch.float64).contiguous()
                g = ctx.mesh.backward(ctx.op, lam, u, scale=scale)
                return g, None, None, None, None

        return _F
