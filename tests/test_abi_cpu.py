"""CPU checks of the boundary: the C-ABI library builds, loads without a GPU and exports
every function include/sfa.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sfa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfa_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2211_06427_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "sfa_form" in names and "sfa_create_mesh" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols():
    from paper_2211_06427_gb300 import sfa
    assert set(_declared()) <= set(sfa.EXPORTED)


def test_invalid_descriptor_rejected_without_gpu_work():
    """Argument validation happens before any CUDA call."""
    from paper_2211_06427_gb300 import build, sfa, synthetic
    build.build()
    lib = sfa.load_library()
    d = synthetic.c1_ball_p2_8()
    bad = sfa.make_desc(dict(d, p=9))
    h = ctypes.c_void_p()
    st = lib.sfa_create_mesh(ctypes.byref(bad), None, ctypes.byref(h))
    assert st == 1 and not h.value
    buf = ctypes.create_string_buffer(256)
    lib.sfa_get_last_error(None, buf, 256)
    assert b"degree" in buf.value
    assert lib.sfa_status_string(5) == b"singular weighted-quadrature system"
