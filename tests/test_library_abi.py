"""The C-ABI library builds, loads and exports every function include/*.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            names.add(m.group(1))
    return names - {"if", "while", "for", "return", "sizeof"}


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["bf_weights", "bf_apply", "cg_filter", "lobpcg_filter", "bf_graph_free",
              "bf_last_error", "bf_simple_filter", "bf_reguided_filter",
              "bf_guided_graph"]:
        assert n in names


def test_library_loads_and_exports_declared_symbols():
    from paper_1509_02468_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    lib.bf_last_error.restype = ctypes.c_char_p
    assert lib.bf_last_error() == b""


def test_argument_validation_needs_no_gpu():
    """Argument checks return BF_EINVAL before touching the device."""
    from paper_1509_02468_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.bf_apply.restype = ctypes.c_int
    assert lib.bf_apply(None, 1, None, 1, 1, None, 1, None, None) == -1
    lib.bf_weights.restype = ctypes.c_int
    assert lib.bf_weights(None, None, None, None) == -1
    lib.cg_filter.restype = ctypes.c_int
    assert lib.cg_filter(None, None, 3, None, None, None, None) == -1
    lib.bf_reguided_filter.restype = ctypes.c_int
    assert lib.bf_reguided_filter(None, None, 2, None, None) == -1
    lib.bf_guided_graph.restype = ctypes.c_int
    assert lib.bf_guided_graph(None, None, None, None) == -1


def test_guided_graph_parameter_checks_need_no_gpu():
    """bf_guided_graph rejects bad parameters with BF_EINVAL before touching the device."""
    from paper_1509_02468_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.bf_guided_graph.restype = ctypes.c_int

    class P(ctypes.Structure):
        _fields_ = [("ndim", ctypes.c_int32), ("radius", ctypes.c_int32),
                    ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                    ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                    ("eps", ctypes.c_double)]

    fake_guide = ctypes.c_void_p(256)            # never dereferenced: the checks come first
    out = ctypes.c_void_p()
    good = dict(ndim=2, radius=2, nx=64, ny=48, dtype=0, reserved=0, eps=0.01)
    bad = [dict(ndim=3), dict(radius=0), dict(radius=9), dict(nx=0), dict(ndim=1, ny=2),
           dict(dtype=7), dict(reserved=1), dict(eps=0.0), dict(eps=float("inf")), dict(eps=float("nan"))]
    for change in bad:
        p = P(**{**good, **change})
        assert lib.bf_guided_graph(ctypes.byref(p), fake_guide, ctypes.byref(out), None) == -1, change
        assert not out.value


def test_spd_preconditioner_checks_need_no_gpu():
    """bf_spd_create rejects a half-width outside 1..4 and NULL output with BF_EINVAL, and
    the SPD entry points reject NULL arguments, before touching the device."""
    from paper_1509_02468_gb300 import build
    lib = ctypes.CDLL(build.build())
    for fn in ("bf_spd_create", "bf_spd_apply", "bf_spd_accumulate", "bf_spd_grad", "bf_spd_adam",
               "bf_spd_zero_grad", "bf_spd_weights", "bf_spd_size"):
        getattr(lib, fn).restype = ctypes.c_int
    out = ctypes.c_void_p()
    for half in (0, 5, -1):
        assert lib.bf_spd_create(half, None, ctypes.byref(out)) == -1
        assert not out.value
    assert lib.bf_spd_create(3, None, None) == -1
    assert lib.bf_spd_size(None) == 0
    assert lib.bf_spd_apply(None, None, None, 1, 1, None, 1, None) == -1
    assert lib.bf_spd_accumulate(None, None, ctypes.c_double(0.01), None, None, None) == -1
    assert lib.bf_spd_grad(None, None, None, None) == -1
    assert lib.bf_spd_adam(None, ctypes.c_float(1e-3), ctypes.c_float(1.0), None) == -1
    assert lib.bf_spd_zero_grad(None, None) == -1
    assert lib.bf_spd_weights(None, None) == -1
