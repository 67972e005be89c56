"""The C-ABI library loads and exports every entry point declared in include/*.h (CPU only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**\s*([A-Za-z_]\w*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bf_build", "bf_apply", "hss_build_from_samples", "hss_ulv_factor", "hss_solve", "fio_solve",
                     "bf_free", "hss_free", "fio_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    build = __graft_entry__._build_module()
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2609_11520_b300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_invalid_arguments_are_rejected_without_a_gpu():
    """Argument checks run before any CUDA call and return FIO_EINVAL."""
    from paper_2609_11520_b300 import _lib
    h = ctypes.c_void_p()
    ph = _lib.Phase(1, 1.0)
    assert _lib.lib.bf_build(ctypes.byref(ph), 1000, 1, 16, None, ctypes.byref(h)) == _lib.FIO_EINVAL
    assert b"power of two" in _lib.lib.fio_last_error()
    assert _lib.lib.bf_build(ctypes.byref(ph), 1024, 1, 40, None, ctypes.byref(h)) == _lib.FIO_EINVAL
    assert _lib.lib.bf_apply(None, None, None, 1024, 1, 0, None) == _lib.FIO_EINVAL
    sm = _lib.Sampler(0, None, None, 0)
    assert _lib.lib.hss_build_from_samples(ctypes.byref(sm), 1000, 64, 10, 1e-3, 0, None,
                                           ctypes.byref(h)) == _lib.FIO_EINVAL
    assert _lib.lib.hss_solve(None, None, None, 1, 1, None) == _lib.FIO_EINVAL
