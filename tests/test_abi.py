"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/pod2g.h declares (no device calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pod2g.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pod2g_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2207_02543_gb300 as pkg
    return pkg.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pod2g_create", "pod2g_set_values", "pod2g_solve", "pod2g_solve_batch", "pod2g_submit",
                 "pod2g_poll", "pod2g_destroy", "pod2g_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    import paper_2207_02543_gb300 as pkg
    assert sorted(pkg.EXPORTS) == _declared()


def test_host_only_calls(lib):
    import paper_2207_02543_gb300 as pkg
    o = pkg.Opts()
    lib.pod2g_default_opts(ctypes.byref(o))
    assert abs(o.omega - 2 / 3) < 1e-15 and o.pre == 1 and o.post == 1 and o.chunk == 8
    assert pkg.strerror(pkg.NOT_SPD).startswith("not SPD")
    assert pkg.strerror(999) == "unknown status"
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert lib.pod2g_create(None, None, 0, None, ctypes.byref(h)) == pkg.INVALID_ARG
    assert lib.pod2g_info(None, None, None, None, None) == pkg.INVALID_ARG
    assert lib.pod2g_launch_count(None) == 0
    lib.pod2g_destroy(None)


def test_opts_struct_layout_matches(lib):
    """pod2g_default_opts fills exactly sizeof(pod2g_opts) bytes: a sentinel placed right
    after the binding's struct must survive, and the appended fields read back their defaults."""
    import paper_2207_02543_gb300 as pkg
    size = ctypes.sizeof(pkg.Opts)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    lib.pod2g_default_opts(ctypes.cast(buf, ctypes.POINTER(pkg.Opts)))
    assert all(b == 0xAB for b in bytes(buf)[size:])
    o = ctypes.cast(buf, ctypes.POINTER(pkg.Opts)).contents
    assert o.method == pkg.PCG and o.smoother == pkg.SMOOTHER_JACOBI and o.precision == pkg.MIXED_FP32PHI


def test_noalloc_rejects_options_it_does_not_offer(lib):
    """pod2g_solve_noalloc runs the damped-Jacobi PCG solve only: a Gauss-Seidel or stationary
    request is refused with INVALID_ARG during argument validation, before any device work."""
    import paper_2207_02543_gb300 as pkg
    fake = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    it, rr, st = ctypes.c_int(0), ctypes.c_double(0.0), ctypes.c_int(0)
    for field, value in (("smoother", pkg.SMOOTHER_SGS), ("method", pkg.STATIONARY)):
        o = pkg.Opts()
        lib.pod2g_default_opts(ctypes.byref(o))
        setattr(o, field, value)
        rc = lib.pod2g_solve_noalloc(4, 1, 4, fake, fake, fake, fake, 1, ctypes.byref(o), fake, None, 1e-8, 10,
                                     fake, ctypes.byref(it), ctypes.byref(rr), ctypes.byref(st), None)
        assert rc == pkg.INVALID_ARG, field
