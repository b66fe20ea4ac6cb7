"""The C ABI library loads without a GPU and exports every entry point that
include/nb.h declares; the header and the Python binding agree on the
struct layouts."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libnb():
    from paper_2106_11143_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_core_calls():
    names = declared_functions()
    for core in ("nb_forces", "nb_step", "nb_energy", "nb_forces_vjp", "nb_strerror"):
        assert core in names


def test_library_exports_all_declared(libnb):
    for name in declared_functions():
        assert hasattr(libnb, name), name


def test_strerror_and_version_without_gpu(libnb):
    libnb.nb_strerror.restype = ctypes.c_char_p
    libnb.nb_version.restype = ctypes.c_char_p
    assert libnb.nb_strerror(0) == b"success"
    assert libnb.nb_strerror(1) == b"invalid argument"
    assert b"sm_103a" in libnb.nb_version()


def test_struct_layout_matches_header():
    from paper_2106_11143_gb300 import api
    # nb_params: 4 doubles, 2 int32, 6 doubles, 7 doubles, uint64, 2 uint32
    assert ctypes.sizeof(api.NbParams) == 4 * 8 + 8 + 6 * 8 + 7 * 8 + 8 + 8
    assert api.NbParams.seed.offset == 4 * 8 + 8 + 6 * 8 + 7 * 8
    # n, 9 state pointers, q, step, m
    assert ctypes.sizeof(api.NbSystem) == 8 + 10 * 8 + 8 + 8
    assert api.NbSystem.m.offset == 8 + 10 * 8 + 8


def test_invalid_arguments_rejected_on_host(libnb):
    """Validation happens before any CUDA call, so it works without a GPU."""
    libnb.nb_forces.restype = ctypes.c_int
    libnb.nb_step.restype = ctypes.c_int
    assert libnb.nb_forces(None, None, None, 0, None) == 1
    assert libnb.nb_step(None, None, 1, None) == 1
    # the arithmetic probes validate before touching the device
    libnb.nb_rinv3_probe.restype = ctypes.c_int
    libnb.nb_rinv3_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    libnb.nb_rsqrt_seed_probe.restype = ctypes.c_int
    libnb.nb_rsqrt_seed_probe.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert libnb.nb_rinv3_probe(99, 4, None, None, None, 0.0, None, None) == 1   # unknown precision
    assert libnb.nb_rinv3_probe(0, -1, None, None, None, 0.0, None, None) == 1   # n < 0
    assert libnb.nb_rinv3_probe(0, 4, None, None, None, 0.0, None, None) == 1    # NULL arrays
    assert libnb.nb_rinv3_probe(0, 4, 8, 8, 8, -1.0, 8, None) == 1               # soft2 < 0
    assert libnb.nb_rinv3_probe(0, 0, None, None, None, 0.0, None, None) == 0    # n == 0: nothing to do
    assert libnb.nb_rsqrt_seed_probe(-1, None, None, None) == 1
