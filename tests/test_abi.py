"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point include/sht.h declares, and
rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import pytest

from sht_testutil import built_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(sht_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = built_lib()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "sht_forward" in names and "sht_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_match_header(lib):
    from paper_1711_11296_gb300 import _native
    assert sorted(_native.EXPORTED) == _declared()


@pytest.mark.parametrize("args,code", [
    ((-1, 3, 4, 1, 0), -1),        # N < 0
    ((3, 8, 16, 1, 0), -1),        # J even
    ((10, 21, 20, 1, 0), -1),      # I <= 2N
    ((10, 21, 21, 1, 0), -1),      # I odd
    ((10, 21, 28, 1, 0), -1),      # I/2 = 14 has the factor 7
    ((10, 21, 24, 0, 0), -1),      # nfields < 1
    ((10, 21, 24, 1, 9), -1),      # unknown precision
    ((10, 21, 16384, 1, 0), -1),   # I too large
])
def test_invalid_plan_arguments_rejected_on_host(lib, args, code):
    h = ctypes.c_void_p()
    lib.sht_plan_create.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_void_p)]
    assert lib.sht_plan_create(*args, ctypes.byref(h)) == code
    lib.sht_last_error.restype = ctypes.c_char_p
    assert lib.sht_last_error()


def test_null_and_foreign_handles(lib):
    vp = ctypes.c_void_p
    lib.sht_forward.argtypes = [vp, vp, vp, vp]
    lib.sht_plan_destroy.argtypes = [vp]
    assert lib.sht_plan_destroy(None) == 0
    assert lib.sht_forward(None, None, None, None) == -6
    bogus = ctypes.create_string_buffer(256)
    assert lib.sht_forward(ctypes.addressof(bogus), None, None, None) == -6
    assert lib.sht_plan_destroy(ctypes.addressof(bogus)) == -6


def _lat(pts):
    return (ctypes.c_int * len(pts))(*pts)


@pytest.mark.parametrize("N,J,pts", [
    (15, 7, None),                                  # NULL I_lat
    (15, 8, [32] * 8),                              # J even
    (15, 7, [16, 24, 32, 40, 32, 24, 18]),          # not symmetric
    (15, 7, [16, 25, 32, 40, 32, 25, 16]),          # odd count
    (15, 7, [16, 24, 32, 16384, 32, 24, 16]),       # count above 8192
    (15, 7, [16, 24, 30, 30, 30, 24, 16]),          # widest row does not exceed 2N
])
def test_invalid_reduced_grids_rejected_on_host(lib, N, J, pts):
    h = ctypes.c_void_p()
    lib.sht_plan_create_reduced.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_void_p)]
    arg = None if pts is None else ctypes.cast(_lat(pts), ctypes.c_void_p)
    assert lib.sht_plan_create_reduced(N, J, arg, 1, 0, ctypes.byref(h)) == -1
    assert not h.value
    lib.sht_last_error.restype = ctypes.c_char_p
    assert lib.sht_last_error()


def test_newer_entry_points_reject_null_handles(lib):
    vp = ctypes.c_void_p
    lib.sht_reduced_grid_sizes.argtypes = [vp, ctypes.c_int, vp]
    lib.sht_plan_grid_points.argtypes = [vp, vp]
    lib.sht_profile_read_kernels.argtypes = [vp, vp, vp, vp]
    lib.sht_prolong_spectral_add.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    buf = ctypes.create_string_buffer(1024)
    assert lib.sht_reduced_grid_sizes(None, 0, buf) == -6
    assert lib.sht_plan_grid_points(None, buf) == -6
    assert lib.sht_profile_read_kernels(None, buf, buf, buf) == -6
    assert lib.sht_prolong_spectral_add(None, buf, 0, buf, None) == -6


@pytest.mark.parametrize("shift", [
    [0, 0, 2, 0, 2, 0, 0],                          # not 0 or 1
    [0, 1, 0, 0, 0, 0, 0],                          # not symmetric
])
def test_invalid_shifts_rejected_on_host(lib, shift):
    h = ctypes.c_void_p()
    vp = ctypes.c_void_p
    lib.sht_plan_create_reduced_shifted.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp,
                                                    ctypes.c_int, ctypes.c_int,
                                                    ctypes.POINTER(vp)]
    pts = [16, 24, 32, 40, 32, 24, 16]
    assert lib.sht_plan_create_reduced_shifted(15, 7, ctypes.cast(_lat(pts), vp),
                                               ctypes.cast(_lat(shift), vp), 1, 0,
                                               ctypes.byref(h)) == -1
    assert not h.value
    assert lib.sht_plan_create_reduced_shifted(15, 7, ctypes.cast(_lat(pts), vp), None, 1, 0,
                                               ctypes.byref(h)) == -1


@pytest.mark.parametrize("J", [1, 9, 47, 1281])
def test_octahedral_and_icositetrahedral_counts_match_the_oracle(lib, J):
    # host-only entry points against the oracle's own restatement
    import oracle as O
    buf = (ctypes.c_int * J)()
    lib.sht_octahedral_grid_sizes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_void_p]
    assert lib.sht_octahedral_grid_sizes(J, 20, 4, buf) == 0
    assert list(buf) == O.octahedral_sizes(J).tolist()
    sh = (ctypes.c_int * J)()
    lib.sht_icositetrahedral_grid_sizes.argtypes = [ctypes.c_int, ctypes.c_void_p,
                                                    ctypes.c_void_p]
    assert lib.sht_icositetrahedral_grid_sizes(J, buf, sh) == 0
    Ij, s = O.icositetrahedral_sizes(J)
    assert list(buf) == Ij.tolist()
    assert list(sh) == [int(2 * v) for v in s]
    assert lib.sht_octahedral_grid_sizes(J + 1, 20, 4, buf) == -1
    assert lib.sht_octahedral_grid_sizes(J, 21, 4, buf) == -1
