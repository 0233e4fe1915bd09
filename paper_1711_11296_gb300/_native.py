"""ctypes binding of the C ABI in ``include/sht.h`` (argument marshalling only).

The shared library is built in-tree (``libsht.so`` next to this file) by
``paper_1711_11296_gb300.build``.  If it is missing, importing this module
raises: there is no host fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsht.so")

# C ABI symbols (kept in the order of include/sht.h)
EXPORTED = [
    "sht_plan_create", "sht_plan_destroy", "sht_plan_query", "sht_forward",
    "sht_inverse", "sht_adjoint", "sht_restrict_nested", "sht_plan_copy_tables",
    "sht_profile_enable", "sht_profile_read", "sht_last_error", "sht_version",
    "sht_forward_noalloc", "sht_plan_status", "sht_group_create",
    "sht_group_destroy", "sht_group_forward", "sht_group_inverse",
    "sht_plan_set_tuning", "sht_plan_get_tuning", "sht_plan_autotune",
    "sht_plan_create_grid", "sht_plan_set_reduced", "sht_prolong_spectral",
    "sht_inject_nested", "sht_reduced_grid_sizes", "sht_plan_create_reduced",
    "sht_plan_grid_points", "sht_profile_read_kernels", "sht_prolong_spectral_add",
    "sht_measure_fma_peak", "sht_alias_products", "sht_plan_create_reduced_shifted",
    "sht_octahedral_grid_sizes", "sht_icositetrahedral_grid_sizes",
]
PROFILE_STAGES = 8
STAGE_NAMES = ["fft_forward", "legendre_forward", "legendre_inverse",
               "fft_inverse", "split_convert", "", "", ""]

SHT_OK = 0
SHT_WARN_INEXACT = 1
STATUS = {
    -1: "SHT_ERR_ARG", -2: "SHT_ERR_ALLOC", -3: "SHT_ERR_CUDA",
    -4: "SHT_ERR_NOT_NESTED", -5: "SHT_ERR_TIMEOUT", -6: "SHT_ERR_HANDLE",
    -7: "SHT_ERR_UNSUPPORTED",
}
PRECISION = {"fp64": 0, "bf16x2": 1, "bf16x3": 2, "fp16x2": 3, "fp16x3": 4}
GRID = {"cc": 0, "fejer1": 1}
REDUCED_RULE = {"smooth": 0, "fast": 1}


class SHTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libsht.so is not built (run paper_1711_11296_gb300.build.build()); "
            "this library has no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int
    lib.sht_plan_create.argtypes = [i, i, i, i, i, ctypes.POINTER(vp)]
    lib.sht_plan_create_grid.argtypes = [i, i, i, i, i, i, ctypes.POINTER(vp)]
    lib.sht_plan_set_reduced.argtypes = [vp, i]
    lib.sht_prolong_spectral.argtypes = [vp, vp, i, vp, vp]
    lib.sht_prolong_spectral_add.argtypes = [vp, vp, i, vp, vp]
    lib.sht_inject_nested.argtypes = [vp, vp, i, vp, vp]
    lib.sht_plan_destroy.argtypes = [vp]
    lib.sht_plan_query.argtypes = [vp, ip, ip, ip, ip, ip, ip,
                                   ctypes.POINTER(ctypes.c_size_t)]
    lib.sht_forward.argtypes = [vp, vp, vp, vp]
    lib.sht_inverse.argtypes = [vp, vp, vp, vp]
    lib.sht_adjoint.argtypes = [vp, i, vp, vp, vp]
    lib.sht_restrict_nested.argtypes = [vp, vp, i, vp, vp]
    dp = ctypes.POINTER(ctypes.c_double)
    lib.sht_plan_copy_tables.argtypes = [vp, dp, dp, dp]
    lib.sht_profile_enable.argtypes = [vp, i]
    lib.sht_profile_read.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong)]
    lib.sht_profile_read_kernels.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(ctypes.c_longlong)]
    lib.sht_forward_noalloc.argtypes = [i, i, i, i, vp, vp, vp]
    lib.sht_plan_status.argtypes = [vp]
    vpp = ctypes.POINTER(vp)
    lib.sht_group_create.argtypes = [vpp, i, ctypes.POINTER(vp)]
    lib.sht_group_destroy.argtypes = [vp]
    lib.sht_group_forward.argtypes = [vp, vpp, vpp, vp]
    lib.sht_group_inverse.argtypes = [vp, vpp, vpp, vp]
    lib.sht_plan_set_tuning.argtypes = [vp, i, i]
    lib.sht_plan_get_tuning.argtypes = [vp, ip, ip]
    lib.sht_plan_autotune.argtypes = [vp, i, vp, ip, ip, ctypes.POINTER(ctypes.c_float)]
    lib.sht_reduced_grid_sizes.argtypes = [vp, i, ip]
    lib.sht_plan_create_reduced.argtypes = [i, i, ip, i, i, ctypes.POINTER(vp)]
    lib.sht_plan_grid_points.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.sht_measure_fma_peak.argtypes = [i, i, vp, dp]
    lib.sht_alias_products.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.sht_plan_create_reduced_shifted.argtypes = [i, i, ip, ip, i, i, ctypes.POINTER(vp)]
    lib.sht_octahedral_grid_sizes.argtypes = [i, i, i, ip]
    lib.sht_icositetrahedral_grid_sizes.argtypes = [i, ip, ip]
    lib.sht_last_error.restype = ctypes.c_char_p
    lib.sht_version.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("sht_last_error", "sht_version"):
            getattr(lib, name).restype = i
    return lib


lib = _load()


def check(rc):
    """Raise SHTError for a negative status; return the status otherwise."""
    if rc < 0:
        raise SHTError(rc, lib.sht_last_error().decode())
    return rc
