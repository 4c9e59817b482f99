"""ctypes binding of the C ABI declared in include/mp3pcf.h (argument marshalling only).

The library is the in-tree ``libmp3pcf.so`` built for sm_103a; there is no fallback. Loading
fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESINGULAR, EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ESINGULAR",
                6: "EUNSUPPORTED"}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16x3": 2, "tf32x3": 3}


class Config(C.Structure):
    """Mirror of ``mp3pcf_config``."""
    _fields_ = [("n_bins", C.c_int32), ("theta_min", C.c_double), ("theta_max", C.c_double),
                ("n_max", C.c_int32), ("n_phi", C.c_int32), ("n_z", C.c_int32),
                ("quantum", C.c_double), ("precision", C.c_int32), ("norm_truncate", C.c_int32),
                ("radial_nodes", C.c_int32), ("cell_occupancy", C.c_int32),
                ("contract_slices", C.c_int32), ("exclude_degenerate", C.c_int32),
                ("grid_fft", C.c_int32), ("reserved", C.c_int32)]


P = C.c_void_p
I64 = C.c_int64
I32 = C.c_int32
# every entry point of include/mp3pcf.h with its argument types
SIGNATURES = {
    "mp3pcf_create": ([P, P, P], C.c_int),
    "mp3pcf_destroy": ([P], C.c_int),
    "mp3pcf_last_error": ([P], C.c_char_p),
    "mp3pcf_bin_edges": ([P, P, P], C.c_int),
    "mp3pcf_accumulate_moments": ([P, I64, P, P, P, P, P, P, P], C.c_int),
    "mp3pcf_counts": ([P, P, P], C.c_int),
    "mp3pcf_copy_moments": ([P, P, P], C.c_int),
    "mp3pcf_contract_multipoles": ([P, P, P], C.c_int),
    "mp3pcf_edge_correct": ([P, P, P, P, P], C.c_int),
    "mp3pcf_to_gamma": ([P, P, I32, P], C.c_int),
    "mp3pcf_to_map3": ([P, P, I64, P, P, P], C.c_int),
    "mp3pcf_to_map3_four": ([P, P, I64, P, P], C.c_int),
    "mp3pcf_map3_direct": ([P, I64, P, P, P, P, P, I64, P, I64, P, C.c_double, P], C.c_int),
    "mp3pcf_grid_catalog": ([P, I64, P, P, P, P, P, P, P, I64, I32, I32, P, P, P, P, P, P, P], C.c_int),
    "mp3pcf_accumulate_moments_combined": ([P, I64, P, P, P, P, P, P, P, I32, P, P], C.c_int),
    "mp3pcf_set_timing": ([P, I32], C.c_int),
    "mp3pcf_stage_times": ([P, P, P, I32], C.c_int),
    "mp3pcf_to_map3_noalloc": ([P, P, P, I64, P, P, P], C.c_int),
    "mp3pcf_measure_peak": ([I32, P, P, P], C.c_int),
    "mp3pcf_to_map3_adjoint": ([P, I64, P, P, P, P], C.c_int),
    "mp3pcf_to_gamma_adjoint": ([P, I32, P, P], C.c_int),
    "mp3pcf_edge_correct_adjoint": ([P, P, P, P, P, P], C.c_int),
    "mp3pcf_moments_adjoint": ([P, P, P, I64, P, P, P, P, P, P], C.c_int),
    "mp3pcf_set_extent": ([P, P], C.c_int),
    "mp3pcf_run_batch": ([P, P, I64, P, I64, P, P, I32], C.c_int),
    "mp3pcf_graph_stats": ([P, P, P], C.c_int),
    "mp3pcf_inject": ([P, I32, I32], C.c_int),
}
INJECT_WAIT_TIMEOUT, INJECT_ALLOC_FAILURE = 1, 2


class CatalogView(C.Structure):
    _fields_ = [("n", C.c_int64), ("xq", C.c_void_p), ("yq", C.c_void_p), ("g1", C.c_void_p),
                ("g2", C.c_void_p), ("w", C.c_void_p), ("zbin", C.c_void_p)]

_lib = None


class Mp3pcfError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__("%s failed with %s%s" % (where, STATUS_NAMES.get(status, status),
                                                   (": " + detail) if detail else ""))


def lib_path() -> str:
    return LIB


def lib():
    """The loaded library; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libmp3pcf.so is not built (run __graft_entry__.build()); "
                               "this package has no CPU fallback")
        _lib = C.CDLL(LIB)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = res
    return _lib


def check(status: int, where: str, ctx=None, ok=(OK,)):
    if status not in ok:
        detail = ""
        if ctx is not None:
            msg = lib().mp3pcf_last_error(ctx)
            detail = msg.decode() if msg else ""
        raise Mp3pcfError(status, where, detail)
    return status


def make_config(n_bins, theta_min, theta_max, n_max, n_phi=100, n_z=1, quantum=2.0 ** -13,
                precision="fp32", norm_truncate=False, radial_nodes="arithmetic", cell_occupancy=0,
                contract_slices=0, exclude_degenerate=False, grid_fft=False) -> Config:
    return Config(int(n_bins), float(theta_min), float(theta_max), int(n_max), int(n_phi), int(n_z),
                  float(quantum), PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                  int(bool(norm_truncate)),
                  {"arithmetic": 0, "geometric": 1}[radial_nodes] if isinstance(radial_nodes, str)
                  else int(radial_nodes), int(cell_occupancy), int(contract_slices),
                  int(bool(exclude_degenerate)), int(bool(grid_fft)), 0)
