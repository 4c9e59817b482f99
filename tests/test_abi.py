"""The C-ABI library loads, exports what include/mp3pcf.h declares, and validates on the host
(no GPU needed: nothing here launches a kernel)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_08601_gb300.build import build_native
    from paper_2309_08601_gb300 import native
    build_native()
    return native


def _declared():
    txt = open(os.path.join(ROOT, "include", "mp3pcf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mp3pcf_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "mp3pcf_accumulate_moments" in names and len(names) >= 11
    so = C.CDLL(lib.lib_path())
    for name in names:
        assert hasattr(so, name), name
    # the binding covers the whole header
    assert set(names) <= set(lib.SIGNATURES)


def test_bin_edge_table_matches_the_oracle(lib, orc):
    for (nb, tmin, tmax) in [(10, 0.5, 30.0), (20, 0.5, 120.0), (30, 0.5, 240.0), (7, 0.1, 3.3)]:
        cfg = lib.make_config(nb, tmin, tmax, 10)
        e = np.zeros(nb + 1)
        e2 = np.zeros(nb + 1, dtype=np.int64)
        st = lib.lib().mp3pcf_bin_edges(C.byref(cfg), e.ctypes.data_as(C.c_void_p),
                                        e2.ctypes.data_as(C.c_void_p))
        assert st == lib.OK
        oe, oe2 = orc.edges(orc.Setup(n_bins=nb, theta_min=tmin, theta_max=tmax, n_max=10))
        np.testing.assert_array_equal(e2, oe2)  # identical pair-to-bin decisions
        np.testing.assert_array_equal(e, oe)


@pytest.mark.parametrize("field,value", [("n_bins", 0), ("n_bins", 65), ("theta_min", 0.0),
                                         ("theta_max", 0.2), ("n_max", -1), ("n_max", 51),
                                         ("n_z", 0), ("n_z", 9), ("quantum", 0.0),
                                         ("precision", 7), ("n_phi", 0), ("norm_truncate", 2)])
def test_bad_configurations_are_rejected_before_any_cuda_call(lib, field, value):
    cfg = lib.make_config(10, 0.5, 30.0, 10)
    setattr(cfg, field, value)
    ctx = C.c_void_p()
    assert lib.lib().mp3pcf_create(C.byref(cfg), None, C.byref(ctx)) == lib.EINVAL
    assert not ctx
    assert lib.lib().mp3pcf_bin_edges(C.byref(cfg), None, None) == lib.EINVAL


def test_reserved_fields_must_be_zero(lib):
    cfg = lib.make_config(10, 0.5, 30.0, 10)
    cfg.reserved = 1
    ctx = C.c_void_p()
    assert lib.lib().mp3pcf_create(C.byref(cfg), None, C.byref(ctx)) == lib.EINVAL


@pytest.mark.parametrize("field,value", [("cell_occupancy", 65), ("cell_occupancy", -1),
                                         ("contract_slices", 65), ("exclude_degenerate", 2),
                                         ("grid_fft", 2)])
def test_tuning_and_variant_fields_are_validated(lib, field, value):
    cfg = lib.make_config(10, 0.5, 30.0, 10)
    setattr(cfg, field, value)
    assert lib.lib().mp3pcf_bin_edges(C.byref(cfg), None, None) == lib.EINVAL


def test_null_context_calls_fail_cleanly(lib):
    L = lib.lib()
    assert L.mp3pcf_destroy(None) == lib.OK
    assert L.mp3pcf_accumulate_moments(None, 0, None, None, None, None, None, None, None) == lib.EINVAL
    assert L.mp3pcf_counts(None, None, None) == lib.EINVAL
    assert L.mp3pcf_last_error(None) == b"null context"


def test_a_plain_c99_caller_builds_and_runs(lib, orc, tmp_path):
    """tests/c/abi_host.c includes only include/mp3pcf.h (compiled as strict C99, warnings as
    errors) and links the library; its host-only calls agree with the oracle's edge table."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    so = lib.lib_path()
    exe = str(tmp_path / "abi_host")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_host.c"),
                    "-L", os.path.dirname(so), "-l:" + os.path.basename(so),
                    "-Wl,-rpath," + os.path.dirname(so), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [r.split() for r in out if r.strip()]
    e = np.array([float(r[1]) for r in rows])
    e2 = np.array([int(r[2]) for r in rows])
    oe, oe2 = orc.edges(orc.Setup(n_bins=20, theta_min=0.5, theta_max=120.0, n_max=30))
    np.testing.assert_array_equal(e2, oe2)
    np.testing.assert_array_equal(e, oe)
