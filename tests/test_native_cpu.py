"""Host-side checks of the C-ABI library: it builds, loads, and exports every
entry point include/kdfmm.h declares (no compute calls; no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2502_01496_gb300 import build
    return build.build_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kdfmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kdfmm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("kdfmm_tree_build", "kdfmm_tree_moments", "kdfmm_fmm_accel",
                 "kdfmm_fmm_accel_vjp", "kdfmm_total_momentum"):
        assert want in names


def test_library_loads_and_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.kdfmm_last_error.restype = ctypes.c_char_p
    assert lib.kdfmm_last_error() == b""


def test_binding_rejects_null_handles_without_a_gpu(libpath):
    from paper_2502_01496_gb300 import native
    L = native.lib()
    p = native.make_params()
    assert L.kdfmm_tree_build(None, None, None, None, 10, ctypes.byref(p), None) == -1
    assert "NULL" in native.last_error()
    assert L.kdfmm_fmm_accel(None, None, None, None) == -1
    assert L.kdfmm_tree_stats(None, None) == -1


def test_params_struct_layout_matches_header():
    from paper_2502_01496_gb300 import native
    assert ctypes.sizeof(native.Params) == 48
    assert native.Params.n_leaf.offset == 24 and native.Params.expansion.offset == 36
    assert native.Params.walk.offset == 40 and native.Params.reserved.offset == 44


def test_forest_arguments_are_checked_on_the_host(libpath):
    """Bad system tables are refused before the handle or any device pointer
    is looked at, so this runs without a GPU."""
    import numpy as np
    from paper_2502_01496_gb300 import native
    L = native.lib()
    p = native.make_params()

    def call(off, theta=None, nleaf=None):
        off = np.asarray(off, dtype=np.int64)
        th = None if theta is None else np.asarray(theta, dtype=np.float64)
        nl = None if nleaf is None else np.asarray(nleaf, dtype=np.int32)
        ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        return L.kdfmm_forest_build(None, None, None, None, ptr(off), len(off) - 1, ptr(th), None,
                                    ptr(nl), ctypes.byref(p), None)

    assert call([0, 5, 5, 9]) == -1 and "empty" in native.last_error()
    assert call([1, 5]) == -1 and "sys_offset[0]" in native.last_error()
    assert call([0, 5, 9], theta=[0.5, 1.5]) == -1 and "theta[1]" in native.last_error()
    assert call([0, 5, 9], nleaf=[16, 33]) == -1 and "n_leaf[1]" in native.last_error()
    assert call([0, 5, 9]) == -1 and "tree is NULL" in native.last_error()


def test_measure_peaks_rejects_null_output_without_a_gpu(libpath):
    from paper_2502_01496_gb300 import native
    assert native.lib().kdfmm_measure_peaks(None, None) == -1
    assert "NULL" in native.last_error()


def test_stat_and_phase_names_match_header():
    """The binding names one statistic per KDFMM_STAT_* index (in index
    order, KDFMM_NSTATS of them) and one phase per KDFMM_PHASE_*."""
    from paper_2502_01496_gb300 import native
    src = open(os.path.join(ROOT, "include", "kdfmm.h")).read()
    stats = dict((k, int(v)) for k, v in re.findall(r"#define KDFMM_STAT_([A-Z0-9_]+)\s+(\d+)", src))
    nstats = int(re.search(r"#define KDFMM_NSTATS\s+(\d+)", src).group(1))
    assert nstats == len(native.STAT_NAMES) == len(stats)
    assert [k.lower() for k, _ in sorted(stats.items(), key=lambda kv: kv[1])] == list(native.STAT_NAMES)
    phases = re.findall(r"#define KDFMM_PHASE_([A-Z0-9_]+)\s+(\d+)", src)
    assert [k.lower() for k, _ in sorted(phases, key=lambda kv: int(kv[1]))] == list(native.PHASES)
