"""The C-ABI library builds, loads and exports every symbol include/gpss.h
declares; host-side validation runs without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2601_02527_gb300 as gp
from paper_2601_02527_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gp.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gpss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_ss_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert sorted(gp.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_status_strings(lib):
    for code in range(9):
        assert lib.gp_ss_status_string(code).decode()
    assert lib.gp_ss_status_string(7).decode().startswith("non-positive")


def _build(lib, t_start, t_end, inst=None, offsets=None, terms=(1,), layout=0, opts=None):
    n = len(t_start)
    offs = np.asarray(offsets if offsets is not None else [0, n], np.int64)
    ts = np.ascontiguousarray(t_start, np.float64)
    te = np.ascontiguousarray(t_end, np.float64)
    y = np.zeros(n, np.float32)
    ye = np.zeros(n, np.float32)
    spec, keep = gp._spec(terms, layout)
    opts = opts if opts is not None else gp._Options(32, 0, 0, 0, 0, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    ii = None if inst is None else np.ascontiguousarray(inst, np.int32)
    rc = lib.gp_ss_build_model(ctypes.byref(spec), len(offs) - 1, offs.ctypes.data,
                               ts.ctypes.data, te.ctypes.data, y.ctypes.data, ye.ctypes.data,
                               None if ii is None else ii.ctypes.data, ctypes.byref(opts),
                               ctypes.byref(h))
    if rc == 0:
        lib.gp_ss_free_model(h)
    return rc


def test_host_validation_without_gpu(lib):
    # unsorted offsets
    assert _build(lib, [0.0, 1.0], [0.5, 1.5], offsets=[0, 2, 1]) == 2
    # negative exposure
    assert _build(lib, [0.0, 1.0], [0.5, 0.9]) == 1
    # instantaneous (zero-length) and integrated measurements in one model get
    # past validation (without a GPU the build then stops at the device copy)
    assert _build(lib, [0.0, 1.0], [0.5, 1.0]) not in (1, 2, 3, 4)
    # one instrument overlapping itself
    assert _build(lib, [0.0, 0.4], [0.5, 0.9], inst=[0, 0]) == 3
    # more than 3 concurrently open exposures (greedy slots) is not compiled
    assert _build(lib, [0.0, 0.1, 0.2, 0.3], [5.0, 5.0, 5.0, 5.0]) == 4
    # more than two terms
    assert _build(lib, [0.0], [1.0], terms=(1, 1, 1)) == 4
    # a product term: compiled first only, and on instantaneous measurements only
    assert _build(lib, [0.0, 1.0], [0.0, 1.0], terms=(1, 3)) == 4
    assert _build(lib, [0.0, 1.0], [0.5, 1.5], terms=(3,)) == 4
    # an unknown term kind
    assert _build(lib, [0.0], [1.0], terms=(4,)) == 1
    # option values outside their ranges
    for bad in (gp._Options(32, 0, 0, 0, 12, 0, 0, 0, 0), gp._Options(32, 0, 0, 0, 0, 0, 0, 2),
                gp._Options(16, 0, 0, 0, 0, 0, 0, 0, 0), gp._Options(32, 4, 0, 0, 0, 0, 0, 0),
                gp._Options(32, 0, 0, 0, 0, 0, 3, 0), gp._Options(32, 0, 0, 0, 0, 0, 0, 0, 16)):
        assert _build(lib, [0.0], [1.0], opts=bad) == 1


def test_mixed_event_build_host_only(lib):
    # an exposure [0, 1], an instant at 1.0 (the exposure's end), an exposure
    # starting at 1.0 and an instant at 2.5: at t = 1 the end comes first,
    # then the instant, then the start (every read before a reset)
    gp = pytest.importorskip("paper_2601_02527_gb300")
    dt, tag, meas, n_slots = gp.build_events([0.0, 1.0, 1.0, 2.5], [1.0, 1.0, 2.0, 2.5],
                                             [1.0, 2.0, 3.0, 4.0], [0.1, 0.2, 0.3, 0.4])
    inst = 0x10
    assert n_slots == 1
    assert list(tag) == [0, 1, 1 | inst, 0, 1, 1 | inst]
    np.testing.assert_allclose(dt, [0.0, 1.0, 0.0, 0.0, 1.0, 0.5])
    # measurement records in event order: (y, yerr^2, 1/delta), 1/delta = 1 for instants
    np.testing.assert_allclose(meas[:, 0], [1.0, 2.0, 3.0, 4.0])
    np.testing.assert_allclose(meas[:, 2], [1.0, 1.0, 1.0, 1.0])
    np.testing.assert_allclose(meas[:, 1], np.float32([0.1, 0.2, 0.3, 0.4]) ** 2, rtol=1e-6)
