"""Host-side tests of the C-ABI library: symbols, validation, layer schedules.

No GPU is touched: code creation and schedule queries are host-only calls.
"""
import re

import numpy as np
import pytest

from tests import helpers


@pytest.fixture(scope="module")
def q():
    from paper_2004_09084_gb300 import build
    build.build()
    import paper_2004_09084_gb300 as q
    return q


def _header_symbols():
    with open(f"{helpers.GOLDEN}/../../include/qcmet.h") as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(qcmet_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(q):
    declared = _header_symbols()
    assert "qcmet_decode" in declared and "qcmet_code_create" in declared
    for name in declared:
        assert hasattr(q.lib, name), f"{name} declared in qcmet.h but not exported"
    assert set(declared) == set(q.EXPORTS)
    assert q.lib.qcmet_version() == 100


def test_status_strings(q):
    for st in range(0, -9, -1):
        assert q.lib.qcmet_status_string(st)
    assert q.lib.qcmet_status_string(-99) == b"unknown status"


def test_code_info_of_the_rate_0_1_construction(q):
    import synth
    c = synth.make_code("0.1", 12500)
    info = q.Code(c.base, c.shifts, c.Z).info()
    assert info["n"] == 1_000_000 and info["m"] == 900_000
    assert info["circulants"] == 300 and info["edges"] == 3_750_000
    assert info["msg_slots"] == 230 and info["degree1_columns"] == 70
    assert info["max_row_degree"] == 10


def test_validation_errors(q):
    base = np.ones((2, 3), np.int8)
    shifts = np.zeros((2, 3), np.int32)
    with pytest.raises(q.QcmetError) as e:
        q.Code(base, shifts, 0)
    assert e.value.status == q.ERR_INVALID_ARG
    bad = shifts.copy()
    bad[1, 2] = 5
    with pytest.raises(q.QcmetError) as e:
        q.Code(base, bad, 5)
    assert e.value.status == q.ERR_SHIFT_RANGE and "row 1" in str(e.value)
    bad[1, 2] = -1
    with pytest.raises(q.QcmetError) as e:
        q.Code(base, bad, 5)
    assert e.value.status == q.ERR_SHIFT_RANGE
    b2 = base.copy()
    b2[0, 0] = 2
    with pytest.raises(q.QcmetError) as e:
        q.Code(b2, shifts, 5)
    assert e.value.status == q.ERR_INVALID_ARG
    wide = np.ones((1, 17), np.int8)
    with pytest.raises(q.QcmetError) as e:
        q.Code(wide, np.zeros((1, 17), np.int32), 4)
    assert e.value.status == q.ERR_DEGREE_LIMIT
    q.Code(np.ones((1, 16), np.int8), np.zeros((1, 16), np.int32), 4)   # at the limit
    with pytest.raises(q.QcmetError) as e:
        q.Code(np.ones((1, 2), np.int8), np.zeros((1, 2), np.int32), 2 ** 30)
    assert e.value.status == q.ERR_INVALID_ARG


def test_null_arguments_are_errors_not_crashes(q):
    import ctypes
    h = ctypes.c_void_p()
    assert q.lib.qcmet_code_create(None, None, 1, 1, 1, ctypes.byref(h)) == q.ERR_INVALID_ARG
    assert q.lib.qcmet_code_get_info(None, None) == q.ERR_INVALID_ARG
    assert q.lib.qcmet_decode(None, None, None, 1, 1, None, None, None, None) == q.ERR_INVALID_ARG
    q.lib.qcmet_code_destroy(None)


@pytest.mark.parametrize("name,M,groups", helpers.read_merge_examples())
def test_greedy_merge_reproduces_the_papers_examples(q, name, M, groups):
    code = q.Code.from_shift_matrix(M, Z=4, merge="greedy")
    _, layers = code.schedule()
    assert layers == groups, f"Eq. ({name})"


def test_exact_merge_keeps_related_rows_in_order(q):
    ex = {name: (M, g) for name, M, g in helpers.read_merge_examples()}
    # Eq. (m1): rows 0 and 1 are unrelated and adjacent: merged
    _, layers = q.Code.from_shift_matrix(ex["m1"][0], 4, merge="exact").schedule()
    assert layers == [[0, 1], [2]]
    # Eq. (m2): row 2 is related to row 1, so the exact schedule may not move it first
    _, layers = q.Code.from_shift_matrix(ex["m2"][0], 4, merge="exact").schedule()
    assert layers == [[0], [1], [2]]
    _, layers = q.Code.from_shift_matrix(ex["m"][0], 4, merge="exact").schedule()
    assert layers == [[0], [1], [2]]
    _, layers = q.Code.from_shift_matrix(ex["m2"][0], 4, merge="none").schedule()
    assert layers == [[0], [1], [2]]


def test_exact_schedule_layers_are_unrelated_and_preserve_related_order(q):
    import synth
    c = synth.make_code("0.1", 16)
    code = q.Code(c.base, c.shifts, c.Z, merge="exact")
    rows, layers = code.schedule()
    assert sorted(rows.tolist()) == list(range(c.mb))
    pos = {r: k for k, layer in enumerate(layers) for r in layer}
    for layer in layers:
        cols = np.concatenate([np.flatnonzero(c.base[r]) for r in layer])
        assert len(cols) == len(set(cols.tolist())), "rows of one layer share a column"
    for a in range(c.mb):
        for b in range(a + 1, c.mb):
            if np.any(c.base[a] & c.base[b]):
                assert pos[a] < pos[b]
    assert len(layers) < c.mb


def test_zero_rows_are_not_scheduled(q):
    base = np.array([[1, 1], [0, 0], [0, 1]], np.int8)
    code = q.Code(base, np.zeros((3, 2), np.int32), 3, merge="none")
    rows, layers = code.schedule()
    assert rows.tolist() == [0, 2]
    assert layers == [[0], [2]]


def test_release_build_has_no_index_checks(q):
    # qcmet_debug_checks answers without touching a GPU in the release build
    with pytest.raises(q.QcmetError) as e:
        q.debug_checks()
    assert e.value.status == q.ERR_UNSUPPORTED
