"""C-ABI checks that need no GPU: the library builds and loads, exports every symbol that
include/apex.h declares, counts compounds like the oracle, and rejects malformed descriptors
before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import csl_gen
from oracle import oracle as O
from paper_2510_24380_b300 import apex, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dll():
    build.build()
    return apex.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "apex.h")).read()
    return sorted(set(re.findall(r"^\s*(?:apex_status|const char \*)\s*(apex_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(dll):
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(dll, n), n
    # and the binding covers every one of them
    assert set(names) == set(apex.SYMBOLS)


@pytest.mark.parametrize("name", ["t_ragged", "c1_tiny", "c2_10m", "c3_real"])
def test_count_matches_oracle(dll, name):
    lib, head, spec = csl_gen.build_workload(name, materialize=False)
    assert apex.apex_count_compounds(lib.n_slots, lib.slot_sizes) == O.count(lib)


def test_count_rejects_bad_shapes(dll):
    with pytest.raises(apex.ApexError) as e:
        apex.apex_count_compounds([2], [2 ** 32, 2 ** 32])
    assert e.value.code == -1
    with pytest.raises(apex.ApexError):
        apex.apex_count_compounds([2], [3, 0])
    with pytest.raises(apex.ApexError):
        apex.apex_count_compounds([0], [])


def _desc(n_slots, sizes, d, dims, act=2, n_obj=1, n_prop=None, prec=1):
    keep = []
    ns = np.asarray(n_slots, np.int32)
    ss = np.asarray(sizes, np.int64)
    U = np.zeros((max(1, int(ss.sum())), d), np.float32)
    dm = np.asarray(dims, np.int32)
    W = [np.zeros((dims[l + 1], dims[l]), np.float32) for l in range(len(dims) - 1)]
    b = [np.zeros(dims[l + 1], np.float32) for l in range(len(dims) - 1)]
    Wp = (C.POINTER(C.c_float) * len(W))(*[w.ctypes.data_as(C.POINTER(C.c_float)) for w in W])
    bp = (C.POINTER(C.c_float) * len(b))(*[x.ctypes.data_as(C.POINTER(C.c_float)) for x in b])
    keep += [ns, ss, U, dm, W, b, Wp, bp]
    D = apex.LibraryDesc()
    D.n_reactions = len(n_slots)
    D.n_slots = ns.ctypes.data_as(C.POINTER(C.c_int32))
    D.slot_sizes = ss.ctypes.data_as(C.POINTER(C.c_int64))
    D.d = d
    D.U = U.ctypes.data_as(C.POINTER(C.c_float))
    D.n_layers = len(dims) - 1
    D.dims = dm.ctypes.data_as(C.POINTER(C.c_int32))
    D.W = C.cast(Wp, C.POINTER(C.POINTER(C.c_float)))
    D.b = C.cast(bp, C.POINTER(C.POINTER(C.c_float)))
    D.activation = act
    D.n_objectives = n_obj
    D.n_properties = dims[-1] - n_obj if n_prop is None else n_prop
    D.precisions = (1 << 0) | ((1 << 1) if prec else 0) if prec in (True, False) else prec
    return D, keep


@pytest.mark.parametrize("case,code", [
    (dict(n_slots=[], sizes=[], d=8, dims=[8, 4]), -1),                         # no reactions
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[7, 4]), -1),                    # dims[0] != d
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 4], n_prop=5), -1),          # n_obj + n_prop != outputs
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 4], act=9), -1),             # unknown activation
    (dict(n_slots=[2], sizes=[3, 0], d=8, dims=[8, 4]), -1),                    # empty slot
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 300, 4]), -1),               # hidden width > 256
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 64]), -1),                   # more than 32 outputs
    (dict(n_slots=[5], sizes=[2, 2, 2, 2, 2], d=8, dims=[8, 4]), -9),           # more than 4 slots
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 128, 256, 4]), -9),          # BF16 needs 256-wide hidden
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 128, 256, 4], prec=(1 << 0) | (1 << 3)), -9),  # so does FP16
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 4], prec=(1 << 0) | (1 << 2)), -1),  # FP64 is not a pass precision
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 128, 256, 4], prec=(1 << 0) | (1 << 4)), -9),  # FP8 needs 256-wide
    (dict(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 4], prec=(1 << 0) | (1 << 5)), -1),  # undefined bit
])
def test_load_rejects_before_touching_the_gpu(dll, case, code):
    D, keep = _desc(**case)
    h = C.c_void_p()
    rc = dll.apex_load_library(C.byref(D), C.byref(h))
    assert rc == code, dll.apex_last_error()
    assert not h.value
    assert len(dll.apex_last_error()) > 0


def test_load_rejects_ids_at_or_above_2_61(dll):
    """Candidate ids carry two flag bits above bit 60, so a library of 2^61 or more compounds is
    refused (before U is read: the descriptor's U here holds far fewer rows than its slots)."""
    D, keep = _desc(n_slots=[2], sizes=[3, 4], d=8, dims=[8, 4])
    for big, code in (([2 ** 31, 2 ** 30], -1), ([2 ** 30, 2 ** 30], None)):
        ss = np.asarray(big, np.int64)
        keep.append(ss)
        D.slot_sizes = ss.ctypes.data_as(C.POINTER(C.c_int64))
        if code is None:  # 2^60 compounds: past the id check (a GPU-less box then fails later)
            assert apex.apex_count_compounds([2], big) == 2 ** 60
            continue
        h = C.c_void_p()
        assert dll.apex_load_library(C.byref(D), C.byref(h)) == code
        assert not h.value and b"2^61" in dll.apex_last_error()


def test_null_arguments(dll):
    h = C.c_void_p()
    assert dll.apex_load_library(None, C.byref(h)) == -1
    assert dll.apex_free_library(None) == 0
    n = C.c_int64()
    assert dll.apex_topk_select(None, None, 10, 0, None, None, C.byref(n), None) == -1
    assert dll.apex_set_launch_shape(None, 1 << 20, 32) == -1
    cpu = C.c_int32()
    assert dll.apex_worker_cpu(None, C.byref(cpu)) == -1
    assert dll.apex_set_finalize_cover(None, 0) == -1


def test_library_file_rejected_before_the_gpu(dll, tmp_path):
    """Files that are missing, not library files, or truncated are refused with APEX_EINVAL
    before any device call."""
    h = C.c_void_p()
    assert dll.apex_load_library_file(str(tmp_path / "missing.apx").encode(), 0, None, 0, C.byref(h)) == -1
    bad = tmp_path / "bad.apx"
    bad.write_bytes(b"NOTAPEX!" + bytes(64))
    assert dll.apex_load_library_file(str(bad).encode(), 0, None, 0, C.byref(h)) == -1
    trunc = tmp_path / "trunc.apx"
    trunc.write_bytes(b"APEXLIB1" + np.array([1, 1, 8, 1, 0, 1, 0, 1], np.int32).tobytes() + bytes(8)
                      + np.array([2], np.int32).tobytes())  # stops inside the slot sizes
    assert dll.apex_load_library_file(str(trunc).encode(), 0, None, 0, C.byref(h)) == -1
    assert not h.value
