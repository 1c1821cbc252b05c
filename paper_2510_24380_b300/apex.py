"""Thin ctypes binding of libapex_b300.so (include/apex.h): argument marshalling only.

Every computation runs in the CUDA library; this module only converts numpy arrays and
Python values into the C structs and back. It fails loudly when the library is missing.
The functions keep the C names; ``Library`` wraps them for csl_gen inputs.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libapex_b300.so")

APEX_OK = 0
STATUS = {0: "APEX_OK", -1: "APEX_EINVAL", -2: "APEX_ENOMEM", -3: "APEX_EBUSY", -4: "APEX_EAGAIN",
          -5: "APEX_ETIMEDOUT", -6: "APEX_ECANCELED", -7: "APEX_ECUDA", -8: "APEX_ENOTFOUND",
          -9: "APEX_EUNSUPPORTED"}
APEX_EAGAIN = -4
ACT = {"identity": 0, "relu": 1, "silu": 2}
PREC = {"fp32": 0, "bf16": 1, "fp64": 2, "fp16": 3, "fp8": 4}
MAX_SLOTS = 4
MAX_OUTPUTS = 32


class ApexError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class LibraryDesc(C.Structure):
    _fields_ = [
        ("n_reactions", C.c_int32), ("n_slots", C.POINTER(C.c_int32)), ("slot_sizes", C.POINTER(C.c_int64)),
        ("d", C.c_int32), ("U", C.POINTER(C.c_float)), ("U_on_device", C.c_int32), ("n_layers", C.c_int32),
        ("dims", C.POINTER(C.c_int32)), ("W", C.POINTER(C.POINTER(C.c_float))), ("b", C.POINTER(C.POINTER(C.c_float))),
        ("activation", C.c_int32), ("n_objectives", C.c_int32), ("n_properties", C.c_int32),
        ("precisions", C.c_uint32), ("device_mem_budget", C.c_uint64), ("cuda_stream", C.c_void_p),
        ("device", C.c_int32), ("seed", C.c_uint64),
    ]


class QueryDesc(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("objective_weights", C.POINTER(C.c_float)), ("n_constraints", C.c_int32),
        ("output_index", C.POINTER(C.c_int32)), ("lower", C.POINTER(C.c_double)), ("upper", C.POINTER(C.c_double)),
        ("k", C.c_int64), ("n_reaction_subset", C.c_int32), ("reactions", C.POINTER(C.c_int32)),
    ]


class LibraryInfo(C.Structure):
    _fields_ = [
        ("n_compounds", C.c_int64), ("n_synthon_rows", C.c_int64), ("max_slots", C.c_int32),
        ("n_outputs", C.c_int32), ("device_bytes", C.c_uint64), ("precisions", C.c_uint32),
        ("n_calibration", C.c_int32), ("err_bf16", C.c_double * MAX_OUTPUTS), ("err_fp16", C.c_double * MAX_OUTPUTS),
        ("err_fp8", C.c_double * MAX_OUTPUTS),
        ("err_fp32", C.c_double * MAX_OUTPUTS),
        ("rms", C.c_double * MAX_OUTPUTS),
    ]


AUTOTUNE_MAX = 8


class AutotuneDesc(C.Structure):
    _fields_ = [("precision", C.c_int32), ("n_queries", C.c_int32), ("k", C.c_int64), ("n_reaction_subset", C.c_int32),
                ("reactions", C.POINTER(C.c_int32))]


class AutotuneResult(C.Structure):
    _fields_ = [("n_chunk_candidates", C.c_int32), ("chunk_compounds", C.c_int64 * AUTOTUNE_MAX),
                ("chunk_ms", C.c_double * AUTOTUNE_MAX), ("fp32_id_tile_ms", C.c_double * 2),
                ("chosen_chunk_compounds", C.c_int64), ("chosen_fp32_id_tile", C.c_int32)]


class QueryStats(C.Structure):
    _fields_ = [
        ("n_scope", C.c_int64), ("n_scored", C.c_int64), ("n_candidates", C.c_int64), ("n_rescored_fp64", C.c_int64),
        ("n_feasible_lower", C.c_int64), ("n_restarts", C.c_int32), ("n_launches", C.c_int32),
        ("queue_ms", C.c_double), ("latency_ms", C.c_double), ("gpu_ms", C.c_double), ("enumerate_ms", C.c_double),
        ("host_start_ms", C.c_double), ("host_pass_ms", C.c_double), ("host_finalize_ms", C.c_double),
        ("n_margin_reruns", C.c_int32), ("n_compactions", C.c_int32), ("pass_err_ratio", C.c_double),
        ("fp32_err_ratio", C.c_double), ("first_item", C.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServingStats(C.Structure):
    _fields_ = [
        ("n_queries", C.c_int64), ("n_failed", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
        ("max_ms", C.c_double), ("mean_ms", C.c_double), ("queue_p50_ms", C.c_double), ("queue_p99_ms", C.c_double),
        ("wall_ms", C.c_double), ("query_compounds", C.c_double), ("head_evaluations", C.c_double),
        ("query_compounds_per_s", C.c_double), ("head_evaluations_per_s", C.c_double),
        ("enumerate_ms", C.c_double), ("n_enumeration_launches", C.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_dll = None

SYMBOLS = {
    "apex_count_compounds": [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "apex_load_library": [C.POINTER(LibraryDesc), C.POINTER(C.c_void_p)],
    "apex_free_library": [C.c_void_p],
    "apex_library_info": [C.c_void_p, C.POINTER(LibraryInfo)],
    "apex_query": [C.c_void_p, C.POINTER(QueryDesc), C.POINTER(C.c_int64)],
    "apex_topk_fetch": [C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                        C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64),
                        C.c_int32],
    "apex_cancel": [C.c_void_p, C.c_int64],
    "apex_query_stats": [C.c_void_p, C.c_int64, C.POINTER(QueryStats)],
    "apex_stats": [C.c_void_p, C.POINTER(ServingStats)],
    "apex_stats_reset": [C.c_void_p],
    "apex_worker_cpu": [C.c_void_p, C.POINTER(C.c_int32)],
    "apex_set_finalize_cover": [C.c_void_p, C.c_int64],
    "apex_score_ids": [C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_double)],
    "apex_dump_outputs": [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_float), C.c_int64],
    "apex_decode_ids": [C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int64)],
    "apex_topk_select": [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64),
                         C.c_void_p],
    "apex_topk_select_noalloc": [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                 C.POINTER(C.c_int64), C.c_void_p],
    "apex_kernel_launches": [C.POINTER(C.c_int64)],
    "apex_selftest_wait_timeout": [C.c_void_p, C.c_int32],
    "apex_autotune": [C.c_void_p, C.POINTER(AutotuneDesc), C.POINTER(AutotuneResult)],
    "apex_set_launch_shape": [C.c_void_p, C.c_int64, C.c_int32],
    "apex_save_library": [C.c_void_p, C.c_char_p],
    "apex_load_library_file": [C.c_char_p, C.c_int32, C.c_void_p, C.c_uint64, C.POINTER(C.c_void_p)],
    "apex_associative_embeddings": [C.c_int64, C.POINTER(C.c_int64), C.c_int32, C.c_int32, C.POINTER(C.c_float),
                                    C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int32, C.c_void_p],
    "apex_last_error": [],
}


def load(path: str = LIB_PATH):
    """Loads the CUDA library (never falls back to anything else)."""
    global _dll
    if _dll is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with `python -m paper_2510_24380_b300.build`")
        dll = C.CDLL(path)
        for name, args in SYMBOLS.items():
            fn = getattr(dll, name)
            fn.argtypes = args
            fn.restype = C.c_int32
        dll.apex_last_error.restype = C.c_char_p
        _dll = dll
    return _dll


def associative_embeddings(slot_sizes, K, V, stream=None):
    """Eq. assoc_embeds on the GPU: U[row] = K[slot(row)] @ V[row] (host numpy in and out)."""
    sizes = np.ascontiguousarray(slot_sizes, np.int64)
    K = np.ascontiguousarray(K, np.float32)
    V = np.ascontiguousarray(V, np.float32)
    n, d, d_u = K.shape
    U = np.empty((V.shape[0], d), np.float32)
    _check(load().apex_associative_embeddings(int(n), _p(sizes, C.c_int64), int(d), int(d_u), _p(K, C.c_float),
                                              _p(V, C.c_float), _p(U, C.c_float), 0, C.c_void_p(stream or 0)),
           "apex_associative_embeddings")
    return U


def last_error() -> str:
    """The calling thread's last error message from the library."""
    return load().apex_last_error().decode(errors="replace")


def _check(code, what=""):
    if code != APEX_OK:
        msg = load().apex_last_error().decode(errors="replace")
        raise ApexError(code, f"{what}: {msg}")


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ---------------------------------------------------------------- C-named thin wrappers
def apex_count_compounds(n_slots, slot_sizes) -> int:
    ns = np.ascontiguousarray(n_slots, np.int32)
    ss = np.ascontiguousarray(slot_sizes, np.int64)
    out = C.c_int64()
    _check(load().apex_count_compounds(int(ns.shape[0]), _p(ns, C.c_int32), _p(ss, C.c_int64), C.byref(out)),
           "apex_count_compounds")
    return out.value


class Library:
    """A loaded library (apex_load_library) built from csl_gen's CSL and Head."""

    def __init__(self, lib, head, precisions=("fp32", "bf16", "fp16"), device: int = 0, stream=None, budget: int = 0,
                 seed: int = 0, U_device=None):
        dll = load()
        self._keep = []
        ns = np.ascontiguousarray(lib.n_slots, np.int32)
        ss = np.ascontiguousarray(lib.slot_sizes, np.int64)
        dims = np.asarray(head.dims, np.int32)
        W = [np.ascontiguousarray(w, np.float32) for w in head.W]
        b = [np.ascontiguousarray(x, np.float32) for x in head.b]
        Wp = (C.POINTER(C.c_float) * len(W))(*[_p(w, C.c_float) for w in W])
        bp = (C.POINTER(C.c_float) * len(b))(*[_p(x, C.c_float) for x in b])
        self._keep += [ns, ss, dims, W, b, Wp, bp]
        D = LibraryDesc()
        D.n_reactions = int(ns.shape[0])
        D.n_slots = _p(ns, C.c_int32)
        D.slot_sizes = _p(ss, C.c_int64)
        D.d = int(lib.d)
        if U_device is not None:
            D.U = C.cast(C.c_void_p(int(U_device)), C.POINTER(C.c_float))
            D.U_on_device = 1
        else:
            U = np.ascontiguousarray(lib.U, np.float32)
            self._keep.append(U)
            D.U = _p(U, C.c_float)
            D.U_on_device = 0
        D.n_layers = len(W)
        D.dims = _p(dims, C.c_int32)
        D.W = C.cast(Wp, C.POINTER(C.POINTER(C.c_float)))
        D.b = C.cast(bp, C.POINTER(C.POINTER(C.c_float)))
        D.activation = ACT[head.activation]
        D.n_objectives = int(head.n_objectives)
        D.n_properties = int(head.n_properties)
        D.precisions = sum(1 << PREC[p] for p in set(precisions))
        D.device_mem_budget = int(budget)
        D.cuda_stream = stream
        D.device = int(device)
        D.seed = int(seed)
        h = C.c_void_p()
        _check(dll.apex_load_library(C.byref(D), C.byref(h)), "apex_load_library")
        self._keep = [dims]
        self.h = h
        self.n_outputs = int(head.dims[-1])
        self.n_objectives = int(head.n_objectives)

    @classmethod
    def from_file(cls, path: str, n_objectives: int, device: int = 0, stream=None, budget: int = 0) -> "Library":
        """A library rebuilt from a file written by save() (apex_load_library_file)."""
        self = cls.__new__(cls)
        self._keep = []
        h = C.c_void_p()
        _check(load().apex_load_library_file(str(path).encode(), int(device), C.c_void_p(stream or 0), int(budget),
                                             C.byref(h)), "apex_load_library_file")
        self.h = h
        self.n_outputs = int(self.info().n_outputs)
        self.n_objectives = int(n_objectives)
        return self

    def save(self, path: str):
        """Writes the library (shapes, U, head, margins) to a file (apex_save_library)."""
        _check(load().apex_save_library(self.h, str(path).encode()), "apex_save_library")

    def close(self):
        if self.h:
            load().apex_free_library(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> LibraryInfo:
        out = LibraryInfo()
        _check(load().apex_library_info(self.h, C.byref(out)), "apex_library_info")
        return out

    def query(self, q) -> int:
        """apex_query for a csl_gen.Query; returns the query id."""
        w = np.ascontiguousarray(q.weights, np.float32)
        idx = np.ascontiguousarray(q.cons_idx, np.int32)
        lo = np.ascontiguousarray(q.lo, np.float64)
        hi = np.ascontiguousarray(q.hi, np.float64)
        sub = None if q.subset is None else np.ascontiguousarray(q.subset, np.int32)
        D = QueryDesc()
        D.precision = PREC[q.precision]
        D.objective_weights = _p(w, C.c_float)
        D.n_constraints = int(idx.shape[0])
        D.output_index = _p(idx, C.c_int32)
        D.lower = _p(lo, C.c_double)
        D.upper = _p(hi, C.c_double)
        D.k = int(q.k)
        D.n_reaction_subset = 0 if sub is None else int(sub.shape[0])
        D.reactions = _p(sub, C.c_int32) if sub is not None else C.POINTER(C.c_int32)()
        qid = C.c_int64()
        _check(load().apex_query(self.h, C.byref(D), C.byref(qid)), "apex_query")
        return qid.value

    def fetch(self, qid: int, capacity: int, timeout_ms: int = -1):
        """apex_topk_fetch into fresh host arrays; returns a dict (or None on EAGAIN)."""
        cap = int(capacity)
        ids = np.empty(cap, np.int64)
        rxn = np.empty(cap, np.int32)
        syn = np.empty((cap, MAX_SLOTS), np.int64)
        obj = np.empty(cap, np.float64)
        out = np.empty((cap, self.n_outputs), np.float64)
        n = C.c_int64()
        code = load().apex_topk_fetch(self.h, int(qid), cap, _p(ids, C.c_int64), _p(rxn, C.c_int32),
                                      _p(syn, C.c_int64), _p(obj, C.c_double), _p(out, C.c_double), C.byref(n),
                                      int(timeout_ms))
        if code == APEX_EAGAIN:
            return None
        _check(code, "apex_topk_fetch")
        m = min(n.value, cap)
        return {"ids": ids[:m], "reaction": rxn[:m], "synthons": syn[:m], "objective": obj[:m],
                "outputs": out[:m], "n": n.value}

    def run(self, q, timeout_ms: int = -1):
        qid = self.query(q)
        return self.fetch(qid, int(q.k), timeout_ms)

    def cancel(self, qid: int):
        _check(load().apex_cancel(self.h, int(qid)), "apex_cancel")

    def stats(self, qid: int = -1) -> dict:
        s = QueryStats()
        _check(load().apex_query_stats(self.h, int(qid), C.byref(s)), "apex_query_stats")
        return s.as_dict()

    def serving_stats(self) -> dict:
        """Latency percentiles and throughput over the queries fetched since load or reset (apex_stats)."""
        s = ServingStats()
        _check(load().apex_stats(self.h, C.byref(s)), "apex_stats")
        return s.as_dict()

    def reset_serving_stats(self):
        _check(load().apex_stats_reset(self.h), "apex_stats_reset")

    def score_ids(self, ids, precision: str = "fp32"):
        ids = np.ascontiguousarray(ids, np.int64)
        out = np.empty((ids.shape[0], self.n_outputs), np.float64)
        _check(load().apex_score_ids(self.h, PREC[precision], int(ids.shape[0]), _p(ids, C.c_int64),
                                     _p(out, C.c_double)), "apex_score_ids")
        return out

    def dump_outputs(self, reaction: int, n_compounds: int, precision: str = "bf16"):
        out = np.empty((int(n_compounds), self.n_outputs), np.float32)
        _check(load().apex_dump_outputs(self.h, PREC[precision], int(reaction), _p(out, C.c_float),
                                        int(n_compounds)), "apex_dump_outputs")
        return out

    def autotune(self, precision: str = "fp16", n_queries: int = 8, k: int = 1000, subset=None) -> dict:
        """Times trial queries to pick the launch shapes (compounds per launch, FP32 id tile)."""
        d = AutotuneDesc()
        d.precision = PREC[precision]
        d.n_queries = int(n_queries)
        d.k = int(k)
        sub = None if subset is None else np.ascontiguousarray(subset, np.int32)
        d.n_reaction_subset = 0 if sub is None else int(sub.shape[0])
        d.reactions = None if sub is None else _p(sub, C.c_int32)
        r = AutotuneResult()
        _check(load().apex_autotune(self.h, C.byref(d), C.byref(r)), "apex_autotune")
        n = r.n_chunk_candidates
        return {"chunk_compounds": list(r.chunk_compounds)[:n], "chunk_ms": [round(x, 3) for x in list(r.chunk_ms)[:n]],
                "fp32_id_tile_ms": [round(x, 3) for x in r.fp32_id_tile_ms],
                "chosen_chunk_compounds": int(r.chosen_chunk_compounds), "chosen_fp32_id_tile": int(r.chosen_fp32_id_tile)}

    def set_launch_shape(self, chunk_compounds: int, fp32_id_tile: int = 32):
        """Compounds per enumeration launch and FP32 id-list tile rows, by hand (what autotune picks)."""
        _check(load().apex_set_launch_shape(self.h, int(chunk_compounds), int(fp32_id_tile)), "apex_set_launch_shape")

    def set_finalize_cover(self, cover: int = 0):
        """Candidates the queued finalization covers before the count is known (0: default)."""
        _check(load().apex_set_finalize_cover(self.h, int(cover)), "apex_set_finalize_cover")

    def worker_cpu(self) -> int:
        """CPU the library's worker thread is pinned to (-1: not pinned)."""
        c = C.c_int32()
        _check(load().apex_worker_cpu(self.h, C.byref(c)), "apex_worker_cpu")
        return c.value

    def keep_caller_off_worker_cpu(self) -> int:
        """Moves the calling thread off the worker's CPU (when it is pinned and other CPUs are
        allowed), so that the caller's polling and Python work never share a core with the thread
        that issues the CUDA calls. Returns the worker's CPU."""
        cpu = self.worker_cpu()
        if cpu >= 0 and hasattr(os, "sched_getaffinity"):
            allowed = os.sched_getaffinity(0)
            if cpu in allowed and len(allowed) > 1:
                os.sched_setaffinity(0, allowed - {cpu})
        return cpu

    def selftest_wait_timeout(self, limit_ms: int = 50) -> int:
        """Runs the device-wait self-test; returns the status code (APEX_ETIMEDOUT = -5 expected)."""
        return int(load().apex_selftest_wait_timeout(self.h, int(limit_ms)))

    def decode(self, ids):
        ids = np.ascontiguousarray(ids, np.int64)
        t = np.empty(ids.shape[0], np.int32)
        s = np.empty((ids.shape[0], MAX_SLOTS), np.int64)
        _check(load().apex_decode_ids(self.h, int(ids.shape[0]), _p(ids, C.c_int64), _p(t, C.c_int32),
                                      _p(s, C.c_int64)), "apex_decode_ids")
        return t, s


def apex_kernel_launches() -> int:
    out = C.c_int64()
    _check(load().apex_kernel_launches(C.byref(out)), "apex_kernel_launches")
    return out.value


def apex_topk_select(keys_ptr: int, ids_ptr: int, n: int, k: int, out_keys_ptr: int, out_ids_ptr: int,
                     stream: int | None = None) -> int:
    """Device pointers in, device pointers out; returns n_out."""
    n_out = C.c_int64()
    _check(load().apex_topk_select(C.c_void_p(keys_ptr), C.c_void_p(ids_ptr), int(n), int(k), C.c_void_p(out_keys_ptr),
                                   C.c_void_p(out_ids_ptr), C.byref(n_out), C.c_void_p(stream or 0)),
           "apex_topk_select")
    return n_out.value


NOALLOC_MAX_K = 65536


def apex_topk_select_noalloc(keys_ptr: int, ids_ptr: int, n: int, k: int, out_keys_ptr: int, out_ids_ptr: int,
                             stream: int | None = None) -> int:
    """apex_topk_select with static device scratch (no allocation); device pointers; returns n_out."""
    n_out = C.c_int64()
    _check(load().apex_topk_select_noalloc(C.c_void_p(keys_ptr), C.c_void_p(ids_ptr), int(n), int(k),
                                           C.c_void_p(out_keys_ptr), C.c_void_p(out_ids_ptr), C.byref(n_out),
                                           C.c_void_p(stream or 0)), "apex_topk_select_noalloc")
    return n_out.value
