"""ctypes front end of the FP64 CPU oracle (apex_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg. It imports nothing from the CUDA package; inputs come from ``csl_gen``.
Every function computes in double precision what Sec. 3 (Eq. orig_topk / apex_topk) and
Sec. 3.2 (Eq. factorizer) define; see the header of apex_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from types import SimpleNamespace

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "apex_oracle.c")
LIB = os.path.join(HERE, "libapex_oracle.so")
ACT = {"identity": 0, "relu": 1, "silu": 2}


GCC_FLAGS = ["-O3", "-march=x86-64-v3", "-std=c11", "-fPIC", "-shared", "-pthread"]


def _source_hash() -> str:
    import hashlib

    h = hashlib.sha256(" ".join(GCC_FLAGS).encode())
    with open(SRC, "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (x86-64-v3 so the binary runs on any AVX2 host). Rebuilt whenever
    the source or the flags differ from those of the last build (sha256 stamp beside the binary)."""
    stamp = LIB + ".sha256"
    want = _source_hash()
    have = open(stamp).read().strip() if os.path.exists(stamp) else ""
    if force or not os.path.exists(LIB) or have != want:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *GCC_FLAGS, SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
        with open(stamp + f".tmp{os.getpid()}", "w") as f:
            f.write(want + "\n")
        os.replace(stamp + f".tmp{os.getpid()}", stamp)
    return LIB


class _Lib(C.Structure):
    _fields_ = [
        ("n_reactions", C.c_int32),
        ("n_slots", C.POINTER(C.c_int32)),
        ("slot_sizes", C.POINTER(C.c_int64)),
        ("d", C.c_int32),
        ("U", C.POINTER(C.c_float)),
        ("n_layers", C.c_int32),
        ("dims", C.POINTER(C.c_int32)),
        ("W", C.POINTER(C.POINTER(C.c_float))),
        ("b", C.POINTER(C.POINTER(C.c_float))),
        ("activation", C.c_int32),
    ]


class _Query(C.Structure):
    _fields_ = [
        ("n_weights", C.c_int32),
        ("weights", C.POINTER(C.c_double)),
        ("n_constraints", C.c_int32),
        ("output_index", C.POINTER(C.c_int32)),
        ("lower", C.POINTER(C.c_double)),
        ("upper", C.POINTER(C.c_double)),
        ("k", C.c_int64),
        ("n_subset", C.c_int32),
        ("subset", C.POINTER(C.c_int32)),
    ]


_dll = None


def _load():
    global _dll
    if _dll is None:
        _dll = C.CDLL(build())
        _dll.orc_count.restype = C.c_int64
        _dll.orc_count.argtypes = [C.POINTER(_Lib)]
        for name in ("orc_decode", "orc_head", "orc_score_ids", "orc_topk", "orc_linear_cost", "orc_assoc"):
            getattr(_dll, name).restype = C.c_int
    return _dll


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class OracleLibrary:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, lib, head=None):
        self.keep = []
        self.n_slots = np.ascontiguousarray(lib.n_slots, dtype=np.int32)
        self.slot_sizes = np.ascontiguousarray(lib.slot_sizes, dtype=np.int64)
        s = _Lib()
        s.n_reactions = int(self.n_slots.shape[0])
        s.n_slots = _p(self.n_slots, C.c_int32)
        s.slot_sizes = _p(self.slot_sizes, C.c_int64)
        s.d = int(lib.d)
        if getattr(lib, "U", None) is not None:
            self.U = np.ascontiguousarray(lib.U, dtype=np.float32)
            s.U = _p(self.U, C.c_float)
        if head is not None:
            self.dims = np.asarray(head.dims, dtype=np.int32)
            self.W = [np.ascontiguousarray(w, dtype=np.float32) for w in head.W]
            self.b = [np.ascontiguousarray(x, dtype=np.float32) for x in head.b]
            Wp = (C.POINTER(C.c_float) * len(self.W))(*[_p(w, C.c_float) for w in self.W])
            bp = (C.POINTER(C.c_float) * len(self.b))(*[_p(x, C.c_float) for x in self.b])
            self.keep += [Wp, bp]
            s.n_layers = len(self.W)
            s.dims = _p(self.dims, C.c_int32)
            s.W = C.cast(Wp, C.POINTER(C.POINTER(C.c_float)))
            s.b = C.cast(bp, C.POINTER(C.POINTER(C.c_float)))
            s.activation = ACT[head.activation]
            self.n_outputs = int(head.dims[-1])
        self.s = s


def count(lib) -> int:
    """N = sum_t prod_j |slot_{t,j}| (App. A.1)."""
    L = OracleLibrary(lib)
    return int(_load().orc_count(C.byref(L.s)))


def linear_cost(n_slots, slot_sizes, d):
    """Sec. 3.3 cost model for a linear-probe head: (cache bytes, precompute flops, total flops, N)."""
    n_slots = np.ascontiguousarray(n_slots, dtype=np.int32)
    slot_sizes = np.ascontiguousarray(slot_sizes, dtype=np.int64)
    cb, pf, tf = C.c_double(), C.c_double(), C.c_double()
    n = C.c_int64()
    rc = _load().orc_linear_cost(int(n_slots.shape[0]), _p(n_slots, C.c_int32), _p(slot_sizes, C.c_int64), int(d),
                                 C.byref(cb), C.byref(pf), C.byref(tf), C.byref(n))
    if rc != 0:
        raise ValueError(f"orc_linear_cost failed ({rc})")
    return cb.value, pf.value, tf.value, n.value


def decode(lib, ids, max_slots: int = 8):
    """Global ids -> (reaction [n], synthon indices [n, max_slots], -1 padded)."""
    L = OracleLibrary(lib)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    t = np.empty(ids.shape[0], dtype=np.int32)
    s = np.empty((ids.shape[0], max_slots), dtype=np.int64)
    rc = _load().orc_decode(C.byref(L.s), int(ids.shape[0]), _p(ids, C.c_int64), _p(t, C.c_int32),
                            _p(s, C.c_int64), int(max_slots))
    if rc != 0:
        raise ValueError(f"orc_decode failed ({rc})")
    return t, s


def head_eval(head, g):
    """Head applied to given embeddings g [n, d] in FP64 -> [n, n_outputs]."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    shape = SimpleNamespace(n_slots=np.array([1], np.int32), slot_sizes=np.array([1], np.int64), d=head.dims[0],
                            U=None)
    L = OracleLibrary(shape, head)
    out = np.empty((g.shape[0], head.dims[-1]), dtype=np.float64)
    rc = _load().orc_head(C.byref(L.s), int(g.shape[0]), _p(g, C.c_double), _p(out, C.c_double))
    if rc != 0:
        raise ValueError(f"orc_head failed ({rc})")
    return out


def score_ids(lib, head, ids, threads: int = 0):
    """FP64 outputs of the given compounds, [n, n_outputs]."""
    L = OracleLibrary(lib, head)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    out = np.empty((ids.shape[0], L.n_outputs), dtype=np.float64)
    rc = _load().orc_score_ids(C.byref(L.s), int(ids.shape[0]), _p(ids, C.c_int64), _p(out, C.c_double),
                               int(threads))
    if rc != 0:
        raise ValueError(f"orc_score_ids failed ({rc})")
    return out


class TopK:
    def __init__(self, ids, scores, outputs, n_feasible, n_enumerated):
        self.ids, self.scores, self.outputs = ids, scores, outputs
        self.n_feasible, self.n_enumerated = n_feasible, n_enumerated


def topk(lib, head, query, threads: int = 0) -> TopK:
    """Exhaustive FP64 top-k of Eq. apex_topk under the query (csl_gen.Query)."""
    L = OracleLibrary(lib, head)
    w = np.ascontiguousarray(query.weights, dtype=np.float64)
    idx = np.ascontiguousarray(query.cons_idx, dtype=np.int32)
    lo = np.ascontiguousarray(query.lo, dtype=np.float64)
    hi = np.ascontiguousarray(query.hi, dtype=np.float64)
    sub = None if query.subset is None else np.ascontiguousarray(query.subset, dtype=np.int32)
    q = _Query()
    q.n_weights = int(w.shape[0])
    q.weights = _p(w, C.c_double)
    q.n_constraints = int(idx.shape[0])
    q.output_index = _p(idx, C.c_int32)
    q.lower = _p(lo, C.c_double)
    q.upper = _p(hi, C.c_double)
    q.k = int(query.k)
    q.n_subset = 0 if sub is None else int(sub.shape[0])
    q.subset = _p(sub, C.c_int32) if sub is not None else C.POINTER(C.c_int32)()
    k = int(query.k)
    ids = np.empty(k, dtype=np.int64)
    scores = np.empty(k, dtype=np.float64)
    outs = np.empty((k, L.n_outputs), dtype=np.float64)
    n_out, n_feas, n_en = C.c_int64(), C.c_int64(), C.c_int64()
    rc = _load().orc_topk(C.byref(L.s), C.byref(q), int(threads), _p(ids, C.c_int64), _p(scores, C.c_double),
                          _p(outs, C.c_double), C.byref(n_out), C.byref(n_feas), C.byref(n_en))
    if rc != 0:
        raise ValueError(f"orc_topk failed ({rc})")
    n = n_out.value
    return TopK(ids[:n].copy(), scores[:n].copy(), outs[:n].copy(), n_feas.value, n_en.value)


def assoc_embeddings(slot_sizes, K, V):
    """Eq. assoc_embeds: u_{r,s} = K_r v_s for every synthon row of every slot (FP64).
    slot_sizes: [n_slots_total]; K: float32 [n_slots_total, d, d_u]; V: float32 [rows, d_u] (rows
    slot-major). Returns float64 [rows, d]."""
    sizes = np.ascontiguousarray(slot_sizes, dtype=np.int64)
    K = np.ascontiguousarray(K, dtype=np.float32)
    V = np.ascontiguousarray(V, dtype=np.float32)
    n_slots, d, d_u = K.shape
    assert sizes.shape[0] == n_slots and V.shape == (int(sizes.sum()), d_u)
    U = np.empty((V.shape[0], d), dtype=np.float64)
    rc = _load().orc_assoc(C.c_int64(n_slots), _p(sizes, C.c_int64), C.c_int32(d), C.c_int32(d_u), _p(K, C.c_float),
                           _p(V, C.c_float), _p(U, C.c_double))
    if rc != 0:
        raise ValueError("orc_assoc failed")
    return U
