"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: the paper's worked
numbers (Sec. 3.3, App. A.1), closed forms, a textbook reduction (Eq. apex for a linear head
is a top-k of X+Y sums, checked by a full numpy sort), brute force on tiny libraries, the
lexicographic (c, f0) priority queue of Sec. 3.3, and invariants (permutations, k, boxes).
"""
import heapq
import itertools
import json
import math
import os

import numpy as np
import pytest

import csl_gen
from csl_gen.library import CSL, Head, make_head, library_from_sizes
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _query(w, idx=(), lo=(), hi=(), k=10, subset=None):
    return csl_gen.Query(np.asarray(w, np.float32), np.asarray(idx, np.int32), np.asarray(lo, np.float64),
                         np.asarray(hi, np.float64), int(k), None if subset is None else np.asarray(subset, np.int32))


def _shape(sizes):
    return library_from_sizes(sizes, d=4, seed=0, materialize=False)


# ---------------------------------------------------------------- counting and cost (App. A.1, Sec. 3.3)
def test_count_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "paper_worked_example.json")))
    n = g["library"]["synthons_per_slot"]
    lib = _shape([[n] * g["library"]["n_slots"]])
    assert O.count(lib) == g["n_compounds"]


def test_linear_cost_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "paper_worked_example.json")))
    n = g["library"]["synthons_per_slot"]
    cache, pre, total, N = O.linear_cost([3], [n, n, n], g["d"])
    assert N == g["n_compounds"]
    assert abs(cache - g["cache_bytes_about"]) <= g["cache_tolerance_rel"] * g["cache_bytes_about"]
    assert pre == g["precompute_flops"]
    assert total == g["total_flops"]
    assert total / N == g["flops_per_compound"]


def test_count_equals_enumerated_and_ids_are_a_permutation():
    lib, head, spec = csl_gen.build_workload("t_ragged")
    N = O.count(lib)
    assert N == sum(math.prod(int(x) for x in s) for s in csl_gen.workload_sizes("t_ragged"))
    r = O.topk(lib, head, _query([1, 0, 0, 0, 0], k=N + 5))
    assert r.n_enumerated == N and r.n_feasible == N and len(r.ids) == N
    assert np.array_equal(np.sort(r.ids), np.arange(N))


def test_count_overflow_rejected():
    lib = _shape([[2 ** 32, 2 ** 32]])
    assert O.count(lib) == -1


# ---------------------------------------------------------------- head: closed forms
def _scalar_head(act):
    # 1 -> 1 -> 1 head with unit weights: z = 0 * 1 + x (bias carries x), o = act(z)
    return Head(dims=[1, 1, 1], activation=act, W=[np.ones((1, 1), np.float32), np.ones((1, 1), np.float32)],
                b=[np.zeros(1, np.float32), np.zeros(1, np.float32)], n_objectives=1)


@pytest.mark.parametrize("act", ["relu", "silu", "identity"])
def test_activation_closed_forms(act):
    pts = json.load(open(os.path.join(GOLDEN, "activation_points.json")))[act]
    h = _scalar_head(act)
    for x, y in pts:
        out = O.head_eval(h, np.array([[x]]))[0, 0]
        assert out == pytest.approx(y, rel=1e-15, abs=1e-300), (act, x, out, y)


def test_identity_activation_collapses_to_one_affine_map():
    dims = [5, 7, 6, 3]
    h = make_head(dims, "identity", seed=3, n_objectives=1, n_properties=2)
    W = [w.astype(np.float64) for w in h.W]
    b = [x.astype(np.float64) for x in h.b]
    A = W[2] @ W[1] @ W[0]
    c = W[2] @ (W[1] @ b[0] + b[1]) + b[2]
    g = np.random.default_rng(0).standard_normal((20, 5))
    assert np.allclose(O.head_eval(h, g), g @ A.T + c, rtol=1e-12, atol=1e-12)


def test_relu_head_on_positive_orthant_is_affine():
    # with all weights/biases >= 0 and inputs >= 0 every ReLU is the identity
    h = make_head([4, 6, 2], "relu", seed=5, n_objectives=1, n_properties=1)
    h.W = [np.abs(w) for w in h.W]
    h.b = [np.abs(x) for x in h.b]
    g = np.abs(np.random.default_rng(1).standard_normal((9, 4)))
    W0, W1 = (w.astype(np.float64) for w in h.W)
    ref = (g @ W0.T + h.b[0]) @ W1.T + h.b[1]
    assert np.allclose(O.head_eval(h, g), ref, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- Eq. apex: linear head = X + Y sums
def test_linear_head_reduces_to_eq_apex_xy_sums():
    lib = library_from_sizes([[40, 60]], d=16, seed=21)
    h = make_head([16, 3], "identity", seed=22, n_objectives=1, n_properties=2)
    w0 = h.W[0][0].astype(np.float64)
    U = lib.U.astype(np.float64)
    X = U[:40] @ w0               # synthon contributions v_{0,r,s} of slot 1 (Eq. apex)
    Y = U[40:] @ w0               # slot 2
    scores = (X[:, None] + Y[None, :] + float(h.b[0][0])).ravel()   # id = s1 * 60 + s2
    order = np.lexsort((np.arange(scores.size), -scores))
    k = 37
    r = O.topk(lib, h, _query([1.0], k=k))
    assert np.array_equal(r.ids, order[:k])
    assert np.allclose(r.scores, scores[order[:k]], rtol=0, atol=1e-12)


def test_one_slot_reactions_are_a_plain_sort():
    lib = library_from_sizes([[50], [30]], d=8, seed=4)
    h = make_head([8, 5, 2], "silu", seed=6, n_objectives=1, n_properties=1)
    per = O.head_eval(h, lib.U.astype(np.float64))[:, 0]
    order = np.lexsort((np.arange(80), -per))
    r = O.topk(lib, h, _query([1.0], k=25))
    assert np.array_equal(r.ids, order[:25])


# ---------------------------------------------------------------- brute force on tiny libraries
def _brute(lib, h, w, idx, lo, hi):
    """Materialize every compound by itertools.product in id order; numpy head; returns all rows."""
    U = lib.U.astype(np.float64)
    rows = []
    rf = lib.row_first
    sf = lib.slot_first
    for t in range(lib.n_reactions):
        sizes = lib.sizes_of(t)
        for combo in itertools.product(*[range(int(n)) for n in sizes]):
            g = sum(U[rf[sf[t] + j] + s] for j, s in enumerate(combo))
            a = g
            for l in range(len(h.W)):
                z = h.W[l].astype(np.float64) @ a + h.b[l].astype(np.float64)
                if l < len(h.W) - 1:
                    z = {"relu": np.maximum(z, 0), "silu": z / (1 + np.exp(-z)), "identity": z}[h.activation]
                a = z
            rows.append(a)
    o = np.array(rows)
    f = o[:, : len(w)] @ np.asarray(w, np.float32).astype(np.float64)
    feas = np.ones(len(o), bool)
    for i, l, u in zip(idx, lo, hi):
        feas &= (o[:, i] >= l) & (o[:, i] <= u)
    return o, f, feas


TINY = [[3, 4], [2, 3, 2], [5], [1, 1, 2]]


@pytest.mark.parametrize("act", ["silu", "relu"])
@pytest.mark.parametrize("k", [1, 7, 100])
def test_brute_force_tiny(act, k):
    lib = library_from_sizes(TINY, d=8, seed=30)
    h = make_head([8, 6, 5, 4], act, seed=31, n_objectives=2, n_properties=2)
    w = [0.7, -0.3]
    o, f, feas = _brute(lib, h, w, [2, 3], [-0.5, -1.0], [0.5, 0.3])
    ids = np.flatnonzero(feas)
    order = ids[np.lexsort((ids, -f[ids]))][:k]
    r = O.topk(lib, h, _query(w, [2, 3], [-0.5, -1.0], [0.5, 0.3], k=k))
    assert r.n_enumerated == len(o)
    assert r.n_feasible == int(feas.sum())
    assert np.array_equal(r.ids, order)
    assert np.allclose(r.scores, f[order], rtol=0, atol=1e-12)
    assert np.allclose(r.outputs, o[order], rtol=0, atol=1e-12)


def test_lexicographic_queue_equivalence():
    """Sec. 3.3: a size-k priority queue on (c, f0) in lexicographic order, then removal of
    c < 0, yields the same set as filtering feasible compounds and taking the top-k."""
    lib = library_from_sizes(TINY, d=8, seed=40)
    h = make_head([8, 6, 4], "silu", seed=41, n_objectives=1, n_properties=3)
    idx, lo, hi = [1, 2, 3], [-0.4, -0.3, -np.inf], [0.4, 0.5, 0.2]
    o, f, _ = _brute(lib, h, [1.0], idx, lo, hi)
    c = np.zeros(len(o))
    for i, l, u in zip(idx, lo, hi):
        c -= np.maximum(0.0, l - o[:, i]) + np.maximum(0.0, o[:, i] - u)
    for k in (1, 5, 12, 60):
        heap = []  # min-heap of (c, f0, -id): root = lexicographically smallest
        for i in range(len(o)):
            item = (c[i], f[i], -i)
            if len(heap) < k:
                heapq.heappush(heap, item)
            elif item > heap[0]:
                heapq.heapreplace(heap, item)
        kept = sorted([it for it in heap if it[0] >= 0], key=lambda it: (-it[1], -it[2]))
        r = O.topk(lib, h, _query([1.0], idx, lo, hi, k=k))
        assert [-it[2] for it in kept] == list(r.ids)


# ---------------------------------------------------------------- special cases
def test_infinite_bounds_equal_unconstrained():
    lib, head, _ = csl_gen.build_workload("t_ragged")
    a = O.topk(lib, head, _query([1, 0, 0, 0, 0], [5, 6], [-np.inf, -np.inf], [np.inf, np.inf], k=40))
    b = O.topk(lib, head, _query([1, 0, 0, 0, 0], k=40))
    assert np.array_equal(a.ids, b.ids) and np.array_equal(a.scores, b.scores)


def test_k_above_feasible_returns_all_feasible_sorted_and_empty_box():
    lib = library_from_sizes(TINY, d=8, seed=50)
    h = make_head([8, 4, 3], "silu", seed=51, n_objectives=1, n_properties=2)
    o, f, feas = _brute(lib, h, [1.0], [1], [0.0], [np.inf])
    r = O.topk(lib, h, _query([1.0], [1], [0.0], [np.inf], k=1000))
    assert len(r.ids) == int(feas.sum()) == r.n_feasible
    assert np.all(np.diff(r.scores) <= 0)
    empty = O.topk(lib, h, _query([1.0], [1], [1e9], [2e9], k=10))
    assert len(empty.ids) == 0 and empty.n_feasible == 0


def test_subset_restricts_to_those_reactions():
    lib, head, _ = csl_gen.build_workload("t_ragged")
    full = O.topk(lib, head, _query([1, 0, 0, 0, 0], k=lib.n_rows * 100))
    t_of, _ = O.decode(lib, full.ids)
    sub = [5, 2]
    r = O.topk(lib, head, _query([1, 0, 0, 0, 0], k=30, subset=sub))
    expect = full.ids[np.isin(t_of, sub)][:30]
    assert np.array_equal(r.ids, expect)


# ---------------------------------------------------------------- invariants
def test_permutation_of_synthons_and_reactions():
    lib = library_from_sizes([[13, 9], [4, 5, 6], [21]], d=8, seed=60)
    h = make_head([8, 8, 3], "silu", seed=61, n_objectives=1, n_properties=2)
    q = _query([1.0], [1], [-0.2], [0.6], k=30)
    base = O.topk(lib, h, q)
    rng = np.random.default_rng(0)
    # permute synthons inside every slot
    perms = [rng.permutation(int(n)) for n in lib.slot_sizes]
    U2 = np.empty_like(lib.U)
    rf = lib.row_first
    for s, p in enumerate(perms):
        U2[rf[s] : rf[s + 1]] = lib.U[rf[s] : rf[s + 1]][p]   # new row i holds old row p[i]
    lib2 = CSL(lib.n_slots.copy(), lib.slot_sizes.copy(), lib.d, lib.seed, U2)
    r2 = O.topk(lib2, h, q)
    t2, s2 = O.decode(lib2, r2.ids)
    sf = lib.slot_first
    mapped = []
    for t, ss in zip(t2, s2):
        old = [int(perms[sf[t] + j][ss[j]]) for j in range(int(lib.n_slots[t]))]
        strides = np.cumprod([1] + [int(x) for x in lib.sizes_of(t)[::-1][:-1]])[::-1]
        off = sum(math.prod(int(x) for x in lib.sizes_of(u)) for u in range(t))
        mapped.append(off + int(np.dot(old, strides)))
    assert sorted(mapped) == sorted(base.ids.tolist())
    assert np.array_equal(np.sort(r2.scores), np.sort(base.scores))
    # reverse the reaction order
    order = [2, 1, 0]
    lib3 = lib.subset(order)
    r3 = O.topk(lib3, h, q)
    t3, s3 = O.decode(lib3, r3.ids)
    back = []
    for t, ss in zip(t3, s3):
        told = order[t]
        sizes = lib.sizes_of(told)
        strides = np.cumprod([1] + [int(x) for x in sizes[::-1][:-1]])[::-1]
        off = sum(math.prod(int(x) for x in lib.sizes_of(u)) for u in range(told))
        back.append(off + int(np.dot(ss[: len(sizes)], strides)))
    assert sorted(back) == sorted(base.ids.tolist())


def test_monotone_in_k_and_box_widening():
    lib, head, _ = csl_gen.build_workload("t_ragged")
    q = lambda k, lo, hi: _query([0.5, 0.5, 0, 0, 0], [5, 7], lo, hi, k=k)
    a = O.topk(lib, head, q(20, [-0.1, -0.1], [0.1, 0.1]))
    b = O.topk(lib, head, q(27, [-0.1, -0.1], [0.1, 0.1]))
    assert np.array_equal(b.ids[:20], a.ids)
    wide = O.topk(lib, head, q(20, [-0.2, -0.2], [0.2, 0.2]))
    assert wide.n_feasible >= a.n_feasible
    kth = wide.scores[-1]
    for i, s in zip(a.ids, a.scores):   # an old result is kept unless displaced by better ones
        assert i in set(wide.ids.tolist()) or s <= kth


def test_decode_roundtrip_beyond_32_bits():
    lib = _shape([[7], [3000, 3000, 3001], [11, 13]])
    N = O.count(lib)
    assert N > 2 ** 34
    ids = np.concatenate([[0, 6, 7, N - 1, N - 144, 2 ** 33 + 12345], np.random.default_rng(2).integers(0, N, 200)])
    t, s = O.decode(lib, ids)
    off = [0, 7, 7 + 3000 * 3000 * 3001, N]
    for i, tt, ss in zip(ids, t, s):
        sizes = lib.sizes_of(tt)
        assert all(0 <= ss[j] < sizes[j] for j in range(len(sizes)))
        v = 0
        for j, n in enumerate(sizes):
            v = v * int(n) + int(ss[j])
        assert off[tt] + v == i
    with pytest.raises(ValueError):
        O.decode(lib, np.array([N]))


def test_assoc_embeddings_pins():
    """Eq. assoc_embeds, u_{r,s} = K_r v_s, pinned by closed forms: identity keys return the
    values; a basis value picks a column of the key; scaling and adding values act linearly;
    each slot uses its own key."""
    rng = np.random.default_rng(3)
    sizes = np.array([3, 1, 4], np.int64)
    d = d_u = 5
    K = np.stack([np.eye(d, dtype=np.float32)] * 3)
    V = rng.standard_normal((8, d_u)).astype(np.float32)
    assert np.array_equal(O.assoc_embeddings(sizes, K, V), V.astype(np.float64))
    d, d_u = 6, 4
    K = rng.standard_normal((3, d, d_u)).astype(np.float32)
    E = np.zeros((8, d_u), np.float32)
    rows_slot = np.repeat(np.arange(3), sizes)
    for row in range(8):
        E[row, row % d_u] = 1.0
    U = O.assoc_embeddings(sizes, K, E)
    for row in range(8):  # u = column (row mod d_u) of the key of the row's own slot
        assert np.array_equal(U[row], K[rows_slot[row]][:, row % d_u].astype(np.float64))
    A = rng.integers(-3, 4, (8, d_u)).astype(np.float32)
    B = rng.integers(-3, 4, (8, d_u)).astype(np.float32)
    Ki = rng.integers(-3, 4, (3, d, d_u)).astype(np.float32)  # small integers: exact in FP64
    ua, ub, uab = (O.assoc_embeddings(sizes, Ki, X) for X in (A, B, 2 * A + B))
    assert np.array_equal(uab, 2 * ua + ub)
