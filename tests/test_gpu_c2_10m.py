"""GPU parity at full size: the ~1e7-compound workload (40 reactions, 256-256-256-13 SiLU head).

Unlike the small test libraries, here every CTA of an enumeration launch walks hundreds of tiles
(the outer-row ring and the TMEM double buffer wrap many times, cost-weighted CTA ranges cross
reactions), and queries span many launches with threshold raises between them. Checked against
the FP64 oracle:
  - the workload's single query, every pass precision, at the default launch shape and cut into
    many launches, against the oracle's full enumeration (about 10^7 compounds);
  - raw outputs of the production enumeration kernel over the whole library, on a seeded sample
    of 10^4 compounds plus every reaction's first and last compound;
  - a 16-query mixed batch (k up to 10^5, reaction subsets, four pass precisions) in one shared
    pass: every returned member rescored by the oracle, and the reaction-decomposed check on a
    seeded sample of reactions;
  - continuous batching: a query that joins while another one's pass is half done returns what it
    returns alone; admission by memory budget (the second query waits for the first one's
    memory; a query that can never fit fails with APEX_ENOMEM);
  - three threads fetching the same query id: one gets the rows, the others APEX_ENOTFOUND.
"""
import threading
import time

import numpy as np
import pytest

import csl_gen
from oracle import oracle as O
from paper_2510_24380_b300 import apex

from parity import (BF16_ABS, FP32_REL, assert_fp32_close, check_members_exact, check_reaction_decomposed,
                    check_topk, output_rms, reaction_first_ids, seeded_small_reactions)

pytestmark = pytest.mark.gpu

PRECISIONS = ("fp32", "bf16", "fp16", "fp8")


@pytest.fixture(scope="module")
def c2():
    lib, head, spec = csl_gen.build_workload("c2_10m")
    L = apex.Library(lib, head, precisions=PRECISIONS, seed=0)
    yield lib, head, spec, L, output_rms(lib, head)
    L.close()


@pytest.fixture(scope="module")
def c2_ref(c2):
    """The oracle's full enumeration of the workload's query (the exact top-k does not depend on the
    pass precision)."""
    lib, head, spec, L, rms = c2
    q = csl_gen.query_single("c2_10m", spec, precision="fp64")
    return q, O.topk(lib, head, q)


def _with(q, precision=None, k=None, subset="keep"):
    return csl_gen.Query(q.weights, q.cons_idx, q.lo, q.hi, int(k if k is not None else q.k),
                         q.subset if subset == "keep" else subset, precision or q.precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_single_query_default_launch_shape_full_oracle(c2, c2_ref, precision):
    lib, head, spec, L, rms = c2
    q0, ref = c2_ref
    q = _with(q0, precision)
    res = L.run(q)
    st = L.stats(-1)
    check_topk(res, ref, lib, head, q, rms)
    assert set(res["ids"].tolist()) == set(ref.ids.tolist())
    # every pass scores each compound of the scope once (n_scored counts compounds, not tile rows)
    assert st["n_scored"] == lib_n(lib) * (1 + st["n_restarts"]) and st["n_margin_reruns"] == 0
    # the runtime margin check saw the candidates' errors inside the calibrated margins
    assert 0.0 <= st["pass_err_ratio"] <= 1.0 and 0.0 <= st["fp32_err_ratio"] <= 1.0, st


def lib_n(lib):
    return int(reaction_first_ids(lib)[-1])


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8"])
def test_many_launches_with_threshold_raises(c2, c2_ref, precision):
    """The same query cut into launches of 2^21 compounds: the admission threshold rises after every
    launch (slot selects between launches); the rows equal the one-launch rows exactly."""
    lib, head, spec, L, rms = c2
    q0, ref = c2_ref
    q = _with(q0, precision)
    one = L.run(q)
    try:
        L.set_launch_shape(1 << 21, 32)
        many = L.run(q)
        st = L.stats(-1)
    finally:
        L.set_launch_shape(1 << 25, 32)
    assert st["n_launches"] >= 5, st
    assert np.array_equal(many["ids"], one["ids"]) and np.array_equal(many["objective"], one["objective"])
    check_topk(many, ref, lib, head, q, rms)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_raw_outputs_whole_library_sampled(c2, precision):
    """The production enumeration kernel over the whole library in pass-shaped launches; raw outputs
    of 10^4 seeded compounds and of every reaction's first and last compound against the oracle:
    FP32 within 1e-5 relative; BF16 / FP16 within 2e-2 absolute; FP8 within the library's calibrated
    FP8 margin (the admission bound that exactness relies on)."""
    lib, head, spec, L, rms = c2
    N = lib_n(lib)
    first = reaction_first_ids(lib)
    launches0 = apex.apex_kernel_launches()
    got_all = L.dump_outputs(-1, N, precision)
    assert apex.apex_kernel_launches() > launches0
    ids = np.unique(np.concatenate([np.random.default_rng(17).integers(0, N, 10000), first[:-1], first[1:] - 1]))
    got = got_all[ids].astype(np.float64)
    del got_all
    ref = O.score_ids(lib, head, ids)
    info = L.info()
    if precision == "fp32":
        assert_fp32_close(got, ref, rms)
        return
    err = np.abs(got - ref).max(axis=0)
    margin = np.array(list(getattr(info, "err_" + precision))[: head.dims[-1]])
    assert np.all(err <= margin), (err, margin)
    if precision in ("bf16", "fp16"):
        assert err.max() <= BF16_ABS, err.max()
    else:
        print(f"fp8 raw outputs: max |err| {err.max():.4f} (per output {np.round(err, 4).tolist()})")


def test_mixed_batch_of_16_queries(c2):
    """16 queries with Dirichlet weights, 8 boxes of joint pass rate 1-50 %, k from 10 to 10^5,
    some on reaction subsets, four pass precisions, submitted together (one shared pass)."""
    lib, head, spec, L, rms = c2
    stats = csl_gen.load_stats("c2_10m")
    rng = np.random.default_rng(23)
    ks = [10, 100, 1000, 10000, 100000]
    qs = []
    for i in range(16):
        sub = None if i % 4 else np.sort(rng.choice(lib.n_reactions, size=int(rng.integers(3, 20)), replace=False))
        prec = ("bf16", "bf16", "fp16", "fp8", "fp32")[i % 5]
        qs.append(csl_gen.random_query(rng, stats, 5, 8, k=ks[i % 5], subset=sub, precision=prec))
    ids = [L.query(q) for q in qs]
    res = [L.fetch(i, q.k) for i, q in zip(ids, qs)]
    first = reaction_first_ids(lib)
    sizes = np.diff(first)
    checked = 0
    for j, (q, r) in enumerate(zip(qs, res)):
        assert r["n"] <= q.k
        check_members_exact(r, lib, head, q, rms)
        # a reaction of the result small enough to enumerate, plus seeded small reactions
        rx = np.unique(np.searchsorted(first, r["ids"], side="right") - 1)
        must = [int(t) for t in rx if sizes[t] <= 150000][:1]
        S = seeded_small_reactions(lib, 3, 60000, seed=100 + j, must=must)
        out = check_reaction_decomposed(r, lib, head, q, S, rms)
        checked += out["reactions"]
    assert checked >= 16
    for q, r in list(zip(qs, res))[:3]:  # alone, the same rows
        a = L.run(q)
        assert np.array_equal(a["ids"], r["ids"]) and np.array_equal(a["objective"], r["objective"])


def test_join_mid_cycle_equals_alone(c2, c2_ref):
    """q1 (FP32 pass, launches of 2^21 compounds) is submitted; once its first launches are out, q2
    (the workload's query, BF16) is submitted: q2 joins the circular pass at q1's current position,
    shares q1's remaining launches and completes its own cycle after q1 has left. q2's rows equal its
    rows alone and the oracle's; q1's rows equal q1 alone."""
    lib, head, spec, L, rms = c2
    q0, ref = c2_ref
    stats = csl_gen.load_stats("c2_10m")
    q1 = csl_gen.random_query(np.random.default_rng(31), stats, 5, 8, k=1000, precision="fp32")
    q2 = _with(q0, "bf16")
    alone1, alone2 = L.run(q1), L.run(q2)
    try:
        L.set_launch_shape(1 << 21, 32)
        n0 = apex.apex_kernel_launches()
        t1 = time.perf_counter()
        i1 = L.query(q1)
        while apex.apex_kernel_launches() - n0 < 4 and time.perf_counter() - t1 < 5:
            time.sleep(0.0005)
        time.sleep(0.02)
        t2 = time.perf_counter()
        i2 = L.query(q2)
        r1 = L.fetch(i1, q1.k)
        s1 = L.stats(-1)
        r2 = L.fetch(i2, q2.k)
        s2 = L.stats(-1)
    finally:
        L.set_launch_shape(1 << 25, 32)
    # q2 was admitted while q1's pass ran, at a later position of the circular pass
    assert (t2 - t1) * 1e3 + s2["queue_ms"] < s1["latency_ms"], (t2 - t1, s1, s2)
    assert s2["first_item"] != s1["first_item"], (s1["first_item"], s2["first_item"])
    assert np.array_equal(r1["ids"], alone1["ids"]) and np.array_equal(r1["objective"], alone1["objective"])
    assert np.array_equal(r2["ids"], alone2["ids"]) and np.array_equal(r2["objective"], alone2["objective"])
    check_topk(r2, ref, lib, head, q2, rms)


def test_admission_by_memory_budget():
    """With a device budget that holds the tables and one query's candidate state, a second query
    waits until the first one has finished (then reuses its slot's memory); a query whose candidate
    state can never fit fails with APEX_ENOMEM. Results equal those of an unbudgeted library."""
    lib, head, spec = csl_gen.build_workload("c2_10m")
    stats = csl_gen.load_stats("c2_10m")
    q1 = csl_gen.query_single("c2_10m", spec, stats, precision="fp32")
    q2 = csl_gen.random_query(np.random.default_rng(41), stats, 5, 8, k=1000, precision="fp32")
    L0 = apex.Library(lib, head, precisions=("fp32",), seed=0)
    try:
        tables = int(L0.info().device_bytes)
        ref1, ref2 = L0.run(q1), L0.run(q2)
    finally:
        L0.close()
    slot = (1 << 18) * (4 + 8) * 2  # candidate keys and ids, double-buffered, of a query with k <= 32768
    L = apex.Library(lib, head, precisions=("fp32",), seed=0, budget=tables + slot + (3 << 20))
    try:
        i1, i2 = L.query(q1), L.query(q2)
        r1 = L.fetch(i1, q1.k)
        s1 = L.stats(-1)
        r2 = L.fetch(i2, q2.k)
        s2 = L.stats(-1)
        assert s2["queue_ms"] >= 0.5 * s1["latency_ms"], (s1, s2)  # waited for q1's memory
        assert np.array_equal(r1["ids"], ref1["ids"]) and np.array_equal(r2["ids"], ref2["ids"])
        big = csl_gen.Query(q1.weights, q1.cons_idx, q1.lo, q1.hi, 1 << 24, None, "fp32")
        with pytest.raises(apex.ApexError) as e:
            L.run(big)
        assert e.value.code == -2, e.value
        assert np.array_equal(L.run(q2)["ids"], ref2["ids"])  # and the library keeps serving
        sv = L.serving_stats()
        assert sv["n_queries"] == 3 and sv["n_failed"] == 1
    finally:
        L.close()


def test_concurrent_fetches_of_one_id(c2):
    """Three threads wait on the same query (two watch the completion counter, the third sleeps on
    the condition variable from the start): exactly one receives the rows, the others get
    APEX_ENOTFOUND, and nothing touches the released record."""
    lib, head, spec, L, rms = c2
    stats = csl_gen.load_stats("c2_10m")
    q = csl_gen.random_query(np.random.default_rng(51), stats, 5, 8, k=500, precision="fp32")
    ref = L.run(q)
    for rep in range(4):
        qid = L.query(q)
        out = [None] * 3

        def fetch(i):
            try:
                out[i] = L.fetch(qid, q.k)
            except apex.ApexError as e:
                out[i] = e.code

        th = [threading.Thread(target=fetch, args=(i,)) for i in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join(timeout=60)
        rows = [o for o in out if isinstance(o, dict)]
        codes = [o for o in out if not isinstance(o, dict)]
        assert len(rows) == 1 and codes == [-8, -8], out
        assert np.array_equal(rows[0]["ids"], ref["ids"])


def test_serving_statistics(c2):
    """apex_stats over a reset window: counts, latency percentiles against the per-query latencies
    (linear interpolation between nearest ranks), throughput figures from the same window."""
    lib, head, spec, L, rms = c2
    stats = csl_gen.load_stats("c2_10m")
    rng = np.random.default_rng(61)
    qs = [csl_gen.random_query(rng, stats, 5, 8, k=100, precision="bf16") for _ in range(6)]
    L.reset_serving_stats()
    lat, scope = [], 0
    for q in qs:
        L.run(q)
        lat.append(L.stats(-1)["latency_ms"])
        scope += lib_n(lib)
    sv = L.serving_stats()
    assert sv["n_queries"] == 6 and sv["n_failed"] == 0
    assert abs(sv["p50_ms"] - np.percentile(lat, 50)) < 1e-9 and abs(sv["p99_ms"] - np.percentile(lat, 99)) < 1e-9
    assert abs(sv["max_ms"] - max(lat)) < 1e-9 and sv["query_compounds"] == scope
    assert sv["head_evaluations"] >= 6 * lib_n(lib) and sv["enumerate_ms"] > 0 and sv["n_enumeration_launches"] >= 6
    assert sv["wall_ms"] >= sum(lat) * 0.5 and sv["query_compounds_per_s"] > 0
