"""The comparison rules of the GPU parity tests, checked on the CPU against the FP64 oracle.

The reaction-decomposed check is how results at sizes the oracle cannot enumerate in full are
verified (a sample of reactions, enumerated exactly). Here it must accept the oracle's own exact
answer on every reaction sample and reject answers with a planted mistake: a member dropped, a
member swapped for a worse compound of the same reactions, a member swapped for a compound of
another reaction, a full result that misses a better compound, and a short result that is missing
a feasible compound."""
import numpy as np
import pytest

import csl_gen
from oracle import oracle as O

from parity import check_members_exact, check_reaction_decomposed, output_rms, reaction_first_ids


@pytest.fixture(scope="module")
def ragged():
    lib, head, spec = csl_gen.build_workload("t_ragged")
    return lib, head, spec, output_rms(lib, head)


def _as_result(ref):
    return {"ids": ref.ids.copy(), "objective": ref.scores.copy(), "outputs": ref.outputs.copy(), "n": len(ref.ids)}


def _query(spec, k):
    stats = csl_gen.load_stats("t_ragged")
    q = csl_gen.query_single("t_ragged", spec, stats, precision="fp64")
    return csl_gen.Query(q.weights, q.cons_idx, q.lo, q.hi, k, None, "fp64")


SAMPLES = [[0], [5], [0, 5], [2, 4, 6], [1, 3], list(range(7))]


@pytest.mark.parametrize("k", [5, 60, 100000])
def test_exact_answer_passes_on_every_sample(ragged, k):
    lib, head, spec, rms = ragged
    q = _query(spec, k)
    res = _as_result(O.topk(lib, head, q))
    for S in SAMPLES:
        check_reaction_decomposed(res, lib, head, q, S, rms)
    check_members_exact(res, lib, head, q, rms)


def _raises(res, lib, head, q, S, rms):
    with pytest.raises(AssertionError):
        check_reaction_decomposed(res, lib, head, q, S, rms)


def test_planted_mistakes_are_caught(ragged):
    lib, head, spec, rms = ragged
    q = _query(spec, 60)
    ref = O.topk(lib, head, q)
    first = reaction_first_ids(lib)
    rxn = np.searchsorted(first, ref.ids, side="right") - 1
    t = int(np.bincount(rxn).argmax())  # the reaction holding most members
    members = np.flatnonzero(rxn == t)
    # the oracle's order of reaction t alone, deeper than the result reaches
    deep = O.topk(lib, head, csl_gen.Query(q.weights, q.cons_idx, q.lo, q.hi, 500, np.array([t], np.int32), "fp64"))
    outside = [int(x) for x in deep.ids if int(x) not in set(ref.ids.tolist())]

    def res_with(ids):
        ids = np.asarray(ids, np.int64)
        o = O.score_ids(lib, head, ids)
        f = o[:, :len(q.weights)] @ np.asarray(q.weights, np.float64)
        order = np.lexsort((ids, -f))
        return {"ids": ids[order], "objective": f[order], "outputs": o[order], "n": len(ids)}

    # 1. the best member of reaction t swapped for a worse compound of t
    ids = ref.ids.copy()
    ids[members[0]] = outside[0]
    _raises(res_with(ids), lib, head, q, [t], rms)
    # 2. a member of t dropped (short result, although more than k compounds are feasible)
    _raises(res_with(np.delete(ref.ids, members[-1])), lib, head, q, [t], rms)
    # 3. a member of t replaced by the best compound of another reaction that is not in the result
    other = (t + 1) % lib.n_reactions
    deep_o = O.topk(lib, head, csl_gen.Query(q.weights, q.cons_idx, q.lo, q.hi, 500, np.array([other], np.int32), "fp64"))
    extra = [int(x) for x in deep_o.ids if int(x) not in set(ref.ids.tolist())][0]
    ids = ref.ids.copy()
    ids[members[0]] = extra
    _raises(res_with(ids), lib, head, q, [t], rms)  # seen from t: its best compound is missing
    # 4. a short result (k above the feasible count) missing one feasible compound of t
    qa = _query(spec, 100000)
    full = O.topk(lib, head, qa)
    rx_all = np.searchsorted(first, full.ids, side="right") - 1
    drop = int(np.flatnonzero(rx_all == t)[0])
    short = res_with(np.delete(full.ids, drop))
    short["n"] = len(short["ids"])
    _raises(short, lib, head, qa, [t], rms)
    # 5. a reported objective that is off (exact members, wrong value)
    bad = _as_result(ref)
    bad["objective"][members[0]] += 1e-3
    _raises(bad, lib, head, q, [t], rms)
    with pytest.raises(AssertionError):
        check_members_exact(bad, lib, head, q, rms)
