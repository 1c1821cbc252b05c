"""GPU parity at the ~3e10-compound scale: c3_real (1,000 reactions of 2-3 slots, 30,020,835,564
compounds, 256-256-256-13 SiLU head), BF16 pass, in the bench's launch configuration (2^27
compounds per enumeration launch) and batched form. The host cannot enumerate the library, so
the checks are those that hold at any size (Eq. apex_topk restricted to a set of reactions):
  - one batched step of 9 queries sharing one circular pass: the workload's query and 7 random ones
    on the whole library, and one (k = 1,000) restricted to 5 seeded small reactions. Every
    returned member is rescored by the FP64 oracle; on the sampled reactions each result's members
    are the oracle's first |X n t| of those reactions and no better feasible compound is missing;
    the restricted query's whole top-k, members included, equals the oracle's;
  - the workload's query alone in FP8 (e4m3 layer 2): its wide margins fill 10^5-10^6-entry
    candidate buffers, so its pass runs in-pass compactions every launch and leaves the large
    buffers' selects between launches to them; checked the same way;
  - raw outputs of the production enumeration kernel over one whole reaction of about 10^6
    compounds against the oracle on a seeded sample of its compounds (2e-2 absolute for BF16).
"""
import numpy as np
import pytest

import csl_gen
from oracle import oracle as O
from paper_2510_24380_b300 import apex

from parity import (BF16_ABS, check_members_exact, check_reaction_decomposed, check_topk, output_rms,
                    reaction_first_ids, seeded_small_reactions)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c3():
    lib, head, spec = csl_gen.build_workload("c3_real")
    L = apex.Library(lib, head, precisions=("fp32", "bf16", "fp8"), seed=0)
    L.set_launch_shape(1 << 27, 32)  # the bench's launch shape on this library
    first = reaction_first_ids(lib)
    yield lib, head, spec, L, first
    L.close()


def test_batched_step_at_3e10_compounds_matches_oracle(c3):
    lib, head, spec, L, first = c3
    assert int(first[-1]) > 3 * 10**10
    # the sampled reactions: seeded, at most 4e5 compounds each (about 1.3e6 in all)
    S = seeded_small_reactions(lib, 5, 400000, seed=5)
    assert len(S) == 5
    stats = csl_gen.load_stats("c3_real")
    qs = csl_gen.queries_step("c3_real", spec, 8, seed=1, precision="bf16")
    rng = np.random.default_rng(9)
    qs.append(csl_gen.random_query(rng, stats, spec["n_obj"], spec["n_prop"], 1000,
                                   subset=np.array(S, np.int32), precision="bf16", n_boxes=6))
    rms = np.array(list(L.info().rms)[: head.dims[-1]])
    ids = [L.query(q) for q in qs]
    res = [L.fetch(i, q.k) for i, q in zip(ids, qs)]
    for q, r, i in zip(qs, res, ids):
        assert r["n"] == q.k, (q.k, r["n"])
        check_members_exact(r, lib, head, q, rms)
        check_reaction_decomposed(r, lib, head, q, S, rms)
    # the restricted query: its whole top-k against the oracle's enumeration of its 5 reactions
    q9, r9 = qs[-1], res[-1]
    check_topk(r9, O.topk(lib, head, q9), lib, head, q9, rms)


def test_fp8_query_at_3e10_compounds_matches_oracle(c3):
    lib, head, spec, L, first = c3
    S = seeded_small_reactions(lib, 5, 400000, seed=6)
    q = csl_gen.query_single("c3_real", spec, precision="fp8")
    rms = np.array(list(L.info().rms)[: head.dims[-1]])
    r = L.run(q)
    st = L.stats(-1)
    assert r["n"] == q.k and st["n_compactions"] > 0 and st["n_restarts"] == 0, st
    assert st["pass_err_ratio"] <= 1.0 and st["fp32_err_ratio"] <= 1.0, st
    check_members_exact(r, lib, head, q, rms)
    check_reaction_decomposed(r, lib, head, q, S, rms)


def test_raw_outputs_of_a_whole_reaction(c3):
    lib, head, spec, L, first = c3
    sizes = np.diff(first)
    t = int(np.argmin(np.abs(sizes - 10**6)))  # the reaction closest to 10^6 compounds
    got = L.dump_outputs(t, int(sizes[t]), "bf16")
    local = np.unique(np.concatenate([np.random.default_rng(31).integers(0, sizes[t], 4000), [0, sizes[t] - 1]]))
    ref = O.score_ids(lib, head, first[t] + local)
    err = np.abs(got[local].astype(np.float64) - ref).max(axis=0)
    margin = np.array(list(L.info().err_bf16)[: head.dims[-1]])
    assert np.all(err <= margin), (err, margin)
    assert err.max() <= BF16_ABS, err.max()
