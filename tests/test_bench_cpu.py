"""Host logic of the benchmark's oracle check (no GPU): the seeded sample of small reactions the
FP64 oracle enumerates, the step's extra query restricted to that sample, and which queries the
check enumerates exactly."""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import csl_gen  # noqa: E402


def _args(workload):
    return argparse.Namespace(mode="batched", workload=workload, queries=8, precision="bf16", oracle_compounds=1.1e6)


def test_oracle_sample_is_seeded_small_and_bounded():
    sizes = np.array([5e6, 2e5, 3e5, 9e4, 4e5, 1e5, 2.5e5, 8e6, 3.5e5, 1.5e5], float)
    a = bench.oracle_sample(sizes, 1.1e6, seed=3)
    b = bench.oracle_sample(sizes, 1.1e6, seed=3)
    assert a == b  # seeded
    S, n = a
    assert len(S) >= 5 and n == int(sizes[S].sum()) and n <= 2 * 1.1e6
    assert all(sizes[t] <= 1.1e6 for t in S)
    # nothing small enough: an empty sample
    assert bench.oracle_sample(np.array([5e6, 8e6]), 1.1e6, seed=3) == ([], 0)


def test_batched_step_adds_a_query_on_the_oracle_sample():
    full, head, spec = csl_gen.build_workload("c3_real", materialize=False)
    sizes = bench.compounds_per_reaction(full)
    qs = bench.step_queries(_args("c3_real"), spec, sizes=sizes)
    assert len(qs) == 9 and all(q.subset is None for q in qs[:8])
    S0, n0 = bench.oracle_sample(sizes, 1.1e6, seed=3)
    assert sorted(qs[-1].subset.tolist()) == S0 and qs[-1].k == 1000 and n0 > 10**6
    # the same last query's objective and boxes, on the sample
    assert np.array_equal(qs[-1].weights, qs[-2].weights) and np.array_equal(qs[-1].lo, qs[-2].lo)


def test_no_extra_query_when_no_reaction_is_small_enough():
    full, head, spec = csl_gen.build_workload("c3_slice", materialize=False)
    sizes = bench.compounds_per_reaction(full)
    qs = bench.step_queries(_args("c3_slice"), spec, sizes=sizes)
    assert len(qs) == 8 and all(q.subset is None for q in qs)


def test_member_reactions_prefer_reactions_with_most_rows():
    sizes = np.array([1e5, 2e5, 3e6, 5e4], float)
    results = [{"n": 4, "reaction": np.array([0, 0, 1, 2])}, {"n": 2, "reaction": np.array([3, 0])}]
    M, n = bench.member_reactions(sizes, results, cap=1e6, budget=2.6e5, exclude=())
    assert M == [0, 3] and n == int(1.5e5)  # reaction 2 is too large, reaction 1 exceeds the budget
