"""Query descriptors: objective weights, constraint boxes, k and reaction subset.

A query follows the retrieval problem of Sec. 3 (Eq. orig_topk / apex_topk): maximize the
objective sum_j w_j o_j over at most k compounds whose constrained outputs lie inside
[lower_i, upper_i] (inclusive; +-inf allowed).

Constraint boxes are placed at quantiles of each output's distribution. Those statistics
are data files under ``csl_gen/data`` (written by ``oracle/make_output_stats.py`` from
FP64 oracle scores of a seeded sample of compounds); this module only reads them.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

import numpy as np

from .library import _rng

DATA_DIR = os.path.join(os.path.dirname(__file__), "data")


@dataclass
class Query:
    weights: np.ndarray          # float32 [n_objectives]
    cons_idx: np.ndarray         # int32 [m] output index constrained
    lo: np.ndarray               # float64 [m]
    hi: np.ndarray               # float64 [m]
    k: int
    subset: np.ndarray | None = None   # int32 reaction indices, None = whole library
    precision: str = "bf16"

    @property
    def m(self) -> int:
        return int(self.cons_idx.shape[0])


def load_stats(name: str) -> dict:
    from .configs import WORKLOADS  # a slice of a workload shares its statistics

    name = WORKLOADS.get(name, {}).get("stats", name)
    path = os.path.join(DATA_DIR, f"{name}_stats.json")
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing; write it with: python oracle/make_output_stats.py {name}")
    with open(path) as f:
        return json.load(f)


def quantile(stats: dict, output: int, q: float) -> float:
    qs = np.asarray(stats["quantile_levels"], dtype=np.float64)
    vals = np.asarray(stats["quantiles"][output], dtype=np.float64)
    return float(np.interp(q, qs, vals))


def query_single(name: str, spec: dict, stats: dict | None = None, precision: str | None = None,
                 k: int | None = None, subset=None) -> Query:
    """The single query of a workload (the recipes are listed in the design notes)."""
    stats = stats if stats is not None else load_stats(name)
    n_obj = spec["n_obj"]
    w = np.zeros(n_obj, dtype=np.float32)
    w[0] = 1.0
    k = int(k if k is not None else spec["k"])
    prec = precision or spec["precision"]
    sub = None if subset is None else np.asarray(subset, dtype=np.int32)
    if name == "c1_tiny":
        idx = np.array([1, 2], dtype=np.int32)
        mu = np.array([stats["mean"][i] for i in idx])
        sd = np.array([stats["std"][i] for i in idx])
        return Query(w, idx, mu - 0.5 * sd, mu + 0.5 * sd, k, sub, prec)
    if name in ("c2_10m", "t_ragged"):
        idx = np.arange(n_obj, n_obj + 4, dtype=np.int32)
        lo = np.array([quantile(stats, int(i), 0.15) for i in idx])
        hi = np.array([quantile(stats, int(i), 0.85) for i in idx])
        return Query(w, idx, lo, hi, k, sub, prec)
    if name in ("c3_real", "c3_slice"):
        idx = np.arange(n_obj, n_obj + 6, dtype=np.int32)
        hi = np.array([quantile(stats, int(i), 0.8) for i in idx])
        lo = np.full(idx.shape, -np.inf)
        return Query(w, idx, lo, hi, k, sub, prec)
    if name == "t_linear":
        idx = np.array([1], dtype=np.int32)
        return Query(w, idx, np.array([quantile(stats, 1, 0.2)]), np.array([np.inf]), k, sub, prec)
    if name in ("t_linear_3x200", "linear_1e12"):
        # property 1 above its 0.2 quantile, property 2 below its 0.9 quantile
        idx = np.array([1, 2], dtype=np.int32)
        return Query(w, idx, np.array([quantile(stats, 1, 0.2), -np.inf]), np.array([np.inf, quantile(stats, 2, 0.9)]),
                     k, sub, prec)
    raise KeyError(name)


def random_query(rng: np.random.Generator, stats: dict, n_obj: int, n_prop: int, k: int, subset=None,
                 precision: str = "bf16", n_boxes: int = 8) -> Query:
    """A query with Dirichlet(1) weights over the objectives and n_boxes property boxes whose
    joint pass rate P is log-uniform in [1 %, 50 %]: each box passes P^(1/n_boxes) of its
    marginal, placed at a uniformly random quantile offset."""
    w = rng.dirichlet(np.ones(n_obj)).astype(np.float32)
    P = math.exp(rng.uniform(math.log(0.01), math.log(0.5)))
    nb = min(n_boxes, n_prop)
    p = P ** (1.0 / nb)
    props = rng.choice(n_prop, size=nb, replace=False)
    idx = np.sort(props).astype(np.int32) + n_obj
    lo, hi = [], []
    for i in idx:
        a = rng.uniform(0.0, 1.0 - p)
        lo.append(quantile(stats, int(i), a) if a > 0 else -np.inf)
        hi.append(quantile(stats, int(i), a + p) if a + p < 1 else np.inf)
    sub = None if subset is None else np.asarray(subset, dtype=np.int32)
    return Query(w, idx, np.array(lo), np.array(hi), int(k), sub, precision)


def queries_batched(stats: dict, n_obj: int, n_prop: int, n_queries: int, seed: int, subset=None,
                    ks=(10, 100, 1000, 10000, 100000), precision: str = "bf16"):
    """The multi-query batch: k drawn uniformly from ks, random weights and 8 property boxes."""
    rng = _rng(seed, 5)
    out = []
    for _ in range(n_queries):
        k = int(rng.choice(ks))
        out.append(random_query(rng, stats, n_obj, n_prop, k, subset=subset, precision=precision))
    return out


def serving_stream(stats: dict, n_obj: int, n_prop: int, n_reactions: int, n_queries: int, rate_hz: float,
                   seed: int, k_range=(10, 100000), max_subset: int = 1000, precision: str = "bf16"):
    """Poisson arrivals at rate_hz; each query takes a log-uniform count of 1..max_subset random
    reactions, random weights and boxes, and k log-uniform in k_range. Returns [(t_arrival_s, Query)]."""
    rng = _rng(seed, 6)
    t = 0.0
    out = []
    for _ in range(n_queries):
        t += rng.exponential(1.0 / rate_hz)
        cnt = int(round(math.exp(rng.uniform(0.0, math.log(min(max_subset, n_reactions))))))
        cnt = max(1, min(cnt, n_reactions))
        sub = np.sort(rng.choice(n_reactions, size=cnt, replace=False)).astype(np.int32)
        k = int(round(math.exp(rng.uniform(math.log(k_range[0]), math.log(k_range[1])))))
        out.append((t, random_query(rng, stats, n_obj, n_prop, k, subset=sub, precision=precision)))
    return out


def queries_step(name: str, spec: dict, n_queries: int, seed: int, stats: dict | None = None,
                 precision: str = "bf16", ks=(100, 1000, 10000), n_boxes: int = 6):
    """The queries of one batched step over a workload: the workload's own query first, then
    n_queries - 1 random ones (Dirichlet(1) weights over the objectives, n_boxes property boxes of
    joint pass rate log-uniform in [1 %, 50 %], k drawn from ks), all on the whole library."""
    stats = stats if stats is not None else load_stats(name)
    out = [query_single(name, spec, stats, precision=precision)]
    rng = _rng(seed, 8)
    for _ in range(n_queries - 1):
        k = int(rng.choice(ks))
        out.append(random_query(rng, stats, spec["n_obj"], spec["n_prop"], k, precision=precision, n_boxes=n_boxes))
    return out

