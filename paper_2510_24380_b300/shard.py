"""Sharding a query across ranks: reaction partition and the k-candidate gather merge.

The path partitions without any exchange during enumeration: compounds are independent and the
top-k of Eq. apex_topk decomposes over any partition of the reactions (the exact top-k of the
whole scope, restricted to one part, is that part's own top-|X n part|). So each rank holds the
library, runs every query on its own part of the reactions (the query's reaction subset
intersected with the rank's part), and the one exchange per query is a gather of each rank's
<= k result rows (id, reaction, synthons, FP64/FP32 objective, outputs) to one rank, which keeps
the first k rows under (objective desc, id asc). Reaction batches are the unit the paper's GPU
implementation chains (App. GPU implementation: batches by reaction and first R-group synthon);
here whole reactions are assigned, balanced by compound count.

Host-side only: no library kernel touches another GPU's memory (the gather goes through
torch.distributed: NCCL between GPUs, gloo on the CPU).
"""
from __future__ import annotations

import heapq

import numpy as np

ROW_KEYS = ("ids", "reaction", "synthons", "objective", "outputs")


def partition_reactions(compounds_per_reaction, world: int):
    """Reactions split into `world` parts of near-equal compound count: longest first, each to the
    part with the fewest compounds so far (ties to the lower rank). Returns sorted index lists."""
    sizes = np.asarray(compounds_per_reaction, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda t: (-sizes[t], t))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for t in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(t))
        heapq.heappush(heap, (load + float(sizes[t]), r))
    return [sorted(p) for p in parts]


def local_subset(part, query_subset):
    """Reactions a rank serves for one query: its part, intersected with the query's subset."""
    if query_subset is None:
        return np.asarray(part, dtype=np.int32)
    return np.intersect1d(np.asarray(part, dtype=np.int32), np.asarray(query_subset, dtype=np.int32)).astype(np.int32)


def empty_rows(n_outputs: int, max_slots: int = 4):
    return {"ids": np.zeros(0, np.int64), "reaction": np.zeros(0, np.int32),
            "synthons": np.zeros((0, max_slots), np.int64), "objective": np.zeros(0, np.float64),
            "outputs": np.zeros((0, n_outputs), np.float64), "n": 0}


def merge_topk(parts, k: int):
    """The first k rows of the union of per-rank results under (objective desc, id asc). Each part
    holds min(k, feasible) rows of disjoint reactions, so the merge is the exact top-k."""
    parts = [p for p in parts if p is not None and len(p["ids"])]
    if not parts:
        return None
    cat = {key: np.concatenate([p[key] for p in parts]) for key in ROW_KEYS}
    order = np.lexsort((cat["ids"], -cat["objective"]))[: int(k)]
    out = {key: cat[key][order] for key in ROW_KEYS}
    out["n"] = int(len(order))
    return out


class ShardedRunner:
    """Runs batches of queries with each rank on its part of the reactions and merges on `root`.

    run_local(queries) -> list of row dicts (the rank's results, one per query, in order);
    queries are csl_gen.Query-like (fields weights, cons_idx, lo, hi, k, subset, precision).
    The process group must be initialized (torch.distributed); with world 1 nothing is exchanged.
    """

    def __init__(self, compounds_per_reaction, rank: int, world: int, run_local, n_outputs: int, root: int = 0,
                 group=None):
        self.rank, self.world, self.root, self.group = int(rank), int(world), int(root), group
        self.parts = partition_reactions(compounds_per_reaction, world)
        self.part = self.parts[self.rank]
        self.run_local = run_local
        self.n_outputs = int(n_outputs)

    def local_queries(self, queries):
        """Each query restricted to this rank's reactions; None where the rank holds none of them."""
        import dataclasses

        if self.world == 1:
            return list(queries)
        out = []
        for q in queries:
            sub = local_subset(self.part, q.subset)
            out.append(dataclasses.replace(q, subset=sub) if len(sub) else None)
        return out

    def run(self, queries):
        """Merged results (list, one per query) on the root rank; None on the others."""
        lq = self.local_queries(queries)
        todo = [q for q in lq if q is not None]
        got = iter(self.run_local(todo) if todo else [])
        mine = [next(got) if q is not None else empty_rows(self.n_outputs) for q in lq]
        if self.world == 1:
            return mine
        import torch.distributed as dist

        gathered = [None] * self.world if self.rank == self.root else None
        dist.gather_object(mine, gathered, dst=self.root, group=self.group)
        if self.rank != self.root:
            return None
        return [merge_topk([g[i] for g in gathered], q.k) or empty_rows(self.n_outputs)
                for i, q in enumerate(queries)]
