"""The sharded path on the CPU: reaction partition balanced by compound count, and the k-candidate
gather merge over world_size-2 gloo ranks. Each rank's local answer here is the FP64 oracle's top-k
over the rank's part (the GPU library produces the same rows on a GPU machine); the merged answer must
equal the oracle's top-k over the whole scope, for whole-library and subset queries, including a
query whose subset lies entirely in one rank's part."""
import os
import socket

import numpy as np
import pytest

import csl_gen
from oracle import oracle as O
from paper_2510_24380_b300 import shard

from parity import reaction_first_ids


def _sizes(lib):
    return np.diff(reaction_first_ids(lib))


def test_partition_covers_every_reaction_once_and_balances():
    rng = np.random.default_rng(3)
    sizes = rng.lognormal(12, 1.0, 1000)
    for world in (1, 2, 3, 8):
        parts = shard.partition_reactions(sizes, world)
        flat = sorted(t for p in parts for t in p)
        assert flat == list(range(1000))
        loads = [sizes[p].sum() for p in parts]
        assert max(loads) - min(loads) <= sizes.max() + 1e-6  # greedy longest-first bound
    assert shard.partition_reactions([5, 1, 1], 2) == [[0], [1, 2]]


def _oracle_rows(lib, head, q):
    ref = O.topk(lib, head, q)
    t, s = O.decode(lib, ref.ids, max_slots=4)
    return {"ids": ref.ids, "reaction": t, "synthons": s, "objective": ref.scores, "outputs": ref.outputs,
            "n": len(ref.ids)}


def _queries(lib, spec):
    stats = csl_gen.load_stats("t_ragged")
    base = csl_gen.query_single("t_ragged", spec, stats, precision="fp64")
    rng = np.random.default_rng(9)
    return [
        base,
        csl_gen.Query(base.weights, base.cons_idx, base.lo, base.hi, 100000, None, "fp64"),  # k above feasible
        csl_gen.random_query(rng, stats, 5, 8, k=300, precision="fp64"),
        csl_gen.Query(base.weights, base.cons_idx, base.lo, base.hi, 40, np.array([6, 1], np.int32), "fp64"),
        csl_gen.Query(base.weights, base.cons_idx, base.lo, base.hi, 20, np.array([3], np.int32), "fp64"),
    ]


def _equal(a, b):
    assert a["n"] == b["n"]
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["objective"], b["objective"])
    assert np.array_equal(a["reaction"], b["reaction"]) and np.array_equal(a["synthons"], b["synthons"])


@pytest.mark.parametrize("world", [2, 3])
def test_merge_of_parts_equals_whole_scope(world):
    lib, head, spec = csl_gen.build_workload("t_ragged")
    parts = shard.partition_reactions(_sizes(lib), world)
    for q in _queries(lib, spec):
        whole = _oracle_rows(lib, head, q)
        local = []
        for p in parts:
            sub = shard.local_subset(p, q.subset)
            if len(sub) == 0:
                local.append(shard.empty_rows(head.dims[-1]))
                continue
            local.append(_oracle_rows(lib, head, csl_gen.Query(q.weights, q.cons_idx, q.lo, q.hi, q.k, sub, "fp64")))
        _equal(shard.merge_topk(local, q.k), whole)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lib, head, spec = csl_gen.build_workload("t_ragged")
        qs = _queries(lib, spec)
        runner = shard.ShardedRunner(_sizes(lib), rank, world,
                                     lambda lq: [_oracle_rows(lib, head, q) for q in lq], head.dims[-1])
        merged = runner.run(qs)
        if rank == 0:
            for q, m in zip(qs, merged):
                _equal(m, _oracle_rows(lib, head, q))
            open(os.path.join(out_dir, "ok"), "w").write(str(len(merged)))
        else:
            assert merged is None
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_gloo_world_size_2_gather_merge(tmp_path):
    import torch.multiprocessing as mp

    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assert (tmp_path / "ok").read_text() == "5"
