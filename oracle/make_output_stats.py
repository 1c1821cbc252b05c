"""Write the per-output statistics that place the workloads' constraint boxes.

For each workload this scores compounds with the FP64 oracle (the whole library when it is
small, else a seeded uniform sample of 10^6 compound ids) and writes the mean, standard
deviation and 1001 quantiles of every head output to csl_gen/data/<workload>_stats.json.
It calls nothing but the oracle and the seeded generators.

usage: python oracle/make_output_stats.py c1_tiny c2_10m t_ragged t_linear [c3_real]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import csl_gen  # noqa: E402
from csl_gen.library import _rng  # noqa: E402
from oracle import oracle as O  # noqa: E402

FULL_LIMIT = 200_000
SAMPLE = 1_000_000


def stats_for(name: str) -> dict:
    lib, head, spec = csl_gen.build_workload(name)
    N = O.count(lib)
    if N <= FULL_LIMIT:
        ids = np.arange(N, dtype=np.int64)
        how = f"all {N} compounds"
    else:
        ids = np.sort(_rng(spec["seed"], 7).integers(0, N, size=SAMPLE)).astype(np.int64)
        how = f"seeded uniform sample of {SAMPLE} ids of {N} (PCG64 SeedSequence([{spec['seed']}, 7]))"
    t0 = time.time()
    out = O.score_ids(lib, head, ids)
    levels = np.linspace(0.0, 1.0, 1001)
    return {
        "workload": name,
        "n_compounds": int(N),
        "scored": how,
        "oracle_seconds": round(time.time() - t0, 2),
        "mean": out.mean(axis=0).tolist(),
        "std": out.std(axis=0).tolist(),
        "rms": np.sqrt((out ** 2).mean(axis=0)).tolist(),
        "quantile_levels": levels.tolist(),
        "quantiles": [np.quantile(out[:, i], levels).tolist() for i in range(out.shape[1])],
        "written_by": "oracle/make_output_stats.py (FP64 oracle scores)",
    }


def main(names):
    os.makedirs(csl_gen.queries.DATA_DIR, exist_ok=True)
    for name in names:
        s = stats_for(name)
        path = os.path.join(csl_gen.queries.DATA_DIR, f"{name}_stats.json")
        with open(path, "w") as f:
            json.dump(s, f)
        print(name, s["scored"], f"{s['oracle_seconds']} s", "->", path)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c1_tiny", "c2_10m", "t_ragged", "t_linear"])
