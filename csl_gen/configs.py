"""The synthetic workloads (library shape + head + query recipe), one per benchmark config.

Sizes follow the paper's CSL shapes: 2- and 3-component reactions (Sec. 2 / App. A.2),
libraries of ~1e7 and ~3e10 compounds (Table runtime's 12M / 10B / 70B scale), heads with
5 objective outputs and 8 property outputs, constraint counts like the Lipinski (4) and
Astex (6) sets of App. Table constraints.
"""
from __future__ import annotations

import numpy as np

from .library import CSL, _rng, lognormal_slot_sizes, library_from_sizes, make_head

WORKLOADS = {
    # 2 reactions x 2 slots x 100 synthons; 64 -> 64 -> 5 ReLU head (1 objective + 4 properties)
    "c1_tiny": dict(sizes=[[100, 100], [100, 100]], d=64, dims=[64, 64, 5], act="relu", n_obj=1, n_prop=4,
                    seed=0, k=100, precision="fp32"),
    # ~1e7 compounds: 40 reactions (70 % 2-slot, 30 % 3-slot), lognormal(300) sizes in [20, 3000]
    "c2_10m": dict(lognormal=dict(n_reactions=40, frac3=0.3, median=300, lo=20, hi=3000, target=1.0e7),
                   d=256, dims=[256, 256, 256, 13], act="silu", n_obj=5, n_prop=8, seed=0, k=1000,
                   precision="bf16"),
    # ~3e10 compounds: 1000 reactions, lognormal(2000) sizes, max 20000
    "c3_real": dict(lognormal=dict(n_reactions=1000, frac3=0.3, median=2000, lo=20, hi=20000, target=3.0e10),
                    d=256, dims=[256, 256, 256, 13], act="silu", n_obj=5, n_prop=8, seed=0, k=10000,
                    precision="bf16"),
    # test-sized library with ragged slots, a 1-slot and a 4-slot reaction, same head as c2/c3
    "t_ragged": dict(sizes=[[37, 129], [1, 300], [5, 7, 11], [257], [3, 2, 4, 5], [130, 127], [2, 64, 65]],
                     d=256, dims=[256, 256, 256, 13], act="silu", n_obj=5, n_prop=8, seed=7, k=50,
                     precision="bf16"),
    # test-sized library for the linear (paper-exact, Eq. apex) head
    "t_linear": dict(sizes=[[40, 60], [25, 30, 9], [200]], d=64, dims=[64, 3], act="identity", n_obj=1, n_prop=2,
                     seed=11, k=40, precision="fp32"),
    # 3-slot linear library the oracle enumerates in full (8e6 compounds, d = 1024)
    "t_linear_3x200": dict(sizes=[[200, 200, 200]], d=1024, dims=[1024, 3], act="identity", n_obj=1, n_prop=2,
                           seed=13, k=1000, precision="fp32"),
    # the paper's worked example (Sec. 3.3): 1 reaction x 3 slots x 10^4 synthons = 10^12 compounds,
    # d = 1024, with a linear head (1 objective + 2 properties)
    "linear_1e12": dict(sizes=[[10000, 10000, 10000]], d=1024, dims=[1024, 3], act="identity", n_obj=1, n_prop=2,
                        seed=17, k=1000, precision="fp32"),
}
# the first 12 reactions of c3_real (same seeds: identical synthon embeddings and head), ~4e8
# compounds in runs as long as c3_real's: profiling-sized (tables of a few tens of MB); its query
# recipe and output statistics are c3_real's
WORKLOADS["c3_slice"] = dict(WORKLOADS["c3_real"], slice_of="c3_real", n_slice=12, stats="c3_real")


def workload_sizes(name: str):
    w = WORKLOADS[name]
    if "slice_of" in w:
        return workload_sizes(w["slice_of"])[: w["n_slice"]]
    if "sizes" in w:
        return [list(s) for s in w["sizes"]]
    return lognormal_slot_sizes(seed=w["seed"], **w["lognormal"])


def build_workload(name: str, materialize: bool = True):
    """Returns (CSL, Head, spec) for a named workload."""
    w = WORKLOADS[name]
    sizes = workload_sizes(name)
    lib = library_from_sizes(sizes, d=w["d"], seed=w["seed"], name=name, materialize=materialize)
    head = make_head(w["dims"], w["act"], seed=w["seed"] + 1000, n_objectives=w["n_obj"], n_properties=w["n_prop"])
    return lib, head, w


def subset_prefix(lib: CSL, seed: int, target: float):
    """Reactions of a seeded shuffle of the library, taken in order until they hold >= target compounds."""
    order = np.arange(lib.n_reactions)
    _rng(seed, 4).shuffle(order)
    out, n = [], 0
    for t in order:
        out.append(int(t))
        n += int(np.prod(lib.sizes_of(int(t)).astype(np.float64)))
        if n >= target:
            break
    return sorted(out)
