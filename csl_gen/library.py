"""Synthetic combinatorial synthesis libraries (CSLs) and random-init surrogate heads.

A CSL here is the hierarchy of Sec. 3.2 (reactions -> R-groups -> synthons, App. A.1)
reduced to what enumeration needs: for every reaction t the number of R-group slots
n_t and the size of each slot, plus one d-dimensional associative embedding u_{r,s}
per (slot, synthon) (Eq. assoc_embeds). The embeddings are stored as one row-major
float32 matrix U whose rows are ordered reaction -> slot -> synthon.

Embeddings are drawn N(0, 1) and head weights U(-1/sqrt(fan_in), +1/sqrt(fan_in)),
both from numpy's PCG64 seeded per block, so that any block can be regenerated on its
own (the oracle re-creates only the reactions it samples).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

ACTIVATIONS = ("identity", "relu", "silu")


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


@dataclass
class CSL:
    """Shape and embeddings of one synthetic CSL.

    n_slots:    int32 [T]            number of R-group slots of each reaction
    slot_sizes: int64 [sum n_slots]  number of synthons in each slot, reaction-major
    d:          embedding width
    U:          float32 [sum slot_sizes, d] or None when only the shape is needed
    """

    n_slots: np.ndarray
    slot_sizes: np.ndarray
    d: int
    seed: int
    U: np.ndarray | None = None
    name: str = ""

    @property
    def n_reactions(self) -> int:
        return int(self.n_slots.shape[0])

    @property
    def slot_first(self) -> np.ndarray:
        """Index into slot_sizes of each reaction's first slot, [T+1]."""
        return np.concatenate([[0], np.cumsum(self.n_slots.astype(np.int64))])

    @property
    def row_first(self) -> np.ndarray:
        """First U row of every slot (reaction-major), [sum n_slots + 1]."""
        return np.concatenate([[0], np.cumsum(self.slot_sizes)])

    @property
    def n_rows(self) -> int:
        return int(self.slot_sizes.sum())

    def sizes_of(self, t: int) -> np.ndarray:
        f = self.slot_first
        return self.slot_sizes[f[t] : f[t + 1]]

    def block(self, t: int, j: int) -> np.ndarray:
        """Embeddings of slot j of reaction t, regenerated from the seed (float32 [n, d])."""
        n = int(self.sizes_of(t)[j])
        return _rng(self.seed, 1, t, j).standard_normal((n, self.d), dtype=np.float32)

    def materialize(self, threads: int | None = None) -> "CSL":
        """Fill U with every block (multi-threaded; each block has its own stream)."""
        U = np.empty((self.n_rows, self.d), dtype=np.float32)
        rf = self.row_first
        sf = self.slot_first
        jobs = [(t, j, int(rf[sf[t] + j])) for t in range(self.n_reactions) for j in range(int(self.n_slots[t]))]

        def fill(job):
            t, j, r0 = job
            b = self.block(t, j)
            U[r0 : r0 + b.shape[0]] = b

        nthreads = threads or min(32, os.cpu_count() or 1)
        if len(jobs) == 1 or nthreads == 1:
            for jb in jobs:
                fill(jb)
        else:
            with ThreadPoolExecutor(nthreads) as ex:
                list(ex.map(fill, jobs))
        self.U = U
        return self

    def subset_materialized(self, reactions, threads: int | None = None) -> "CSL":
        """The given reactions as a new CSL whose embeddings are generated directly from the
        original (reaction, slot) seeds, without materializing the whole library."""
        reactions = [int(t) for t in reactions]
        sf = self.slot_first
        sizes = np.concatenate([self.slot_sizes[sf[t] : sf[t + 1]] for t in reactions]).astype(np.int64)
        out = CSL(n_slots=self.n_slots[reactions].copy(), slot_sizes=sizes, d=self.d, seed=self.seed,
                  name=self.name + "[subset]")
        U = np.empty((out.n_rows, self.d), dtype=np.float32)
        jobs, r0 = [], 0
        for t in reactions:
            for j in range(int(self.n_slots[t])):
                n = int(self.sizes_of(t)[j])
                jobs.append((t, j, r0))
                r0 += n

        def fill(job):
            t, j, r = job
            b = self.block(t, j)
            U[r : r + b.shape[0]] = b

        with ThreadPoolExecutor(threads or min(32, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, jobs))
        out.U = U
        return out

    def subset(self, reactions) -> "CSL":
        """A new CSL made of the given reactions (in the given order); U is copied if present."""
        reactions = [int(t) for t in reactions]
        sf = self.slot_first
        sizes = np.concatenate([self.slot_sizes[sf[t] : sf[t + 1]] for t in reactions])
        n_slots = self.n_slots[reactions].copy()
        out = CSL(n_slots=n_slots, slot_sizes=sizes.astype(np.int64), d=self.d, seed=self.seed,
                  name=self.name + "[subset]")
        if self.U is not None:
            rf = self.row_first
            out.U = np.concatenate([self.U[rf[sf[t]] : rf[sf[t + 1]]] for t in reactions])
        return out


@dataclass
class Head:
    """Dense head applied to the compound embedding: dims[0] = d -> ... -> dims[-1] outputs.

    W[l] is float32 [dims[l+1], dims[l]] (row-major, PyTorch Linear layout), b[l] float32
    [dims[l+1]]. The activation follows every layer but the last.
    """

    dims: list
    activation: str
    W: list = field(default_factory=list)
    b: list = field(default_factory=list)
    n_objectives: int = 1
    n_properties: int = 0

    @property
    def n_layers(self) -> int:
        return len(self.dims) - 1

    @property
    def n_outputs(self) -> int:
        return int(self.dims[-1])


def make_head(dims, activation: str, seed: int, n_objectives: int, n_properties: int) -> Head:
    assert activation in ACTIVATIONS
    assert n_objectives + n_properties == dims[-1]
    W, b = [], []
    for l in range(len(dims) - 1):
        fan_in = dims[l]
        bound = 1.0 / math.sqrt(fan_in)
        W.append(_rng(seed, 2, l, 0).uniform(-bound, bound, size=(dims[l + 1], dims[l])).astype(np.float32))
        b.append(_rng(seed, 2, l, 1).uniform(-bound, bound, size=(dims[l + 1],)).astype(np.float32))
    return Head(dims=list(dims), activation=activation, W=W, b=b, n_objectives=n_objectives,
                n_properties=n_properties)


def library_from_sizes(sizes_per_reaction, d: int, seed: int, name: str = "", materialize=True) -> CSL:
    n_slots = np.array([len(s) for s in sizes_per_reaction], dtype=np.int32)
    slot_sizes = np.array([int(x) for s in sizes_per_reaction for x in s], dtype=np.int64)
    assert (slot_sizes >= 1).all() and (n_slots >= 1).all()
    lib = CSL(n_slots=n_slots, slot_sizes=slot_sizes, d=d, seed=seed, name=name)
    return lib.materialize() if materialize else lib


def _n_of(sizes_per_reaction) -> int:
    return int(sum(math.prod(int(x) for x in s) for s in sizes_per_reaction))


def lognormal_slot_sizes(seed: int, n_reactions: int, frac3: float, median: float, lo: int, hi: int,
                         target: float, sigma: float = 0.75):
    """Slot sizes of a synthetic CSL shaped like the paper's 2-/3-component libraries.

    Each size is lognormal(ln median, sigma), rounded and clamped to [lo, hi]. A seeded
    shuffle decides which reactions have 3 slots (round(frac3 * T) of them). The 2-slot
    reactions are kept as drawn; the 3-slot sizes are scaled by one factor alpha, found by
    bisection (each scaled size >= 2), so that the library holds ~target compounds. If the
    2-slot reactions alone already exceed the target, every reaction is scaled.
    """
    rng = _rng(seed, 3)
    n3 = int(round(frac3 * n_reactions))
    kinds = np.array([2] * (n_reactions - n3) + [3] * n3)
    rng.shuffle(kinds)
    raw = []
    for t in range(n_reactions):
        s = np.exp(rng.normal(math.log(median), sigma, size=int(kinds[t])))
        raw.append([int(min(hi, max(lo, round(x)))) for x in s])

    def scaled(alpha, which):
        out = []
        for s in raw:
            if which == "all" or len(s) == 3:
                out.append([max(2, int(round(alpha * x))) for x in s])
            else:
                out.append(list(s))
        return out

    n2 = _n_of([s for s in raw if len(s) == 2])
    which = "three" if (n2 < target and n3 > 0) else "all"
    lo_a, hi_a = 1e-6, 1.0
    while _n_of(scaled(hi_a, which)) < target and hi_a < 1e6:
        hi_a *= 2.0
    best = scaled(hi_a, which)
    for _ in range(200):
        mid = 0.5 * (lo_a + hi_a)
        cand = scaled(mid, which)
        n = _n_of(cand)
        if abs(n - target) < abs(_n_of(best) - target):
            best = cand
        if n < target:
            lo_a = mid
        else:
            hi_a = mid
        if abs(n - target) <= 0.001 * target:
            break
    return best


def make_library(sizes_per_reaction, d: int, seed: int, name: str = "", materialize: bool = True) -> CSL:
    return library_from_sizes(sizes_per_reaction, d, seed, name=name, materialize=materialize)
