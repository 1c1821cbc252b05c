"""Benchmark of the APEX hot path: compounds scored per second of the exhaustive top-k pass.

Default (no flags): the ~3e10-compound synthetic CSL `c3_real` (1,000 reactions of 2-3 slots,
lognormal(2000) slot sizes, d = 256, 256-256-256-13 SiLU head), BF16 tensor-core head with FP32
boundary rescore and FP64 tie-breaking, in the batched form: one step = one shared pass of the
circular enumeration serving 9 queries submitted together through the C ABI (the workload's own
query -- objective 0, six upper bounds at the 0.8 quantile, k = 10^4 -- plus 7 with random convex
weights over the 5 objectives, six property boxes and k in {100, 1000, 10^4}, all on the whole
library, and one more, k = 1000, restricted to the oracle's seeded sample of five small reactions
so that the oracle check below covers one whole top-k, members included). `value` counts
unique compounds scored per second (every compound's head evaluated once per step, whatever the
number of queries); `query_compounds_per_s` counts sum over queries of their scopes.

Beside it on the same JSON line: the FP32 plain single-query path (CUDA cores) on the 1e9-compound
reaction subset of the same library (a full FP32 pass over 3e10 compounds takes minutes); p50/p99
query latency over the timed steps (apex_stats); the roofline of the enumeration kernel; the
FP64 oracle on the host cores over a seeded sample of reactions, which also checks every query of
the last step with the reaction-decomposed rule (exact per sampled reaction); e2e through the C
ABI with host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3_real] [--queries 8]
                  [--precision bf16|fp16|fp8] [--mode batched|single|serving] [--impl ours|reference]

--mode single: one query per step (the workload's own). --mode serving: Poisson arrivals over the
resident library at each rate of --rates (queries on random subsets of 1-1000 reactions), p50/p99
latency and throughput per rate from apex_stats. Under torchrun (N > 1) the reactions are
partitioned across ranks by compound count, each rank serves every query on its part, and rank 0
gathers and merges the <= k rows of every query (strong scaling: the library is fixed).
--impl reference times the FP64 CPU oracle (the only reference this build has) on a bounded
sample of the same workload, per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOP_PER_COMPOUND = 2 * (256 * 256 + 256 * 13)  # layers 2 and 3 of the 256-256-256-13 head (MMA work)
METRIC = "compounds scored/s (BF16/FP8 batched vs FP32 plain), top-k match vs FP64; p99 query ms"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c3_real")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="batched", choices=["batched", "single", "serving"])
    ap.add_argument("--queries", type=int, default=8, help="queries per batched step")
    ap.add_argument("--subset-compounds", type=float, default=0.0,
                    help="batched: run the step's queries on the seeded reaction subset of this many compounds "
                         "(64 queries there, k in {10..10^5} and 8 boxes each, is the multi-query config)")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp16", "fp8", "fp32"],
                    help="pass precision of the enumeration (tensor-core bf16/fp16/fp8, or fp32 CUDA cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 plain leg")
    ap.add_argument("--fp32-subset", type=float, default=1e9, help="compounds of the FP32 plain leg's subset")
    ap.add_argument("--oracle-compounds", type=float, default=1.1e6,
                    help="compounds of the seeded reaction sample the oracle enumerates (per query)")
    ap.add_argument("--autotune", action="store_true", help="autotune the launch shape first (else 2^27 for c3_real)")
    ap.add_argument("--rates", default="5,20,50,100,200", help="serving: arrival rates (queries/s)")
    ap.add_argument("--serve-seconds", type=float, default=12.0, help="serving: arrival window per rate")
    ap.add_argument("--serve-max-queries", type=int, default=160, help="serving: cap on queries per rate")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# MUFU element rates per clock per SM, measured on a B300 with a full-occupancy kernel of independent
# chains timed by CUDA events (per clock at the 2,032 MHz maximum SM clock, so lower bounds):
# tanh.approx.{bf16x2,f16x2} 7.92 instructions (15.84 activations), ex2.approx.{bf16x2,f16x2} twice that
MUFU_SILU_PER_CLK_SM = 15.84
# share of the BF16 pass's layer-2 activations evaluated through ex2 (half the MUFU time of tanh)
EX2_SHARE_L2_BF16 = 3.0 / 8.0


def mufu_bound(N, head, enum_ms, clk, precision):
    """Second bound of the tensor-core kernel: the SiLU activations of every hidden layer on the MUFU
    (one tanh per pair, or one ex2 at half its cost for the BF16 layer-2 share), in tanh-equivalent
    activations, against the measured MUFU rate x 148 SMs x the sampled SM clock."""
    if head.activation != "silu":
        return None
    hidden = [float(x) for x in head.dims[1:-1]]
    acts = float(sum(hidden))
    work = acts
    if precision == "bf16" and len(hidden) >= 2:
        work = acts - hidden[1] * EX2_SHARE_L2_BF16 * 0.5
    mhz = (clk or {}).get("sm_mhz") or 2032.0
    achieved = N * work / (enum_ms * 1e-3) / (148 * mhz * 1e6)
    t_mufu = N * work / MUFU_SILU_PER_CLK_SM / 148 / (mhz * 1e6)
    t_tensor = N / 128 * 2851 / 148 / (mhz * 1e6)  # 2,221 (layer 2) + ~630 (layer 3) cycles per 128-row tile
    return {"bound": "xu", "unit": "tanh-equivalent activations/clk/SM", "achieved": achieved,
            "peak": MUFU_SILU_PER_CLK_SM, "frac": achieved / MUFU_SILU_PER_CLK_SM, "activations_per_compound": acts,
            "mufu_work_per_compound": work,
            "tensor_frac_cap": t_tensor / t_mufu if t_mufu > t_tensor else 1.0,
            "peak_kind": "measured tanh.approx.bf16x2 rate x 2 elements (ex2 counted at half)"}


def linear_roofline(N, q, lib, enum_ms, clk):
    """Linear head (Eq. apex): the work per compound is the scalar sums and compares, ALU-bound:
    (1 + m)(n - 1) additions + 2m comparisons (m constraints, n slots), against the FP32/INT
    lane rate 148 SMs x 128 lanes x the SM clock sampled during the run."""
    m = int(q.m)
    ops = 0.0
    for t in range(lib.n_reactions):
        n = len(lib.sizes_of(t))
        ops += float(np.prod(lib.sizes_of(t).astype(np.float64))) * ((1 + m) * (n - 1) + 2 * m)
    mhz = (clk or {}).get("sm_mhz") or 2032.0
    peak = 148 * 128 * mhz * 1e6 / 1e12  # Tops/s
    achieved = ops / (enum_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_linear (per-synthon scalar sums, Eq. apex)",
            "ops_per_compound": ops / N, "peak_kind": "148 SMs x 128 lanes x sampled SM clock",
            "kernel_ms_per_step": enum_ms}


def recorded_traffic(profile: str = "k_tc_head_c3_real.md"):
    """DRAM bytes per launch of the enumeration kernel from the committed ncu summary, when the
    kernel source is still the one the counters were taken on (sha256 of k_tc.cu + common.cuh +
    tc_sync.cuh);
    None otherwise."""
    import hashlib
    import re

    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        csrc = os.path.join(ROOT, "paper_2510_24380_b300", "csrc")
        h = hashlib.sha256()
        for f in ("k_tc.cu", "common.cuh", "tc_sync.cuh"):
            h.update(open(os.path.join(csrc, f), "rb").read())
        want = re.search(r"sha256\[:16\][^:]*:\s*([0-9a-f]{16})", text).group(1)
        traffic = int(re.search(r"traffic_bytes_per_launch:\s*(\d+)", text).group(1))
        return traffic if h.hexdigest()[:16] == want else None
    except Exception:
        return None


class _Nvml:
    """Read-only NVML queries through ctypes (the driver's libnvidia-ml): SM clock, max SM clock,
    clock-event reasons. Reason bits are the NVML API constants."""

    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, cuda_index: int):
        import ctypes as C

        self.C = C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.lib = lib
        self.h = C.c_void_p()
        import torch

        pr = torch.cuda.get_device_properties(cuda_index)
        bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
        if lib.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(self.h)) != 0:
            if lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(cuda_index), C.byref(self.h)) != 0:
                raise RuntimeError("no NVML handle")
        self.get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def clock(self, kind: str = "cur") -> float:
        C = self.C
        v = C.c_uint()
        fn = self.lib.nvmlDeviceGetClockInfo if kind == "cur" else self.lib.nvmlDeviceGetMaxClockInfo
        if fn(self.h, C.c_int(1), C.byref(v)) != 0:  # NVML_CLOCK_SM = 1
            raise RuntimeError("clock query failed")
        return float(v.value)

    def reasons(self) -> set:
        C = self.C
        v = C.c_ulonglong()
        if self.get_reasons(self.h, C.byref(v)) != 0:
            raise RuntimeError("reason query failed")
        return {n for n, bit in self.REASONS.items() if v.value & bit}


class Clocks:
    """SM clock and clock-event reasons sampled every few ms through NVML during the timed region;
    nvidia-smi at 200 ms when NVML cannot be opened."""

    REASON_NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int, period_s: float = 0.005):
        import threading

        self.samples, self.reasons, self.p, self.nv = [], set(), None, None
        self.stop_ev = threading.Event()
        try:
            self.nv = _Nvml(index)
            self.max_mhz = self.nv.clock("max")
            self.period = period_s
            self.sample()
            self.t = threading.Thread(target=self.loop, daemon=True)
            self.t.start()
        except Exception:
            self.nv = None
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            try:
                self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                          stderr=subprocess.DEVNULL)
            except Exception:
                self.p = None

    def sample(self):
        self.samples.append(self.nv.clock("cur"))
        self.reasons |= self.nv.reasons()

    def loop(self):
        while not self.stop_ev.wait(self.period):
            try:
                self.sample()
            except Exception:
                return

    def stop(self):
        if self.nv is not None:
            self.stop_ev.set()
            self.t.join(timeout=2)
            self.sample()
            return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                    "reasons": sorted(self.reasons), "samples": len(self.samples), "source": "nvml"}
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            if len(r) > 8:
                for n, v in zip(self.REASON_NAMES, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "source": "nvidia-smi"}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        import torch

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


def compounds_per_reaction(lib):
    return np.array([float(np.prod(lib.sizes_of(t).astype(np.float64))) for t in range(lib.n_reactions)])


def step_queries(args, spec, precision=None, sizes=None):
    """The step's queries. The batched form over the whole library adds one more query (the last
    random query's objective and boxes, k = 1,000) restricted to the oracle leg's seeded sample of
    small reactions, so that the oracle check covers one whole top-k, members included: the other
    queries' rows lie in reactions too large to enumerate on the host. (No such query when no
    reaction is small enough, as on c3_slice.)"""
    import csl_gen

    prec = precision or args.precision
    if args.mode == "single":
        return [csl_gen.query_single(args.workload, spec, precision=prec)]
    qs = csl_gen.queries_step(args.workload, spec, args.queries, seed=1, precision=prec)
    if sizes is not None:
        s0, _ = oracle_sample(sizes, args.oracle_compounds, seed=3)
        if s0:  # (an empty reaction list would mean the whole library through the C ABI)
            b = qs[-1]
            qs.append(csl_gen.Query(b.weights, b.cons_idx, b.lo, b.hi, 1000, np.array(s0, np.int32), b.precision))
    return qs


def oracle_sample(sizes, n_target: float, seed: int, min_reactions: int = 5):
    """A seeded sample of small reactions for the oracle: drawn from those no larger than
    max(n_target / 3, the min_reactions-th smallest) and never larger than n_target, until about
    n_target compounds (at least min_reactions reactions when that many fit)."""
    order = np.sort(sizes)
    cap = min(max(n_target / 3.0, order[min(min_reactions, len(order)) - 1]), n_target)
    cand = np.flatnonzero(sizes <= cap)
    np.random.default_rng(seed).shuffle(cand)
    chosen, n = [], 0.0
    for t in cand:
        if n + sizes[t] > n_target and len(chosen) >= min_reactions:
            continue
        chosen.append(int(t))
        n += sizes[t]
        if n >= 0.8 * n_target and len(chosen) >= min_reactions:
            break
    return sorted(chosen), int(n)


def row_bytes(n_out: int) -> int:
    return 8 + 4 + 8 * 4 + 8 + 8 * n_out  # id, reaction, synthons, objective, outputs


def query_upload_bytes(q) -> int:
    sub = 0 if q.subset is None else 4 * len(q.subset)
    return 4 * len(q.weights) + (4 + 8 + 8) * q.m + sub + 880  # descriptor arrays + the device query slot


def member_reactions(sizes, results, cap: float, budget: float, exclude=()):
    """Reactions that hold returned rows (of any query), no larger than `cap` compounds, most rows
    first, until about `budget` compounds: the reaction-decomposed check is exact on them for the
    members themselves (result n t == the oracle's first |result n t| of t), not only for the
    reactions' best non-members. The choice of reactions uses the rows; every expected value is
    the oracle's."""
    cnt = {}
    for r in results:
        for t in np.asarray(r["reaction"][: int(r["n"])]).tolist():
            cnt[int(t)] = cnt.get(int(t), 0) + 1
    cands = sorted((t for t in cnt if sizes[t] <= cap and t not in set(exclude)), key=lambda t: (-cnt[t], t))
    chosen, n = [], 0.0
    for t in cands:
        if n + sizes[t] > budget:
            continue
        chosen.append(int(t))
        n += float(sizes[t])
    return chosen, int(n)


def oracle_leg(L, lib, head, qs, results, n_target, seed=3, scope=None, max_checked=8):
    """The FP64 oracle as it stands, on every host core, over a seeded sample of small reactions
    plus the small reactions that hold the most returned rows: the exact top-(k + 65) of the sample
    for up to `max_checked` queries of the step (all of them when there are that few; else a seeded
    choice, so that the oracle's work stays bounded), timed (cpu_baseline, scaled to all queries),
    then the reaction-decomposed check of the GPU's rows against it for those queries and every
    returned member of every query rescored by the oracle (the top-k match). When no reaction of
    the queries' scope fits the sample budget, the smallest one is taken."""
    import csl_gen
    from oracle import oracle as O

    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import check_members_exact, check_reaction_decomposed, decomposed_query

    sizes = compounds_per_reaction(lib)
    nq = len(qs)
    if scope is not None:  # only the queries' reactions can be checked
        sizes = np.where(np.isin(np.arange(lib.n_reactions), scope), sizes, np.inf)
    S0, n0 = oracle_sample(sizes, n_target, seed)
    if not S0:
        t = int(np.argmin(sizes))
        S0, n0 = [t], int(sizes[t])
    # queries whose whole scope is sampled are always checked (cheap, and their top-k in full);
    # of the others up to max_checked, seeded
    inside = [i for i, q in enumerate(qs) if q.subset is not None and set(np.asarray(q.subset).tolist()) <= set(S0)]
    rest = [i for i in range(nq) if i not in inside]
    if len(rest) > max_checked:
        rest = sorted(np.random.default_rng(seed).choice(rest, max_checked, replace=False).tolist())
    checked = sorted(inside + rest)
    M, nM = member_reactions(sizes, results, cap=max(n_target, 1.0), budget=n_target, exclude=S0)
    S, nS = sorted(S0 + M), n0 + nM
    rms = np.array(list(L.info().rms)[: head.dims[-1]])
    t_or, refs = 0.0, {}
    for i in checked:
        sq = decomposed_query(qs[i], S)
        t0 = time.perf_counter()
        refs[i] = O.topk(lib, head, sq) if sq is not None else None
        t_or += time.perf_counter() - t0
    per, ok = [], True
    for i, (q, r) in enumerate(zip(qs, results)):
        entry = {"k": int(q.k), "n": int(r["n"]), "decomposed": i in refs}
        try:
            if i in refs:
                v = check_reaction_decomposed(r, lib, head, q, S, rms, ref=refs[i])
                entry.update(in_sample=v["in_result"], ambiguous=v["ambiguous"])
            check_members_exact(r, lib, head, q, rms)
            entry["ok"] = True
        except AssertionError as e:
            entry.update(ok=False, why=str(e)[:200])
            ok = False
        per.append(entry)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    t_all = t_or * nq / len(checked)  # the oracle's time for every query of the step over the sample
    sample = (f"{len(S)} of {lib.n_reactions} reactions ({nS} compounds: {len(S0)} drawn at random, {len(M)} "
              f"holding returned rows), {len(checked)} of the {nq} queries of a step enumerated exactly "
              f"({t_or:.1f} s; the value scales that time to all {nq} queries)")
    cpu = {"value": nS / t_all, "unit": "compounds/s", "cores": cores, "kind": "oracle", "sample": sample}
    match = {"passed": ok, "rule": "reaction-decomposed on the sampled reactions (exact per reaction) for the "
                                   "queries marked decomposed + every returned member of every query rescored in "
                                   "FP64 (feasible, objective and outputs within 1e-5)",
             "reactions": S, "member_reactions": M, "sample_compounds": nS, "decomposed_queries": checked,
             "queries": per}
    return cpu, match


def run_reference(args):
    """The FP64 oracle (no other reference exists) on the host cores, timed per step on a bounded
    seeded sample of the workload's reactions: every query of the step over the sample."""
    import csl_gen
    from oracle import oracle as O

    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    full, head, spec = csl_gen.build_workload(args.workload, materialize=False)
    sizes = compounds_per_reaction(full)
    qs = step_queries(args, spec, precision="fp64", sizes=sizes)
    # rate probe on the smallest reaction
    t_small = int(np.argmin(sizes))
    lib1 = full.subset_materialized([t_small])
    t0 = time.perf_counter()
    for q in qs:
        O.topk(lib1, head, csl_gen.Query(q.weights, q.cons_idx, q.lo, q.hi, q.k, None, "fp64"))
    rate = sizes[t_small] / max(time.perf_counter() - t0, 1e-6)  # compounds per second for all queries
    budget = max(2.0, 150.0 / max(1, args.warmup + args.steps))
    vals, ms, last = [], [], None
    for i in range(args.warmup + args.steps):
        S, nS = oracle_sample(sizes, rate * budget, seed=100 + i, min_reactions=1)
        lib_s = full.subset_materialized(S)
        t0 = time.perf_counter()
        for q in qs:  # every query over the sampled reactions of its scope
            sub = None if q.subset is None else np.flatnonzero(np.isin(S, q.subset)).astype(np.int32)
            if sub is None or len(sub):
                O.topk(lib_s, head, csl_gen.Query(q.weights, q.cons_idx, q.lo, q.hi, q.k, sub, "fp64"))
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(nS / dt)
            ms.append(1e3 * float(sizes.sum()) / (nS / dt))
            last = (S, nS, dt)
    v = float(np.mean(vals))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    N = float(sizes.sum())
    line = {"metric": METRIC, "value": v, "unit": "compounds/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(args, full, head, qs, N, world=1), "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "compounds/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step {len(last[0])} seeded reactions (~{last[1]} compounds) x "
                                       f"{len(qs)} queries, ~{last[2]:.1f} s; ms_per_step extrapolated to the "
                                       f"whole library"},
            "e2e": {"value": v, "unit": "compounds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_config(args, lib, head, qs, N, world):
    form = "batched" if args.mode == "batched" else "single query"
    where = f" {N:.3g}-compound reaction subset," if args.subset_compounds > 0 else ""
    n_sub = sum(q.subset is not None for q in qs) if args.subset_compounds <= 0 else 0
    canary = (f" ({len(qs) - n_sub} on the whole library, {n_sub} on the oracle's seeded sample of "
              f"{len(qs[-1].subset)} small reactions, checked in full)") if n_sub else ""
    return {"workload": f"{args.workload}{where} {form}: {len(qs)} quer{'ies' if len(qs) > 1 else 'y'} per shared "
                        f"pass{canary}",
            "n_compounds": int(N), "n_reactions": int(lib.n_reactions), "queries_per_step": len(qs),
            "k": [int(q.k) for q in qs], "n_constraints": [int(q.m) for q in qs],
            "head": "-".join(str(x) for x in head.dims) + f" {head.activation}",
            "precision": f"{args.precision} pass + "
                         f"{'fp16' if args.precision in ('bf16', 'fp8') else 'fp32'} in-pass compaction rescore + "
                         "fp32 boundary rescore + fp64 tie-break",
            "parallelism": f"reactions sharded x{world} (gather merge of <= k rows per query)" if world > 1
            else "1 GPU",
            "l2": "inputs larger than L2 (the 16-bit P table alone is 2.1 GB on c3_real) and a 512 MB write before "
                  "every timed step"}


def run_batched(args):
    import torch

    import csl_gen
    from paper_2510_24380_b300 import apex, shard

    world, rank, local, pg = dist_setup(args)
    t_load0 = time.perf_counter()
    lib, head, spec = csl_gen.build_workload(args.workload)
    sizes = compounds_per_reaction(lib)
    prec = args.precision
    scope = None
    if args.subset_compounds > 0:  # the multi-query form on a reaction subset: random queries only
        scope = np.array(csl_gen.subset_prefix(lib, 0, args.subset_compounds), np.int32)
        qs = csl_gen.queries_batched(csl_gen.load_stats(args.workload), spec["n_obj"], spec["n_prop"], args.queries,
                                     seed=1, subset=scope, precision=prec)
        N = float(sizes[scope].sum())  # every step scores the subset once
    else:
        qs = step_queries(args, spec, sizes=sizes)
        N = float(sizes.sum())
    dev = local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    L = apex.Library(lib, head, precisions=("fp32", prec), device=dev, stream=stream.cuda_stream, seed=0)
    load_s = time.perf_counter() - t_load0
    if args.autotune:
        tune = L.autotune(prec, n_queries=len(qs), k=10000,
                          subset=scope if scope is not None else np.arange(min(30, lib.n_reactions)))
    elif N > 1e9 and len(head.dims) > 2:
        L.set_launch_shape(1 << 27, 32)  # 2^27 compounds per launch: the autotuner's choice on this library
        tune = {"chosen_chunk_compounds": 1 << 27, "how": "fixed (autotuned choice on this workload)"}
    else:
        tune = {"chosen_chunk_compounds": 1 << 25, "how": "library default"}

    qstats = []  # stats of every query of the last run (fetched one after another)

    def run_local(lq):
        ids = [L.query(q) for q in lq]
        out = []
        qstats.clear()
        for i, q in zip(ids, lq):
            out.append(L.fetch(i, q.k))
            qstats.append(L.stats(-1))
        return out

    runner = shard.ShardedRunner(sizes, rank, world, run_local, L.n_outputs)
    n_rank = float(sizes[runner.part].sum())
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    for _ in range(args.warmup):
        runner.run(qs)
    torch.cuda.synchronize()
    barrier(pg)

    # ------------------------------------------------------------- timed region (device events)
    clocks = Clocks(dev) if rank == 0 else None
    L.reset_serving_stats()
    launches0 = apex.apex_kernel_launches()
    dev_ms, e2e_ms, res = [], [], None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        torch.cuda.synchronize()
        barrier(pg)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        res = runner.run(qs)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        dev_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = apex.apex_kernel_launches() - launches0
    sv = L.serving_stats()
    clk = clocks.stop() if clocks else None
    barrier(pg)
    t_dev = max_over_ranks(pg, float(np.sum(dev_ms)))
    t_e2e = max_over_ranks(pg, float(np.sum(e2e_ms)))
    last_stats = [L.stats(-1)]
    if rank != 0:
        barrier(pg)
        L.close()
        return

    # ------------------------------------------------------------- FP32 plain path, same library
    fp32 = None
    if not args.no_fp32:
        sub = csl_gen.subset_prefix(lib, 0, args.fp32_subset)
        n_sub = float(sizes[sub].sum())
        q0 = qs[0]
        q32 = csl_gen.Query(q0.weights, q0.cons_idx, q0.lo, q0.hi, q0.k, np.array(sub, np.int32), "fp32")
        q16 = csl_gen.Query(q0.weights, q0.cons_idx, q0.lo, q0.hi, q0.k, np.array(sub, np.int32), prec)
        L.run(csl_gen.Query(q0.weights, q0.cons_idx, q0.lo, q0.hi, q0.k,
                            np.array([int(np.argmin(sizes))], np.int32), "fp32"))  # warm-up
        times = {}
        rows = {}
        for name, qq in (("fp32", q32), (prec, q16)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rows[name] = L.run(qq)
            e1.record(stream)
            e1.synchronize()
            times[name] = e0.elapsed_time(e1)
        fp32 = {"value": n_sub / (times["fp32"] * 1e-3), "unit": "compounds/s",
                "workload": f"{args.workload} reaction subset of {len(sub)} reactions ({int(n_sub)} compounds; a full "
                            f"FP32 pass over the library takes minutes), the workload's query, single query, FP32 "
                            f"CUDA cores",
                "ms": times["fp32"],
                f"{prec}_single_query_same_subset": n_sub / (times[prec] * 1e-3),
                "same_topk_set_as_tc_pass": bool(set(rows["fp32"]["ids"].tolist()) == set(rows[prec]["ids"].tolist()))}

    P, kind = peaks()
    K = args.steps
    enum_ms = sv["enumerate_ms"] / K
    # compounds the enumeration launches scored per step (the scope once per pass; more when a query
    # had to run its pass again)
    n_enum = sv["head_evaluations"] / K if sv["head_evaluations"] > 0 else n_rank
    achieved = FLOP_PER_COMPOUND * n_enum / (enum_ms * 1e-3) / 1e12
    linear = len(head.dims) == 2
    peak_s = P.get("bf16_tflops_sustained", 1400.0)
    peak_b = P.get("bf16_tflops", 1800.0)
    if prec == "fp8":
        peak_s, peak_b = 2 * peak_s, 2 * peak_b  # layer 2 at the FP8 rate (nominal 2x of BF16)
    if linear:
        roof = linear_roofline(n_rank, qs[0], lib, enum_ms, clk)
    else:
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_s, "unit": "TFLOP/s", "frac": achieved / peak_s,
                "traffic": recorded_traffic(f"k_tc_head_{args.workload}.md"),
                "kernel": "k_tc_head (enumeration: layer-1 sums and SiLU on CUDA cores, layers 2-3 on tcgen05)",
                "flop_per_compound": FLOP_PER_COMPOUND,
                "peak_kind": f"{kind} bf16 sustained (the kernel runs for seconds inside each step); "
                             f"against the {kind} burst peak {peak_b:.0f}: frac {achieved / peak_b:.3f}",
                "frac_vs_burst": achieved / peak_b, "kernel_ms_per_step": enum_ms,
                "launches_per_step": sv["n_enumeration_launches"] / K,
                "compounds_scored_per_step": n_enum,
                "mufu": mufu_bound(n_enum, head, enum_ms, clk, prec)}
    d2h = int(sum(r["n"] for r in res)) * row_bytes(L.n_outputs)
    h2d = int(sum(query_upload_bytes(q) for q in qs))
    qc = float(sum(N if q.subset is None else sizes[q.subset].sum() for q in qs))
    line = {
        "metric": METRIC,
        "value": N * K / (t_dev * 1e-3),
        "unit": "compounds/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": t_dev / K,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": prec,
        "data": "synthetic (seeded N(0,1) synthon embeddings, random-init head; the paper's libraries are unavailable)",
        "config": run_config(args, lib, head, qs, N, world),
        "query_compounds_per_s": qc * K / (t_dev * 1e-3),
        "latency": {"p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "max_ms": sv["max_ms"],
                    "queue_p99_ms": sv["queue_p99_ms"], "n_queries": sv["n_queries"]},
        "e2e": {"value": N * K / (t_e2e * 1e-3), "unit": "compounds/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "p50_ms": float(np.percentile(e2e_ms, 50)),
                "p99_ms": float(np.percentile(e2e_ms, 99))},
        "gpu_launches": int(launches),
        "roofline": roof,
        "fp32_plain": fp32,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cpu, match = oracle_leg(L, lib, head, qs, res, args.oracle_compounds, scope=scope)
        line["topk_match_vs_fp64_oracle"] = match
        line["cpu_baseline"] = cpu
    line["queries"] = [{"k": int(q.k), "n": int(r["n"])} for q, r in zip(qs, res)]
    if qstats:  # the runtime margin check and the candidate traffic of the last step's queries
        line["margin_check"] = {
            "max_pass_err_ratio": round(max(st["pass_err_ratio"] for st in qstats), 4),
            "max_fp32_err_ratio": round(max(st["fp32_err_ratio"] for st in qstats), 4),
            "n_margin_reruns": int(sum(st["n_margin_reruns"] for st in qstats)),
            "n_restarts": int(sum(st["n_restarts"] for st in qstats)),
            "n_compactions": int(sum(st["n_compactions"] for st in qstats)),
            "max_candidates": int(max(st["n_candidates"] for st in qstats)),
            "rule": "observed max |pass - FP32| objective and |FP32 - FP64| output over every candidate / the "
                    "margins the pass used; a ratio above 1 reruns the query with wider margins"}
    st = last_stats[0]
    line["last_query_stats"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()
                                if k in ("n_candidates", "n_rescored_fp64", "n_restarts", "n_margin_reruns",
                                         "pass_err_ratio", "fp32_err_ratio", "n_launches", "enumerate_ms",
                                         "latency_ms", "host_finalize_ms")}
    line["host"] = {"load_s": round(load_s, 1), "launch_shape": tune,
                    "margins": {"pass": [round(x, 5) for x in list(getattr(L.info(), "err_" + prec))[:L.n_outputs]]
                                if prec != "fp32" else None,
                                "fp32": [float("%.3g" % x) for x in list(L.info().err_fp32)[:L.n_outputs]]}}
    line["steps_detail_ms"] = [round(x, 2) for x in dev_ms]
    barrier(pg)
    L.close()
    print(json.dumps(line))


def run_serving(args):
    """Poisson arrivals at each rate over the resident library: each query on a random subset of
    1..1000 reactions (log-uniform count), random weights and boxes, k log-uniform in [10, 10^5];
    p50/p99 latency, queue time and throughput per rate from apex_stats."""
    import threading

    import torch

    import csl_gen
    from paper_2510_24380_b300 import apex

    lib, head, spec = csl_gen.build_workload(args.workload)
    stats = csl_gen.load_stats(args.workload)
    stream = torch.cuda.Stream()
    L = apex.Library(lib, head, precisions=("fp32", args.precision), stream=stream.cuda_stream)
    if lib.n_reactions >= 100:
        L.set_launch_shape(1 << 27, 32)
    out = {"mode": "serving", "workload": f"{args.workload} resident", "precision": args.precision,
           "n_compounds": float(compounds_per_reaction(lib).sum()), "rates": []}
    for i, rate in enumerate(float(x) for x in args.rates.split(",")):
        n_q = int(min(args.serve_max_queries, max(8, rate * args.serve_seconds)))
        arrivals = csl_gen.serving_stream(stats, spec["n_obj"], spec["n_prop"], lib.n_reactions, n_q, rate, seed=2 + i,
                                          precision=args.precision)
        L.reset_serving_stats()
        threads = []
        t0 = time.perf_counter()
        for t_arr, q in arrivals:
            now = time.perf_counter() - t0
            if t_arr > now:
                time.sleep(t_arr - now)
            qid = L.query(q)
            th = threading.Thread(target=L.fetch, args=(qid, int(q.k)))
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        sv = L.serving_stats()
        out["rates"].append({"rate_hz": rate, "queries": sv["n_queries"], "failed": sv["n_failed"],
                             "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"], "max_ms": sv["max_ms"],
                             "queue_p50_ms": sv["queue_p50_ms"], "queue_p99_ms": sv["queue_p99_ms"],
                             "wall_s": sv["wall_ms"] / 1e3, "query_compounds_per_s": sv["query_compounds_per_s"],
                             "head_evaluations_per_s": sv["head_evaluations_per_s"],
                             "mean_scope_compounds": sv["query_compounds"] / max(1, sv["n_queries"])})
    L.close()
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "serving":
        return run_serving(args)
    return run_batched(args)


if __name__ == "__main__":
    main()
