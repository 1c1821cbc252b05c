"""Shared comparison rules for the GPU parity tests.

Tolerances (from the stated targets; near-zero handling as a relative bound with an RMS floor):
  FP32 raw outputs:  |x - x*| <= 1e-5 * max(|x*|, RMS of that output)
  BF16 raw outputs:  |x - x*| <= 2e-2 absolute
  final top-k set:   equal to the FP64 oracle's set, except compounds whose oracle objective is
                     within tol of the oracle's k-th objective or whose constrained outputs are
                     within tol of a bound (ambiguous set A), with tol = 1e-9 * RMS (the FP64
                     rescore decides the boundary); the counts must agree.
"""
import numpy as np

from oracle import oracle as O

FP32_REL = 1e-5
BF16_ABS = 2e-2  # raw BF16, FP16 and FP8 pass outputs (absolute)
SET_TOL_REL = 1e-9


def rel_err(x, ref, rms):
    floor = np.maximum(np.abs(ref), rms[None, :] if ref.ndim == 2 else rms)
    return np.abs(x - ref) / floor


def assert_fp32_close(x, ref, rms):
    if np.asarray(x).size == 0:
        assert np.asarray(ref).size == 0
        return
    e = rel_err(np.asarray(x, np.float64), ref, rms)
    assert e.max() <= FP32_REL, f"max relative error {e.max():.3e}"


def output_rms(lib, head, n=2048, seed=5):
    N = O.count(lib)
    ids = np.random.default_rng(seed).integers(0, N, size=min(n, N))
    o = O.score_ids(lib, head, ids)
    return np.sqrt((o ** 2).mean(axis=0)) + 1e-30


def objective(outputs, w):
    w = np.asarray(w, np.float32).astype(np.float64)
    return outputs[:, : len(w)] @ w


def check_topk(res, ref, lib, head, q, rms):
    """res: GPU fetch dict; ref: oracle TopK. Applies the boundary-tolerance set rule and checks
    order, feasibility, reported objectives and outputs."""
    n = res["n"]
    assert n == len(ref.ids), (n, len(ref.ids))
    gids = res["ids"]
    assert len(set(gids.tolist())) == len(gids), "duplicate ids"
    # order: objective desc, id asc
    obj = res["objective"]
    for i in range(len(gids) - 1):
        assert obj[i] > obj[i + 1] or (obj[i] == obj[i + 1] and gids[i] < gids[i + 1]), i
    # exact oracle values for every id in either set
    union = np.union1d(gids, ref.ids)
    o_u = O.score_ids(lib, head, union) if len(union) else np.zeros((0, head.dims[-1]))
    f_u = objective(o_u, q.weights)
    rms_f = float(np.sqrt(np.mean(f_u ** 2))) if len(f_u) else 1.0
    tol = SET_TOL_REL * max(rms_f, float(rms.max()))
    fk = ref.scores[-1] if len(ref.scores) else -np.inf
    amb = np.abs(f_u - fk) <= tol
    for c, lo, hi in zip(q.cons_idx, q.lo, q.hi):
        v = o_u[:, c]
        amb |= (np.abs(v - lo) <= tol) | (np.abs(v - hi) <= tol)
    A = set(union[amb].tolist())
    g_set = set(gids.tolist()) - A
    r_set = set(ref.ids.tolist()) - A
    assert g_set == r_set, f"{len(g_set ^ r_set)} ids differ outside the ambiguous set ({len(A)} ambiguous)"
    # every GPU result is feasible under FP64 (up to tol) and its reported values match the oracle
    pos = np.searchsorted(union, gids)
    og = o_u[pos]
    for c, lo, hi in zip(q.cons_idx, q.lo, q.hi):
        assert np.all(og[:, c] >= lo - tol) and np.all(og[:, c] <= hi + tol)
    fg = f_u[pos]
    scale = np.maximum(np.abs(fg), rms_f)
    assert np.all(np.abs(obj - fg) <= FP32_REL * scale), np.max(np.abs(obj - fg) / scale)
    assert_fp32_close(res["outputs"], og, rms)
    return len(A)


def reaction_first_ids(lib):
    """First global id of every reaction (library order), [T + 1]."""
    sizes = [int(np.prod(lib.sizes_of(t).astype(np.int64))) for t in range(lib.n_reactions)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def decomposed_query(q, reactions, slack=64):
    """The oracle query of the reaction-decomposed check: q restricted to the given reactions (and
    its own subset), k + 1 + slack deep; None when no sampled reaction lies in q's scope."""
    import csl_gen

    scope = None if q.subset is None else set(int(t) for t in q.subset)
    S = sorted(int(t) for t in reactions if scope is None or int(t) in scope)
    if not S:
        return None
    return csl_gen.Query(q.weights, q.cons_idx, q.lo, q.hi, int(q.k) + 1 + slack, np.array(S, np.int32), "fp64")


def check_reaction_decomposed(res, lib, head, q, reactions, rms, slack=64, ref=None):
    """Reaction-decomposed check of a result against the FP64 oracle (the top-k of Eq. apex_topk
    restricted to a set of reactions), usable at any library size.

    The exact top-k X of the whole scope, restricted to any set S of its reactions, is the first
    |X n S| compounds of S's own order (objective desc, id asc, feasible only); and when |X| = k
    the next feasible compound of S scores at most the k-th objective, while when |X| < k every
    feasible compound of S is in X. So with G = res's ids in S and R = the oracle's order of S
    (top k + 1 + slack), outside the ambiguous set A (FP64 objective within tol of the k-th, or a
    constrained output within tol of a bound; tol = SET_TOL_REL * RMS):
      G \\ A == the first |G \\ A| of R \\ A, and
      if n == k: the next element of R \\ A scores <= f_k + tol; else R \\ A == G \\ A.
    ref: the oracle's answer to decomposed_query(q, reactions, slack), when already computed.
    Returns a summary dict (reactions checked, |G n S|, oracle compounds scored)."""
    k = int(q.k)
    sub = decomposed_query(q, reactions, slack)
    if sub is None:
        return {"reactions": 0, "in_result": 0, "oracle_compounds": 0, "ambiguous": 0}
    S = [int(t) for t in sub.subset]
    first = reaction_first_ids(lib)
    n_S = int(sum(first[t + 1] - first[t] for t in S))
    if ref is None:
        ref = O.topk(lib, head, sub)
    gids = np.asarray(res["ids"], np.int64)
    rxn = np.searchsorted(first, gids, side="right") - 1
    G = gids[np.isin(rxn, S)]
    n = int(res["n"])
    # FP64 values of every compound involved: the GPU's members of S, the oracle's list, the k-th
    extra = gids[-1:] if n == k and n > 0 else np.zeros(0, np.int64)
    union = np.union1d(np.union1d(G, ref.ids), extra)
    o_u = O.score_ids(lib, head, union) if len(union) else np.zeros((0, head.dims[-1]))
    f_u = objective(o_u, q.weights)
    rms_f = float(np.sqrt(np.mean(f_u ** 2))) if len(f_u) else 1.0
    tol = SET_TOL_REL * max(rms_f, float(np.max(rms)))
    fk = float(f_u[np.searchsorted(union, gids[-1])]) if n == k and n > 0 else -np.inf
    amb = np.abs(f_u - fk) <= tol
    for c, lo, hi in zip(q.cons_idx, q.lo, q.hi):
        v = o_u[:, c]
        amb |= (np.abs(v - lo) <= tol) | (np.abs(v - hi) <= tol)
    A = set(union[amb].tolist())
    g = [int(x) for x in G if int(x) not in A]
    r = [int(x) for x in ref.ids if int(x) not in A]
    assert len(r) >= len(g), (len(r), len(g))
    assert set(g) == set(r[: len(g)]), (
        f"{len(set(g) ^ set(r[: len(g)]))} of {len(g)} result members in the sampled reactions differ from the "
        f"oracle's order of those reactions")
    if n == k:
        if len(r) > len(g):
            nxt = int(r[len(g)])
            f_next = float(f_u[np.searchsorted(union, nxt)])
            assert f_next <= fk + tol, f"oracle compound {nxt} of a sampled reaction beats the k-th result ({f_next} > {fk})"
    else:
        assert len(ref.ids) < k + 1 + slack and len(r) == len(g), (
            f"fewer than k results, but the sampled reactions hold {len(r)} feasible compounds against {len(g)} returned")
    # reported values of the members checked here equal the oracle's
    if len(G):
        sel = np.isin(gids, G)
        og = o_u[np.searchsorted(union, gids[sel])]
        fg = objective(og, q.weights)
        scale = np.maximum(np.abs(fg), rms_f)
        obj = np.asarray(res["objective"])[sel]
        assert np.all(np.abs(obj - fg) <= FP32_REL * scale), np.max(np.abs(obj - fg) / scale)
        assert_fp32_close(np.asarray(res["outputs"])[sel], og, rms)
    return {"reactions": len(S), "in_result": int(len(G)), "oracle_compounds": n_S, "ambiguous": len(A)}


def check_members_exact(res, lib, head, q, rms):
    """Every returned compound, rescored by the FP64 oracle: feasible (within tol), reported objective
    and outputs equal to the oracle's, order (objective desc, id asc), no duplicates; any size."""
    gids = np.asarray(res["ids"], np.int64)
    assert len(set(gids.tolist())) == len(gids), "duplicate ids"
    obj = np.asarray(res["objective"])
    for i in range(len(gids) - 1):
        assert obj[i] > obj[i + 1] or (obj[i] == obj[i + 1] and gids[i] < gids[i + 1]), i
    if len(gids) == 0:
        return
    o = O.score_ids(lib, head, gids)
    f = objective(o, q.weights)
    rms_f = float(np.sqrt(np.mean(f ** 2)))
    tol = SET_TOL_REL * max(rms_f, float(np.max(rms)))
    for c, lo, hi in zip(q.cons_idx, q.lo, q.hi):
        assert np.all(o[:, c] >= lo - tol) and np.all(o[:, c] <= hi + tol)
    scale = np.maximum(np.abs(f), rms_f)
    assert np.all(np.abs(obj - f) <= FP32_REL * scale), np.max(np.abs(obj - f) / scale)
    assert_fp32_close(np.asarray(res["outputs"]), o, rms)


def seeded_small_reactions(lib, n, max_compounds, seed, must=()):
    """n reactions drawn (seeded) from those with at most max_compounds compounds, plus `must`."""
    first = reaction_first_ids(lib)
    sizes = np.diff(first)
    small = np.flatnonzero(sizes <= max_compounds)
    rng = np.random.default_rng(seed)
    pick = rng.choice(small, size=min(n, len(small)), replace=False) if len(small) else np.zeros(0, int)
    return sorted(set(int(t) for t in pick) | set(int(t) for t in must))
