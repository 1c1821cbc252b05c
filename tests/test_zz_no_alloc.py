"""The selection entry point for callers that cannot allocate device memory.

apex_topk_select_noalloc keeps its scratch in a fixed device array inside the library, for
callers whose device memory is owned by someone else (an arena or pool that forbids outside
allocations, a framework that owns every allocation) or that cannot afford cudaMalloc's
implicit synchronization. Its output must equal apex_topk_select's on the same input, on two
calls in a row (the shared array keeps the previous call's contents). This file is collected
last so that a stop at the first failure has already run every other test; it also passes
alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2510_24380_b300 import apex, build

pytestmark = pytest.mark.gpu


def _select(fn, keys, ids, k):
    import torch

    dk = torch.from_numpy(keys).cuda()
    di = torch.from_numpy(ids).cuda()
    m = min(k, len(keys))
    ok = torch.full((max(m, 1),), float("nan"), dtype=torch.float32, device="cuda")
    oi = torch.full((max(m, 1),), -1, dtype=torch.int64, device="cuda")
    n = fn(dk.data_ptr(), di.data_ptr(), len(keys), k, ok.data_ptr(), oi.data_ptr())
    torch.cuda.synchronize()
    return n, ok[:m].cpu().numpy(), oi[:m].cpu().numpy()


def test_noalloc_select_matches_allocating_select_twice():
    build.build()
    rng = np.random.default_rng(21)
    # the second call follows a larger one in the same array; the third asks for more than n
    # (k = 9000 > n = 5000: every key comes back, sorted)
    cases = [(200000, 65536), (50000, 777), (5000, 9000)]
    for n, k in cases:
        keys = rng.standard_normal(n).astype(np.float32)
        keys[rng.integers(0, n, n // 20)] = -0.5  # ties broken by the smaller id
        ids = (rng.permutation(n).astype(np.int64) << 3) + 5
        n_ref, k_ref, i_ref = _select(apex.apex_topk_select, keys, ids, k)
        n_got, k_got, i_got = _select(apex.apex_topk_select_noalloc, keys, ids, k)
        assert n_got == n_ref == min(n, k)
        assert np.array_equal(i_got, i_ref)
        assert np.array_equal(k_got, k_ref)  # same keys (exact: selection copies them)
        # and both equal the plain definition: key descending, then id ascending
        order = np.lexsort((ids, -keys.astype(np.float64)))[: min(n, k)]
        assert np.array_equal(i_got, ids[order]) and np.array_equal(k_got, keys[order])


def test_noalloc_select_rejects_k_above_its_limit():
    import torch

    n = apex.NOALLOC_MAX_K + 10
    dk = torch.zeros(n, dtype=torch.float32, device="cuda")
    di = torch.arange(n, dtype=torch.int64, device="cuda")
    with pytest.raises(apex.ApexError) as e:
        apex.apex_topk_select_noalloc(dk.data_ptr(), di.data_ptr(), n, n, dk.data_ptr(), di.data_ptr())
    assert e.value.code == -1 and "APEX_SELECT_NOALLOC_MAX_K" in str(e.value)
