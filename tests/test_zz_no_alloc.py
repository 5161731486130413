"""The allocation-free variant of Alg. 2 (imin_estimate_decrease_noalloc) against the regular
entry point, through the C ABI.

Callers that cannot allocate device memory at call time (stream capture, a foreign allocator
with a fixed budget, latency-critical paths) use the variant; it must return exactly the
counters of imin_estimate_decrease. Two calls in a row check that what the static scratch keeps
from the previous call never leaks into the next. This file is collected last so that a run that
stops at the first failure has already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2302_13529_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_no_alloc_matches_regular_entry_point(cuda_lib):
    import torch
    q = W.tiny_chung_lu_query()
    gh = cuda_lib.load_graph(q.graph)
    blocked = [int(x) for x in np.setdiff1d(np.arange(40), q.seeds)[:5]]
    calls = ((0, [], 10_000), (3, blocked, 7_000))  # two calls in a row, different inputs
    for rnd, bl, theta in calls:
        want = cuda_lib.estimate_decrease(gh, q.seeds, bl, theta, q.key, rnd)
        got = cuda_lib.estimate_decrease_noalloc(gh, q.seeds, bl, theta, q.key, rnd)
        assert np.array_equal(got, want), rnd  # integer counters: tolerance 0
    # device-resident inputs and output, twice in a row
    seeds_d = torch.from_numpy(q.seeds).cuda()
    out = torch.empty(q.graph.n, dtype=torch.uint64, device="cuda")
    for rnd, bl, theta in calls:
        want = cuda_lib.estimate_decrease(gh, q.seeds, bl, theta, q.key, rnd)
        bl_d = torch.tensor(bl, dtype=torch.int32, device="cuda") if bl else None
        cuda_lib.estimate_decrease_noalloc(gh, seeds_d, bl_d, theta, q.key, rnd, out=out)
        assert np.array_equal(out.cpu().numpy(), want), rnd


def test_no_alloc_rejects_requests_beyond_its_limits(cuda_lib):
    from paper_2302_13529_gb300.imin import IminError
    q = W.tiny_chung_lu_query()
    gh = cuda_lib.load_graph(q.graph)
    with pytest.raises(IminError) as e:
        cuda_lib.estimate_decrease_noalloc(gh, q.seeds, [], 1 << 18, q.key, 0)
    assert e.value.code == -1 and "static limit" in str(e.value)
    big = W.Graph(70_000, np.zeros(70_001, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    gbig = cuda_lib.load_graph(big)
    with pytest.raises(IminError) as e:
        cuda_lib.estimate_decrease_noalloc(gbig, [1], [], 10, 1, 0)
    assert e.value.code == -1 and "static limit" in str(e.value)
    with pytest.raises(IminError) as e:
        cuda_lib.estimate_decrease_noalloc(gh, [int(q.seeds[0])] * 2, [], 10, 1, 0)
    assert e.value.code == -1
