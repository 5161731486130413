"""The allocation-free variant of Alg. 2 (imin_estimate_decrease_noalloc) against the regular
entry point and the oracle, through the C ABI.

Callers that cannot allocate device memory at call time (a foreign allocator with a fixed
budget, latency-critical paths where cudaMalloc/cudaFree may synchronize the device) use the
variant; it must return exactly the counters of imin_estimate_decrease. Two calls in a row check
that what the static scratch keeps from the previous call never leaks into the next. This file
is collected last so that a run that stops at the first failure has already run every other
test.
"""
from __future__ import annotations

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import oracle as O
from paper_2302_13529_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

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
        assert np.array_equal(got, O.decrease(q.graph, q.seeds, bl, theta, q.key, rnd)), rnd
    # device-resident inputs and output, twice in a row
    seeds_d = torch.from_numpy(q.seeds).cuda()
    out = torch.empty(q.graph.n, dtype=torch.uint64, device="cuda")
    for rnd, bl, theta in calls:
        want = cuda_lib.estimate_decrease(gh, q.seeds, bl, theta, q.key, rnd)
        bl_d = torch.tensor(bl, dtype=torch.int32, device="cuda") if bl else None
        cuda_lib.estimate_decrease_noalloc(gh, seeds_d, bl_d, theta, q.key, rnd, out=out)
        assert np.array_equal(out.cpu().numpy(), want), rnd


def test_no_alloc_on_a_linear_threshold_graph(cuda_lib):
    """The same call on a graph loaded under the linear-threshold model: equal to the regular
    entry point and to the oracle's LT mode."""
    q = W.tiny_chung_lu_query()
    g = W.Graph(q.graph.n, q.graph.row_ptr, q.graph.col, W.lt_wc_weights(q.graph.col, q.graph.n))
    gh = cuda_lib.load_graph(g, model="lt")
    for rnd, theta in ((0, 3000), (5, 2000)):
        got = cuda_lib.estimate_decrease_noalloc(gh, q.seeds, [], theta, q.key, rnd)
        assert np.array_equal(got, cuda_lib.estimate_decrease(gh, q.seeds, [], theta, q.key, rnd))
        assert np.array_equal(got, O.decrease(g, q.seeds, [], theta, q.key, rnd, model="lt"))


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


_CAPACITY_CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_2302_13529_gb300 import imin, workloads as W
    torch.cuda.set_device(0)
    g = W.graph_rmat_wc(11, 16000, seed=5)
    seeds = W.uniform_seeds(g.n, 12, seed=6)
    gh = imin.load_graph(g)
    try:
        imin.estimate_decrease_noalloc(gh, seeds, [], 3000, 1234, 2)
        print("no error")
        sys.exit(1)
    except imin.IminError as e:
        assert e.code == -4, e
    # the regular entry point hands the same samples to its whole-graph tier
    assert np.array_equal(imin.estimate_decrease(gh, seeds, [], 3000, 1234, 2),
                          O.decrease(g, seeds, [], 3000, 1234, 2))
    # the next call after the failure: an out-tree has no non-tree edges, so it fits
    rng = np.random.default_rng(3)
    parent = [int(rng.integers(0, v)) for v in range(1, 500)]
    t = W.graph_from_edges(500, [(p, v + 1, W.Fraction(1, 2)) for v, p in enumerate(parent)])
    th = imin.load_graph(t)
    got = imin.estimate_decrease_noalloc(th, [0], [], 4000, 99, 1)
    assert np.array_equal(got, imin.estimate_decrease(th, [0], [], 4000, 99, 1))
    assert np.array_equal(got, O.decrease(t, [0], [], 4000, 99, 1))
    print("capacity ok")
""")


def test_no_alloc_capacity_error_then_next_call(cuda_lib):
    """IMIN_ERR_CAPACITY when a sample needs more non-tree edges than the block tier holds (the
    IMIN_CTA_EDGE_CAP hook, set before the first call of a fresh process because the launch plan
    is kept per graph size), and a correct call right after it."""
    env = dict(os.environ, IMIN_CTA_EDGE_CAP="2", IMIN_TIER0_VERTICES="0")
    r = subprocess.run([sys.executable, "-c", _CAPACITY_CHILD.format(root=ROOT)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "capacity ok" in r.stdout, r.stdout + r.stderr
