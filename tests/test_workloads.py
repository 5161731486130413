"""The synthetic inputs (CPU): exact edge counts, no self-loops or duplicates, seeded
determinism, the degree skew each generator is meant to have, and the threshold encodings of the
weighted-cascade and trivalency models."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

from paper_2302_13529_gb300 import workloads as W


def _edges(rp, col):
    n = len(rp) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    return src, col.astype(np.int64)


def _check_simple(rp, col, n, m):
    assert rp[0] == 0 and rp[-1] == m and len(col) == m and len(rp) == n + 1
    assert np.all(np.diff(rp) >= 0)
    src, dst = _edges(rp, col)
    assert np.all((dst >= 0) & (dst < n))
    assert not np.any(src == dst), "self-loop"
    assert len(np.unique(src * n + dst)) == m, "duplicate edge"


@pytest.mark.parametrize("n,m", [(2000, 10000), (20000, 150000)])
def test_chung_lu_is_simple_exact_and_seeded(n, m):
    rp, col = W.chung_lu(n, m, 2.1, seed=5)
    _check_simple(rp, col, n, m)
    rp2, col2 = W.chung_lu(n, m, 2.1, seed=5)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    rp3, _ = W.chung_lu(n, m, 2.1, seed=6)
    assert not np.array_equal(rp, rp3)
    # power-law skew: the heaviest out-degree is a few percent of n, far above the mean
    outdeg = np.diff(rp)
    assert outdeg.max() > 20 * outdeg.mean()
    assert outdeg.max() < 0.2 * n


def test_rmat_is_simple_exact_seeded_and_skewed():
    rp, col = W.rmat(14, 1 << 17, W.RMAT_ABCD, seed=9)
    n, m = 1 << 14, 1 << 17
    _check_simple(rp, col, n, m)
    rp2, col2 = W.rmat(14, 1 << 17, W.RMAT_ABCD, seed=9)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    outdeg = np.diff(rp)
    indeg = np.bincount(col, minlength=n)
    # (0.57, 0.19, 0.19, 0.05): heavy hubs on both sides, many isolated or low-degree vertices
    assert outdeg.max() > 50 * outdeg.mean() and indeg.max() > 50 * indeg.mean()
    assert (outdeg == 0).mean() > 0.2
    # the relabelling spreads the hubs over the id range (raw R-MAT puts them at low ids)
    top = np.argsort(outdeg)[-32:]
    assert top.mean() > n / 8


def test_weighted_cascade_thresholds():
    rp, col = W.chung_lu(3000, 12000, 2.1, seed=2)
    thr = W.wc_thresholds(col, 3000)
    indeg = np.bincount(col, minlength=3000)
    for e in range(0, len(col), 97):
        d = int(indeg[col[e]])
        t = int(thr[e])
        # the smallest multiple of 2^-32 that is >= 1/d: keep probability (t+1)/2^32
        assert (t + 1) * d >= 2 ** 32 > t * d
    assert np.all(thr[indeg[col] == 1] == 0xFFFFFFFF)  # p = 1 is always live


def test_trivalency_thresholds():
    thr = W.tr_thresholds(30000, seed=4)
    allowed = {W.threshold_of(Fraction(1, 10)), W.threshold_of(Fraction(1, 100)),
               W.threshold_of(Fraction(1, 1000))}
    assert set(np.unique(thr).tolist()) == allowed
    counts = np.array([(thr == t).sum() for t in sorted(allowed)])
    assert np.all(np.abs(counts - 10000) < 5 * np.sqrt(10000 * 2 / 9))  # uniform over the three


def test_seed_sets_and_keys():
    s = W.uniform_seeds(1000, 50, 3)
    assert len(set(s.tolist())) == 50 and s.min() >= 0 and s.max() < 1000
    assert np.array_equal(s, W.uniform_seeds(1000, 50, 3))
    assert W.query_key(11) == W.query_key(11) != W.query_key(12)
    assert 0 <= W.query_key(11) < 2 ** 64
    with pytest.raises(ValueError):
        W.uniform_seeds(10, 11, 0)
