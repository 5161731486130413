"""The CPU oracle on all host cores, for full-size parity checks.

Alg. 2's counters and the simulated spread are integer sums over independent samples, so the
oracle's thread-parallel sample loop (oracle.set_threads) returns exactly what its sequential
loop returns; this module only picks the thread count (every core of the host) and runs the
oracle's own entry points with it.
"""
from __future__ import annotations

import os

from oracle import oracle as O


def workers() -> int:
    return max(1, os.cpu_count() or 1)


def decrease(g, seeds, blocked, theta, key, round_, nproc=None, j0=0, model="ic"):
    """Alg. 2 counters over samples [j0, j0 + theta) of call `round_`."""
    with O.threads(nproc or workers()):
        return O.decrease(g, seeds, blocked if blocked is not None else [], theta, key, round_, j0,
                          model=model)


def advanced_greedy(g, seeds, b, theta, key, nproc=None, model="ic"):
    """Alg. 3, every round on all host cores."""
    with O.threads(nproc or workers()):
        return O.advanced_greedy(g, seeds, b, theta, key, model=model)


def greedy_replace(g, seeds, b, theta, key, nproc=None, model="ic"):
    """Alg. 4, every round on all host cores."""
    with O.threads(nproc or workers()):
        return O.greedy_replace(g, seeds, b, theta, key, model=model)


def spread(g, seeds, blocked, theta, key, round_=0, nproc=None, model="ic"):
    with O.threads(nproc or workers()):
        return O.spread(g, seeds, blocked if blocked is not None else [], theta, key, round_,
                        model=model)
