"""Independent oracle evaluations spread over the host's cores.

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle/``: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may use it.

The oracle itself stays single-threaded and unchanged.  Ciphertexts are
independent (every EQ of Eq. 3 is a chain of 16 squarings on one ciphertext,
Sec. 4.3.1), so a sample of them can be checked in separate processes, each
holding its own ``Oracle`` keyed from the same seed: key generation is a
deterministic function of the seed (Philox draws), so every worker holds the
same keys as the caller.  Workers are started with ``spawn``: a pool created
after the calling process has initialised CUDA must not be forked.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

_worker_oracle = None


def _init(logn: int, key_seed: int, dp: int, coarse_from: int) -> None:
    global _worker_oracle
    from oracle import Oracle

    _worker_oracle = Oracle(logn, dp=dp, coarse_from=coarse_from)
    _worker_oracle.keygen(key_seed)


def _eq_one(job):
    x, y, const_val = job
    return _worker_oracle.eq(x, y, const_val=const_val)


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # platforms without affinity masks
        return os.cpu_count() or 1


def eq_many(logn: int, key_seed: int, xs, ys=None, const_val: int = 0, workers: int | None = None, dp: int = 3,
            coarse_from: int = 0):
    """The oracle's EQ (Eq. 3: 1 - (x - y)^(p-1), or against the constant
    ``const_val`` when ``ys`` is None) of each ciphertext ``xs[i]`` (uint64
    [2][L][N]), with the default parameters at ring degree 2^logn, key-switching
    digits of ``dp`` primes (the two-digit key from depth ``coarse_from`` on, 0 =
    never) and the keys of ``keygen(key_seed)``.  Returns the list of result ciphertexts, in the
    order of ``xs``.  ``workers`` defaults to min(len(xs), host cores)."""
    n = len(xs)
    if ys is not None and len(ys) != n:
        raise ValueError("xs and ys differ in length")
    if n == 0:
        return []
    jobs = [(np.ascontiguousarray(xs[i], dtype=np.uint64),
             None if ys is None else np.ascontiguousarray(ys[i], dtype=np.uint64), int(const_val))
            for i in range(n)]
    workers = max(1, min(n, workers or host_cores()))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                             initializer=_init, initargs=(logn, key_seed, dp, coarse_from)) as ex:
        return list(ex.map(_eq_one, jobs))
