"""Seeded synthetic plaintext columns for the equality predicate.

This module holds no arithmetic of the method: it only draws integer columns
shaped like the paper's workloads (16-bit integer columns, Sec. 5.4 "Memory and
Storage Efficiency"; dictionary IDs 1..|D|, Sec. 4.2.2 GROUP BY) with numpy's
seeded generator.  Both the CUDA path and the oracle-based tests consume its
output; neither side's randomness for keys and encryption comes from here.
"""
from __future__ import annotations

import numpy as np


def eq_pair_columns(n: int, seed: int, value_bits: int = 16, p_equal: float = 0.5):
    """Two uint32 columns (x, y) of length n: x uniform in [0, 2^value_bits),
    y = x with probability p_equal, else an independent draw."""
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 1 << value_bits, n, dtype=np.uint32)
    other = rng.integers(0, 1 << value_bits, n, dtype=np.uint32)
    y = np.where(rng.random(n) < p_equal, x, other).astype(np.uint32)
    return x, y


def dictionary_column(n: int, seed: int, n_ids: int = 1 << 15):
    """Dictionary-encoded column: IDs uniform in [1, n_ids]."""
    rng = np.random.default_rng(seed)
    return rng.integers(1, n_ids + 1, n, dtype=np.uint32)


def log_uniform_sizes(count: int, seed: int, lo_log2: int = 8, hi_log2: int = 16):
    """Instance sizes log-uniform in [2^lo_log2, 2^hi_log2] (uneven batched instances)."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(lo_log2, hi_log2, count)
    return np.minimum(np.floor(2.0 ** e).astype(np.int64), 1 << hi_log2)
