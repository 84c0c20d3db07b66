"""LT comparison (Eq. 4) on the GPU: closed form [x < y] on every slot, edge
differences included, and the ciphertext bit for bit against the oracle, which
follows the same baby-step / giant-step schedule."""
import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp

pytestmark = pytest.mark.gpu
LOGN = 12
SEED_KEY = 2024
HALF = 32768


def test_lt_closed_form_and_oracle_parity():
    import torch

    build.build()
    ctx = hp.Context(LOGN, max_tile_ct=3)
    ctx.keygen(SEED_KEY)
    N, n = ctx.N, 4  # 4 ciphertexts: one LT tile of 3 plus a ragged tail of 1
    rng = np.random.default_rng(21)
    x = rng.integers(0, HALF + 1, n * N).astype(np.uint32)
    y = np.where(rng.random(n * N) < 0.3, x, rng.integers(0, HALF + 1, n * N)).astype(np.uint32)
    edges = [(5, 3), (3, 5), (0, HALF), (HALF, 0), (7, 7), (100, 101), (101, 100), (0, 0), (HALF, HALF)]
    for i, (a, b) in enumerate(edges):
        x[i], y[i] = a, b
    cx = ctx.encrypt(x.reshape(n, N), seed=70)
    cy = ctx.encrypt(y.reshape(n, N), seed=70, ct_index0=n)
    out = ctx.run(hp.HP_LT, cx, cy)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(out).reshape(-1), (x < y).astype(np.uint32))
    o = oracle.Oracle(LOGN)
    o.keygen(SEED_KEY)
    c = 3  # the ragged tail's ciphertext
    assert np.array_equal(hp.to_u64(out[c]), o.lt(hp.to_u64(cx[c]), hp.to_u64(cy[c])))
    ctx.close()
