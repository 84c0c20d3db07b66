"""Key switching with per-prime digits for the first levels (ks_fine_depth) on
the GPU against the oracle, at N = 4096:

* the per-prime relinearisation key (15 digits [d2]_{q_i}) is bit-identical to
  the oracle's;
* a squaring of a fresh ciphertext (depth 1) with ks_fine_depth = 1, the EQ
  chain (Eq. 3) with per-prime digits for its first two squarings, and LT
  (Eq. 4) with them up to depth 3 are bit-exact against the oracle, which
  applies the same rule (the LT ciphertext through the SHA-256 written by
  tests/golden/make_n4096_budgets.py);
* SELECT on an EQ mask through hp_select_mask is bit-exact against the oracle's
  product at depth 17, and a request whose estimated budget is below the
  margin is refused with HP_ERR_DEPTH before anything runs."""
import hashlib

import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp
from tests.conftest import read_golden_kv
from tests.golden.make_n4096_budgets import LOGN, SEED_ENC, SEED_KEY, lt_inputs

pytestmark = pytest.mark.gpu


def _digest(ct):
    return hashlib.sha256(np.ascontiguousarray(hp.to_u64(ct), dtype=np.uint64).tobytes()).hexdigest()


def test_fine_key_and_products_match_oracle():
    import torch

    build.build()
    F = 2
    ctx = hp.Context(LOGN, max_tile_ct=2, ks_fine_depth=F)
    ctx.keygen(SEED_KEY)
    o = oracle.Oracle(LOGN, fine_depth=F)
    o.keygen(SEED_KEY)
    # the installed keys: three-prime (returned by keygen) and per-prime
    rk_fine = ctx.keygen_fine(SEED_KEY)
    torch.cuda.synchronize()
    assert np.array_equal(hp.to_u64(rk_fine), o.fine_key())
    N = ctx.N
    rng = np.random.default_rng(9)
    x = rng.integers(0, hp.T, (3, N)).astype(np.uint32)
    y = np.where(rng.random((3, N)) < 0.5, x, rng.integers(0, hp.T, (3, N))).astype(np.uint32)
    cx, cy = ctx.encrypt(x, seed=SEED_ENC), ctx.encrypt(y, seed=SEED_ENC, ct_index0=3)
    # EQ over a tile of 2 and a ragged tail of 1; ciphertext 2 bit for bit
    eq = ctx.run(hp.HP_EQ_CT_CT, cx, cy)
    sq = ctx.run(hp.HP_SQUARE, cx[:1])
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(eq), (x == y).astype(np.uint32))
    hx2, hy2 = hp.to_u64(cx[2]), hp.to_u64(cy[2])
    assert np.array_equal(hp.to_u64(eq[2]), o.eq(hx2, hy2))
    hx0 = hp.to_u64(cx[0])
    assert np.array_equal(hp.to_u64(sq[0]), o.mul_relin(hx0, hx0))
    # SELECT on the EQ masks: column x mask (depth 17) against the oracle's product
    col = ctx.encrypt(y, seed=SEED_ENC + 1)
    p = hp.hp_params(LOGN, hp.L, ctx._q, ctx.P, ctx.t, 17, F)
    mask_bits = hp.budget_estimate(p, hp.HP_BUDGET_EQ)
    sel = ctx.select_mask(col, eq, mask_depth=16, mask_bits=mask_bits)
    torch.cuda.synchronize()
    assert np.array_equal(ctx.decrypt(sel), np.where(x == y, y, 0).astype(np.uint32))
    assert np.array_equal(hp.to_u64(sel[2]), o.mul_relin(hp.to_u64(col[2]), hp.to_u64(eq[2]), 0, 16))
    # a mask whose budget leaves too little after the product: refused, nothing launched
    with pytest.raises(hp.HpError) as e:
        ctx.select_mask(col, eq, mask_depth=16, mask_bits=30.0)
    assert e.value.code == hp.HP_ERR_DEPTH
    assert ctx.launch_count() == 0
    # the allocation-free squaring holds three-prime digits only
    assert ctx.lib.hp_square_noalloc(ctx.h, cx.data_ptr(), sq.data_ptr(), None) == hp.HP_ERR_UNSUPPORTED
    ctx.close()


def test_lt_with_fine_digits_matches_oracle_digest():
    import torch

    build.build()
    gold = read_golden_kv("fine_lt_n4096.txt")
    assert gold["ks_fine_depth"] == 3 and gold["seed_key"] == SEED_KEY
    ctx = hp.Context(LOGN, max_tile_ct=1, ks_fine_depth=3)
    ctx.keygen(SEED_KEY)
    N = ctx.N
    x, y, _ = lt_inputs(N)
    cx = ctx.encrypt(x.reshape(1, N), seed=SEED_ENC, ct_index0=0)
    cy = ctx.encrypt(y.reshape(1, N), seed=SEED_ENC, ct_index0=1)
    out = ctx.run(hp.HP_LT, cx, cy)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(out)[0], (x < y).astype(np.uint32))
    assert _digest(out[0]) == gold["sha256"]
    ctx.close()
