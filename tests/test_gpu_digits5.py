"""Key switching with digits of five primes (ks_digit_primes = 5: three digits
instead of five) on the GPU against the oracle with the same grouping, at
N = 4096:

* the relinearisation key and the Galois keys are bit-identical to the
  oracle's;
* EQ (Eq. 3) over a tile of 2 and a ragged tail of 1 and its constant form are
  bit-exact, and [x == y] in every slot;
* SELECT (Eq. 5) on the EQ mask through hp_select_mask is bit-exact against the
  oracle's product at depth 17;
* the rotate-and-add reduction (COUNT / SUM) of a fresh ciphertext is
  bit-exact;
* LT (Eq. 4) matches the oracle's ciphertext through the SHA-256 that
  tests/golden/make_n4096_budgets.py --digits5 wrote, and BETWEEN gives
  [lo <= x <= hi] in every slot;
* the allocation-free squaring, which holds three-prime digits only, refuses
  the handle;
* with per-prime digits up to depth 2 and five-prime digits below, the
  per-prime key and an EQ chain are bit-exact against the oracle."""
import hashlib

import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp
from tests.conftest import read_golden_kv
from tests.golden.make_n4096_budgets import HI, LO, LOGN, SEED_ENC, SEED_KEY, lt_inputs

pytestmark = pytest.mark.gpu
DP = 5


def _digest(ct):
    return hashlib.sha256(np.ascontiguousarray(hp.to_u64(ct), dtype=np.uint64).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def env():
    import torch

    build.build()
    ctx = hp.Context(LOGN, max_tile_ct=2, ks_digit_primes=DP)
    _, rk = ctx.keygen(SEED_KEY)
    o = oracle.Oracle(LOGN, dp=DP)
    o.keygen(SEED_KEY)
    yield ctx, o, rk
    ctx.close()
    torch.cuda.empty_cache()


def test_keys_match_oracle(env):
    import torch

    ctx, o, rk = env
    torch.cuda.synchronize()
    assert ctx.D == 3 and rk.shape[0] == 3
    assert np.array_equal(hp.to_u64(rk), o.rk)
    gk = ctx.galois_keygen(SEED_KEY + 1, keep=True)
    torch.cuda.synchronize()
    for st, g in enumerate(o.galois_elements()):
        assert np.array_equal(hp.to_u64(gk[st]), o.galois_keygen(SEED_KEY + 1, g)), st


def test_eq_and_select_match_oracle(env):
    import torch

    ctx, o, _ = env
    N = ctx.N
    rng = np.random.default_rng(19)
    x = rng.integers(0, hp.T, (3, N)).astype(np.uint32)
    y = np.where(rng.random((3, N)) < 0.5, x, rng.integers(0, hp.T, (3, N))).astype(np.uint32)
    cx, cy = ctx.encrypt(x, seed=SEED_ENC), ctx.encrypt(y, seed=SEED_ENC, ct_index0=3)
    eq = ctx.run(hp.HP_EQ_CT_CT, cx, cy)
    eqc = ctx.run(hp.HP_EQ_CT_CONST, cx[:1], const_val=int(x[0, 7]))
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(eq), (x == y).astype(np.uint32))
    assert np.array_equal(ctx.decrypt(eqc)[0], (x[0] == x[0, 7]).astype(np.uint32))
    for c in (0, 2):
        assert np.array_equal(hp.to_u64(eq[c]), o.eq(hp.to_u64(cx[c]), hp.to_u64(cy[c]))), c
    assert np.array_equal(hp.to_u64(eqc[0]), o.eq(hp.to_u64(cx[0]), const_val=int(x[0, 7])))
    col = ctx.encrypt(y, seed=SEED_ENC + 1)
    p = hp.hp_params(LOGN, hp.L, ctx._q, ctx.P, ctx.t, 17, 0, DP)
    sel = ctx.select_mask(col, eq, mask_depth=16, mask_bits=hp.budget_estimate(p, hp.HP_BUDGET_EQ))
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(sel), np.where(x == y, y, 0).astype(np.uint32))
    assert np.array_equal(hp.to_u64(sel[2]), o.mul_relin(hp.to_u64(col[2]), hp.to_u64(eq[2]), 0, 16))
    # the allocation-free squaring holds three-prime digits only
    assert ctx.lib.hp_square_noalloc(ctx.h, cx.data_ptr(), sel.data_ptr(), None) == hp.HP_ERR_UNSUPPORTED


def test_rotate_sum_matches_oracle(env):
    import torch

    ctx, o, _ = env
    N = ctx.N
    ctx.galois_keygen(SEED_KEY)
    for g in o.galois_elements():
        o.galois_keygen(SEED_KEY, g)
    x = np.random.default_rng(21).integers(0, 16, N).astype(np.uint32)
    cx = ctx.encrypt(x.reshape(1, N), seed=SEED_ENC, ct_index0=9)
    got = ctx.rotate_sum(cx)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.all(ctx.decrypt(got)[0] == int(x.sum()))
    assert np.array_equal(hp.to_u64(got[0]), o.rotate_sum(hp.to_u64(cx[0])))


def test_lt_digest_and_between(env):
    import torch

    ctx, _, _ = env
    gold = read_golden_kv("digits5_n4096.txt")
    assert gold["ks_digit_primes"] == DP and gold["seed_key"] == SEED_KEY
    N = ctx.N
    x, y, _ = lt_inputs(N)
    cx = ctx.encrypt(x.reshape(1, N), seed=SEED_ENC, ct_index0=0)
    cy = ctx.encrypt(y.reshape(1, N), seed=SEED_ENC, ct_index0=1)
    lt = ctx.run(hp.HP_LT, cx, cy)
    bt = ctx.between(cx, LO, HI)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(lt)[0], (x < y).astype(np.uint32))
    assert _digest(lt[0]) == gold["lt_sha256"]
    assert np.array_equal(ctx.decrypt(bt)[0], ((x >= LO) & (x <= HI)).astype(np.uint32))


def test_per_prime_first_levels_with_five_prime_digits():
    """ks_fine_depth = 2 with five-prime digits below it: the per-prime key and
    an EQ chain (its first two squarings per-prime, the rest five-prime) are
    bit-exact against the oracle with the same rule."""
    import torch

    build.build()
    ctx = hp.Context(LOGN, max_tile_ct=1, ks_digit_primes=DP, ks_fine_depth=2)
    ctx.keygen(SEED_KEY)
    rk_fine = ctx.keygen_fine(SEED_KEY)
    o = oracle.Oracle(LOGN, dp=DP, fine_depth=2)
    o.keygen(SEED_KEY)
    torch.cuda.synchronize()
    assert np.array_equal(hp.to_u64(rk_fine), o.fine_key())
    N = ctx.N
    rng = np.random.default_rng(23)
    x = rng.integers(0, hp.T, (1, N)).astype(np.uint32)
    y = np.where(rng.random((1, N)) < 0.5, x, rng.integers(0, hp.T, (1, N))).astype(np.uint32)
    cx, cy = ctx.encrypt(x, seed=SEED_ENC), ctx.encrypt(y, seed=SEED_ENC, ct_index0=1)
    eq = ctx.run(hp.HP_EQ_CT_CT, cx, cy)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(eq), (x == y).astype(np.uint32))
    assert np.array_equal(hp.to_u64(eq[0]), o.eq(hp.to_u64(cx[0]), hp.to_u64(cy[0])))
    ctx.close()
