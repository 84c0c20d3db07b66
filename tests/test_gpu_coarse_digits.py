"""Key switching with the two-digit key (digits [d2] mod q_0..q_7 and mod
q_8..q_14) for the products at depth ks_coarse_from and beyond, on the GPU
against the oracle with the same rule, at N = 4096, in the benchmark's two
configurations -- five-prime digits with the two-digit key from depth 7 (the
EQ workloads); per-prime digits up to depth 4, five-prime digits, the
two-digit key from depth 10 (LT and BETWEEN) -- and with three-prime digits
below the two-digit key:

* the two-digit key is bit-identical to the oracle's;
* EQ (Eq. 3) over a tile of 2 and a ragged tail of 1 is bit-exact, and
  [x == y] in every slot;
* SELECT (Eq. 5) on the EQ mask (a product at depth 17) is bit-exact;
* LT (Eq. 4) matches the oracle's ciphertext through the SHA-256 that
  tests/golden/make_n4096_budgets.py --coarse wrote, and BETWEEN gives
  [lo <= x <= hi] in every slot;
* with per-prime digits up to depth 2 as well, an EQ chain is bit-exact;
* the allocation-free squaring refuses such a handle."""
import hashlib

import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp
from tests.conftest import read_golden_kv
from tests.golden.make_n4096_budgets import HI, LO, LOGN, SEED_ENC, SEED_KEY, lt_inputs

pytestmark = pytest.mark.gpu


def _digest(ct):
    return hashlib.sha256(np.ascontiguousarray(hp.to_u64(ct), dtype=np.uint64).tobytes()).hexdigest()


@pytest.mark.parametrize("F, dp, cf", [(0, 5, 7), (4, 5, 10), (0, 3, 10)])
def test_two_digit_key_from_depth(F, dp, cf):
    import torch

    build.build()
    gold = read_golden_kv(("coarse_f%dd%dc%d_n4096.txt" % (F, dp, cf)) if F else ("coarse_d%dc%d_n4096.txt" % (dp, cf)))
    assert gold["ks_digit_primes"] == dp and gold["ks_coarse_from"] == cf and gold["seed_key"] == SEED_KEY
    assert gold.get("ks_fine_depth", 0) == F
    ctx = hp.Context(LOGN, max_tile_ct=2, ks_digit_primes=dp, ks_coarse_from=cf, ks_fine_depth=F)
    ctx.keygen(SEED_KEY)
    rk2 = ctx.keygen_coarse(SEED_KEY)
    o = oracle.Oracle(LOGN, dp=dp, coarse_from=cf, fine_depth=F)
    o.keygen(SEED_KEY)
    torch.cuda.synchronize()
    assert np.array_equal(hp.to_u64(rk2), o.coarse_key())
    N = ctx.N
    rng = np.random.default_rng(29)
    x = rng.integers(0, hp.T, (3, N)).astype(np.uint32)
    y = np.where(rng.random((3, N)) < 0.5, x, rng.integers(0, hp.T, (3, N))).astype(np.uint32)
    cx, cy = ctx.encrypt(x, seed=SEED_ENC), ctx.encrypt(y, seed=SEED_ENC, ct_index0=3)
    eq = ctx.run(hp.HP_EQ_CT_CT, cx, cy)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(eq), (x == y).astype(np.uint32))
    for c in (0, 2):
        assert np.array_equal(hp.to_u64(eq[c]), o.eq(hp.to_u64(cx[c]), hp.to_u64(cy[c]))), c
    # SELECT on the mask: a product at depth 17, relinearised with the two-digit key
    col = ctx.encrypt(y, seed=SEED_ENC + 1)
    sel = ctx.select_mask(col, eq, mask_depth=16, mask_bits=hp.budget_estimate(ctx.params(), hp.HP_BUDGET_EQ))
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(sel), np.where(x == y, y, 0).astype(np.uint32))
    assert np.array_equal(hp.to_u64(sel[1]), o.mul_relin(hp.to_u64(col[1]), hp.to_u64(eq[1]), 0, 16))
    # LT (products from depth 1 to 18) against the oracle's digest; BETWEEN's closed form
    xl, yl, _ = lt_inputs(N)
    cxl = ctx.encrypt(xl.reshape(1, N), seed=SEED_ENC, ct_index0=0)
    cyl = ctx.encrypt(yl.reshape(1, N), seed=SEED_ENC, ct_index0=1)
    lt = ctx.run(hp.HP_LT, cxl, cyl)
    bt = ctx.between(cxl, LO, HI)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(lt)[0], (xl < yl).astype(np.uint32))
    assert _digest(lt[0]) == gold["lt_sha256"]
    assert np.array_equal(ctx.decrypt(bt)[0], ((xl >= LO) & (xl <= HI)).astype(np.uint32))
    # the allocation-free squaring holds three-prime digits only
    assert ctx.lib.hp_square_noalloc(ctx.h, cx.data_ptr(), sel.data_ptr(), None) == hp.HP_ERR_UNSUPPORTED
    ctx.close()


def test_per_prime_then_five_prime_then_two_digit():
    """ks_fine_depth = 2, five-prime digits for depths 3..6, the two-digit key
    from depth 7: the three keys side by side, an EQ chain bit-exact."""
    import torch

    build.build()
    ctx = hp.Context(LOGN, max_tile_ct=1, ks_digit_primes=5, ks_fine_depth=2, ks_coarse_from=7)
    ctx.keygen(SEED_KEY)
    o = oracle.Oracle(LOGN, dp=5, fine_depth=2, coarse_from=7)
    o.keygen(SEED_KEY)
    N = ctx.N
    rng = np.random.default_rng(31)
    x = rng.integers(0, hp.T, (1, N)).astype(np.uint32)
    y = np.where(rng.random((1, N)) < 0.5, x, rng.integers(0, hp.T, (1, N))).astype(np.uint32)
    cx, cy = ctx.encrypt(x, seed=SEED_ENC), ctx.encrypt(y, seed=SEED_ENC, ct_index0=1)
    eq = ctx.run(hp.HP_EQ_CT_CT, cx, cy)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(eq), (x == y).astype(np.uint32))
    assert np.array_equal(hp.to_u64(eq[0]), o.eq(hp.to_u64(cx[0]), hp.to_u64(cy[0])))
    ctx.close()
