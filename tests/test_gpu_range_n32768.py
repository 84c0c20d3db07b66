"""Range filter then aggregate at the paper's ring degree N = 32768 (Sec. 5.1),
the shape of TPC-H Q6 (Table 5: the filter, then SUM):

    mask = BETWEEN(x, lo, hi)   (Sec. 4.2.2: (1 - LT(x, lo)) (1 - LT(hi, x)), Eq. 4)
    sel  = col * mask           (SELECT, Eq. 5, through hp_select_mask)
    agg  = rotate-and-add(sel)  (SUM, Sec. 4.2.2)

with per-prime relinearisation up to depth 0 (three-prime key switching
throughout) and 3, and with the benchmark's key switching for LT and BETWEEN
(per-prime digits up to depth 4, five-prime digits, the two-digit key from
depth 10).  Every slot of every result is checked against its closed
form after GPU decryption ([lo <= x <= hi], col where selected, the column's
sum in every slot), and each ciphertext bit for bit against the oracle's
through the SHA-256 that tests/golden/make_range_n32768.py wrote from the
oracle; LT(x, y) on its own likewise.  The library's budget estimate of each
result lies below the budget the oracle measured in it."""
import hashlib

import numpy as np
import pytest

from paper_2602_24271_b300 import build, hp
from tests.conftest import read_golden_kv
from tests.golden.make_range_n32768 import (CT_COL, CT_X, CT_Y, HI, LO, LOGN, MASK_DEPTH, SEED_ENC, SEED_KEY,
                                            range_inputs)

pytestmark = pytest.mark.gpu


def _digest(ct):
    return hashlib.sha256(np.ascontiguousarray(hp.to_u64(ct), dtype=np.uint64).tobytes()).hexdigest()


SCHEDULES = [(0, 3, 0), (3, 3, 0), (4, 5, 10)]  # (per-prime up to, digit primes, two-digit key from)


def _golden(kind, F, dp, cf):
    sfx = ("_d%d" % dp if dp != 3 else "") + ("_c%d" % cf if cf else "")
    if kind == "lt":
        return read_golden_kv("lt_n32768%s.txt" % (("_f%d" % F if F else "") + sfx))
    return read_golden_kv("range_n32768_f%d%s.txt" % (F, sfx))


@pytest.mark.parametrize("fine_depth, dp, cf", SCHEDULES)
def test_between_select_sum_n32768(fine_depth, dp, cf):
    import torch

    build.build()
    gold = _golden("range", fine_depth, dp, cf)
    assert gold["lo"] == LO and gold["hi"] == HI and gold["seed_key"] == SEED_KEY
    assert gold.get("ks_digit_primes", 3) == dp and gold.get("ks_coarse_from", 0) == cf
    ctx = hp.Context(LOGN, max_tile_ct=1, ks_fine_depth=fine_depth, ks_digit_primes=dp, ks_coarse_from=cf)
    ctx.keygen(SEED_KEY)
    ctx.galois_keygen(SEED_KEY)
    N = ctx.N
    x, _, col = range_inputs(N)
    cx = ctx.encrypt(x.reshape(1, N), seed=SEED_ENC, ct_index0=CT_X)
    cc = ctx.encrypt(col.reshape(1, N), seed=SEED_ENC, ct_index0=CT_COL)
    prm = ctx.params()
    bits_between = hp.budget_estimate(prm, hp.HP_BUDGET_BETWEEN)
    mask = ctx.between(cx, LO, HI)
    sel = ctx.select_mask(cc, mask, mask_depth=MASK_DEPTH, mask_bits=bits_between)
    agg = ctx.rotate_sum(sel)
    torch.cuda.synchronize()
    ctx.check_status()
    rows = (x >= LO) & (x <= HI)
    assert np.array_equal(ctx.decrypt(mask)[0], rows.astype(np.uint32))
    assert np.array_equal(ctx.decrypt(sel)[0], np.where(rows, col, 0).astype(np.uint32))
    total = int(col[rows].astype(np.int64).sum() % 65537)
    assert total == gold["sum_value"]
    assert np.all(ctx.decrypt(agg)[0] == total)
    assert _digest(mask[0]) == gold["between_sha256"]
    assert _digest(sel[0]) == gold["select_sha256"]
    assert _digest(agg[0]) == gold["sum_sha256"]
    # the static estimates lie below what the oracle measured in these results
    bits_sel = hp.budget_estimate(prm, hp.HP_BUDGET_PRODUCT, MASK_DEPTH, bits_between)
    bits_sum = hp.budget_estimate(prm, hp.HP_BUDGET_ROTATE_SUM, 0, bits_sel)
    assert 0 < bits_between <= gold["between_budget_bits"]
    assert 0 < bits_sel <= gold["select_budget_bits"]
    assert 0 < bits_sum <= gold["sum_budget_bits"]
    ctx.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("fine_depth, dp, cf", [(0, 3, 0), (4, 5, 10)])
def test_lt_n32768(fine_depth, dp, cf):
    import torch

    build.build()
    gold = _golden("lt", fine_depth, dp, cf)
    assert gold["seed_key"] == SEED_KEY and gold["ks_fine_depth"] == fine_depth
    assert gold.get("ks_digit_primes", 3) == dp and gold.get("ks_coarse_from", 0) == cf
    ctx = hp.Context(LOGN, max_tile_ct=1, ks_fine_depth=fine_depth, ks_digit_primes=dp, ks_coarse_from=cf)
    ctx.keygen(SEED_KEY)
    N = ctx.N
    x, y, _ = range_inputs(N)
    cx = ctx.encrypt(x.reshape(1, N), seed=SEED_ENC, ct_index0=CT_X)
    cy = ctx.encrypt(y.reshape(1, N), seed=SEED_ENC, ct_index0=CT_Y)
    out = ctx.run(hp.HP_LT, cx, cy)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(out)[0], (x < y).astype(np.uint32))
    assert _digest(out[0]) == gold["lt_sha256"]
    assert hp.budget_estimate(ctx.params(), hp.HP_BUDGET_LT) <= gold["lt_budget_bits"]
    ctx.close()
    torch.cuda.empty_cache()
