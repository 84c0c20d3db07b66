"""COUNT / SUM, IN and JOIN (Sec. 4.2.2, Eq. 6) at the paper's ring degree
N = 32768 (Sec. 5.1), with three-prime key-switching digits and with the
benchmark's key switching for these workloads.  Every slot of every result is checked against its closed
form after GPU decryption, and one ciphertext of each against the oracle bit for
bit through the SHA-256 digests that tests/golden/make_aggregates_n32768.py
(with --bench-grouping for the benchmark's key switching) wrote from the oracle:

* SUM over a 2^26-slot column (2048 ciphertexts summed, then reduced by
  rotate-and-add): the column's total mod p in every slot; the reduction of
  ciphertext 0 on its own against the oracle;
* IN against four constants over 64 ciphertexts: [x in S] in every slot;
  ciphertext 0 against the oracle;
* JOIN of 4 A ciphertexts with 3 B rows and one attribute: the matching B row's
  attribute or 0 in every slot; A ciphertext 0 against the oracle."""
import hashlib

import numpy as np
import pytest

from paper_2602_24271_b300 import build, hp
from tests.conftest import read_golden_kv
from tests.golden.make_aggregates_n32768 import (JOIN_ROWS, LOGN, N_A, N_COLUMN, N_IN, SEED_ENC, SEED_KEY, column,
                                                 in_constants, join_tables)

pytestmark = pytest.mark.gpu


def _digest(ct):
    return hashlib.sha256(np.ascontiguousarray(hp.to_u64(ct), dtype=np.uint64).tobytes()).hexdigest()


@pytest.fixture(scope="module", params=[(3, 0), (5, 7)], ids=["three-prime", "bench"])
def agg(request):
    """The handle with three-prime key-switching digits, and with the key
    switching the benchmark's aggregate workloads use (five-prime digits, the
    two-digit key from depth 7 on), each against the digests the oracle wrote
    with the same rule."""
    import torch

    build.build()
    dp, cf = request.param
    gold = read_golden_kv("aggregates_d5c7_n32768.txt" if cf else "aggregates_n32768.txt")
    assert gold["seed_key"] == SEED_KEY and gold["log_n"] == LOGN
    assert gold.get("ks_digit_primes", 3) == dp and gold.get("ks_coarse_from", 0) == cf
    ctx = hp.Context(LOGN, ks_digit_primes=dp, ks_coarse_from=cf)
    ctx.keygen(SEED_KEY)
    ctx.galois_keygen(SEED_KEY)
    ctx.autotune()
    yield ctx, gold
    ctx.close()
    torch.cuda.empty_cache()


def _encrypt(ctx, slots, n_ct, idx0):
    out = ctx.ct_empty(n_ct)
    for c0 in range(0, n_ct, 128):
        c1 = min(n_ct, c0 + 128)
        out[c0:c1] = ctx.encrypt(slots[c0 * ctx.N:c1 * ctx.N].reshape(-1, ctx.N), seed=SEED_ENC, ct_index0=idx0 + c0)
    return out


def test_sum_over_a_2_26_slot_column(agg):
    import torch

    ctx, gold = agg
    N = ctx.N
    x = column(N_COLUMN, N, 11)
    cx = _encrypt(ctx, x, N_COLUMN, 0)
    total = ctx.rotate_sum(cx, group=N_COLUMN)
    one = ctx.rotate_sum(cx[:1])
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.all(ctx.decrypt(total)[0] == int(x.astype(np.int64).sum() % 65537))
    assert np.all(ctx.decrypt(one)[0] == int(x[:N].astype(np.int64).sum() % 65537))
    assert _digest(one[0]) == gold["rotate_sum_sha256"]
    del cx
    torch.cuda.empty_cache()


def test_in_over_64_ciphertexts(agg):
    import torch

    ctx, gold = agg
    N = ctx.N
    x = column(N_IN, N, 12)
    consts = in_constants(x)
    cx = _encrypt(ctx, x, N_IN, 0)
    _, ins = ctx.eq_fanout(cx, consts, masks=False, in_set=True)
    torch.cuda.synchronize()
    ctx.check_status()
    assert np.array_equal(ctx.decrypt(ins).reshape(-1), np.isin(x, consts).astype(np.uint32))
    assert _digest(ins[0]) == gold["in_sha256"]


def test_join_of_4_a_ciphertexts_with_3_b_rows(agg):
    import torch

    ctx, gold = agg
    N = ctx.N
    akey, bkey, battr = join_tables(N)
    ca = _encrypt(ctx, akey, N_A, 100)
    cbk = ctx.encrypt(bkey.reshape(1, N), seed=SEED_ENC, ct_index0=200)
    cba = ctx.encrypt(battr.reshape(1, N), seed=SEED_ENC, ct_index0=201)
    out = ctx.join(ca, cbk, [cba], JOIN_ROWS)
    torch.cuda.synchronize()
    ctx.check_status()
    want = np.zeros(N_A * N, dtype=np.uint32)
    for r in range(JOIN_ROWS):
        want[akey == bkey[r]] = battr[r]
    assert np.array_equal(ctx.decrypt(out[0]).reshape(-1), want)
    assert _digest(out[0][0]) == gold["join_sha256"]
