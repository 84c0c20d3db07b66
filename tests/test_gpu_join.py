"""GPU parity of Extract + Broadcast and the equi-join built on it (Sec.
4.2.2): broadcasts of single rows and of row ranges that cross a ciphertext
boundary over tiles of 3 with a ragged tail, bit for bit against the oracle;
key-foreign-key joins with two attributes and the semi-join against the closed
forms; a small join bit for bit against the oracle's composition; errors."""
import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp

pytestmark = pytest.mark.gpu
T = 65537
LOGN = 12
SEED_KEY, SEED_GK = 111, 112


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available()
    build.build()
    ctx = hp.Context(LOGN, max_tile_ct=3)
    ctx.keygen(SEED_KEY)
    ctx.galois_keygen(SEED_GK)
    o = oracle.Oracle(LOGN)
    o.keygen(SEED_KEY)
    for g in o.galois_elements():
        o.galois_keygen(SEED_GK, g)
    yield ctx, o
    ctx.close()


def test_extract_broadcast_matches_oracle(env):
    ctx, o = env
    N = ctx.N
    rng = np.random.default_rng(113)
    x = rng.integers(0, T, 2 * N).astype(np.uint32)
    col = ctx.encrypt(x.reshape(2, N), seed=114)
    ocol = hp.to_u64(col)
    for r in (5, N + 7):
        got = ctx.extract_broadcast(col, r)
        ctx.check_status()
        assert np.all(ctx.decrypt(got) == x[r])
        assert np.array_equal(hp.to_u64(got[0]), o.extract_broadcast(ocol, r)), r
    rng_rows = ctx.extract_broadcast(col, N - 2, n_rows=4)  # crosses into the second ciphertext
    dec = ctx.decrypt(rng_rows)
    for k in range(4):
        assert np.all(dec[k] == x[N - 2 + k])
    assert np.array_equal(hp.to_u64(rng_rows[3]), hp.to_u64(ctx.extract_broadcast(col, N + 1)[0]))


def join_tables(N, rng):
    bkey = np.zeros(N, dtype=np.uint32)
    bkey[:5] = [3, 99, 4242, 60000, T - 1]
    size = np.zeros(N, dtype=np.uint32)
    size[:5] = [10, 20, 30, 40, 50]
    brand = np.zeros(N, dtype=np.uint32)
    brand[:5] = [7, 8, 9, 1000, 65000]
    akey = rng.choice([3, 99, 4242, 60000, T - 1, 5, 6], 2 * N).astype(np.uint32)
    return bkey, size, brand, akey


def test_join_closed_form(env):
    ctx, _ = env
    N = ctx.N
    bkey, size, brand, akey = join_tables(N, np.random.default_rng(115))
    ca = ctx.encrypt(akey.reshape(2, N), seed=116)
    cb = ctx.encrypt(bkey.reshape(1, N), seed=116, ct_index0=2)
    cs = ctx.encrypt(size.reshape(1, N), seed=116, ct_index0=3)
    cbr = ctx.encrypt(brand.reshape(1, N), seed=116, ct_index0=4)
    out = ctx.join(ca, cb, [cs, cbr], 5)
    ctx.check_status()
    assert out.shape[:2] == (2, 2) and ctx.launch_count() > 0
    for k, attr in enumerate((size, brand)):
        ref = np.zeros(2 * N, dtype=np.uint32)
        for r in range(5):
            ref[akey == bkey[r]] = attr[r]
        assert np.array_equal(ctx.decrypt(out[k]).reshape(-1), ref), k
    semi = ctx.join(ca, cb, [], 5)
    assert semi.shape[0] == 1
    assert np.array_equal(ctx.decrypt(semi[0]).reshape(-1), np.isin(akey, bkey[:5]).astype(np.uint32))


def test_join_matches_oracle(env):
    ctx, o = env
    N = ctx.N
    bkey, size, _, akey = join_tables(N, np.random.default_rng(117))
    ca = ctx.encrypt(akey[:N].reshape(1, N), seed=118)
    cb = ctx.encrypt(bkey.reshape(1, N), seed=118, ct_index0=1)
    cs = ctx.encrypt(size.reshape(1, N), seed=118, ct_index0=2)
    got = ctx.join(ca, cb, [cs], 2)
    ref = o.join(hp.to_u64(ca), hp.to_u64(cb), [hp.to_u64(cs)], 2)
    assert np.array_equal(hp.to_u64(got), ref)


def test_join_errors(env):
    ctx, _ = env
    N = ctx.N
    c = ctx.encrypt(np.zeros((1, N), dtype=np.uint32), seed=119)
    with pytest.raises(hp.HpError) as e:
        ctx.join(c, c, [], 0)
    assert e.value.code == hp.HP_ERR_ARG
    with pytest.raises(hp.HpError) as e:
        ctx.extract_broadcast(c, N)  # row beyond the column
    assert e.value.code == hp.HP_ERR_ARG
    other = hp.Context(LOGN, max_tile_ct=2)
    try:
        other.keygen(SEED_KEY)
        with pytest.raises(hp.HpError) as e:
            other.join(c, c, [], 1)
        assert e.value.code == hp.HP_ERR_STATE
    finally:
        other.close()
