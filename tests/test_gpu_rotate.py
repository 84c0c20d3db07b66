"""GPU parity of rotations and the rotate-and-add reduction behind COUNT and
SUM (Sec. 4.2.2): Galois keys bit for bit against the oracle's, reductions of
fresh ciphertexts, of EQ masks (COUNT) and of SELECT products (SUM, Eq. 5)
against the oracle's reduction and the closed forms; groups of ciphertexts
with a ragged last group over tiles of 2 with a ragged tail; in-place use;
error cases."""
import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp

pytestmark = pytest.mark.gpu
T = 65537
LOGN = 12
SEED_KEY, SEED_GK = 91, 92


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available()
    build.build()
    ctx = hp.Context(LOGN, max_tile_ct=2)
    ctx.keygen(SEED_KEY)
    gk = ctx.galois_keygen(SEED_GK, keep=True)
    o = oracle.Oracle(LOGN)
    o.keygen(SEED_KEY)
    ogk = [o.galois_keygen(SEED_GK, g) for g in o.galois_elements()]
    yield ctx, o, gk, ogk
    ctx.close()


def test_galois_keys_match_oracle(env):
    ctx, o, gk, ogk = env
    assert hp.galois_elements(LOGN) == o.galois_elements()
    for st in range(LOGN):
        assert np.array_equal(hp.to_u64(gk[st]), ogk[st]), st


def test_rotate_sum_fresh_matches_oracle(env):
    ctx, o, _, _ = env
    N = ctx.N
    rng = np.random.default_rng(93)
    x = rng.integers(0, 16, 3 * N).astype(np.uint32)  # per-ciphertext sums < t
    cx = ctx.encrypt(x.reshape(3, N), seed=94)
    got = ctx.rotate_sum(cx)
    ctx.check_status()
    assert ctx.launch_count() > 0
    dec = ctx.decrypt(got)
    for c in range(3):
        assert np.all(dec[c] == int(x[c * N:(c + 1) * N].sum()))
    for c in (0, 2):
        assert np.array_equal(hp.to_u64(got[c]), o.rotate_sum(hp.to_u64(cx[c]))), c


def test_groups_over_ragged_tiles(env):
    """5 ciphertexts in groups of 2: outputs {0,1}, {2,3}, {4}; tiles of 2 leave a tail of 1."""
    ctx, o, _, _ = env
    N = ctx.N
    rng = np.random.default_rng(95)
    x = rng.integers(0, T, 5 * N).astype(np.uint32)
    cx = ctx.encrypt(x.reshape(5, N), seed=96)
    got = ctx.rotate_sum(cx, group=2)
    assert got.shape[0] == 3
    dec = ctx.decrypt(got)
    ox = hp.to_u64(cx)
    for k, (c0, c1) in enumerate([(0, 2), (2, 4), (4, 5)]):
        assert np.all(dec[k] == int(x[c0 * N:c1 * N].astype(np.int64).sum() % T)), k
        ref = o.rotate_sum(o.linear(ox[c0:c1], [1] * (c1 - c0)))
        assert np.array_equal(hp.to_u64(got[k]), ref), k


def test_ct_sum_matches_oracle(env):
    ctx, o, _, _ = env
    N = ctx.N
    rng = np.random.default_rng(103)
    x = rng.integers(0, T, 3 * N).astype(np.uint32)
    cx = ctx.encrypt(x.reshape(3, N), seed=104)
    got = ctx.ct_sum(cx, group=2)
    ox = hp.to_u64(cx)
    assert np.array_equal(hp.to_u64(got[0]), o.linear(ox[:2], [1, 1]))
    assert np.array_equal(hp.to_u64(got[1]), ox[2])
    assert np.array_equal(ctx.decrypt(got[0:1])[0], ((x[:N].astype(np.int64) + x[N:2 * N]) % T).astype(np.uint32))


def test_in_place_equals_out_of_place(env):
    ctx, _, _, _ = env
    N = ctx.N
    rng = np.random.default_rng(97)
    cx = ctx.encrypt(rng.integers(0, T, 3 * N).astype(np.uint32).reshape(3, N), seed=98)
    ref = ctx.rotate_sum(cx)
    ctx.rotate_sum(cx, out=cx)
    assert np.array_equal(hp.to_u64(cx), hp.to_u64(ref))


def test_count_and_sum_queries(env):
    """COUNT(*) WHERE key = 2 and SUM(price) WHERE key = 2 over 3 ciphertexts."""
    ctx, o, _, _ = env
    N, n_ct, cval = ctx.N, 3, 2
    rng = np.random.default_rng(99)
    key = rng.integers(0, 4, n_ct * N).astype(np.uint32)
    price = rng.integers(0, 1000, n_ct * N).astype(np.uint32)
    ck = ctx.encrypt(key.reshape(n_ct, N), seed=100)
    cp = ctx.encrypt(price.reshape(n_ct, N), seed=100, ct_index0=n_ct)
    mask = ctx.eq(ck, None, const_val=cval)
    count = ctx.rotate_sum(mask, group=n_ct)
    assert np.all(ctx.decrypt(count) == int((key == cval).sum()))
    sel = ctx.run(hp.HP_SELECT, ck, cp, cval)
    total = ctx.rotate_sum(sel, group=n_ct)
    assert np.all(ctx.decrypt(total) == int(price[key == cval].astype(np.int64).sum() % T))
    # bit for bit: COUNT of ciphertext 1 alone and SUM of ciphertext 0 alone
    om = o.eq(hp.to_u64(ck[1]), None, const_val=cval)
    assert np.array_equal(hp.to_u64(mask[1]), om)
    assert np.array_equal(hp.to_u64(ctx.rotate_sum(mask[1:2])[0]), o.rotate_sum(om))
    assert np.array_equal(hp.to_u64(ctx.rotate_sum(sel[0:1])[0]), o.rotate_sum(hp.to_u64(sel[0])))


def test_set_galois_keys_and_errors(env):
    ctx, _, gk, _ = env
    N = ctx.N
    rng = np.random.default_rng(101)
    cx = ctx.encrypt(rng.integers(0, T, 2 * N).astype(np.uint32).reshape(2, N), seed=102)
    ref = ctx.rotate_sum(cx)
    other = hp.Context(LOGN, max_tile_ct=2)
    try:
        other.keygen(SEED_KEY)
        with pytest.raises(hp.HpError) as e:  # no Galois keys yet
            other.rotate_sum(cx)
        assert e.value.code == hp.HP_ERR_STATE
        other.set_galois_keys(gk)
        assert np.array_equal(hp.to_u64(other.rotate_sum(cx)), hp.to_u64(ref))
    finally:
        other.close()
    with pytest.raises(hp.HpError) as e:
        ctx.rotate_sum(cx, group=0)
    assert e.value.code == hp.HP_ERR_ARG
    big = ctx.ct_empty(4)
    with pytest.raises(hp.HpError) as e:  # overlapping output with group > 1
        ctx.rotate_sum(big, group=2, out=big[1:3])
    assert e.value.code == hp.HP_ERR_ARG
