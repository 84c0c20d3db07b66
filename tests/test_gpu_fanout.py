"""GPU parity of the fan-out of one column against many constants
(hp_eq_fanout): GROUP BY masks EQ(x, c_k) (Sec. 4.2.2) and IN(x, S) (Eq. 6).
Tiles of 4 over 15 chains leave a ragged tail and make tiles that start and end
in the middle of a constant's run.  Masks are compared bit for bit with
hp_run's constant form and with the oracle; the IN sums with the oracle's
linear combination; everything decrypts to the closed forms."""
import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp

pytestmark = pytest.mark.gpu
T = 65537
LOGN = 12
SEED_KEY = 77


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available()
    build.build()
    ctx = hp.Context(LOGN, max_tile_ct=4)
    ctx.keygen(SEED_KEY)
    o = oracle.Oracle(LOGN)
    o.keygen(SEED_KEY)
    yield ctx, o
    ctx.close()


def column(ctx, n_ct, seed):
    rng = np.random.default_rng(seed)
    dictionary = np.array([0, 3, 17, 4242, T - 1, 60000], dtype=np.uint32)
    x = dictionary[rng.integers(0, len(dictionary), n_ct * ctx.N)]
    return x, ctx.encrypt(x.reshape(n_ct, ctx.N), seed=seed)


def test_group_by_masks_and_in(env):
    ctx, o = env
    N, n_ct = ctx.N, 3
    consts = [3, 4242, 0, 5, T - 1]  # 5 is absent from the column
    x, cx = column(ctx, n_ct, 81)
    masks, ins = ctx.eq_fanout(cx, consts)
    assert masks.shape == (len(consts), n_ct, 2, ctx.L, N)
    ctx.check_status()
    assert ctx.launch_count() > 0
    for k, c in enumerate(consts):
        ref = ctx.eq(cx, None, const_val=c)
        assert np.array_equal(hp.to_u64(masks[k]), hp.to_u64(ref)), k
        assert np.array_equal(ctx.decrypt(masks[k]).reshape(-1), (x == c).astype(np.uint32))
    assert np.array_equal(ctx.decrypt(ins).reshape(-1), np.isin(x, consts).astype(np.uint32))
    # oracle: all masks of ciphertext 2, then their sum
    ox = hp.to_u64(cx[2])
    om = o.group_by_masks(ox, consts)
    assert np.array_equal(hp.to_u64(masks[:, 2]), om)
    assert np.array_equal(hp.to_u64(ins[2]), o.in_set(ox, consts, masks=om))


def test_in_only_and_masks_only_agree(env):
    ctx, _ = env
    consts = [17, 60000, 3]
    _, cx = column(ctx, 2, 82)
    masks, ins = ctx.eq_fanout(cx, consts)
    m2, none = ctx.eq_fanout(cx, consts, in_set=False)
    assert none is None and np.array_equal(hp.to_u64(m2), hp.to_u64(masks))
    none, i2 = ctx.eq_fanout(cx, consts, masks=False)
    assert none is None and np.array_equal(hp.to_u64(i2), hp.to_u64(ins))


def test_single_constant_in_equals_eq(env):
    ctx, _ = env
    _, cx = column(ctx, 2, 83)
    _, ins = ctx.eq_fanout(cx, [17], masks=False)
    assert np.array_equal(hp.to_u64(ins), hp.to_u64(ctx.eq(cx, None, const_val=17)))


def test_fanout_errors_and_empty(env):
    ctx, _ = env
    cx = ctx.ct_empty(1)
    with pytest.raises(hp.HpError) as e:
        ctx.eq_fanout(cx, [T])
    assert e.value.code == hp.HP_ERR_ARG
    with pytest.raises(hp.HpError) as e:
        ctx.eq_fanout(cx, [1], masks=False, in_set=False)
    assert e.value.code == hp.HP_ERR_ARG
    m, i = ctx.eq_fanout(cx, [])
    assert m.shape[0] == 0 and ctx.launch_count() == 0
