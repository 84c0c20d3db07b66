"""GPU parity: the CUDA path through the C ABI against the oracle, bit-exact
(integer work), at N = 4096 (several NTT tiles per polynomial, ragged
ciphertext tiles) — plus decrypted closed forms."""
import math

import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp
from paper_2602_24271_b300.inputs import eq_pair_columns

pytestmark = pytest.mark.gpu
T = 65537
SEED_KEY = 2024
LOGN = 12


@pytest.fixture(scope="module")
def ctx():
    import torch

    assert torch.cuda.is_available()
    build.build()
    c = hp.Context(LOGN, max_tile_ct=3)
    c.keygen(SEED_KEY)
    yield c
    c.close()


@pytest.fixture(scope="module")
def orc():
    o = oracle.Oracle(LOGN)
    o.keygen(SEED_KEY)
    return o


def u64(t):
    return hp.to_u64(t)


def dev(a):
    return hp.from_u64(a)


def edge_ct(o, seed=0):
    """A ciphertext-shaped array whose c0 coefficients sit at the centring
    boundary (Q - 1)/2, (Q + 1)/2 and 0, Q - 1 (exercise the exact fallback of
    the lift), c1 random."""
    Q = math.prod(o.q)
    rng = np.random.default_rng(seed)
    ct = np.zeros((2, o.L, o.N), dtype=np.uint64)
    vals = [(Q - 1) // 2, (Q + 1) // 2, 0, Q - 1, (Q - 3) // 2, (Q + 3) // 2]
    for k in range(o.N):
        v = vals[k % len(vals)] if k % 3 == 0 else int(rng.integers(0, 2**62)) * int(rng.integers(0, 2**62)) % Q
        for i, qi in enumerate(o.q):
            ct[0, i, k] = v % qi
    for i, qi in enumerate(o.q):
        ct[1, i, :] = rng.integers(0, qi, o.N, dtype=np.uint64)
    return ct


def test_keygen_parity(ctx, orc):
    sk = ctx.sk.cpu().numpy()
    assert np.array_equal(sk, orc.s)
    _, rk = ctx.keygen(SEED_KEY)
    assert np.array_equal(u64(rk), orc.rk)


def test_encrypt_decrypt_parity(ctx, orc):
    x, y = eq_pair_columns(2 * ctx.N, seed=1)
    slots = x.reshape(2, ctx.N)
    ct = ctx.encrypt(slots, seed=10, ct_index0=0)
    for c in range(2):
        assert np.array_equal(u64(ct[c]), orc.encrypt(slots[c], 10, c))
    assert np.array_equal(ctx.decrypt(ct), slots)
    # GPU decrypts oracle ciphertexts
    oc = orc.encrypt(y[: ctx.N], 77, 5)
    assert np.array_equal(ctx.decrypt(dev(oc[None]))[0], y[: ctx.N])


def test_square_parity(ctx, orc):
    rng = np.random.default_rng(3)
    a = orc.encrypt(rng.integers(0, T, ctx.N).astype(np.uint32), 11, 0)
    e = edge_ct(orc)
    for ct in (a, e):
        got = u64(ctx.run(hp.HP_SQUARE, dev(ct[None])))[0]
        assert np.array_equal(got, orc.mul_relin(ct, ct))
    ctx.check_status()


def test_eq_parity_config1(ctx, orc):
    x, y = eq_pair_columns(ctx.N, seed=0)
    # edge pairs: equal, +-1, +-(p-1)/2, 0 vs p-1
    edges = [(5, 5), (6, 5), (5, 6), (0, T - 1), (T - 1, 0), ((T - 1) // 2, 0), (0, (T - 1) // 2), (1, 0)]
    for i, (a, b) in enumerate(edges):
        x[i], y[i] = a, b
    cx, cy = orc.encrypt(x, 20, 0), orc.encrypt(y, 20, 1)
    got = u64(ctx.eq(dev(cx[None]), dev(cy[None])))[0]
    ref = orc.eq(cx, cy)
    assert np.array_equal(got, ref)
    assert np.array_equal(orc.decrypt(got), (x == y).astype(np.uint32))
    ctx.check_status()


def test_eq_const_and_select_parity(ctx, orc):
    rng = np.random.default_rng(4)
    x = rng.integers(0, 8, ctx.N).astype(np.uint32)
    col = rng.integers(0, T, ctx.N).astype(np.uint32)
    cx, ccol = orc.encrypt(x, 30, 0), orc.encrypt(col, 30, 1)
    got = u64(ctx.eq(dev(cx[None]), None, const_val=3))[0]
    assert np.array_equal(got, orc.eq(cx, None, const_val=3))
    assert np.array_equal(orc.decrypt(got), (x == 3).astype(np.uint32))
    sel = u64(ctx.run(hp.HP_SELECT, dev(cx[None]), dev(ccol[None]), const_val=3))[0]
    mask = orc.eq(cx, None, const_val=3)
    assert np.array_equal(sel, orc.mul_relin(mask, ccol))
    assert np.array_equal(orc.decrypt(sel), np.where(x == 3, col, 0).astype(np.uint32))


def test_ragged_tiles_and_aliasing(ctx, orc):
    """5 ciphertexts through tiles of 3 (3 + 2); output aliases the input."""
    n = 5
    x, y = eq_pair_columns(n * ctx.N, seed=7)
    xs, ys = x.reshape(n, ctx.N), y.reshape(n, ctx.N)
    cx = ctx.encrypt(xs, seed=40, ct_index0=0)
    cy = ctx.encrypt(ys, seed=40, ct_index0=n)
    ox = u64(cx)
    oy = u64(cy)
    ctx.eq(cx, cy, out=cx)  # in place
    got = u64(cx)
    assert np.array_equal(ctx.decrypt(cx), (xs == ys).astype(np.uint32))
    for c in (0, 3, 4):  # one per tile plus the ragged tail
        assert np.array_equal(got[c], orc.eq(ox[c], oy[c]))


def test_host_pointer_path_matches_device(ctx):
    n = 4
    x, y = eq_pair_columns(n * ctx.N, seed=8)
    cx = ctx.encrypt(x.reshape(n, ctx.N), seed=50)
    cy = ctx.encrypt(y.reshape(n, ctx.N), seed=50, ct_index0=n)
    dres = u64(ctx.eq(cx, cy))
    hx, hy = u64(cx), u64(cy)
    hres = np.empty_like(hx)
    ctx.run(hp.HP_EQ_CT_CT, hx, hy, 0, out=hres)
    assert np.array_equal(hres, dres)


def test_argument_errors(ctx):
    import torch

    cx = ctx.ct_empty(1)
    ctx.run(hp.HP_EQ_CT_CT, cx[:0], cx[:0])  # n = 0: no-op
    with pytest.raises(hp.HpError) as e:
        ctx.run(hp.HP_EQ_CT_CONST, cx, None, const_val=T)
    assert e.value.code == hp.HP_ERR_ARG
    with pytest.raises(hp.HpError) as e:
        ctx.run(hp.HP_EQ_CT_CT, cx, None)
    assert e.value.code == hp.HP_ERR_ARG
    with pytest.raises(hp.HpError) as e:
        ctx.run(7, cx, cx)
    assert e.value.code == hp.HP_ERR_ARG
    fresh = hp.Context(LOGN, max_tile_ct=1)
    with pytest.raises(hp.HpError) as e:
        fresh.run(hp.HP_EQ_CT_CT, cx, cx)
    assert e.value.code == hp.HP_ERR_STATE
    fresh.close()
    assert ctx.backward(hp.HP_EQ_CT_CT, cx, cx, 1) == hp.HP_ERR_UNSUPPORTED
    torch.cuda.synchronize()
