"""GPU parity of the batched form (hp_run_batched): uneven instances, packed
into shared ciphertexts or one group of ciphertexts each, graph-replayed tiles,
autotuned tile size — bit-exact against hp_run and the oracle, and against the
closed form per instance after decryption; with key-switching digits of three
and of five primes."""
import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp
from paper_2602_24271_b300.inputs import log_uniform_sizes

pytestmark = pytest.mark.gpu
T = 65537
LOGN = 12
SEED_KEY = 2024


@pytest.fixture(scope="module", params=[3, 5])
def ctx(request):
    import torch

    assert torch.cuda.is_available()
    build.build()
    c = hp.Context(LOGN, max_tile_ct=3, ks_digit_primes=request.param)
    c.keygen(SEED_KEY)
    yield c
    c.close()


@pytest.fixture(scope="module")
def orc(ctx):
    o = oracle.Oracle(LOGN, dp=ctx.ks_digit_primes)
    o.keygen(SEED_KEY)
    return o


def packed_layout(sizes, N):
    """Instances laid out back to back in one global slot space."""
    inst, off = [], 0
    for n in sizes:
        ct0, so = off // N, off % N
        nct = (so + int(n) + N - 1) // N
        inst.append((ct0, nct, so, int(n), 0, 0))
        off += int(n)
    return inst, (off + N - 1) // N


def test_batched_packed_ctct_matches_plain_and_closed_form(ctx):
    N = ctx.N
    sizes = log_uniform_sizes(14, seed=2, lo_log2=4, hi_log2=13)
    inst, n_ct = packed_layout(sizes, N)
    rng = np.random.default_rng(3)
    x = rng.integers(1, 1 << 15, n_ct * N).astype(np.uint32)
    y = np.where(rng.random(n_ct * N) < 0.5, x, rng.integers(1, 1 << 15, n_ct * N)).astype(np.uint32)
    cx = ctx.encrypt(x.reshape(n_ct, N), seed=60)
    cy = ctx.encrypt(y.reshape(n_ct, N), seed=60, ct_index0=n_ct)
    got = ctx.run_batched(hp.HP_EQ_CT_CT, inst, cx, cy)
    ref = ctx.eq(cx, cy)
    assert np.array_equal(hp.to_u64(got), hp.to_u64(ref))
    dec = ctx.decrypt(got).reshape(-1)
    for (ct0, nct, so, n, _, _) in inst:
        g0 = ct0 * N + so
        assert np.array_equal(dec[g0:g0 + n], (x[g0:g0 + n] == y[g0:g0 + n]).astype(np.uint32))
    assert ctx.launch_count() > 0
    ctx.check_status()


def test_batched_per_instance_ciphertexts(ctx):
    N = ctx.N
    sizes = [17, N, N + 5, 300, 2 * N]
    inst, c = [], 0
    for n in sizes:
        nct = (n + N - 1) // N
        inst.append((c, nct, 0, n, 0, 0))
        c += nct
    n_ct = c
    rng = np.random.default_rng(4)
    x = rng.integers(0, 1 << 16, n_ct * N).astype(np.uint32)
    y = np.where(rng.random(n_ct * N) < 0.5, x, rng.integers(0, 1 << 16, n_ct * N)).astype(np.uint32)
    cx = ctx.encrypt(x.reshape(n_ct, N), seed=61)
    cy = ctx.encrypt(y.reshape(n_ct, N), seed=61, ct_index0=n_ct)
    got = ctx.run_batched(hp.HP_EQ_CT_CT, inst, cx, cy)
    assert np.array_equal(hp.to_u64(got), hp.to_u64(ctx.eq(cx, cy)))


def test_batched_packed_const_matches_oracle(ctx, orc):
    N = ctx.N
    sizes = [100, 2000, 1500, 700, 900, 3000]  # the fourth instance crosses the first ciphertext boundary
    consts = [3, 7, 3, 0, 5, 9]
    inst, off = [], 0
    for n, cval in zip(sizes, consts):
        ct0, so = off // N, off % N
        inst.append((ct0, (so + n + N - 1) // N, so, n, 0, cval))
        off += n
    n_ct = (off + N - 1) // N
    rng = np.random.default_rng(5)
    x = rng.integers(0, 10, n_ct * N).astype(np.uint32)
    cx = ctx.encrypt(x.reshape(n_ct, N), seed=62)
    got = ctx.run_batched(hp.HP_EQ_CT_CONST, inst, cx, None)
    cslots = np.zeros(n_ct * N, dtype=np.uint32)
    for (ct0, nct, so, n, _, cval) in inst:
        g0 = ct0 * N + so
        cslots[g0:g0 + n] = cval
    dec = ctx.decrypt(got).reshape(-1)
    assert np.array_equal(dec, (x == cslots).astype(np.uint32))
    g = hp.to_u64(got)
    ox = hp.to_u64(cx)
    for c in range(n_ct):
        assert np.array_equal(g[c], orc.eq_plain(ox[c], cslots[c * N:(c + 1) * N]))


def test_batched_uniform_const_equals_broadcast_form(ctx):
    N = ctx.N
    rng = np.random.default_rng(6)
    x = rng.integers(0, 4, 2 * N).astype(np.uint32)
    cx = ctx.encrypt(x.reshape(2, N), seed=63)
    got = ctx.run_batched(hp.HP_EQ_CT_CONST, [(0, 2, 0, 2 * N, 0, 2)], cx, None)
    assert np.array_equal(hp.to_u64(got), hp.to_u64(ctx.eq(cx, None, const_val=2)))


def test_batched_descriptor_errors(ctx):
    N = ctx.N
    cx = ctx.ct_empty(2)
    with pytest.raises(hp.HpError) as e:  # ciphertext 1 uncovered
        ctx.run_batched(hp.HP_EQ_CT_CT, [(0, 1, 0, N, 0, 0)], cx, cx)
    assert e.value.code == hp.HP_ERR_ARG
    with pytest.raises(hp.HpError) as e:  # overlapping slot ranges
        ctx.run_batched(hp.HP_EQ_CT_CT, [(0, 2, 0, 100, 0, 0), (0, 2, 50, 100, 0, 0)], cx, cx)
    assert e.value.code == hp.HP_ERR_ARG
    with pytest.raises(hp.HpError) as e:  # outside the batch
        ctx.run_batched(hp.HP_EQ_CT_CT, [(0, 3, 0, 100, 0, 0)], cx, cx)
    assert e.value.code == hp.HP_ERR_ARG


def test_autotune_keeps_results_exact(ctx):
    N = ctx.N
    t = ctx.autotune()
    assert 1 <= t <= 3 and ctx.tile() == t
    rng = np.random.default_rng(7)
    x = rng.integers(0, 1 << 16, 5 * N).astype(np.uint32)
    cx = ctx.encrypt(x.reshape(5, N), seed=64)
    cy = ctx.encrypt(x.reshape(5, N), seed=64, ct_index0=5)
    got = ctx.run_batched(hp.HP_EQ_CT_CT, [(0, 5, 0, 5 * N, 0, 0)], cx, cy)
    assert np.all(ctx.decrypt(got) == 1)
    assert np.array_equal(hp.to_u64(got), hp.to_u64(ctx.eq(cx, cy)))
