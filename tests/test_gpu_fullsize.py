"""Full-size parity at N = 32768 in the benchmark's launch configuration
(autotuned tiles, key-switching digits of five primes, the two-digit key from
depth 7 on): the plain workload
(2^26 slots = 2048 ciphertext pairs) and the constant form at 2^28 slots (8192
ciphertexts).  Every slot of every
result is checked against the closed form [x == y] after GPU decryption (whose
own parity with the oracle is tested at N = 4096 and again here on samples),
and 16 seeded sampled ciphertexts of each workload (the first and the last
among them) are compared with the oracle bit for bit; the oracle evaluates the
samples in parallel processes on the host's cores (one EQ at N = 32768 is
about half a minute of single-threaded oracle time)."""
import numpy as np
import pytest

import oracle
from oracle.parallel import eq_many
from paper_2602_24271_b300 import build, hp
from paper_2602_24271_b300.inputs import eq_pair_columns

pytestmark = pytest.mark.gpu
LOGN = 15
SEED_KEY = 1
N_SAMPLES = 16
DP, COARSE = 5, 7  # key switching as the benchmark's EQ workloads use it


def sample_indices(n_ct: int, seed: int):
    """N_SAMPLES distinct ciphertext indices: the first, the last and seeded
    uniform draws."""
    rng = np.random.default_rng(seed)
    idx = {0, n_ct - 1}
    while len(idx) < N_SAMPLES:
        idx.add(int(rng.integers(0, n_ct)))
    return sorted(idx)


@pytest.fixture(scope="module")
def big():
    import torch

    build.build()
    ctx = hp.Context(LOGN, ks_digit_primes=DP, ks_coarse_from=COARSE)
    ctx.keygen(SEED_KEY)
    ctx.autotune()
    o = oracle.Oracle(LOGN, dp=DP, coarse_from=COARSE)
    o.keygen(SEED_KEY)
    yield ctx, o
    ctx.close()
    torch.cuda.empty_cache()


def encrypt_chunked(ctx, slots, n_ct, seed, idx0):
    out = ctx.ct_empty(n_ct)
    for c0 in range(0, n_ct, 128):
        c1 = min(n_ct, c0 + 128)
        out[c0:c1] = ctx.encrypt(slots[c0 * ctx.N:c1 * ctx.N].reshape(-1, ctx.N), seed=seed, ct_index0=idx0 + c0)
    return out


def decrypt_chunked(ctx, ct):
    return np.concatenate([ctx.decrypt(ct[c0:c0 + 256]) for c0 in range(0, ct.shape[0], 256)])


def test_keygen_parity_n32768(big):
    ctx, o = big
    sk, rk = ctx.keygen(SEED_KEY)
    assert np.array_equal(sk.cpu().numpy(), o.s)
    assert np.array_equal(hp.to_u64(rk), o.rk)


def test_plain_workload_2048_pairs(big):
    ctx, o = big
    n_ct, N = 2048, ctx.N
    x, y = eq_pair_columns(n_ct * N, seed=1)
    cx = encrypt_chunked(ctx, x, n_ct, 1, 0)
    cy = encrypt_chunked(ctx, y, n_ct, 1, n_ct)
    out = ctx.eq(cx, cy)
    dec = decrypt_chunked(ctx, out)
    assert np.array_equal(dec.reshape(-1), (x == y).astype(np.uint32))
    ctx.check_status()
    idx = sample_indices(n_ct, 101)
    want = eq_many(LOGN, SEED_KEY, [hp.to_u64(cx[c]) for c in idx], [hp.to_u64(cy[c]) for c in idx], dp=DP,
                   coarse_from=COARSE)
    for c, w in zip(idx, want):  # sampled ciphertexts, bit for bit
        assert np.array_equal(hp.to_u64(out[c]), w), c
    import torch

    del cx, cy, out
    torch.cuda.empty_cache()


def test_const_workload_2_28_slots(big):
    import torch

    ctx, o = big
    n_ct, N, cval = 8192, ctx.N, 4242
    rng = np.random.default_rng(3)
    x = rng.integers(0, 1 << 16, n_ct * N, dtype=np.uint32)
    x[rng.random(n_ct * N) < 0.25] = cval
    cx = encrypt_chunked(ctx, x, n_ct, 3, 0)
    out = ctx.eq(cx, None, const_val=cval)
    ctx.check_status()
    for c0 in range(0, n_ct, 512):
        c1 = min(n_ct, c0 + 512)
        dec = decrypt_chunked(ctx, out[c0:c1])
        assert np.array_equal(dec.reshape(-1), (x[c0 * N:c1 * N] == cval).astype(np.uint32))
    idx = sample_indices(n_ct, 103)
    want = eq_many(LOGN, SEED_KEY, [hp.to_u64(cx[c]) for c in idx], None, const_val=cval, dp=DP, coarse_from=COARSE)
    for c, w in zip(idx, want):  # sampled ciphertexts, bit for bit
        assert np.array_equal(hp.to_u64(out[c]), w), c
    del cx, out
    torch.cuda.empty_cache()
