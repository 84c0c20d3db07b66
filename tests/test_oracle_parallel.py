"""The oracle's process pool (oracle/parallel.py) on CPU: spreading independent
EQ evaluations (Eq. 3) over worker processes, each keyed from the same seed,
returns exactly the ciphertexts the single-process oracle returns, in order,
for the ciphertext-ciphertext and the constant form.  The full-size GPU tests
use the pool to compare a larger sample of ciphertexts with the oracle."""
import numpy as np

from oracle.parallel import eq_many

LOGN, KEY_SEED = 12, 2024  # the orc4096 fixture's ring degree and key seed


def test_pool_matches_single_process_oracle(orc4096):
    o = orc4096
    rng = np.random.default_rng(5)
    x = rng.integers(0, 1 << 16, (2, o.N)).astype(np.uint32)
    y = np.where(rng.random((2, o.N)) < 0.5, x, rng.integers(0, 1 << 16, (2, o.N))).astype(np.uint32)
    cx = [o.encrypt(x[i], 11, i) for i in range(2)]
    cy = [o.encrypt(y[i], 11, 2 + i) for i in range(2)]
    got = eq_many(LOGN, KEY_SEED, cx, cy, workers=2)
    assert len(got) == 2
    for i in range(2):
        assert np.array_equal(got[i], o.eq(cx[i], cy[i]))
        assert np.array_equal(o.decrypt(got[i]), (x[i] == y[i]).astype(np.uint32))
    got_c = eq_many(LOGN, KEY_SEED, cx[:1], None, const_val=int(x[0][3]))
    assert np.array_equal(got_c[0], o.eq(cx[0], None, const_val=int(x[0][3])))


def test_pool_argument_checks():
    assert eq_many(LOGN, KEY_SEED, []) == []
    try:
        eq_many(LOGN, KEY_SEED, [np.zeros(1, np.uint64)], [])
    except ValueError:
        pass
    else:
        raise AssertionError("mismatched xs / ys accepted")
