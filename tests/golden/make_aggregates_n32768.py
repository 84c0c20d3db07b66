"""Writes tests/golden/aggregates_n32768.txt: SHA-256 digests of ciphertexts the
oracle computes at the paper's ring degree N = 32768 (Sec. 5.1) for the
aggregate and membership operators of Sec. 4.2.2, on one ciphertext each, so
that the full-size GPU test (tests/test_gpu_aggregates_n32768.py) compares bit
for bit without re-running the oracle:

    COUNT / SUM   the rotate-and-add reduction of ciphertext 0 of the column
    IN (Eq. 6)    sum_k EQ(x, c_k) over the constants of in_constants(), ciphertext 0
    JOIN          A.key = B.key over the first JOIN_ROWS rows of B with one
                  attribute (Extract + Broadcast, EQ masks, products, sums), A ciphertext 0

With --bench-grouping the oracle uses the benchmark's key switching for these
workloads (digits of five data primes, the two-digit key from depth 7 on) and
the digests go to tests/golden/aggregates_d5c7_n32768.txt.

Calls only oracle/ and the seeded input recipe below (a few minutes of
single-threaded CPU, most of it in the Galois keys and the EQ chains).

    python tests/golden/make_aggregates_n32768.py [--bench-grouping]
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

LOGN, SEED_KEY, SEED_ENC = 15, 2028, 95
N_COLUMN = 2048      # column ciphertexts of the COUNT / SUM test (2^26 slots)
N_IN = 64            # ciphertexts of the IN test
N_A, JOIN_ROWS = 4, 3  # A ciphertexts and joined B rows of the JOIN test


def column(n_ct, N, seed):
    """16-bit column values (COUNT / SUM, IN) for n_ct ciphertexts."""
    return np.random.default_rng(seed).integers(0, 1 << 16, n_ct * N).astype(np.uint32)


def in_constants(x):
    """Four IN constants: three drawn from the column's first slots, one absent from the first ciphertext."""
    first = set(int(v) for v in x[:1 << LOGN])
    absent = next(v for v in range(1, 1 << 16) if v not in first)
    return [int(x[3]), int(x[100]), int(x[5000]), absent]


def join_tables(N):
    """A keys (N_A ciphertexts), B keys (distinct, drawn from A's first ciphertext) and one B attribute."""
    rng = np.random.default_rng(97)
    akey = rng.integers(1, 1 << 15, N_A * N).astype(np.uint32)
    bkey = np.zeros(N, dtype=np.uint32)
    bkey[:JOIN_ROWS] = [akey[7], akey[9], 1 << 15]  # the last matches no row of A (keys < 2^15)
    battr = rng.integers(0, 1 << 16, N).astype(np.uint32)
    return akey, bkey, battr


def digest(ct):
    return hashlib.sha256(np.ascontiguousarray(ct, dtype=np.uint64).tobytes()).hexdigest()


def main(argv):
    t0 = time.time()
    bench = "--bench-grouping" in argv
    dp, cf = (5, 7) if bench else (3, 0)
    o = oracle.Oracle(LOGN, dp=dp, coarse_from=cf)
    o.keygen(SEED_KEY)
    N = o.N
    for g in o.galois_elements():
        o.galois_keygen(SEED_KEY, g)
    # COUNT / SUM: reduction of ciphertext 0 of the column
    x = column(N_COLUMN, N, 11)
    c0 = o.encrypt(x[:N], SEED_ENC, 0)
    red = o.rotate_sum(c0)
    assert np.all(o.decrypt(red) == int(x[:N].astype(np.int64).sum() % 65537))
    # IN: ciphertext 0 of the IN column against four constants
    xi = column(N_IN, N, 12)
    consts = in_constants(xi)
    ci = o.encrypt(xi[:N], SEED_ENC, 0)
    ins = o.in_set(ci, consts)
    assert np.array_equal(o.decrypt(ins), np.isin(xi[:N], consts).astype(np.uint32))
    # JOIN: A ciphertext 0 against the first JOIN_ROWS rows of B, one attribute
    akey, bkey, battr = join_tables(N)
    ca = o.encrypt(akey[:N], SEED_ENC, 100)
    cbk = o.encrypt(bkey, SEED_ENC, 200)
    cba = o.encrypt(battr, SEED_ENC, 201)
    jn = o.join([ca], [cbk], [[cba]], JOIN_ROWS)[0, 0]
    want = np.zeros(N, dtype=np.uint32)
    for r in range(JOIN_ROWS):
        want[akey[:N] == bkey[r]] = battr[r]
    assert np.array_equal(o.decrypt(jn), want)
    name = "aggregates_d5c7_n32768.txt" if bench else "aggregates_n32768.txt"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    with open(path, "w") as f:
        f.write("# COUNT/SUM, IN and JOIN at N = 32768: SHA-256 of the oracle's ciphertexts (uint64 [2][15][32768],\n")
        f.write("# little endian); written by tests/golden/make_aggregates_n32768.py%s\n"
                % (" --bench-grouping" if bench else ""))
        f.write("log_n = %d\nseed_key = %d\nseed_enc = %d\n" % (LOGN, SEED_KEY, SEED_ENC))
        if bench:
            f.write("ks_digit_primes = %d\nks_coarse_from = %d\n" % (dp, cf))
        f.write("rotate_sum_sha256 = %s\nin_sha256 = %s\njoin_sha256 = %s\n" % (digest(red), digest(ins), digest(jn)))
        f.write("oracle_seconds = %.0f\n" % (time.time() - t0))
    print(path)


if __name__ == "__main__":
    main(sys.argv[1:])
