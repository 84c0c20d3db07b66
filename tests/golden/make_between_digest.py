"""Writes tests/golden/between_n4096.txt: the SHA-256 of the ciphertext the
oracle computes for BETWEEN (Sec. 4.2.2: the product (1 - LT(x, lo)) (1 - LT(hi, x))
of the two comparisons) on the GPU test's inputs, so that the GPU test compares
bit for bit without re-running the oracle's two LT evaluations (about ten
minutes of CPU at N = 4096).  Calls only oracle/ and the seeded input recipe of
tests/test_gpu_between.py.

    python tests/golden/make_between_digest.py
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

LOGN, SEED_KEY, SEED_ENC, LO, HI, HALF, N_CT, CT = 12, 2025, 71, 1000, 20000, 32768, 4, 3


def between_inputs(N):
    """The test's column: 4 ciphertexts' slots from a seeded generator, edge values first."""
    rng = np.random.default_rng(31)
    x = rng.integers(0, HALF + 1, N_CT * N).astype(np.uint32)
    x[:8] = [LO, HI, LO - 1, HI + 1, 0, HALF, (LO + HI) // 2, LO + 1]
    return x


def main():
    o = oracle.Oracle(LOGN)
    o.keygen(SEED_KEY)
    N = o.N
    x = between_inputs(N)
    ct = o.encrypt(x[CT * N:(CT + 1) * N], SEED_ENC, CT)
    out = o.between(ct, LO, HI)
    digest = hashlib.sha256(np.ascontiguousarray(out, dtype=np.uint64).tobytes()).hexdigest()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "between_n4096.txt")
    with open(path, "w") as f:
        f.write("# SHA-256 of the oracle's BETWEEN ciphertext (uint64 [2][15][4096], little endian) for the\n")
        f.write("# inputs of tests/test_gpu_between.py; written by tests/golden/make_between_digest.py\n")
        f.write("log_n = %d\nseed_key = %d\nseed_enc = %d\nlo = %d\nhi = %d\nciphertext = %d\n" % (LOGN, SEED_KEY, SEED_ENC, LO, HI, CT))
        f.write("sha256 = %s\n" % digest)
    print(digest)


if __name__ == "__main__":
    main()
