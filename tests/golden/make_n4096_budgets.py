"""Writes tests/golden/budgets_n4096.txt and tests/golden/fine_lt_n4096.txt
(or, with --digits5, tests/golden/digits5_n4096.txt; with --coarse DP:C,
tests/golden/coarse_d<DP>c<C>_n4096.txt).

budgets_n4096.txt: the invariant-noise budgets the oracle measures at N = 4096
(same primes and plaintext modulus as the paper's N = 32768, Sec. 5.1) in the
results of EQ (Eq. 3, 16 squarings), LT (Eq. 4), BETWEEN (Sec. 4.2.2, product
of two comparisons), SELECT on the BETWEEN mask (Eq. 5) and the SUM of that
product (rotate-and-add, Sec. 4.2.2), with per-prime relinearisation up to
depth 0 and 3.  The CPU test of the library's static budget estimate
(tests/test_budget_cpu.py) checks that every estimate lies below these.

fine_lt_n4096.txt: the SHA-256 of the oracle's LT ciphertext with per-prime
relinearisation up to depth 3, for the GPU parity test of that key-switching
path (tests/test_gpu_fine_digits.py), so the test does not re-run the oracle's
LT (about five minutes of CPU).

digits5_n4096.txt (--digits5): the same budgets and the LT digest with
key-switching digits of five primes (three digits) instead of three, for the
budget test and the GPU parity test of that grouping
(tests/test_gpu_digits5.py).

coarse_d<DP>c<C>_n4096.txt (--coarse DP:C): the same with digits of DP primes
and the two-digit key from depth C on (tests/test_gpu_coarse_digits.py);
coarse_f<F>d<DP>c<C>_n4096.txt (--coarse F:DP:C) with per-prime digits up to
depth F as well.

Calls only oracle/ and the seeded inputs below.

    python tests/golden/make_n4096_budgets.py [--digits5 | --coarse [F:]DP:C]
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

LOGN, SEED_KEY, SEED_ENC, LO, HI, HALF = 12, 2027, 93, 5000, 25000, 32768
FINE_DEPTHS = (0, 3)


def lt_inputs(N):
    """x, y in [0, 2^15] with edge pairs first, and a 16-bit column to sum."""
    rng = np.random.default_rng(55)
    x = rng.integers(0, HALF + 1, N).astype(np.uint32)
    y = np.where(rng.random(N) < 0.2, x, rng.integers(0, HALF + 1, N)).astype(np.uint32)
    x[:6], y[:6] = [5, 3, 0, HALF, 7, LO], [3, 5, HALF, 0, 7, LO]
    col = rng.integers(0, 1 << 16, N).astype(np.uint32)
    return x, y, col


def measure(F, dp, here, coarse_from=0):
    """Budgets of EQ, LT, BETWEEN, SELECT and SUM with per-prime relinearisation
    up to depth F, the two-digit key from depth coarse_from on (0 = never) and
    digits of dp primes elsewhere; returns them with the SHA-256 of the LT
    ciphertext."""
    o = oracle.Oracle(LOGN, fine_depth=F, dp=dp, coarse_from=coarse_from)
    o.keygen(SEED_KEY)
    N = o.N
    x, y, col = lt_inputs(N)
    cx, cy, cc = o.encrypt(x, SEED_ENC, 0), o.encrypt(y, SEED_ENC, 1), o.encrypt(col, SEED_ENC, 2)
    eq, nb_eq = o.decrypt(o.eq(cx, cy), with_noise=True)
    assert np.array_equal(eq, (x == y).astype(np.uint32))
    lt = o.lt(cx, cy)
    got, nb_lt = o.decrypt(lt, with_noise=True)
    assert np.array_equal(got, (x < y).astype(np.uint32))
    lt_sha = hashlib.sha256(np.ascontiguousarray(lt, dtype=np.uint64).tobytes()).hexdigest()
    mask = o.between(cx, LO, HI)
    got, nb_bt = o.decrypt(mask, with_noise=True)
    rows_in = (x >= LO) & (x <= HI)
    assert np.array_equal(got, rows_in.astype(np.uint32))
    sel = o.mul_relin(cc, mask, depth_a=0, depth_b=19)
    got, nb_sel = o.decrypt(sel, with_noise=True)
    assert np.array_equal(got, np.where(rows_in, col, 0).astype(np.uint32))
    for g in o.galois_elements():
        o.galois_keygen(SEED_KEY, g)
    got, nb_sum = o.decrypt(o.rotate_sum(sel), with_noise=True)
    assert np.all(got == int(col[rows_in].astype(np.int64).sum() % 65537))
    row = (nb_eq, nb_lt, nb_bt, nb_sel, nb_sum)
    print(F, dp, row, flush=True)
    return row, lt_sha


NAMES = ("eq", "lt", "between", "select", "sum")


def main(argv):
    here = os.path.dirname(os.path.abspath(__file__))
    if "--coarse" in argv:
        spec = [int(v) for v in argv[argv.index("--coarse") + 1].split(":")]
        F, dp, cf = spec if len(spec) == 3 else [0] + spec
        row, lt_sha = measure(F, dp, here, cf)
        name = ("coarse_f%dd%dc%d_n4096.txt" % (F, dp, cf)) if F else ("coarse_d%dc%d_n4096.txt" % (dp, cf))
        with open(os.path.join(here, name), "w") as f:
            f.write("# %sDigits of %d primes with the two-digit key from depth %d on, at N = 4096: the noise budgets\n"
                    % ("Per-prime digits up to depth %d, then " % F if F else "", dp, cf))
            f.write("# (bits) the oracle measures in the results of EQ, LT, BETWEEN, SELECT on the BETWEEN mask and its\n")
            f.write("# SUM, and the SHA-256 of its LT ciphertext (uint64 [2][15][4096], little endian); written by\n")
            f.write("# tests/golden/make_n4096_budgets.py --coarse %s (inputs: its lt_inputs, ciphertext indices 0, 1)\n"
                    % ":".join(str(v) for v in spec))
            f.write("log_n = %d\nseed_key = %d\nseed_enc = %d\nks_fine_depth = %d\nks_digit_primes = %d\n"
                    "ks_coarse_from = %d\n" % (LOGN, SEED_KEY, SEED_ENC, F, dp, cf))
            for name, b in zip(NAMES, row):
                f.write("%s = %.2f\n" % (name, b))
            f.write("lt_sha256 = %s\n" % lt_sha)
        return
    if "--digits5" in argv:
        row, lt_sha = measure(0, 5, here)
        with open(os.path.join(here, "digits5_n4096.txt"), "w") as f:
            f.write("# Five-prime key-switching digits at N = 4096: the noise budgets (bits) the oracle measures in the\n")
            f.write("# results of EQ, LT, BETWEEN, SELECT on the BETWEEN mask and its SUM, and the SHA-256 of its LT\n")
            f.write("# ciphertext (uint64 [2][15][4096], little endian); written by\n")
            f.write("# tests/golden/make_n4096_budgets.py --digits5 (inputs: its lt_inputs, ciphertext indices 0 and 1)\n")
            f.write("log_n = %d\nseed_key = %d\nseed_enc = %d\nks_digit_primes = 5\n" % (LOGN, SEED_KEY, SEED_ENC))
            for name, b in zip(NAMES, row):
                f.write("%s = %.2f\n" % (name, b))
            f.write("lt_sha256 = %s\n" % lt_sha)
        return
    rows = []
    for F in FINE_DEPTHS:
        row, lt_sha = measure(F, 3, here)
        if F == 3:
            with open(os.path.join(here, "fine_lt_n4096.txt"), "w") as f:
                f.write("# LT(x, y) (Eq. 4) at N = 4096 with per-prime relinearisation up to depth 3: SHA-256 of the\n")
                f.write("# oracle's ciphertext (uint64 [2][15][4096], little endian); written by\n")
                f.write("# tests/golden/make_n4096_budgets.py (inputs: its lt_inputs, ciphertext indices 0 and 1)\n")
                f.write("log_n = %d\nseed_key = %d\nseed_enc = %d\nks_fine_depth = 3\n" % (LOGN, SEED_KEY, SEED_ENC))
                f.write("sha256 = %s\n" % lt_sha)
        rows.append((F,) + row)
    with open(os.path.join(here, "budgets_n4096.txt"), "w") as f:
        f.write("# Noise budgets (bits, log2(Q / (2 |v|))) the oracle measures at N = 4096 in the results of EQ, LT,\n")
        f.write("# BETWEEN (product form), SELECT on the BETWEEN mask and the SUM of that product, with per-prime\n")
        f.write("# relinearisation up to depth F; written by tests/golden/make_n4096_budgets.py\n")
        f.write("log_n = %d\n" % LOGN)
        for F, *v in rows:
            for name, b in zip(NAMES, v):
                f.write("f%d_%s = %.2f\n" % (F, name, b))


if __name__ == "__main__":
    main(sys.argv[1:])
