"""Writes tests/golden/range_n32768_f<F>.txt (and, with --lt, lt_n32768.txt;
with --digit-primes 5 and --coarse-from C > 0 the names end in _d5, _c<C>):
the SHA-256 digests of the ciphertexts the oracle computes at the paper's ring
degree N = 32768 for a range filter followed by an aggregate, the pattern of
TPC-H Q6 (Table 5: filter, then SUM):

    mask = BETWEEN(x, LO, HI)        (Sec. 4.2.2: the product of two comparisons, Eq. 4)
    sel  = col * mask                (SELECT, Eq. 5; the mask at depth 19)
    agg  = rotate-and-add(sel)       (SUM, Sec. 4.2.2: every slot holds the column's sum)

and, with --lt, LT(x, y) (Eq. 4) on its own, together with the noise budget
the oracle measures in each result.  --digit-primes sets the key-switching
digits between the per-prime ones (up to --fine-depth) and the two-digit key
(data primes 0..7 and 8..14) that relinearises the products at depth
--coarse-from and beyond.  The GPU test (tests/test_gpu_range_n32768.py)
compares its own ciphertexts with these digests bit for bit, so it does not
re-run the oracle (each LT is about forty minutes of single-threaded CPU at this
ring degree).  Calls only oracle/ and the seeded input recipe below.

    python tests/golden/make_range_n32768.py --fine-depth 0
    python tests/golden/make_range_n32768.py --fine-depth 3
    python tests/golden/make_range_n32768.py --lt
    python tests/golden/make_range_n32768.py --fine-depth 4 --digit-primes 5 --coarse-from 10
    python tests/golden/make_range_n32768.py --lt --fine-depth 4 --digit-primes 5 --coarse-from 10
"""
import argparse
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

LOGN, SEED_KEY, SEED_ENC = 15, 2026, 91
LO, HI, HALF = 12000, 20000, 32768
CT_X, CT_Y, CT_COL = 0, 1, 2  # encryption object indices
MASK_DEPTH = 19  # BETWEEN: two LT results (depth 18) multiplied


def range_inputs(N):
    """x in [0, 2^15] with the bounds and the values around them first; y for
    LT (equal to x in about a tenth of the slots); col uniform 16-bit values
    (the summed column)."""
    rng = np.random.default_rng(77)
    x = rng.integers(0, HALF + 1, N).astype(np.uint32)
    x[:10] = [LO, HI, LO - 1, HI + 1, 0, HALF, (LO + HI) // 2, LO + 1, HI - 1, 1]
    y = np.where(rng.random(N) < 0.1, x, rng.integers(0, HALF + 1, N)).astype(np.uint32)
    y[:4] = [LO + 1, HI - 1, LO - 1, 0]
    col = rng.integers(0, 1 << 16, N).astype(np.uint32)
    return x, y, col


def digest(ct):
    return hashlib.sha256(np.ascontiguousarray(ct, dtype=np.uint64).tobytes()).hexdigest()


def write(name, header, kv):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    with open(path, "w") as f:
        for line in header:
            f.write("# %s\n" % line)
        for k, v in kv:
            f.write("%s = %s\n" % (k, v))
    print(path)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--fine-depth", type=int, default=0)
    ap.add_argument("--lt", action="store_true")
    ap.add_argument("--coarse-from", type=int, default=0)
    ap.add_argument("--digit-primes", type=int, default=3)
    a = ap.parse_args()
    F, C, dp = a.fine_depth, a.coarse_from, a.digit_primes
    sfx = ("_d%d" % dp if dp != 3 else "") + ("_c%d" % C if C else "")
    t0 = time.time()
    o = oracle.Oracle(LOGN, fine_depth=F, coarse_from=C, dp=dp)
    o.keygen(SEED_KEY)
    opts = "".join([" --lt" if a.lt else "", " --fine-depth %d" % F if (F or not a.lt) else "",
                    " --digit-primes %d" % dp if dp != 3 else "", " --coarse-from %d" % C if C else ""])
    N = o.N
    x, y, col = range_inputs(N)
    cx = o.encrypt(x, SEED_ENC, CT_X)
    if a.lt:
        cy = o.encrypt(y, SEED_ENC, CT_Y)
        lt = o.lt(cx, cy)
        got, nb = o.decrypt(lt, with_noise=True)
        assert np.array_equal(got, (x < y).astype(np.uint32))
        write("lt_n32768%s.txt" % (("_f%d" % F if F else "") + sfx),
              ["LT(x, y) (Eq. 4) at N = 32768: SHA-256 of the oracle's ciphertext (uint64 [2][15][32768],",
               "little endian) and its measured noise budget; written by tests/golden/make_range_n32768.py%s"
               % opts],
              [("log_n", LOGN), ("seed_key", SEED_KEY), ("seed_enc", SEED_ENC), ("ks_fine_depth", F)]
              + ([("ks_digit_primes", dp)] if dp != 3 else []) + ([("ks_coarse_from", C)] if C else []) + [
               ("lt_sha256", digest(lt)), ("lt_budget_bits", "%.2f" % nb),
               ("oracle_seconds", "%.0f" % (time.time() - t0))])
        return
    ccol = o.encrypt(col, SEED_ENC, CT_COL)
    mask = o.between(cx, LO, HI)
    got, nb_mask = o.decrypt(mask, with_noise=True)
    sel_rows = (x >= LO) & (x <= HI)
    assert np.array_equal(got, sel_rows.astype(np.uint32))
    sel = o.mul_relin(ccol, mask, depth_a=0, depth_b=MASK_DEPTH)
    got, nb_sel = o.decrypt(sel, with_noise=True)
    assert np.array_equal(got, np.where(sel_rows, col, 0).astype(np.uint32))
    for g in o.galois_elements():
        o.galois_keygen(SEED_KEY, g)
    agg = o.rotate_sum(sel)
    got, nb_agg = o.decrypt(agg, with_noise=True)
    total = int(col[sel_rows].astype(np.int64).sum() % 65537)
    assert np.all(got == total)
    write("range_n32768_f%d%s.txt" % (F, sfx),
          ["BETWEEN -> SELECT -> SUM at N = 32768 with per-prime relinearisation up to depth %d%s:"
           % (F, "".join([", digits of %d primes" % dp if dp != 3 else "", ", two-digit from depth %d" % C if C else ""])),
           "SHA-256 of the oracle's ciphertexts (uint64 [2][15][32768], little endian) and their measured",
           "noise budgets; written by tests/golden/make_range_n32768.py%s" % opts],
          [("log_n", LOGN), ("seed_key", SEED_KEY), ("seed_enc", SEED_ENC), ("ks_fine_depth", F)]
          + ([("ks_digit_primes", dp)] if dp != 3 else []) + ([("ks_coarse_from", C)] if C else []) + [("lo", LO),
           ("hi", HI), ("mask_depth", MASK_DEPTH), ("between_sha256", digest(mask)),
           ("between_budget_bits", "%.2f" % nb_mask), ("select_sha256", digest(sel)),
           ("select_budget_bits", "%.2f" % nb_sel), ("sum_sha256", digest(agg)), ("sum_budget_bits", "%.2f" % nb_agg),
           ("sum_value", total), ("oracle_seconds", "%.0f" % (time.time() - t0))])


if __name__ == "__main__":
    main()
