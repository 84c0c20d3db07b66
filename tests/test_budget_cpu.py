"""CPU check of the library's static noise-budget estimate (hp_budget_estimate,
the depth guard of every operation) against the budgets the oracle measured.
No GPU needed: the estimate is host code."""
import ctypes

from paper_2602_24271_b300 import hp


def _budget(logn, fine_depth, op, in_depth=0, in_bits=0.0, dp=3, cf=0):
    q, P, t = hp.default_params()
    qa = (ctypes.c_uint64 * len(q))(*q)
    return hp.budget_estimate(hp.hp_params(logn, len(q), qa, P, t, 17, fine_depth, dp, cf), op, in_depth, in_bits)


def test_budget_estimate_lies_below_the_oracle_measurements():
    """The library's static noise-budget estimate (the depth guard of every
    operation) never promises more than the oracle measured: EQ, LT, BETWEEN,
    SELECT on the BETWEEN mask and its SUM at N = 4096 and N = 32768, with
    three-prime key switching throughout, with per-prime digits up to depth 3,
    with five-prime digits and with the two-digit key from a given depth on
    (measurements written by tests/golden/make_n4096_budgets.py and
    make_range_n32768.py).  It is not vacuous either: within 80 bits of each."""
    from tests.conftest import read_golden_kv

    hp.load()
    E, LT, BT, PR, RS = hp.HP_BUDGET_EQ, hp.HP_BUDGET_LT, hp.HP_BUDGET_BETWEEN, hp.HP_BUDGET_PRODUCT, hp.HP_BUDGET_ROTATE_SUM
    pairs = []
    g = read_golden_kv("budgets_n4096.txt")
    for F in (0, 3):
        bt = _budget(12, F, BT)
        sel = _budget(12, F, PR, 19, bt)
        pairs += [(_budget(12, F, E), g["f%d_eq" % F]), (_budget(12, F, LT), g["f%d_lt" % F]), (bt, g["f%d_between" % F]),
                  (sel, g["f%d_select" % F]), (_budget(12, F, RS, 0, sel), g["f%d_sum" % F])]
    for name, F, dp, cf in (("coarse_d5c7_n4096.txt", 0, 5, 7), ("coarse_d3c10_n4096.txt", 0, 3, 10),
                            ("coarse_f4d5c10_n4096.txt", 4, 5, 10)):
        g = read_golden_kv(name)
        bt = _budget(12, F, BT, dp=dp, cf=cf)
        sel = _budget(12, F, PR, 19, bt, dp=dp, cf=cf)
        pairs += [(_budget(12, F, E, dp=dp, cf=cf), g["eq"]), (_budget(12, F, LT, dp=dp, cf=cf), g["lt"]),
                  (bt, g["between"]), (sel, g["select"]), (_budget(12, F, RS, 0, sel, dp=dp, cf=cf), g["sum"])]
    d5 = read_golden_kv("digits5_n4096.txt")
    bt = _budget(12, 0, BT, dp=5)
    sel = _budget(12, 0, PR, 19, bt, dp=5)
    pairs += [(_budget(12, 0, E, dp=5), d5["eq"]), (_budget(12, 0, LT, dp=5), d5["lt"]), (bt, d5["between"]),
              (sel, d5["select"]), (_budget(12, 0, RS, 0, sel, dp=5), d5["sum"])]
    for F in (0, 3):
        r = read_golden_kv("range_n32768_f%d.txt" % F)
        bt = _budget(15, F, BT)
        sel = _budget(15, F, PR, 19, bt)
        pairs += [(bt, r["between_budget_bits"]), (sel, r["select_budget_bits"]),
                  (_budget(15, F, RS, 0, sel), r["sum_budget_bits"])]
    pairs.append((_budget(15, 0, LT), read_golden_kv("lt_n32768.txt")["lt_budget_bits"]))
    # the benchmark's LT / BETWEEN key switching: per-prime up to depth 4, five-prime, two-digit from depth 10
    r = read_golden_kv("range_n32768_f4_d5_c10.txt")
    bt = _budget(15, 4, BT, dp=5, cf=10)
    sel = _budget(15, 4, PR, 19, bt, dp=5, cf=10)
    pairs += [(bt, r["between_budget_bits"]), (sel, r["select_budget_bits"]),
              (_budget(15, 4, RS, 0, sel, dp=5, cf=10), r["sum_budget_bits"]),
              (_budget(15, 4, LT, dp=5, cf=10), read_golden_kv("lt_n32768_f4_d5_c10.txt")["lt_budget_bits"])]
    for est, measured in pairs:
        assert 0 < est <= measured < est + 80, (est, measured)
    # the guard's margin: a product on a mask with too little budget left is refused
    assert _budget(15, 0, PR, 19, 35.0) < hp.HP_BUDGET_MARGIN
