"""The oracle's pins have teeth (CPU only).

Each case builds a separate copy of the oracle with one plausible mistake
planted in it (bfv_oracle.cpp, ORC_MUTANT = k; the normal build has none) and
runs a pin from test_oracle_pins.py on that copy: the pin must fail.  The pins
compare the oracle with things other than itself -- Python big-integer brute
force with a schoolbook product, direct evaluation of the encoding, the
closed form of the predicate -- so a mistake in any of these steps shows up
there and not only as a disagreement with the GPU.  The same pins pass on the
normal build in test_oracle_pins.py."""
import pytest

import oracle
from tests import test_oracle_pins as pins

# (planted mistake, the pin that must catch it)
CASES = [
    (1, "round(t d / Q) truncated toward zero", pins.test_tensor_and_rounding_bruteforce),
    (2, "cross term a1 b0 dropped from d1", pins.test_tensor_and_rounding_bruteforce),
    (3, "mod-down remainder not centred", pins.test_relinearisation_bruteforce),
    (4, "negacyclic twist left out", pins.test_encoding_closed_forms),
    (4, "negacyclic twist left out", pins.test_tensor_and_rounding_bruteforce),
    (5, "sign of (a s + e) in the key flipped", pins.test_keygen_relation_bruteforce),
    (6, "slots in natural transform order", pins.test_encoding_closed_forms),
    (7, "digit taken mod its first prime only", pins.test_relinearisation_bruteforce),
    (8, "one squaring too few", pins.test_eq_const_closed_form),
    (9, "LT coefficients from the even powers", pins.test_lt_polynomial_is_the_paper_sum),
    (10, "automorphism without the negacyclic sign", lambda o: pins.test_automorphism_permutes_slots(o, 5)),
    (11, "reduction without the row exchange", pins.test_count_and_sum_closed_form_n16),
    (12, "BETWEEN's first factor a instead of 1 - a", pins.test_between_closed_form_n16),
    (13, "first giant step w^128", pins.test_lt_closed_form_n16),
    (14, "noise budget without its factor 2", pins.test_noise_budget_bruteforce),
    (15, "per-prime key only below the fine depth", lambda o: pins.check_fine_depth_selection(oracle.build_mutant(15))),
    (16, "two-digit key from one level late", lambda o: pins.check_coarse_selection(oracle.build_mutant(16))),
]


def _name(pin):
    if pin.__name__.startswith("test_"):
        return pin.__name__[5:]
    names = pin.__code__.co_names
    if "check_fine_depth_selection" in names:
        return "fine_depth_selection"
    if "check_coarse_selection" in names:
        return "coarse_selection"
    return "automorphism_permutes_slots"


def _oracle16(lib_path=None):
    o = oracle.Oracle(4, lib_path=lib_path)  # the orc16 fixture's parameters and key seed
    o.keygen(7)
    return o


@pytest.mark.parametrize("k, mistake, pin", CASES, ids=["%d-%s" % (k, _name(p)) for k, _, p in CASES])
def test_pin_catches_planted_mistake(k, mistake, pin):
    o = _oracle16(oracle.build_mutant(k))
    with pytest.raises(AssertionError):
        pin(o)
