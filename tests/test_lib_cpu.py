"""CPU checks of the C-ABI library: it loads, exports every symbol the header
declares, and its host-side parameter logic agrees with the paper and the
oracle's independent prime search.  No compute call needs a GPU here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2602_24271_b300 import build, hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hp.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "hp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hp_\w+)\s*\(", src, flags=re.M)))


def test_header_symbols_exported(lib):
    names = header_functions()
    assert "hp_run" in names and "hp_create" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(hp.EXPORTED) == names


def test_default_params_match_oracle(lib):
    q, P, t = hp.default_params()
    qo, Po = oracle.default_primes(15)
    assert q == qo and P == Po and t == 65537
    assert round(sum(math.log2(x) for x in q) + math.log2(P)) == 881


def test_default_params_bad_args(lib):
    q = (ctypes.c_uint64 * 16)()
    P, t = ctypes.c_uint64(), ctypes.c_uint64()
    assert lib.hp_default_params(0, q, ctypes.byref(P), ctypes.byref(t)) == hp.HP_ERR_ARG
    assert lib.hp_default_params(16, q, ctypes.byref(P), ctypes.byref(t)) == hp.HP_ERR_ARG


def _create(lib, log_n=15, max_depth=16, q=None, P=None, t=65537, dp=0, fine=0, coarse=0):
    if q is None:
        q, P, t = hp.default_params()
    qa = (ctypes.c_uint64 * len(q))(*q)
    prm = hp.hp_params(log_n, len(q), qa, P, t, max_depth, fine, dp, coarse)
    h = ctypes.c_void_p()
    rc = lib.hp_create(ctypes.byref(prm), None, 1, ctypes.byref(h))
    return rc, h


def test_create_rejects_bad_parameters(lib):
    rc, _ = _create(lib, log_n=11)
    assert rc == hp.HP_ERR_UNSUPPORTED
    rc, _ = _create(lib, max_depth=40)  # beyond the static noise estimate
    assert rc == hp.HP_ERR_DEPTH
    assert b"depth" in lib.hp_last_error(None)
    q, P, t = hp.default_params()
    rc, _ = _create(lib, q=[q[0] + 2] + q[1:], P=P)  # not prime / not 1 mod 2^16
    assert rc == hp.HP_ERR_ARG
    rc, _ = _create(lib, q=q, P=P, t=257)
    assert rc == hp.HP_ERR_UNSUPPORTED
    for dp in (1, 2, 4, 15):  # key-switching digits of 3 or 5 primes only
        rc, _ = _create(lib, dp=dp)
        assert rc == hp.HP_ERR_UNSUPPORTED
        assert b"ks_digit_primes" in lib.hp_last_error(None)
    for fine, coarse in ((3, 3), (3, 1)):  # the two-digit key starts above the fine depth
        rc, _ = _create(lib, fine=fine, coarse=coarse)
        assert rc == hp.HP_ERR_ARG
        assert b"ks_coarse_from" in lib.hp_last_error(None)


def test_backward_is_unsupported(lib):
    assert lib.hp_backward(None, 0, None, None, 0, None) == hp.HP_ERR_UNSUPPORTED


def test_static_depth_estimate_is_conservative_against_oracle():
    """hp_create's depth estimate must not promise more squarings than the
    oracle's measured noise budget allows (3-prime modulus, N = 16)."""
    lib = hp.load()
    # the estimate for the paper's parameters covers EQ + SELECT
    est = {}
    for logn in (12, 15):
        est[logn] = lib_depth(logn, *hp.default_params()[:2])
        assert est[logn] >= 17
    q, P = oracle.default_primes(15)
    o = oracle.Oracle(4, q=q[:3], P=P)
    o.keygen(3)
    x = np.arange(o.N, dtype=np.uint32) + 2
    cx = o.encrypt(x, 5, 0)
    d = lib_depth(4, q[:3], P)
    _, nb = o.decrypt(o.square_chain(cx, d), with_noise=True)
    assert nb > 0


def lib_depth(logn, q, P):
    # mirror of the C estimate (hp_host.cpp supported_depth): fresh budget
    # log2 Q - log2 t - log N - 8, per squaring log2 t + log N + 2; the budget
    # after the first squaring is also bounded by the key-switching noise
    # |digit| sqrt(N) 2^4 / P (digits: groups of 3 data primes)
    lq = sum(math.log2(x) for x in q)
    lt = math.log2(65537)
    fresh = lq - lt - logn - 8
    per = lt + logn + 2
    if fresh <= 0:
        return 0
    dbits = max(sum(math.log2(x) for x in q[a:a + 3]) for a in range(0, len(q), 3))
    b1 = min(fresh - per, (lq - lt) - (dbits + 0.5 * logn + 4 - math.log2(P)))
    return 1 + int((b1 - 1) // per) if b1 > 1 else 0


def test_lt_coefficients_match_oracle(lib):
    """The library's LT coefficients (one length-2^16 transform over F_65537)
    equal the oracle's (plain power sums); computed independently."""
    got = hp.lt_coefficients()
    o = oracle.Oracle(4)
    assert np.array_equal(got, o.lt_coefficients())


def test_galois_elements_match_oracle(lib):
    """The library's rotate-and-add schedule equals the oracle's (elements and order)."""
    for logn in (4, 12, 15):
        assert hp.galois_elements(logn) == oracle.galois_elements(logn)
    g = (ctypes.c_uint64 * 2)()
    assert lib.hp_galois_elements(2, g) == hp.HP_ERR_ARG
    assert lib.hp_galois_elements(12, None) == hp.HP_ERR_ARG

