"""Pins of the textbook-BFV oracle to things other than itself (CPU only).

Each test names what fixes the expected value: a published known-answer
vector, a closed form from the paper, a number-theoretic invariant, or a
brute-force computation on tiny inputs with Python's own big integers and a
schoolbook negacyclic product (a different algorithm from the oracle's
multi-modular transform + CRT).
"""
import math

import numpy as np
import pytest
import sympy

import oracle
from tests.conftest import golden_path, read_golden_kv

T = 65537


# --------------------------------------------------------------------------
# helpers: plain Python big-integer reference pieces for tiny N
# --------------------------------------------------------------------------
def negacyclic_schoolbook(a, b, N):
    r = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                r[k] += a[i] * b[j]
            else:
                r[k - N] -= a[i] * b[j]
    return r


def to_ints(res, moduli):
    """residues [len(moduli)][N] -> list of integers in [0, prod)"""
    N = res.shape[-1]
    return [oracle.crt_to_int([int(res[i][j]) for i in range(len(moduli))], moduli) for j in range(N)]


def brv(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2) if bits else 0


# --------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# --------------------------------------------------------------------------
def test_philox_known_answer_vectors():
    rows = []
    with open(golden_path("philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert oracle.philox_raw(r[0:4], r[4:6]) == r[6:10]


def test_philox_draw_uses_seed_as_key_and_counter_fields():
    seed = 0x0123456789ABCDEF
    w = oracle.philox(seed, 5, 6, 7, 8)
    assert w == oracle.philox_raw([5, 6, 7, 8], [seed & 0xFFFFFFFF, seed >> 32])


# --------------------------------------------------------------------------
# parameters (Sec. 5.1)
# --------------------------------------------------------------------------
def test_default_primes_match_their_definition_and_the_paper():
    q, P = oracle.default_primes(15)
    assert len(q) == 15 and len(set(q)) == 15
    step = 1 << 16
    for x in q:
        assert sympy.isprime(x) and x < 2**55 and x % step == 1
    assert sympy.isprime(P) and P < 2**56 and P % step == 1 and P >= 2**55
    assert q == sorted(q, reverse=True)
    # "largest": every skipped candidate k*2^16 + 1 between q_14 and 2^55 is composite
    cands = [k * step + 1 for k in range(q[-1] // step, (2**55 - 2) // step + 1)]
    primes_found = [c for c in cands if sympy.isprime(c)]
    assert primes_found == sorted(q)
    cands_P = [k * step + 1 for k in range(P // step, (2**56 - 2) // step + 1)]
    assert [c for c in cands_P if sympy.isprime(c)] == [P]
    g = read_golden_kv("paper_parameters.txt")
    logqp = sum(math.log2(x) for x in q) + math.log2(P)
    assert round(logqp) == g["log2_QP"]
    # every prime supports the negacyclic transform of the paper's ring degree
    for x in q + [P]:
        assert (x - 1) % (2 * g["ring_degree"]) == 0
    assert (g["plaintext_modulus"] - 1) % (2 * g["ring_degree"]) == 0
    # ciphertext size: 2 polynomials x 15 limbs x N words of 8 bytes ~ the paper's 7.4 MB
    size_mb = 2 * 15 * g["ring_degree"] * 8 / 2**20
    assert abs(size_mb - g["ciphertext_megabytes"]) / g["ciphertext_megabytes"] < 0.05


def test_oracle_constants(orc16):
    o = orc16
    Q = math.prod(o.q)
    assert o.Q == Q
    assert o.QP == Q * o.P
    assert o.Delta == Q // T
    assert Q % 2 == 1 and math.gcd(Q, T) == 1  # no rounding ties (t d / Q never half-integral)


# --------------------------------------------------------------------------
# the method's arithmetic fact: 16 squarings give the Fermat exponent
# --------------------------------------------------------------------------
def test_fermat_sixteen_squarings_exhaustive():
    g = read_golden_kv("paper_parameters.txt")
    p = g["plaintext_modulus"]
    assert math.ceil(math.log2(p - 1)) == g["eq_multiplications"]
    a = np.arange(p, dtype=np.int64)
    for _ in range(g["eq_multiplications"]):
        a = (a * a) % p
    assert a[0] == 0 and np.all(a[1:] == 1)  # a^(p-1) = [a != 0]


# --------------------------------------------------------------------------
# negacyclic transform
# --------------------------------------------------------------------------
@pytest.mark.parametrize("logn", [3, 4, 6])
def test_ntt_product_matches_schoolbook(logn):
    N = 1 << logn
    m = 2305843009213554689  # a 61-bit prime = 1 mod 2^17 (checked below)
    assert sympy.isprime(m) and (m - 1) % (2 * N) == 0
    rng = np.random.default_rng(logn)
    a = [int(x) for x in rng.integers(0, m, N, dtype=np.uint64)]
    b = [int(x) for x in rng.integers(0, m, N, dtype=np.uint64)]
    A = oracle.ntt_forward(logn, m, a)
    B = oracle.ntt_forward(logn, m, b)
    C = [(int(x) * int(y)) % m for x, y in zip(A, B)]
    c = oracle.ntt_inverse(logn, m, C)
    ref = [v % m for v in negacyclic_schoolbook(a, b, N)]
    assert [int(x) for x in c] == ref
    assert [int(x) for x in oracle.ntt_inverse(logn, m, A)] == a


def test_ntt_is_evaluation_at_odd_powers():
    logn, N, m = 3, 8, 65537
    g = 3  # smallest quadratic non-residue mod 65537
    assert pow(2, (m - 1) // 2, m) == 1 and pow(3, (m - 1) // 2, m) == m - 1
    psi = pow(g, (m - 1) // (2 * N), m)
    a = list(range(1, N + 1))
    A = oracle.ntt_forward(logn, m, a)
    for j in range(N):
        assert int(A[j]) == sum(a[k] * pow(psi, (2 * j + 1) * k, m) for k in range(N)) % m


# --------------------------------------------------------------------------
# batch encoding (slots <-> plaintext polynomial mod t)
# --------------------------------------------------------------------------
def test_encoding_closed_forms(orc16):
    o = orc16
    N = o.N
    ones = np.ones(N, dtype=np.uint32)
    m = o.encode(ones)
    assert int(m[0]) == 1 and not np.any(m[1:])  # all-ones slots = constant polynomial 1
    c = np.full(N, 4242, dtype=np.uint32)
    m = o.encode(c)
    assert int(m[0]) == 4242 and not np.any(m[1:])
    rng = np.random.default_rng(1)
    x = rng.integers(0, T, N).astype(np.uint32)
    assert np.array_equal(o.decode(o.encode(x)), x)
    # slot j is the evaluation at psi^(2 brv(j) + 1), psi = 3^((t-1)/2N)
    psi = pow(3, (T - 1) // (2 * N), T)
    mm = [int(v) for v in o.encode(x)]
    for j in range(N):
        e = 2 * brv(j, o.logn) + 1
        assert sum(mm[k] * pow(psi, e * k, T) for k in range(N)) % T == int(x[j])
    # ring homomorphism: slot-wise product <-> negacyclic product mod t
    y = rng.integers(0, T, N).astype(np.uint32)
    prod = [v % T for v in negacyclic_schoolbook([int(v) for v in o.encode(x)], [int(v) for v in o.encode(y)], N)]
    assert np.array_equal(o.decode(np.array(prod, dtype=np.uint64)), (x.astype(np.int64) * y % T).astype(np.uint32))


# --------------------------------------------------------------------------
# keys, encryption, decryption
# --------------------------------------------------------------------------
def test_keygen_relation_bruteforce(orc16):
    o = orc16
    N, L, P = o.N, o.L, o.P
    s, rk = o.s, o.rk
    assert set(np.unique(s)).issubset({-1, 0, 1})
    Q = math.prod(o.q)
    QP = Q * P
    sl = [int(v) for v in s]
    s2 = negacyclic_schoolbook(sl, sl, N)
    assert o.D == (L + 2) // 3 and rk.shape[0] == o.D
    for a in range(o.D):
        rk0 = to_ints(rk[a][0], o.q + [P])
        rk1 = to_ints(rk[a][1], o.q + [P])
        Qa = math.prod(o.q[3 * a:3 * a + 3])  # digit a: the group of primes 3a, 3a+1, 3a+2
        qh = Q // Qa
        g_a = qh * pow(qh, -1, Qa)
        lhs = [(a_ + b) % QP for a_, b in zip(rk0, negacyclic_schoolbook(rk1, sl, N))]
        err = [(v - P * g_a * w) % QP for v, w in zip(lhs, s2)]
        err = [e - QP if e > QP // 2 else e for e in err]
        assert max(abs(e) for e in err) <= 21  # centred binomial, eta = 21


def test_encrypt_relation_bruteforce(orc16):
    o = orc16
    N = o.N
    Q = math.prod(o.q)
    x = np.arange(N, dtype=np.uint32) * 977 % T
    ct = o.encrypt(x, seed=99, ct_index=3)
    c0, c1 = to_ints(ct[0], o.q), to_ints(ct[1], o.q)
    sl = [int(v) for v in o.s]
    m = [int(v) for v in o.encode(x)]
    ph = [(a + b) % Q for a, b in zip(c0, negacyclic_schoolbook(c1, sl, N))]
    err = [(v - (Q // T) * mm) % Q for v, mm in zip(ph, m)]
    err = [e - Q if e > Q // 2 else e for e in err]
    assert max(abs(e) for e in err) <= 21
    assert np.array_equal(o.decrypt(ct), x)
    # different ciphertext index -> different randomness, same plaintext
    ct2 = o.encrypt(x, seed=99, ct_index=4)
    assert not np.array_equal(ct, ct2) and np.array_equal(o.decrypt(ct2), x)


def _budget_bruteforce(o, ct):
    """Invariant noise budget from its definition with Python integers:
    log2(Q) - 1 - log2 max_k |[t (c0 + c1 s)_k]_Q| (centred), the phase taken
    with a schoolbook negacyclic product."""
    N, Q = o.N, math.prod(o.q)
    c0, c1 = to_ints(ct[0], o.q), to_ints(ct[1], o.q)
    ph = [(a + b) % Q for a, b in zip(c0, negacyclic_schoolbook(c1, [int(v) for v in o.s], N))]
    y = [(T * v) % Q for v in ph]
    worst = max(abs(v - Q if v > Q // 2 else v) for v in y)
    return math.log2(Q) - 1 - math.log2(worst), worst


def test_noise_budget_bruteforce(orc16):
    """The decryption's noise budget equals its definition, for a fresh
    ciphertext and after one product.  For a fresh ciphertext the closed form
    bounds it: c0 + c1 s = Delta m - e gives [t (c0 + c1 s)]_Q = -(Q mod t) m - t e,
    so |.| <= (Q mod t)(t - 1) + 21 t."""
    o = orc16
    Q = math.prod(o.q)
    rng = np.random.default_rng(31)
    x, y = rng.integers(0, T, o.N).astype(np.uint32), rng.integers(0, T, o.N).astype(np.uint32)
    cx, cy = o.encrypt(x, 32, 0), o.encrypt(y, 32, 1)
    _, nb = o.decrypt(cx, with_noise=True)
    want, worst = _budget_bruteforce(o, cx)
    assert abs(nb - want) < 1e-6
    assert worst <= (Q % T) * (T - 1) + 21 * T
    prod = o.mul_relin(cx, cy)
    _, nb2 = o.decrypt(prod, with_noise=True)
    assert abs(nb2 - _budget_bruteforce(o, prod)[0]) < 1e-6
    assert nb2 < nb


# --------------------------------------------------------------------------
# textbook multiplication and relinearisation: brute force on N = 16
# --------------------------------------------------------------------------
def _centered(v, Q):
    return v - Q if v > (Q - 1) // 2 else v


def test_tensor_and_rounding_bruteforce(orc16):
    o = orc16
    N, Q = o.N, math.prod(o.q)
    rng = np.random.default_rng(5)
    a = o.encrypt(rng.integers(0, T, N).astype(np.uint32), seed=1, ct_index=0)
    b = o.encrypt(rng.integers(0, T, N).astype(np.uint32), seed=1, ct_index=1)
    # also an adversarial pair: coefficients at the centring boundary (Q +- 1)/2
    edge = np.zeros_like(a)
    for i, qi in enumerate(o.q):
        edge[0, i, :] = ((Q - 1) // 2) % qi
        edge[1, i, :] = ((Q + 1) // 2) % qi
    for (x, y) in [(a, b), (a, a), (edge, a), (edge, edge)]:
        got = o.tensor_round(x, y)
        A0 = [_centered(v, Q) for v in to_ints(x[0], o.q)]
        A1 = [_centered(v, Q) for v in to_ints(x[1], o.q)]
        B0 = [_centered(v, Q) for v in to_ints(y[0], o.q)]
        B1 = [_centered(v, Q) for v in to_ints(y[1], o.q)]
        d = [negacyclic_schoolbook(A0, B0, N),
             [u + v for u, v in zip(negacyclic_schoolbook(A0, B1, N), negacyclic_schoolbook(A1, B0, N))],
             negacyclic_schoolbook(A1, B1, N)]
        for k in range(3):
            # round(t d / Q) with exact rationals (no ties: Q odd, gcd(Q, t) = 1)
            ref = []
            for v in d[k]:
                n2, den = 2 * T * v + Q, 2 * Q
                ref.append((n2 // den) % Q)
            assert to_ints(got[k], o.q) == ref


def test_relinearisation_bruteforce(orc16):
    o = orc16
    N, L, P = o.N, o.L, o.P
    Q = math.prod(o.q)
    QP = Q * P
    rng = np.random.default_rng(6)
    d3 = np.stack([np.stack([rng.integers(0, qi, N, dtype=np.uint64) for qi in o.q]) for _ in range(3)])
    got = o.relin(d3)
    D = [to_ints(d3[k], o.q) for k in range(3)]
    RK = [[to_ints(o.rk[a][c], o.q + [P]) for c in range(2)] for a in range(o.D)]
    out = []
    for c in range(2):
        u = [0] * N
        for a in range(o.D):
            Qa = math.prod(o.q[3 * a:3 * a + 3])
            dig = [v % Qa for v in D[2]]  # digit a = [d2]_{Q_a}
            u = [x + y for x, y in zip(u, negacyclic_schoolbook(dig, RK[a][c], N))]
        u = [v % QP for v in u]
        ks = []
        for v in u:
            r = v % P
            r = r - P if r > (P - 1) // 2 else r
            assert (v - r) % P == 0
            ks.append((v - r) // P)
        out.append([(a + b) % Q for a, b in zip(D[c], ks)])
    assert to_ints(got[0], o.q) == out[0]
    assert to_ints(got[1], o.q) == out[1]


def _relin_bruteforce(o, d3, rk, groups):
    """(d0, d1) + round(sum_a [d2]_{Q_a} rk_a / P) mod Q with Python integers and a
    schoolbook product; `groups`: the data-prime indices of each digit."""
    N, P, Q = o.N, o.P, math.prod(o.q)
    QP = Q * P
    D = [to_ints(d3[k], o.q) for k in range(3)]
    out = []
    for c in range(2):
        u = [0] * N
        for a, grp in enumerate(groups):
            Qa = math.prod(o.q[i] for i in grp)
            dig = [v % Qa for v in D[2]]
            u = [x + y for x, y in zip(u, negacyclic_schoolbook(dig, to_ints(rk[a][c], o.q + [P]), N))]
        ks = []
        for v in u:
            v %= QP
            r = v % P
            r = r - P if r > (P - 1) // 2 else r
            ks.append((v - r) // P)
        out.append([(a + b) % Q for a, b in zip(D[c], ks)])
    return out


def _key_relation_ok(o, rk, groups, s2):
    """rk_a0 + rk_a1 s = -e_a + P g_a s^2 mod QP with |e_a| <= 21, g_a = (Q/Q_a) [(Q/Q_a)^{-1}]_{Q_a}."""
    N, P, Q = o.N, o.P, math.prod(o.q)
    QP = Q * P
    sl = [int(v) for v in o.s]
    for a, grp in enumerate(groups):
        Qa = math.prod(o.q[i] for i in grp)
        g_a = (Q // Qa) * pow(Q // Qa, -1, Qa)
        rk0, rk1 = to_ints(rk[a][0], o.q + [P]), to_ints(rk[a][1], o.q + [P])
        lhs = [(x + y) % QP for x, y in zip(rk0, negacyclic_schoolbook(rk1, sl, N))]
        err = [(v - P * g_a * w) % QP for v, w in zip(lhs, s2)]
        if max(abs(e - QP if e > QP // 2 else e) for e in err) > 21:
            return False
    return True


@pytest.mark.parametrize("dp", [1, 2, 3, 5, 8])
def test_digit_groupings_keys_and_relinearisation_bruteforce(dp):
    """Key switching with digits of dp consecutive data primes (the last group
    shorter when dp does not divide L = 15): the keys satisfy their defining
    relation and relinearisation equals its integer definition, for each
    grouping."""
    o = oracle.Oracle(4, dp=dp)
    o.keygen(7)
    groups = [list(range(a * dp, min(o.L, (a + 1) * dp))) for a in range(o.D)]
    assert o.D == -(-o.L // dp) and o.rk.shape[0] == o.D
    sl = [int(v) for v in o.s]
    assert _key_relation_ok(o, o.rk, groups, negacyclic_schoolbook(sl, sl, o.N))
    rng = np.random.default_rng(60 + dp)
    d3 = np.stack([np.stack([rng.integers(0, qi, o.N, dtype=np.uint64) for qi in o.q]) for _ in range(3)])
    got = o.relin(d3)
    want = _relin_bruteforce(o, d3, o.rk, groups)
    assert to_ints(got[0], o.q) == want[0] and to_ints(got[1], o.q) == want[1]


def test_fine_depth_selects_the_per_prime_key_bruteforce():
    """With fine_depth F = 1 the oracle keeps a second relinearisation key of one
    prime per digit (its own relation holds) and relinearises a product of fresh
    ciphertexts (depth 1) with it, a product at depth 2 with the three-prime
    key: each equals tensor-and-round followed by the integer key switching of
    its key, by brute force."""
    check_fine_depth_selection()


def check_fine_depth_selection(lib_path=None):
    o = oracle.Oracle(4, fine_depth=1, lib_path=lib_path)
    o.keygen(7)
    fine = o.fine_key()
    sl = [int(v) for v in o.s]
    s2 = negacyclic_schoolbook(sl, sl, o.N)
    per_prime = [[i] for i in range(o.L)]
    three = [[3 * a, 3 * a + 1, 3 * a + 2] for a in range(5)]
    assert _key_relation_ok(o, fine, per_prime, s2)
    rng = np.random.default_rng(61)
    a = o.encrypt(rng.integers(0, T, o.N).astype(np.uint32), seed=3, ct_index=0)
    b = o.encrypt(rng.integers(0, T, o.N).astype(np.uint32), seed=3, ct_index=1)
    d3 = o.tensor_round(a, b)
    for depth_a, key, groups in [(0, fine, per_prime), (1, o.rk, three)]:
        got = o.mul_relin(a, b, depth_a=depth_a)
        want = _relin_bruteforce(o, d3, key, groups)
        assert to_ints(got[0], o.q) == want[0] and to_ints(got[1], o.q) == want[1], depth_a


def test_coarse_from_selects_the_two_digit_key_bruteforce():
    """With coarse_from C = 2 the oracle keeps a third relinearisation key of two
    digits (data primes 0..7 and 8..14; its own relation holds) and relinearises
    a product of fresh ciphertexts (depth 1) with the three-prime key, products
    at depth 2 and 3 with the two-digit key: each equals tensor-and-round
    followed by the integer key switching of its key, by brute force."""
    check_coarse_selection()


def check_coarse_selection(lib_path=None):
    o = oracle.Oracle(4, coarse_from=2, lib_path=lib_path)
    o.keygen(7)
    coarse = o.coarse_key()
    sl = [int(v) for v in o.s]
    s2 = negacyclic_schoolbook(sl, sl, o.N)
    two = [list(range(8)), list(range(8, o.L))]
    three = [[3 * a, 3 * a + 1, 3 * a + 2] for a in range(5)]
    assert _key_relation_ok(o, coarse, two, s2)
    rng = np.random.default_rng(62)
    a = o.encrypt(rng.integers(0, T, o.N).astype(np.uint32), seed=3, ct_index=0)
    b = o.encrypt(rng.integers(0, T, o.N).astype(np.uint32), seed=3, ct_index=1)
    d3 = o.tensor_round(a, b)
    for depth_a, key, groups in [(0, o.rk, three), (1, coarse, two), (2, coarse, two)]:
        got = o.mul_relin(a, b, depth_a=depth_a)
        want = _relin_bruteforce(o, d3, key, groups)
        assert to_ints(got[0], o.q) == want[0] and to_ints(got[1], o.q) == want[1], depth_a


def test_homomorphic_product_closed_form(orc16):
    o = orc16
    rng = np.random.default_rng(8)
    x = rng.integers(0, T, o.N).astype(np.uint32)
    y = rng.integers(0, T, o.N).astype(np.uint32)
    cx, cy = o.encrypt(x, 3, 0), o.encrypt(y, 3, 1)
    got, nb = o.decrypt(o.mul_relin(cx, cy), with_noise=True)
    assert np.array_equal(got, (x.astype(np.int64) * y % T).astype(np.uint32))
    # one product leaves most of the ~793-bit budget: key switching adds about
    # |digit| sqrt(N) / P = 2^(165 + 2 - 56) of noise, i.e. ~110 bits below Delta = 2^808
    assert nb > 680


# --------------------------------------------------------------------------
# EQ (Eq. equality) against the closed form [x == y]
# --------------------------------------------------------------------------
def _edge_pairs(N, rng):
    x = rng.integers(0, 2**16, N).astype(np.int64)
    y = np.where(rng.random(N) < 0.5, x, rng.integers(0, 2**16, N))
    cases = [(5, 5), (0, 0), (T - 1, T - 1), (6, 5), (5, 6), (0, T - 1), (T - 1, 0),
             ((T - 1) // 2, 0), (0, (T - 1) // 2), ((T + 1) // 2, 0), (1, 0), (0, 1), (65535, 65536)]
    for i, (a, b) in enumerate(cases):
        x[i], y[i] = a, b
    return x.astype(np.uint32), y.astype(np.uint32)


def test_eq_closed_form_n4096(orc4096):
    o = orc4096
    rng = np.random.default_rng(0)
    x, y = _edge_pairs(o.N, rng)
    cx, cy = o.encrypt(x, 10, 0), o.encrypt(y, 10, 1)
    ce = o.eq(cx, cy)
    got, nb = o.decrypt(ce, with_noise=True)
    assert np.array_equal(got, (x == y).astype(np.uint32))
    assert nb > 100  # 16 squarings stay well inside the budget (no bootstrapping)


def test_eq_const_closed_form(orc16):
    o = orc16
    x = np.array([7, 8, 7, 0, T - 1, 7, 6, 7] * (o.N // 8), dtype=np.uint32)
    cx = o.encrypt(x, 10, 0)
    got = o.decrypt(o.eq(cx, None, const_val=7))
    assert np.array_equal(got, (x == 7).astype(np.uint32))


def test_eq_plain_per_slot_constants(orc16):
    """Per-slot constants: closed form [x_j == c_j]; a uniform constant gives
    the same ciphertext as the broadcast form (encode(c, ..., c) = c)."""
    o = orc16
    rng = np.random.default_rng(9)
    x = rng.integers(0, 6, o.N).astype(np.uint32)
    c = rng.integers(0, 6, o.N).astype(np.uint32)
    cx = o.encrypt(x, 12, 0)
    got = o.decrypt(o.eq_plain(cx, c))
    assert np.array_equal(got, (x == c).astype(np.uint32))
    uni = np.full(o.N, 4, dtype=np.uint32)
    assert np.array_equal(o.eq_plain(cx, uni), o.eq(cx, None, const_val=4))


def test_eq_depth_is_sixteen(orc16):
    """Fewer squarings do not give the predicate: (x - y)^(2^k) for k < 16."""
    o = orc16
    x = np.full(o.N, 3, dtype=np.uint32)
    y = np.full(o.N, 1, dtype=np.uint32)
    cx, cy = o.encrypt(x, 4, 0), o.encrypt(y, 4, 1)
    got = o.decrypt(o.eq(cx, cy, squarings=4))
    assert np.all(got == (1 - pow(2, 16, T)) % T)
    got = o.decrypt(o.eq(cx, cy, squarings=16))
    assert np.all(got == 0)


def test_depth_overflow_decrypts_wrongly():
    """With a 3-prime modulus the noise budget runs out after a few squarings and
    decryption stops matching the plaintext closed form (leveled HE, Sec. 2.1.1-2.1.2)."""
    q, P = oracle.default_primes(15)
    o = oracle.Oracle(4, q=q[:3], P=P)
    o.keygen(3)
    x = np.arange(o.N, dtype=np.uint32) + 2
    cx = o.encrypt(x, 5, 0)
    ok_at = {}
    for k in [1, 2, 8]:
        got, nb = o.decrypt(o.square_chain(cx, k), with_noise=True)
        ok_at[k] = np.array_equal(got, np.array([pow(int(v), 2**k, T) for v in x], dtype=np.uint32))
    assert ok_at[1] and ok_at[2]
    assert not ok_at[8]


# --------------------------------------------------------------------------
# LT comparison (Eq. 4) -- the first row beyond equality
# --------------------------------------------------------------------------
def _lt_poly(h, z, p=T):
    """f(z) = z h(z^2) - ((p-1)/2) z^(p-1), by Horner over the odd coefficients."""
    w = z * z % p
    acc = 0
    for m in range(len(h) - 1, -1, -1):
        acc = (acc * w + int(h[m])) % p
    return (z * acc - (p - 1) // 2 * pow(w, (p - 1) // 2, p)) % p


def test_lt_polynomial_is_the_paper_sum(orc16):
    """The coefficients reproduce Eq. 4 as a function on F_p: f(z) = [z in {-(p-1)/2..-1}]."""
    h = orc16.lt_coefficients()
    assert len(h) == (T - 1) // 2
    rng = np.random.default_rng(11)
    zs = [0, 1, 2, T - 1, T - 2, (T - 1) // 2, (T + 1) // 2, (T - 3) // 2, (T + 3) // 2]
    zs += [int(v) for v in rng.integers(0, T, 12)]
    for z in zs:
        assert _lt_poly(h, z) == (1 if z >= (T + 1) // 2 else 0), z
    # direct evaluation of Eq. 4 (sum over a of 1 - (z - a)^(p-1)) at a few points
    for z in (0, 3, T - 3):
        direct = sum(1 - pow((z - a) % T, T - 1, T) for a in range(-(T - 1) // 2, 0)) % T
        assert _lt_poly(h, z) == direct


def test_linear_combination_closed_form(orc16):
    o = orc16
    rng = np.random.default_rng(12)
    xs = [rng.integers(0, T, o.N).astype(np.uint32) for _ in range(3)]
    cts = np.stack([o.encrypt(x, 13, i) for i, x in enumerate(xs)])
    coef = [5, T - 1, 40000]
    got = o.decrypt(o.linear(cts, coef, coef0=7))
    ref = (sum(int(k) * x.astype(object) for k, x in zip(coef, xs)) + 7) % T
    assert np.array_equal(got, ref.astype(np.uint32))


def test_lt_closed_form_n16(orc16):
    """Oracle LT decrypts to [x < y] for x, y in [0, 2^15] (the valid domain:
    the true difference must lie in [-(p-1)/2, (p-1)/2])."""
    o = orc16
    rng = np.random.default_rng(13)
    x = rng.integers(0, (T - 1) // 2 + 1, o.N).astype(np.uint32)
    y = rng.integers(0, (T - 1) // 2 + 1, o.N).astype(np.uint32)
    pairs = [(5, 3), (3, 5), (0, 32768), (32768, 0), (7, 7), (100, 101), (101, 100), (0, 0)]
    for i, (a, b) in enumerate(pairs):
        x[i], y[i] = a, b
    cx, cy = o.encrypt(x, 14, 0), o.encrypt(y, 14, 1)
    got, nb = o.decrypt(o.lt(cx, cy), with_noise=True)
    assert np.array_equal(got, (x < y).astype(np.uint32))
    assert nb > 0


def test_group_by_and_in_closed_form_n16(orc16):
    """GROUP BY masks decrypt to [x == c_k] per constant and IN (Eq. 6) to
    [x in S] for a set of distinct constants, including one absent value, the
    value 0 and p - 1; a repeated constant counts twice (the sum is a count)."""
    o = orc16
    rng = np.random.default_rng(15)
    consts = [0, 9, T - 1, 12345]
    x = rng.choice([0, 9, T - 1, 1, 2], o.N).astype(np.uint32)
    cx = o.encrypt(x, 16, 0)
    masks = o.group_by_masks(cx, consts)
    for k, c in enumerate(consts):
        assert np.array_equal(o.decrypt(masks[k]), (x == c).astype(np.uint32))
    got = o.decrypt(o.in_set(cx, consts, masks=masks))
    assert np.array_equal(got, np.isin(x, consts).astype(np.uint32))
    twice = o.decrypt(o.in_set(cx, [9, 9], masks=masks[[1, 1]]))
    assert np.array_equal(twice, 2 * (x == 9).astype(np.uint32))


# ---- rotations and the rotate-and-add reduction (COUNT / SUM, Sec. 4.2.2) ----
def _slot_exponents(logn):
    """Slot j is the evaluation at psi^(2 brv(j) + 1) (the batch-encoding order)."""
    N = 1 << logn
    return np.array([2 * int(format(j, "0%db" % logn)[::-1], 2) + 1 for j in range(N)])


def _slot_permutation(logn, g):
    """tau_g(m)(psi^e) = m(psi^(e g)): new slot j takes old slot of exponent e_j g mod 2N."""
    e = _slot_exponents(logn)
    where = {int(v): j for j, v in enumerate(e)}
    return np.array([where[int(v) * g % (2 << logn)] for v in e])


def _secret_automorph(s, g):
    N = len(s)
    out = np.zeros(N, dtype=np.int64)
    for j in range(N):
        e = j * g % (2 * N)
        if e < N:
            out[e] += s[j]
        else:
            out[e - N] -= s[j]
    return out.astype(np.int8)


@pytest.mark.parametrize("g", [3, 9, 5, 31])
def test_automorphism_permutes_slots(orc16, g):
    """tau_g(ct) decrypts under tau_g(s) to the slots permuted by e -> e g (mod 2N);
    tau_g(s) and the permutation are computed here from their definitions."""
    o = orc16
    rng = np.random.default_rng(20 + g)
    x = rng.integers(0, T, o.N).astype(np.uint32)
    ct = o.encrypt(x, 21, 0)
    got = o.decrypt(o.automorphism(ct, g), s=_secret_automorph(o.s, g))
    assert np.array_equal(got, x[_slot_permutation(o.logn, g)])


def test_rotation_with_galois_key(orc16):
    """Key switching with a Galois key brings tau_g(ct) back under s; the slots
    are the same permutation and the noise budget stays positive."""
    o = orc16
    rng = np.random.default_rng(22)
    x = rng.integers(0, T, o.N).astype(np.uint32)
    ct = o.encrypt(x, 23, 0)
    for g in o.galois_elements():
        o.galois_keygen(5, g)
        got, nb = o.decrypt(o.rotate(ct, g), with_noise=True)
        assert np.array_equal(got, x[_slot_permutation(o.logn, g)]), g
        assert nb > 0
    with pytest.raises(RuntimeError):
        o.rotate(ct, 7)  # no key for 7


def test_galois_elements_generate_the_rows():
    """3 has order N/2 mod 2N (one row), -1 is outside <3> (the other row)."""
    for logn in (4, 12, 15):
        twoN = 2 << logn
        powers, v = set(), 1
        for _ in range(twoN):
            powers.add(v)
            v = v * 3 % twoN
        assert len(powers) == (1 << logn) // 2 and twoN - 1 not in powers


def test_rotate_sum_paper_worked_example_n16(orc16):
    """Sec. 4.2.2's 8-slot example on one row of N = 16 (a row holds 8 slots,
    position r at exponent 3^r): rotate by 4 and add gives v_r + v_(r+4); by 2,
    v_r + v_(r+2) + v_(r+4) + v_(r+6); by 1, the row sum.  The row exchange then
    puts the sum of all 16 slots in every slot."""
    o = orc16
    N, twoN = o.N, 2 * o.N
    for g in o.galois_elements():
        o.galois_keygen(5, g)
    e = _slot_exponents(o.logn)
    where = {int(v): j for j, v in enumerate(e)}
    row0 = [where[pow(3, r, twoN)] for r in range(8)]
    row1 = [where[twoN - pow(3, r, twoN)] for r in range(8)]
    v = np.array([1, 10, 100, 1000, 7, 70, 700, 7000])
    w = np.array([3, 5, 11, 13, 17, 19, 23, 29])
    x = np.zeros(N, dtype=np.uint32)
    x[row0], x[row1] = v, w
    ct = o.encrypt(x, 24, 0)
    r = np.arange(8)
    step1 = o.decrypt(o.rotate_sum(ct, row_steps=1, swap=False))
    assert np.array_equal(step1[row0], v + v[(r + 4) % 8])
    step2 = o.decrypt(o.rotate_sum(ct, row_steps=2, swap=False))
    assert np.array_equal(step2[row0], v + v[(r + 2) % 8] + v[(r + 4) % 8] + v[(r + 6) % 8])
    step3 = o.decrypt(o.rotate_sum(ct, row_steps=3, swap=False))
    assert np.all(step3[row0] == v.sum()) and np.all(step3[row1] == w.sum())
    full = o.decrypt(o.rotate_sum(ct))
    assert np.all(full == (v.sum() + w.sum()) % T)


def test_count_and_sum_closed_form_n16(orc16):
    """COUNT = rotate-sum of an EQ mask, SUM = rotate-sum of column x mask (Eq. 5),
    both mod p in every slot."""
    o = orc16
    for g in o.galois_elements():
        o.galois_keygen(5, g)
    rng = np.random.default_rng(25)
    key = rng.integers(0, 4, o.N).astype(np.uint32)
    price = rng.integers(0, T, o.N).astype(np.uint32)
    ck, cp = o.encrypt(key, 26, 0), o.encrypt(price, 26, 1)
    mask = o.eq(ck, None, const_val=2)
    count, nb = o.decrypt(o.rotate_sum(mask), with_noise=True)
    assert np.all(count == int((key == 2).sum())) and nb > 0
    total = o.decrypt(o.rotate_sum(o.mul_relin(cp, mask)))
    assert np.all(total == int(price[key == 2].astype(np.int64).sum() % T))


# ---- JOIN by Extract + Broadcast (Sec. 4.2.2) ----
def test_mul_plain_is_slotwise_product(orc16):
    o = orc16
    rng = np.random.default_rng(30)
    x = rng.integers(0, T, o.N).astype(np.uint32)
    v = rng.integers(0, T, o.N).astype(np.uint32)
    v[:3] = [0, 1, T - 1]
    got = o.decrypt(o.mul_plain(o.encrypt(x, 31, 0), o.encode(v)))
    assert np.array_equal(got, (x.astype(np.int64) * v % T).astype(np.uint32))


def test_extract_broadcast_n16(orc16):
    o = orc16
    for g in o.galois_elements():
        o.galois_keygen(5, g)
    rng = np.random.default_rng(32)
    x = rng.integers(0, T, 2 * o.N).astype(np.uint32)
    col = np.stack([o.encrypt(x[:o.N], 33, 0), o.encrypt(x[o.N:], 33, 1)])
    for row in (0, 5, o.N - 1, o.N + 3):
        got, nb = o.decrypt(o.extract_broadcast(col, row), with_noise=True)
        assert np.all(got == x[row]) and nb > 0, row


def test_join_closed_form_n16(orc16):
    """SELECT size, brand FROM A, B WHERE A.key = B.key with unique B keys:
    each A row gets the attributes of its matching B row, 0 without a match;
    the attribute-free form (semi-join) gives the number of matches."""
    o = orc16
    for g in o.galois_elements():
        o.galois_keygen(5, g)
    N = o.N
    rng = np.random.default_rng(34)
    bkey = np.zeros(N, dtype=np.uint32)
    bkey[:3] = [7, 42, 65000]
    size = np.zeros(N, dtype=np.uint32)
    size[:3] = [11, 22, 33]
    brand = np.zeros(N, dtype=np.uint32)
    brand[:3] = [100, 200, 300]
    akey = rng.choice([7, 42, 65000, 5], N).astype(np.uint32)
    ca = o.encrypt(akey, 35, 0)[None]
    cb = o.encrypt(bkey, 35, 1)[None]
    cs, cbr = o.encrypt(size, 35, 2)[None], o.encrypt(brand, 35, 3)[None]
    out = o.join(ca, cb, [cs, cbr], 3)
    for k, attr in enumerate((size, brand)):
        ref = np.zeros(N, dtype=np.uint32)
        for r in range(3):
            ref[akey == bkey[r]] = attr[r]
        got, nb = o.decrypt(out[k, 0], with_noise=True)
        assert np.array_equal(got, ref) and nb > 0, k
    semi = o.join(ca, cb, [], 3)
    assert np.array_equal(o.decrypt(semi[0, 0]), np.isin(akey, bkey[:3]).astype(np.uint32))


def test_between_closed_form_n16(orc16):
    """BETWEEN (Sec. 4.2.2) decrypts to [lo <= x <= hi] on 15-bit inputs,
    including both bounds and lo = hi, and equals the product (1 - LT(x, lo))
    (1 - LT(hi, x)) of the two comparisons slot by slot, checked here after
    decryption; an empty range (lo > hi) is rejected."""
    o = orc16
    rng = np.random.default_rng(40)
    x = rng.integers(0, (T - 1) // 2 + 1, o.N).astype(np.uint32)
    x[:6] = [100, 200, 99, 201, 0, 32768]
    cx = o.encrypt(x, 41, 0)
    for lo, hi in [(100, 200), (0, 32768), (150, 150)]:
        got, nb = o.decrypt(o.between(cx, lo, hi), with_noise=True)
        assert np.array_equal(got, ((x >= lo) & (x <= hi)).astype(np.uint32)), (lo, hi)
        assert nb > 0
        a = o.decrypt(o.lt(cx, o.encrypt(np.full(o.N, lo, dtype=np.uint32), 42, 1)))
        b = o.decrypt(o.lt(o.encrypt(np.full(o.N, hi, dtype=np.uint32), 42, 2), cx))
        assert np.array_equal(got, ((1 - a.astype(np.int64)) * (1 - b.astype(np.int64)) % T).astype(np.uint32))
    with pytest.raises(RuntimeError):
        o.between(cx, 300, 200)
