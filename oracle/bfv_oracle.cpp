// Textbook BFV oracle for the homomorphic equality predicate of NSHEDB.
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
// this file; only the tests, the smoke check and the CPU-baseline leg of the
// benchmark do.  It shares no code, header, table or constant generator with
// the CUDA library.
//
// What it computes (paper: Sec. 2.1.7 "Basic logical comparisons", Eq. 3;
// Sec. 4.3.1 "Equality checks" for exponentiation by squaring; Sec. 5.1 for the
// parameters N = 32768, log QP = 881, p = 65537):
//
//   EQ(ct_x, ct_y) = 1 - (ct_x - ct_y)^(p-1),  p - 1 = 2^16  =>  16 squarings.
//
// Every ciphertext operation is written as its plain integer definition
// (Fan-Vercauteren 2012 textbook BFV; relinearisation with digits over groups of
// three data primes and one special prime, Gentry-Halevi-Smart 2012):
//
//   * coefficients are big integers in [0, Q) (Q = q_0 ... q_{L-1});
//   * multiplication lifts every coefficient to (-Q/2, Q/2], forms the exact
//     integer negacyclic products d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1,
//     then maps d -> round(t d / Q) mod Q;
//   * relinearisation: digit_a = [d2]_{Q_a} with Q_a = q_3a q_3a+1 q_3a+2 (five
//     digits for L = 15), u = sum_a digit_a rk_a mod QP, (c0, c1) += round(u / P)
//     mod Q (the paper fixes only log QP = 881, Sec. 5.1; SEAL's own
//     decomposition is internal to it).
//
// The exact integer polynomial products are computed by a multi-modular
// negacyclic NTT over the oracle's OWN 61-bit primes followed by Garner CRT
// reconstruction; a product is exact because the CRT modulus exceeds twice
// the largest possible coefficient.  Big-integer arithmetic is a small
// fixed-width sign-magnitude type written here.  Plain, slow, single-threaded.
// Planted mistakes (mutation tests).  The normal build leaves ORC_MUTANT at 0
// and none of them is compiled in.  tests/test_oracle_mutants.py builds separate
// copies with -DORC_MUTANT=k, each containing one plausible mistake, and checks
// that a pin of this oracle fails on that copy:
//   1 round(t d / Q) truncated toward zero instead of rounded
//   2 the cross term a1 b0 dropped from d1
//   3 the mod-down remainder taken in [0, P) instead of centred
//   4 the negacyclic twist left out (cyclic products)
//   5 the sign of (a s + e) in the key-switching keys flipped
//   6 slots read in natural instead of bit-reversed transform order
//   7 key-switching digit a taken mod q_3a alone instead of mod Q_a
//   8 one squaring too few in the EQ chain
//   9 LT coefficients taken from the even powers (b^(p-1-2m) for c_{2m+1})
//  10 the automorphism's negacyclic sign dropped (X^N taken as +1)
//  11 the rotate-and-add reduction without its row exchange
//  12 BETWEEN's first factor taken as a instead of 1 - a
//  13 LT's first giant step taken as w^128 instead of w^256
//  14 the noise budget without the factor 2 of its definition
//  15 the per-prime relinearisation key used only below the fine depth, not at it
//  16 the two-digit relinearisation key used from one level after its first depth
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <cstdio>
#include <cmath>
#include <map>
#include <vector>
#include <algorithm>

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// word-size modular arithmetic
// ---------------------------------------------------------------------------
// (hi 2^64 + lo) = q d + r with hi < d, so the quotient fits in 64 bits
static inline uint64_t div_2by1(uint64_t hi, uint64_t lo, uint64_t d, uint64_t* r) {
#if defined(__x86_64__)
  uint64_t q, rr;
  __asm__("divq %4" : "=a"(q), "=d"(rr) : "a"(lo), "d"(hi), "rm"(d));
  *r = rr;
  return q;
#else
  u128 cur = ((u128)hi << 64) | lo;
  *r = (uint64_t)(cur % d);
  return (uint64_t)(cur / d);
#endif
}
// a b mod m for a, b < m < 2^63
static inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) {
  u128 x = (u128)a * b;
  uint64_t r;
  div_2by1((uint64_t)(x >> 64), (uint64_t)x, m, &r);
  return r;
}
static inline uint64_t addmod(uint64_t a, uint64_t b, uint64_t m) {
  uint64_t r = a + b;  // a, b < m < 2^63
  return r >= m ? r - m : r;
}
static inline uint64_t submod(uint64_t a, uint64_t b, uint64_t m) {
  return a >= b ? a - b : a + m - b;
}
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod(r, a, m);
    a = mulmod(a, a, m);
    e >>= 1;
  }
  return r;
}
static uint64_t invmod(uint64_t a, uint64_t m) {  // m prime
  return powmod(a, m - 2, m);
}

// Shoup's precomputed-quotient multiplication by a fixed w (< m):
// wp = floor(w 2^64 / m).  Result is reduced to [0, m).
struct Shoup {
  uint64_t w, wp;
};
static inline Shoup shoup_make(uint64_t w, uint64_t m) {
  Shoup s;
  s.w = w;
  s.wp = (uint64_t)(((u128)w << 64) / m);
  return s;
}
static inline uint64_t mulmod_shoup(uint64_t a, const Shoup& s, uint64_t m) {
  uint64_t qh = (uint64_t)(((u128)a * s.wp) >> 64);
  uint64_t r = a * s.w - qh * m;
  while (r >= m) r -= m;
  return r;
}

// Deterministic Miller-Rabin for n < 2^64 (bases: first twelve primes).
static bool is_prime_u64(uint64_t n) {
  if (n < 2) return false;
  static const uint64_t small[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (uint64_t p : small) {
    if (n % p == 0) return n == p;
  }
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; ++s; }
  for (uint64_t a : small) {
    uint64_t x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = mulmod(x, x, n);
      if (x == n - 1) { comp = false; break; }
    }
    if (comp) return false;
  }
  return true;
}

// Largest `count` primes strictly below 2^bits with p = 1 (mod 2^mod_log2),
// in descending order.
static std::vector<uint64_t> primes_below(int bits, int mod_log2, int count) {
  std::vector<uint64_t> out;
  uint64_t step = 1ULL << mod_log2;
  uint64_t top = 1ULL << bits;
  uint64_t k = (top - 2) / step;  // largest k with k*step + 1 < top
  for (; k > 0 && (int)out.size() < count; --k) {
    uint64_t c = k * step + 1;
    if (is_prime_u64(c)) out.push_back(c);
  }
  return out;
}

// Smallest quadratic non-residue g mod prime m (g^((m-1)/2) = -1).  For
// 2N | m - 1, psi = g^((m-1)/(2N)) then satisfies psi^N = -1, i.e. it is a
// primitive 2N-th root of unity.  For m = 65537 this gives g = 3.
static uint64_t smallest_qnr(uint64_t m) {
  for (uint64_t g = 2;; ++g)
    if (powmod(g, (m - 1) / 2, m) == m - 1) return g;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), restated from its
// published definition: ten rounds of two 32x32->64 multiplies and a Weyl
// key schedule.
// ---------------------------------------------------------------------------
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Sampling domains: every random draw of the scheme is philox(seed; counter =
// (coefficient k, prime index j, object index, domain)).
// Galois keys (domains 6, 7) use object index (g << 5) | digit for Galois
// element g, so a key does not depend on which other elements are generated.
enum { DOM_S = 1, DOM_E_ENC = 2, DOM_A_ENC = 3, DOM_E_RK = 4, DOM_A_RK = 5, DOM_E_GK = 6, DOM_A_GK = 7 };

static void draw(uint64_t seed, uint32_t k, uint32_t j, uint32_t obj, uint32_t dom, uint32_t w[4]) {
  uint32_t ctr[4] = {k, j, obj, dom};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox4x32_10(ctr, key, w);
}
// ternary secret coefficient in {-1, 0, 1}: floor(3 w0 / 2^32) - 1
static int sample_ternary(const uint32_t w[4]) { return (int)(((uint64_t)w[0] * 3) >> 32) - 1; }
// centred binomial, eta = 21: popcount of 21 bits minus popcount of 21 bits
static int sample_cbd21(const uint32_t w[4]) {
  return __builtin_popcount(w[0] & 0x1FFFFFu) - __builtin_popcount(w[1] & 0x1FFFFFu);
}
// uniform residue mod m: floor(r m / 2^128), r = w3:w2:w1:w0 (128 bits)
static uint64_t sample_uniform(const uint32_t w[4], uint64_t m) {
  uint64_t lo = ((uint64_t)w[1] << 32) | w[0];
  uint64_t hi = ((uint64_t)w[3] << 32) | w[2];
  u128 a = (u128)lo * m;  // r m = hi m 2^64 + lo m
  u128 b = (u128)hi * m;
  u128 s = b + (a >> 64);
  return (uint64_t)(s >> 64);
}

// ---------------------------------------------------------------------------
// Fixed-width sign-magnitude big integers (64-bit limbs, little endian).
// ---------------------------------------------------------------------------
enum { BW = 34 };  // 2176 bits: enough for every exact product used here
struct Big {
  uint64_t w[BW];
  int n;    // number of significant limbs, 0 = zero
  int neg;  // 1 if negative (only when n > 0)
};

static void fail(const char* msg) {
  fprintf(stderr, "oracle: %s\n", msg);
  abort();
}
static inline void big_norm(Big& a) {
  while (a.n > 0 && a.w[a.n - 1] == 0) --a.n;
  if (a.n == 0) a.neg = 0;
}
static inline Big big_zero() {
  Big r;
  r.n = 0;
  r.neg = 0;
  return r;
}
static inline Big big_u64(uint64_t v) {
  Big r = big_zero();
  if (v) { r.w[0] = v; r.n = 1; }
  return r;
}
static inline bool big_is_zero(const Big& a) { return a.n == 0; }
static int mag_cmp(const Big& a, const Big& b) {
  if (a.n != b.n) return a.n < b.n ? -1 : 1;
  for (int i = a.n - 1; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}
static Big mag_add(const Big& a, const Big& b) {
  Big r = big_zero();
  int n = std::max(a.n, b.n);
  uint64_t carry = 0;
  for (int i = 0; i < n; ++i) {
    u128 s = (u128)(i < a.n ? a.w[i] : 0) + (i < b.n ? b.w[i] : 0) + carry;
    r.w[i] = (uint64_t)s;
    carry = (uint64_t)(s >> 64);
  }
  if (carry) {
    if (n >= BW) fail("big overflow (add)");
    r.w[n++] = carry;
  }
  r.n = n;
  big_norm(r);
  return r;
}
static Big mag_sub(const Big& a, const Big& b) {  // |a| >= |b|
  Big r = big_zero();
  uint64_t borrow = 0;
  for (int i = 0; i < a.n; ++i) {
    uint64_t bi = i < b.n ? b.w[i] : 0;
    uint64_t d = a.w[i] - bi - borrow;
    borrow = (a.w[i] < bi || (a.w[i] == bi && borrow)) ? 1 : 0;
    r.w[i] = d;
  }
  if (borrow) fail("big underflow (sub)");
  r.n = a.n;
  big_norm(r);
  return r;
}
static Big big_add(const Big& a, const Big& b) {
  Big r;
  if (a.neg == b.neg) {
    r = mag_add(a, b);
    r.neg = a.n || b.n ? a.neg : 0;
  } else {
    int c = mag_cmp(a, b);
    if (c == 0) return big_zero();
    if (c > 0) { r = mag_sub(a, b); r.neg = a.neg; }
    else { r = mag_sub(b, a); r.neg = b.neg; }
  }
  big_norm(r);
  return r;
}
static Big big_neg(Big a) {
  if (a.n) a.neg ^= 1;
  return a;
}
static Big big_sub(const Big& a, const Big& b) { return big_add(a, big_neg(b)); }
static Big big_mul_u64(const Big& a, uint64_t m) {
  Big r = big_zero();
  if (a.n == 0 || m == 0) return r;
  uint64_t carry = 0;
  for (int i = 0; i < a.n; ++i) {
    u128 p = (u128)a.w[i] * m + carry;
    r.w[i] = (uint64_t)p;
    carry = (uint64_t)(p >> 64);
  }
  r.n = a.n;
  if (carry) {
    if (r.n >= BW) fail("big overflow (mul_u64)");
    r.w[r.n++] = carry;
  }
  r.neg = a.neg;
  big_norm(r);
  return r;
}
static Big big_mul(const Big& a, const Big& b) {
  Big r = big_zero();
  if (a.n == 0 || b.n == 0) return r;
  if (a.n + b.n > BW) fail("big overflow (mul)");
  for (int i = 0; i < a.n + b.n; ++i) r.w[i] = 0;
  for (int i = 0; i < a.n; ++i) {
    uint64_t carry = 0;
    for (int j = 0; j < b.n; ++j) {
      u128 p = (u128)a.w[i] * b.w[j] + r.w[i + j] + carry;
      r.w[i + j] = (uint64_t)p;
      carry = (uint64_t)(p >> 64);
    }
    r.w[i + b.n] = carry;
  }
  r.n = a.n + b.n;
  r.neg = a.neg ^ b.neg;
  big_norm(r);
  return r;
}
// quotient of |a| by d; remainder in *rem (of |a|)
static Big mag_divmod_u64(const Big& a, uint64_t d, uint64_t* rem) {
  Big q = big_zero();
  uint64_t r = 0;
  for (int i = a.n - 1; i >= 0; --i) q.w[i] = div_2by1(r, a.w[i], d, &r);
  q.n = a.n;
  big_norm(q);
  if (rem) *rem = r;
  return q;
}
// residue of signed a modulo m, in [0, m)
static uint64_t big_mod_u64(const Big& a, uint64_t m) {
  uint64_t r = 0;
  for (int i = a.n - 1; i >= 0; --i) div_2by1(r, a.w[i], m, &r);
  if (a.neg && r) r = m - r;
  return r;
}
static int big_bits(const Big& a) {
  if (a.n == 0) return 0;
  return 64 * (a.n - 1) + (64 - __builtin_clzll(a.w[a.n - 1]));
}
// log2 |a| as a double (for noise reporting only)
static double big_log2(const Big& a) {
  if (a.n == 0) return -INFINITY;
  double top = (double)a.w[a.n - 1];
  if (a.n >= 2) top += (double)a.w[a.n - 2] / 18446744073709551616.0;
  return std::log2(top) + 64.0 * (a.n - 1);
}
// floor(|a| / (m_0 m_1 ... m_{k-1})) by successive single-word divisions
static Big mag_floordiv_primes(const Big& a, const std::vector<uint64_t>& ms) {
  Big q = a;
  q.neg = 0;
  for (uint64_t m : ms) q = mag_divmod_u64(q, m, nullptr);
  return q;
}

// ---------------------------------------------------------------------------
// Garner CRT reconstruction over a fixed list of word primes.
// ---------------------------------------------------------------------------
struct Crt {
  std::vector<uint64_t> m;                 // moduli
  std::vector<std::vector<Shoup>> inv;     // inv[i][j] = m_i^{-1} mod m_j (i < j)
  Big M, Mhalf;                            // product, floor(M/2)
  void init(const std::vector<uint64_t>& mods) {
    m = mods;
    size_t k = m.size();
    inv.assign(k, std::vector<Shoup>(k));
    for (size_t i = 0; i < k; ++i)
      for (size_t j = i + 1; j < k; ++j) inv[i][j] = shoup_make(invmod(m[i] % m[j], m[j]), m[j]);
    M = big_u64(1);
    for (uint64_t x : m) M = big_mul_u64(M, x);
    uint64_t r;
    Mhalf = mag_divmod_u64(M, 2, &r);
  }
  // residues r[i] in [0, m_i)  ->  X in [0, M)
  Big reconstruct(const uint64_t* r) const {
    size_t k = m.size();
    uint64_t a[64];
    for (size_t j = 0; j < k; ++j) {
      uint64_t t = r[j];
      for (size_t i = 0; i < j; ++i) t = mulmod_shoup(submod(t, a[i] % m[j], m[j]), inv[i][j], m[j]);
      a[j] = t;
    }
    Big x = big_u64(a[k - 1]);
    for (size_t j = k - 1; j-- > 0;) {  // x = x m_j + a_j
      uint64_t carry = a[j];
      for (int i = 0; i < x.n; ++i) {
        u128 p = (u128)x.w[i] * m[j] + carry;
        x.w[i] = (uint64_t)p;
        carry = (uint64_t)(p >> 64);
      }
      if (carry) {
        if (x.n >= BW) fail("big overflow (crt)");
        x.w[x.n++] = carry;
      }
    }
    return x;
  }
  // same, mapped to the symmetric range (-M/2, M/2]
  Big reconstruct_centered(const uint64_t* r) const {
    Big x = reconstruct(r);
    if (mag_cmp(x, Mhalf) > 0) x = big_sub(x, M);
    return x;
  }
};

// ---------------------------------------------------------------------------
// Negacyclic NTT over a word prime m with 2N | m - 1:
//   forward:  A_j = sum_k a_k psi^{(2j+1) k}   (j in natural order)
//   inverse:  a_k = N^{-1} psi^{-k} sum_j A_j psi^{-2jk}
// implemented as twist by psi^k, then a textbook iterative radix-2 cyclic
// transform with omega = psi^2 (bit-reversal permutation, then butterflies).
// ---------------------------------------------------------------------------
struct NttPlan {
  int logn, n;
  uint64_t m;
  std::vector<Shoup> tw, itw;   // twist psi^k, psi^{-k} * N^{-1}
  std::vector<Shoup> w, iw;     // omega^k, omega^{-k}, k < N/2
  void init(int logn_, uint64_t mod) {
    logn = logn_;
    n = 1 << logn;
    m = mod;
    if ((m - 1) % (2ULL * n) != 0) fail("prime does not support this ring degree");
    uint64_t g = smallest_qnr(m);
    uint64_t psi = powmod(g, (m - 1) / (2ULL * n), m);
    uint64_t ipsi = invmod(psi, m);
    uint64_t omega = mulmod(psi, psi, m), iomega = invmod(omega, m);
    uint64_t ninv = invmod((uint64_t)n % m, m);
    tw.resize(n); itw.resize(n);
    uint64_t p = 1, ip = ninv;
    for (int k = 0; k < n; ++k) {
      tw[k] = shoup_make(p, m);
      itw[k] = shoup_make(ip, m);
      p = mulmod(p, psi, m);
      ip = mulmod(ip, ipsi, m);
    }
    w.resize(n / 2); iw.resize(n / 2);
    uint64_t x = 1, ix = 1;
    for (int k = 0; k < n / 2; ++k) {
      w[k] = shoup_make(x, m);
      iw[k] = shoup_make(ix, m);
      x = mulmod(x, omega, m);
      ix = mulmod(ix, iomega, m);
    }
  }
  void cyclic(uint64_t* a, const std::vector<Shoup>& ws) const {
    for (int i = 1, j = 0; i < n; ++i) {  // bit-reversal permutation
      int bit = n >> 1;
      for (; j & bit; bit >>= 1) j ^= bit;
      j ^= bit;
      if (i < j) std::swap(a[i], a[j]);
    }
    for (int len = 2; len <= n; len <<= 1) {
      int half = len >> 1, stride = n / len;
      for (int s = 0; s < n; s += len)
        for (int k = 0; k < half; ++k) {
          uint64_t u = a[s + k];
          uint64_t v = mulmod_shoup(a[s + k + half], ws[k * stride], m);
          a[s + k] = addmod(u, v, m);
          a[s + k + half] = submod(u, v, m);
        }
    }
  }
  void forward(uint64_t* a) const {
#if ORC_MUTANT != 4
    for (int k = 0; k < n; ++k) a[k] = mulmod_shoup(a[k], tw[k], m);
#endif
    cyclic(a, w);
  }
  void inverse(uint64_t* a) const {
    cyclic(a, iw);
#if ORC_MUTANT == 4
    for (int k = 0; k < n; ++k) a[k] = mulmod_shoup(a[k], itw[0], m);  // N^{-1} only
#else
    for (int k = 0; k < n; ++k) a[k] = mulmod_shoup(a[k], itw[k], m);
#endif
  }
};

static int brv(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// ---------------------------------------------------------------------------
// Oracle context
// ---------------------------------------------------------------------------
typedef std::vector<Big> Poly;  // N big-integer coefficients

// A key-switching key from a secret s' to s: k_a = (-(a_a s + e_a) + P g_a s',
// a_a) mod QP for the digits a < D, one special prime.  Digit a is the residue
// modulo Q_a, the product of the a-th group of `dp` consecutive data primes (the
// last group is shorter when dp does not divide L).  The key is kept in
// big-integer form and transformed over the oracle primes used for the exact
// products.
struct KsKey {
  int dp = 0, D = 0;                        // data primes per digit, digits
  std::vector<std::vector<uint64_t>> grp;   // the primes of each digit
  std::vector<Big> Qa;                      // their products
  std::vector<Poly> k0, k1;
  int nprimes = 0;
  std::vector<uint64_t> ntt;      // [i][comp][prime][N]
};

// Key-switching digit groupings.  The relinearisation and Galois keys use
// groups of c.dp data primes (3 unless set otherwise).  Products whose output
// lies at multiplicative depth <= c.fine_depth are relinearised with a second
// key of one prime per digit (the decomposition of SEAL): its key-switching
// noise |digit| sqrt(N) / P is about 2^-110 of the three-prime key's, which
// matters only while the product's own noise is still small, i.e. at the first
// levels of a chain.
enum { DIGIT_PRIMES_DEFAULT = 3, FINE_OBJ = 16 };  // fine key digits draw with object index 16 + i
// Products whose output lies at depth >= c.coarse_from (0 = never) are
// relinearised with a third key of two digits, the data primes 0..7 and 8..14:
// its key-switching noise |digit| sqrt(N) / P (|digit| < 2^440) is far above the
// other keys', which matters only while it is not below the product's own noise,
// i.e. it costs nothing once a chain is deep enough.
enum { COARSE_DIGIT_PRIMES = 8, COARSE_OBJ = 48 };  // coarse key digits draw with object index 48 + a

struct Ctx {
  int logn, N, L;
  uint64_t t, P;
  std::vector<uint64_t> q;        // data primes (Q = prod q)
  std::vector<uint64_t> qp;       // q_0..q_{L-1}, P
  Big Q, QP, Qhalf, Delta;        // Qhalf = (Q-1)/2, Delta = floor(Q/t)
  Crt crtQ, crtQP;                // reconstruction from the scheme's own primes
  std::vector<uint64_t> om;       // oracle product primes (61-bit)
  std::vector<NttPlan> plans;     // one per oracle prime
  NttPlan tplan;                  // plaintext-modulus transform (batch encoding)
  std::vector<Crt> crt_prefix;    // crt over the first k oracle primes, k = 1..
  // key-switching digit groupings (see KsKey): dp data primes per digit for the
  // relinearisation and Galois keys; products at output depth <= fine_depth
  // use the per-prime relinearisation key rk1
  int dp = DIGIT_PRIMES_DEFAULT, fine_depth = 0;
  // products at output depth >= coarse_from (0 = never) use the two-digit key rk2
  int coarse_from = 0;
  // relinearisation keys and Galois keys (switching from s^2, resp. tau_g(s), to s)
  bool have_rk = false, have_rk1 = false, have_rk2 = false;
  KsKey rk, rk1, rk2;
  std::map<uint64_t, KsKey> gk;   // by Galois element g
  std::vector<uint32_t> lt_h;     // LT polynomial's odd coefficients (computed on first use)
};

static int primes_needed(const Ctx& c, int bound_bits) {
  // smallest k such that prod of first k oracle primes > 2^(bound_bits + 1)
  double acc = 0;
  for (size_t k = 0; k < c.om.size(); ++k) {
    acc += std::log2((double)c.om[k]);
    if (acc > bound_bits + 2) return (int)k + 1;
  }
  fail("not enough oracle primes for exact product");
  return 0;
}
static int poly_max_bits(const Poly& a) {
  int b = 0;
  for (const Big& x : a) b = std::max(b, big_bits(x));
  return b;
}

// A sum of products  sum_t a_t * b_t  in Z[X]/(X^N + 1).
typedef std::vector<std::pair<const Poly*, const Poly*>> Terms;

// Exact values of several such sums (signed big-integer coefficients).  The
// sums share the transforms of repeated operands; otherwise each is computed
// independently: residues mod each oracle prime, forward transform, pointwise
// multiply-accumulate, inverse transform, CRT.
static std::vector<Poly> poly_sums_exact(const Ctx& c, const std::vector<Terms>& sums) {
  int N = c.N;
  std::vector<const Poly*> ops;
  auto slot = [&](const Poly* p) {
    for (size_t u = 0; u < ops.size(); ++u)
      if (ops[u] == p) return (int)u;
    ops.push_back(p);
    return (int)ops.size() - 1;
  };
  int bound = 0;
  std::vector<std::vector<std::pair<int, int>>> idx(sums.size());
  for (size_t s = 0; s < sums.size(); ++s) {
    int ba = 0, bb = 0;
    for (auto& tm : sums[s]) {
      ba = std::max(ba, poly_max_bits(*tm.first));
      bb = std::max(bb, poly_max_bits(*tm.second));
      idx[s].push_back({slot(tm.first), slot(tm.second)});
    }
    int terms = (int)sums[s].size();
    bound = std::max(bound, ba + bb + c.logn + (int)std::ceil(std::log2((double)terms + 1)) + 1);
  }
  int k = primes_needed(c, bound);
  std::vector<std::vector<uint64_t>> res(sums.size(), std::vector<uint64_t>((size_t)k * N));
  std::vector<std::vector<uint64_t>> T(ops.size(), std::vector<uint64_t>(N));
  std::vector<uint64_t> acc(N);
  for (int pi = 0; pi < k; ++pi) {
    uint64_t m = c.om[pi];
    for (size_t u = 0; u < ops.size(); ++u) {
      for (int j = 0; j < N; ++j) T[u][j] = big_mod_u64((*ops[u])[j], m);
      c.plans[pi].forward(T[u].data());
    }
    for (size_t s = 0; s < sums.size(); ++s) {
      std::fill(acc.begin(), acc.end(), 0);
      for (auto& ab : idx[s]) {
        const uint64_t* A = T[ab.first].data();
        const uint64_t* B = T[ab.second].data();
        for (int j = 0; j < N; ++j) acc[j] = addmod(acc[j], mulmod(A[j], B[j], m), m);
      }
      c.plans[pi].inverse(acc.data());
      for (int j = 0; j < N; ++j) res[s][(size_t)j * k + pi] = acc[j];
    }
  }
  std::vector<Poly> out(sums.size(), Poly(N));
  const Crt& crt = c.crt_prefix[k - 1];
  for (size_t s = 0; s < sums.size(); ++s)
    for (int j = 0; j < N; ++j) out[s][j] = crt.reconstruct_centered(&res[s][(size_t)j * k]);
  return out;
}
static Poly poly_mul_exact(const Ctx& c, const Poly& a, const Poly& b) {
  return poly_sums_exact(c, {Terms{{&a, &b}}})[0];
}
// exact tensor of (a0, a1) and (b0, b1): d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1
static std::vector<Poly> tensor_exact(const Ctx& c, const Poly& a0, const Poly& a1, const Poly& b0, const Poly& b1) {
#if ORC_MUTANT == 2
  return poly_sums_exact(c, {Terms{{&a0, &b0}}, Terms{{&a0, &b1}}, Terms{{&a1, &b1}}});
#else
  return poly_sums_exact(c, {Terms{{&a0, &b0}}, Terms{{&a0, &b1}, {&a1, &b0}}, Terms{{&a1, &b1}}});
#endif
}

// canonical representative in [0, M) of a signed integer, M = prod(ms)
static Big mod_primes(const Big& x, const Big& M, const std::vector<uint64_t>& ms) {
  Big a = x;
  a.neg = 0;
  Big quo = mag_floordiv_primes(a, ms);
  Big r = big_sub(a, big_mul(quo, M));  // |x| mod M
  if (x.neg && !big_is_zero(r)) r = big_sub(M, r);
  return r;
}
static Big mod_Q(const Ctx& c, const Big& x) { return mod_primes(x, c.Q, c.q); }
static Big mod_QP(const Ctx& c, const Big& x) { return mod_primes(x, c.QP, c.qp); }
// representative of x in [0, Q) mapped to (-Q/2, Q/2]
static Big center_Q(const Ctx& c, const Big& x) {
  if (mag_cmp(x, c.Qhalf) > 0) return big_sub(x, c.Q);
  return x;
}
// round(t d / Q) for a signed integer d (Q odd and coprime to t: no ties)
static Big round_t_over_Q(const Ctx& c, const Big& d) {
  Big a = d;
  a.neg = 0;
#if ORC_MUTANT == 1
  Big num = big_mul_u64(a, 2 * c.t);
#else
  Big num = big_add(big_mul_u64(a, 2 * c.t), c.Q);  // 2 t |d| + Q
#endif
  uint64_t r;
  Big h = mag_divmod_u64(num, 2, &r);               // floor(num / 2)
  Big w = mag_floordiv_primes(h, c.q);              // floor(num / (2Q))
  if (d.neg) w = big_neg(w);
  return w;
}

// ---- ciphertext <-> residue arrays (layout [2][L][N], canonical residues) ----
struct Ct {
  Poly c0, c1;    // coefficients in [0, Q)
  int depth = 0;  // multiplicative depth from fresh inputs (selects the relinearisation key)
};
static Poly poly_from_rns(const Ctx& c, const uint64_t* res /*[L][N]*/) {
  Poly p(c.N);
  std::vector<uint64_t> r(c.L);
  for (int j = 0; j < c.N; ++j) {
    for (int i = 0; i < c.L; ++i) {
      r[i] = res[(size_t)i * c.N + j];
      if (r[i] >= c.q[i]) fail("residue out of range");
    }
    p[j] = c.crtQ.reconstruct(r.data());
  }
  return p;
}
static void poly_to_rns(const Ctx& c, const Poly& p, uint64_t* res) {
  for (int i = 0; i < c.L; ++i)
    for (int j = 0; j < c.N; ++j) res[(size_t)i * c.N + j] = big_mod_u64(p[j], c.q[i]);
}
static Ct ct_from_rns(const Ctx& c, const uint64_t* a) {
  Ct ct;
  ct.c0 = poly_from_rns(c, a);
  ct.c1 = poly_from_rns(c, a + (size_t)c.L * c.N);
  return ct;
}
static void ct_to_rns(const Ctx& c, const Ct& ct, uint64_t* a) {
  poly_to_rns(c, ct.c0, a);
  poly_to_rns(c, ct.c1, a + (size_t)c.L * c.N);
}

// ---- batch encoding (slots <-> plaintext polynomial mod t) ----
// decode:  slot_j = m(psi_t^(2 brv(j) + 1))  =  negacyclic transform output at brv(j)
static void decode_poly(const Ctx& c, const uint64_t* m, uint32_t* slots) {
  std::vector<uint64_t> a(m, m + c.N);
  c.tplan.forward(a.data());
#if ORC_MUTANT == 6
  for (int j = 0; j < c.N; ++j) slots[j] = (uint32_t)a[j];
#else
  for (int j = 0; j < c.N; ++j) slots[j] = (uint32_t)a[brv(j, c.logn)];
#endif
}
static void encode_slots(const Ctx& c, const uint32_t* slots, uint64_t* m) {
  std::vector<uint64_t> a(c.N);
#if ORC_MUTANT == 6
  for (int j = 0; j < c.N; ++j) a[j] = slots[j] % c.t;
#else
  for (int j = 0; j < c.N; ++j) a[brv(j, c.logn)] = slots[j] % c.t;
#endif
  c.tplan.inverse(a.data());
  for (int j = 0; j < c.N; ++j) m[j] = a[j];
}

// ---- scheme operations ----
static Ct ct_sub(const Ctx& c, const Ct& x, const Ct& y) {
  Ct r;
  r.depth = std::max(x.depth, y.depth);
  r.c0.resize(c.N);
  r.c1.resize(c.N);
  for (int j = 0; j < c.N; ++j) {
    r.c0[j] = mod_Q(c, big_sub(x.c0[j], y.c0[j]));
    r.c1[j] = mod_Q(c, big_sub(x.c1[j], y.c1[j]));
  }
  return r;
}
// ct - (Delta * v, 0) where v in [0, t) is broadcast to every slot (constant poly)
static Ct ct_sub_const(const Ctx& c, const Ct& x, uint64_t v) {
  Ct r = x;
  r.c0[0] = mod_Q(c, big_sub(x.c0[0], big_mul_u64(c.Delta, v % c.t)));
  return r;
}
// 1 - ct = (Delta - c0, -c1)
static Ct ct_one_minus(const Ctx& c, const Ct& x) {
  Ct r;
  r.depth = x.depth;
  r.c0.resize(c.N);
  r.c1.resize(c.N);
  for (int j = 0; j < c.N; ++j) {
    r.c0[j] = mod_Q(c, big_neg(x.c0[j]));
    r.c1[j] = mod_Q(c, big_neg(x.c1[j]));
  }
  r.c0[0] = mod_Q(c, big_add(r.c0[0], c.Delta));
  return r;
}

// Key switching of (d0, d1, d2), coefficients in [0, Q), where d2 is to be
// multiplied by the key's source secret: (d0, d1) + round(sum_a [d2]_{Q_a} k_a / P)
// mod Q, digits a < D over the key's groups of data primes.  With a
// relinearisation key this is relinearisation (source s^2); with a Galois key
// it completes an automorphism (source tau_g(s)).
static Ct key_switch(const Ctx& c, const KsKey& K, const Poly& d0, const Poly& d1, const Poly& d2) {
  int N = c.N, D = K.D, k = K.nprimes;
  // u = sum_a digit_a * k_a  (exact integer negacyclic products, then mod QP)
  std::vector<uint64_t> res0((size_t)k * N), res1((size_t)k * N);
  std::vector<Big> digit((size_t)D * N);  // digit_a = [d2]_{Q_a}
  for (int a = 0; a < D; ++a)
#if ORC_MUTANT == 7
    for (int j = 0; j < N; ++j)
      digit[(size_t)a * N + j] = mod_primes(d2[j], big_u64(K.grp[a][0]), std::vector<uint64_t>{K.grp[a][0]});
#else
    for (int j = 0; j < N; ++j) digit[(size_t)a * N + j] = mod_primes(d2[j], K.Qa[a], K.grp[a]);
#endif
  std::vector<uint64_t> Dg(N), acc0(N), acc1(N);
  for (int pi = 0; pi < k; ++pi) {
    uint64_t m = c.om[pi];
    std::fill(acc0.begin(), acc0.end(), 0);
    std::fill(acc1.begin(), acc1.end(), 0);
    for (int a = 0; a < D; ++a) {
      for (int j = 0; j < N; ++j) Dg[j] = big_mod_u64(digit[(size_t)a * N + j], m);
      c.plans[pi].forward(Dg.data());
      const uint64_t* K0 = &K.ntt[(((size_t)a * 2 + 0) * k + pi) * N];
      const uint64_t* K1 = &K.ntt[(((size_t)a * 2 + 1) * k + pi) * N];
      for (int j = 0; j < N; ++j) {
        acc0[j] = addmod(acc0[j], mulmod(Dg[j], K0[j], m), m);
        acc1[j] = addmod(acc1[j], mulmod(Dg[j], K1[j], m), m);
      }
    }
    c.plans[pi].inverse(acc0.data());
    c.plans[pi].inverse(acc1.data());
    for (int j = 0; j < N; ++j) {
      res0[(size_t)j * k + pi] = acc0[j];
      res1[(size_t)j * k + pi] = acc1[j];
    }
  }
  const Crt& crt = c.crt_prefix[k - 1];
  Ct out;
  out.c0.resize(N);
  out.c1.resize(N);
  uint64_t Phalf = (c.P - 1) / 2;
  for (int comp = 0; comp < 2; ++comp) {
    const std::vector<uint64_t>& res = comp ? res1 : res0;
    const Poly& base = comp ? d1 : d0;
    Poly& dst = comp ? out.c1 : out.c0;
    for (int j = 0; j < N; ++j) {
      // exact signed sum (the negacyclic wrap can make it negative)
      Big u = crt.reconstruct_centered(&res[(size_t)j * k]);
      u = mod_QP(c, u);
      uint64_t rp = big_mod_u64(u, c.P);             // [u]_P, centred below
#if ORC_MUTANT == 3
      Big cen = big_u64(rp);
      (void)Phalf;
#else
      Big cen = rp > Phalf ? big_neg(big_u64(c.P - rp)) : big_u64(rp);
#endif
      uint64_t rem;
      Big ks = mag_divmod_u64(big_sub(u, cen), c.P, &rem);  // (u - [u]_P) / P, exact
      if (rem != 0) fail("mod-down not exact");
      dst[j] = mod_Q(c, big_add(base[j], ks));
    }
  }
  return out;
}

// Relinearisation of a product at multiplicative depth `depth`: the per-prime
// key when depth <= fine_depth, the two-digit key when depth >= coarse_from
// (coarse_from > 0), else the key of dp-prime digits.
static Ct relinearize(const Ctx& c, const Poly& d0, const Poly& d1, const Poly& d2, int depth) {
  if (!c.have_rk) fail("relinearisation key not set");
#if ORC_MUTANT == 15
  if (depth < c.fine_depth) {
#else
  if (depth <= c.fine_depth) {
#endif
    if (!c.have_rk1) fail("per-prime relinearisation key not set");
    return key_switch(c, c.rk1, d0, d1, d2);
  }
#if ORC_MUTANT == 16
  if (c.coarse_from > 0 && depth > c.coarse_from) {
#else
  if (c.coarse_from > 0 && depth >= c.coarse_from) {
#endif
    if (!c.have_rk2) fail("two-digit relinearisation key not set");
    return key_switch(c, c.rk2, d0, d1, d2);
  }
  return key_switch(c, c.rk, d0, d1, d2);
}

// textbook multiplication + relinearisation; the product lies one level below
// the deeper operand
static Ct ct_mul_relin(const Ctx& c, const Ct& a, const Ct& b) {
  int N = c.N;
  Poly a0(N), a1(N), b0(N), b1(N);
  for (int j = 0; j < N; ++j) {
    a0[j] = center_Q(c, a.c0[j]);
    a1[j] = center_Q(c, a.c1[j]);
    b0[j] = center_Q(c, b.c0[j]);
    b1[j] = center_Q(c, b.c1[j]);
  }
  std::vector<Poly> d = tensor_exact(c, a0, a1, b0, b1);
  Poly &d0 = d[0], &d1 = d[1], &d2 = d[2];
  for (int j = 0; j < N; ++j) {
    d0[j] = mod_Q(c, round_t_over_Q(c, d0[j]));
    d1[j] = mod_Q(c, round_t_over_Q(c, d1[j]));
    d2[j] = mod_Q(c, round_t_over_Q(c, d2[j]));
  }
  Ct r = relinearize(c, d0, d1, d2, std::max(a.depth, b.depth) + 1);
  r.depth = std::max(a.depth, b.depth) + 1;
  return r;
}

static Poly secret_poly(const Ctx& c, const int8_t* s) {
  Poly p(c.N);
  for (int j = 0; j < c.N; ++j) {
    p[j] = big_u64((uint64_t)std::abs((int)s[j]));
    if (s[j] < 0) p[j] = big_neg(p[j]);
  }
  return p;
}

// [c0 + c1 s]_Q in [0, Q)
static Poly phase(const Ctx& c, const Ct& ct, const int8_t* s) {
  Poly sp = secret_poly(c, s);
  Poly c1c(c.N);
  for (int j = 0; j < c.N; ++j) c1c[j] = center_Q(c, ct.c1[j]);
  Poly prod = poly_mul_exact(c, c1c, sp);
  Poly x(c.N);
  for (int j = 0; j < c.N; ++j) x[j] = mod_Q(c, big_add(ct.c0[j], prod[j]));
  return x;
}

// ---------------------------------------------------------------------------
// extern "C" interface (consumed by oracle/__init__.py through ctypes)
// ---------------------------------------------------------------------------
// Key-switching key from source secret `src` (an integer polynomial: s^2 or
// tau_g(s)) to s: k_a = (-(a_a s + e_a) + P g_a src, a_a) mod QP for digit a,
// with g_a = (Q/Q_a) [(Q/Q_a)^{-1}]_{Q_a} = sum over the group's primes q_i of
// (Q/q_i) [(Q/q_i)^{-1}]_{q_i} (both are 1 mod Q_a and 0 mod Q/Q_a); a_a
// uniform mod QP (residue j drawn with counter (k, j, obj_base | a, dom_a)),
// e_a centred binomial (counter (k, 0, obj_base | a, dom_e)).
// `out` (may be null): uint64 [D][2][L+1][N].
// The digit groups of a key with dp data primes per digit: primes
// q_{a dp} .. q_{min(L, (a+1) dp) - 1} form digit a.
static void set_digit_groups(const Ctx& c, int dp, KsKey& K) {
  K.dp = dp;
  K.D = (c.L + dp - 1) / dp;
  K.grp.assign(K.D, {});
  K.Qa.assign(K.D, big_u64(1));
  for (int a = 0; a < K.D; ++a)
    for (int i = a * dp; i < std::min(c.L, (a + 1) * dp); ++i) {
      K.grp[a].push_back(c.q[i]);
      K.Qa[a] = big_mul_u64(K.Qa[a], c.q[i]);
    }
}

static void make_ks_key(const Ctx& c, uint64_t seed, const Poly& s, const Poly& src, uint32_t dom_a, uint32_t dom_e,
                        uint32_t obj_base, int dp, KsKey& K, uint64_t* out) {
  set_digit_groups(c, dp, K);
  int N = c.N, L = c.L, D = K.D;
  uint32_t w[4];
  K.k0.assign(D, Poly(N));
  K.k1.assign(D, Poly(N));
  std::vector<uint64_t> res(L + 1);
  for (int a = 0; a < D; ++a) {
    Big g = big_zero();
    for (int i = a * dp; i < std::min(L, (a + 1) * dp); ++i) {
      uint64_t rr;
      Big qhat = mag_divmod_u64(c.Q, c.q[i], &rr);
      uint64_t qhat_inv = invmod(big_mod_u64(qhat, c.q[i]), c.q[i]);
      g = big_add(g, big_mul_u64(qhat, qhat_inv));
    }
    Big Pg = big_mul_u64(g, c.P);
    Poly av(N), e(N);
    for (int k = 0; k < N; ++k) {
      for (int j = 0; j <= L; ++j) {
        draw(seed, k, j, obj_base | (uint32_t)a, dom_a, w);
        res[j] = sample_uniform(w, c.qp[j]);
      }
      av[k] = c.crtQP.reconstruct(res.data());
      draw(seed, k, 0, obj_base | (uint32_t)a, dom_e, w);
      int ev = sample_cbd21(w);
      e[k] = big_u64((uint64_t)std::abs(ev));
      if (ev < 0) e[k] = big_neg(e[k]);
    }
    Poly as = poly_mul_exact(c, av, s);
    for (int k = 0; k < N; ++k) {
#if ORC_MUTANT == 5
      Big v = big_add(as[k], e[k]);
#else
      Big v = big_neg(big_add(as[k], e[k]));
#endif
      v = big_add(v, big_mul(Pg, src[k]));
      K.k0[a][k] = mod_QP(c, v);
      K.k1[a][k] = av[k];
    }
    if (out)
      for (int comp = 0; comp < 2; ++comp)
        for (int j = 0; j <= L; ++j)
          for (int k = 0; k < N; ++k) {
            const Big& v = comp ? K.k1[a][k] : K.k0[a][k];
            out[((((size_t)a * 2 + comp) * (L + 1)) + j) * N + k] = big_mod_u64(v, c.qp[j]);
          }
  }
  // transforms over the oracle primes: |u| < D N max(Q_a) QP
  int dbits = 0;
  for (const Big& M : K.Qa) dbits = std::max(dbits, big_bits(M));
  int bound = dbits + big_bits(c.QP) + c.logn + (int)std::ceil(std::log2((double)D + 1)) + 1;
  int k = primes_needed(c, bound);
  K.nprimes = k;
  K.ntt.assign((size_t)D * 2 * k * N, 0);
  for (int a = 0; a < D; ++a)
    for (int comp = 0; comp < 2; ++comp)
      for (int pi = 0; pi < k; ++pi) {
        uint64_t* dst = &K.ntt[(((size_t)a * 2 + comp) * k + pi) * N];
        const Poly& srcp = comp ? K.k1[a] : K.k0[a];
        for (int j = 0; j < N; ++j) dst[j] = big_mod_u64(srcp[j], c.om[pi]);
        c.plans[pi].forward(dst);
      }
}

// Galois automorphism tau_g: a(X) -> a(X^g) mod X^N + 1 (g odd).  Coefficient j
// moves to j g mod 2N; landing at N + r means -X^r.  `M` null: signed
// integer coefficients (negation), else residues in [0, M) (negation mod M).
static Poly automorph(const Ctx& c, const Poly& a, uint64_t g, const Big* M) {
  const uint64_t twoN = 2 * (uint64_t)c.N;
  Poly out(c.N);
  for (int j = 0; j < c.N; ++j) {
    uint64_t e = ((uint64_t)j * g) % twoN;
    if (e < (uint64_t)c.N) {
      out[e] = a[j];
    } else {
      const Big& v = a[j];
#if ORC_MUTANT == 10
      out[e - c.N] = v;
#else
      out[e - c.N] = M ? (big_is_zero(v) ? v : big_sub(*M, v)) : big_neg(v);
#endif
    }
  }
  return out;
}

// ct -> tau_g(ct), which decrypts under tau_g(s) to tau_g(m)
static Ct ct_automorph(const Ctx& c, const Ct& x, uint64_t g) {
  Ct r;
  r.depth = x.depth;
  r.c0 = automorph(c, x.c0, g, &c.Q);
  r.c1 = automorph(c, x.c1, g, &c.Q);
  return r;
}

// Rotation (slot permutation) by g: tau_g(ct) switched back to s with the
// Galois key of g: (tau_g(c0), 0) + round(sum_i [tau_g(c1)]_{q_i} gk_i / P).
static Ct ct_rotate(const Ctx& c, const Ct& x, uint64_t g) {
  auto it = c.gk.find(g);
  if (it == c.gk.end()) fail("Galois key not generated");
  Ct t = ct_automorph(c, x, g);
  Poly zero(c.N, big_zero());
  Ct r = key_switch(c, it->second, t.c0, zero, t.c1);
  r.depth = x.depth;
  return r;
}

extern "C" {

// Largest `L` primes below 2^55 and the largest prime below 2^56, all = 1 mod 2^16.
int orc_default_primes(int L, uint64_t* q_out, uint64_t* P_out) {
  std::vector<uint64_t> q = primes_below(55, 16, L);
  std::vector<uint64_t> P = primes_below(56, 16, 1);
  if ((int)q.size() != L || P.size() != 1) return -1;
  for (int i = 0; i < L; ++i) q_out[i] = q[i];
  *P_out = P[0];
  return 0;
}

void* orc_create(int logn, int L, const uint64_t* q, uint64_t P, uint64_t t) {
  Ctx* c = new Ctx();
  c->logn = logn;
  c->N = 1 << logn;
  c->L = L;
  c->t = t;
  c->P = P;
  c->q.assign(q, q + L);
  c->qp = c->q;
  c->qp.push_back(P);
  for (uint64_t x : c->qp)
    if (!is_prime_u64(x)) fail("modulus is not prime");
  if (!is_prime_u64(t)) fail("plaintext modulus is not prime");
  c->crtQ.init(c->q);
  c->crtQP.init(c->qp);
  c->Q = c->crtQ.M;
  c->QP = c->crtQP.M;
  uint64_t r;
  c->Qhalf = mag_divmod_u64(c->Q, 2, &r);  // Q odd: (Q-1)/2
  c->Delta = mag_divmod_u64(c->Q, t, &r);
  // oracle product primes: 61-bit, = 1 mod 2^17; enough for 2176-bit products
  c->om = primes_below(61, 17, 34);
  for (uint64_t m : c->om)
    for (uint64_t x : c->qp)
      if (m == x) fail("oracle prime collides with a scheme prime");
  c->plans.resize(c->om.size());
  for (size_t i = 0; i < c->om.size(); ++i) c->plans[i].init(logn, c->om[i]);
  c->crt_prefix.resize(c->om.size());
  for (size_t k = 1; k <= c->om.size(); ++k)
    c->crt_prefix[k - 1].init(std::vector<uint64_t>(c->om.begin(), c->om.begin() + k));
  c->tplan.init(logn, t);
  return c;
}

// Digits of the relinearisation and Galois keys: ceil(L / dp).
int orc_num_digits(void* h) {
  Ctx* c = (Ctx*)h;
  return (c->L + c->dp - 1) / c->dp;
}

// Key-switching digit groupings (before orc_keygen): dp data primes per digit
// for the relinearisation and Galois keys (1 .. L), and the depth up to which
// products are relinearised with the per-prime key instead (0 = never).
int orc_set_digits(void* h, int dp, int fine_depth) {
  Ctx* c = (Ctx*)h;
  if (dp < 1 || dp > c->L || fine_depth < 0) return -1;
  c->dp = dp;
  c->fine_depth = fine_depth;
  c->have_rk = c->have_rk1 = c->have_rk2 = false;
  c->gk.clear();
  return 0;
}

// The depth from which products are relinearised with the two-digit key (before
// orc_keygen; 0 = never; above the fine depth when both are set).
int orc_set_coarse(void* h, int coarse_from) {
  Ctx* c = (Ctx*)h;
  if (coarse_from < 0 || (coarse_from > 0 && coarse_from <= c->fine_depth)) return -1;
  c->coarse_from = coarse_from;
  c->have_rk = c->have_rk1 = c->have_rk2 = false;
  c->gk.clear();
  return 0;
}

void orc_destroy(void* h) { delete (Ctx*)h; }

// Q, QP, Delta as little-endian 64-bit limbs (for tests); returns limb count
int orc_export_big(void* h, int which, uint64_t* out, int cap) {
  Ctx* c = (Ctx*)h;
  const Big& b = which == 0 ? c->Q : which == 1 ? c->QP : c->Delta;
  if (b.n > cap) return -1;
  for (int i = 0; i < b.n; ++i) out[i] = b.w[i];
  return b.n;
}

void orc_philox(uint64_t seed, uint32_t k, uint32_t j, uint32_t obj, uint32_t dom, uint32_t* out4) {
  draw(seed, k, j, obj, dom, out4);
}
void orc_philox_raw(const uint32_t* ctr4, const uint32_t* key2, uint32_t* out4) {
  philox4x32_10(ctr4, key2, out4);
}

// plain negacyclic transform over an oracle-chosen prime m (tests only)
int orc_ntt_forward(int logn, uint64_t m, uint64_t* a) {
  NttPlan p;
  p.init(logn, m);
  p.forward(a);
  return 0;
}
int orc_ntt_inverse(int logn, uint64_t m, uint64_t* a) {
  NttPlan p;
  p.init(logn, m);
  p.inverse(a);
  return 0;
}

// exact product of two signed small-coefficient polynomials (tests only):
// a, b int64 [N]; out int64 [N] (must fit)
int orc_polymul_small(void* h, const int64_t* a, const int64_t* b, int64_t* out) {
  Ctx* c = (Ctx*)h;
  Poly A(c->N), B(c->N);
  for (int j = 0; j < c->N; ++j) {
    A[j] = big_u64((uint64_t)std::llabs(a[j]));
    if (a[j] < 0) A[j] = big_neg(A[j]);
    B[j] = big_u64((uint64_t)std::llabs(b[j]));
    if (b[j] < 0) B[j] = big_neg(B[j]);
  }
  Poly C = poly_mul_exact(*c, A, B);
  for (int j = 0; j < c->N; ++j) {
    if (C[j].n > 1 || (C[j].n == 1 && C[j].w[0] >> 63)) return -1;
    int64_t v = C[j].n ? (int64_t)C[j].w[0] : 0;
    out[j] = C[j].neg ? -v : v;
  }
  return 0;
}

int orc_encode(void* h, const uint32_t* slots, uint64_t* m) {
  encode_slots(*(Ctx*)h, slots, m);
  return 0;
}
int orc_decode(void* h, const uint64_t* m, uint32_t* slots) {
  decode_poly(*(Ctx*)h, m, slots);
  return 0;
}

// secret key s (int8 [N]) and relinearisation key rk (uint64 [D][2][L+1][N],
// residues mod q_0..q_{L-1}, P), both from `seed`.  The key is also kept in
// the context for later multiplications.
int orc_keygen(void* h, uint64_t seed, int8_t* s_out, uint64_t* rk_out) {
  Ctx& c = *(Ctx*)h;
  uint32_t w[4];
  for (int k = 0; k < c.N; ++k) {
    draw(seed, k, 0, 0, DOM_S, w);
    s_out[k] = (int8_t)sample_ternary(w);
  }
  Poly s = secret_poly(c, s_out);
  Poly s2 = poly_mul_exact(c, s, s);
  make_ks_key(c, seed, s, s2, DOM_A_RK, DOM_E_RK, 0, c.dp, c.rk, rk_out);
  c.have_rk = true;
  if (c.fine_depth > 0) {
    make_ks_key(c, seed, s, s2, DOM_A_RK, DOM_E_RK, FINE_OBJ, 1, c.rk1, nullptr);
    c.have_rk1 = true;
  }
  if (c.coarse_from > 0) {
    make_ks_key(c, seed, s, s2, DOM_A_RK, DOM_E_RK, COARSE_OBJ, COARSE_DIGIT_PRIMES, c.rk2, nullptr);
    c.have_rk2 = true;
  }
  return 0;
}

// The per-prime relinearisation key made by orc_keygen when fine_depth > 0:
// uint64 [L][2][L+1][N] (digit i = [d2]_{q_i}, drawn with object index 16 + i).
int orc_fine_key(void* h, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk1) return -2;
  for (int a = 0; a < c.rk1.D; ++a)
    for (int comp = 0; comp < 2; ++comp)
      for (int j = 0; j <= c.L; ++j)
        for (int k = 0; k < c.N; ++k) {
          const Big& v = comp ? c.rk1.k1[a][k] : c.rk1.k0[a][k];
          out[((((size_t)a * 2 + comp) * (c.L + 1)) + j) * c.N + k] = big_mod_u64(v, c.qp[j]);
        }
  return 0;
}

// The two-digit relinearisation key made by orc_keygen when coarse_from > 0:
// uint64 [2][2][L+1][N] (digits [d2] mod q_0..q_7 and mod q_8..q_14, drawn with
// object index 48 + a).
int orc_coarse_key(void* h, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk2) return -2;
  for (int a = 0; a < c.rk2.D; ++a)
    for (int comp = 0; comp < 2; ++comp)
      for (int j = 0; j <= c.L; ++j)
        for (int k = 0; k < c.N; ++k) {
          const Big& v = comp ? c.rk2.k1[a][k] : c.rk2.k0[a][k];
          out[((((size_t)a * 2 + comp) * (c.L + 1)) + j) * c.N + k] = big_mod_u64(v, c.qp[j]);
        }
  return 0;
}

// Symmetric encryption of `slots` (uint32 [N], values mod t):
// ct = (-(a s + e) + Delta m, a) mod Q; a, e drawn with object index ct_index.
int orc_encrypt(void* h, const int8_t* s, const uint32_t* slots, uint64_t seed, uint32_t ct_index, uint64_t* ct_out) {
  Ctx& c = *(Ctx*)h;
  int N = c.N, L = c.L;
  std::vector<uint64_t> m(N);
  encode_slots(c, slots, m.data());
  Poly sp = secret_poly(c, s);
  Poly a(N), e(N);
  std::vector<uint64_t> res(L);
  uint32_t w[4];
  for (int k = 0; k < N; ++k) {
    for (int j = 0; j < L; ++j) {
      draw(seed, k, j, ct_index, DOM_A_ENC, w);
      res[j] = sample_uniform(w, c.q[j]);
    }
    a[k] = c.crtQ.reconstruct(res.data());
    draw(seed, k, 0, ct_index, DOM_E_ENC, w);
    int ev = sample_cbd21(w);
    e[k] = big_u64((uint64_t)std::abs(ev));
    if (ev < 0) e[k] = big_neg(e[k]);
  }
  Poly as = poly_mul_exact(c, a, sp);
  Ct ct;
  ct.c0.resize(N);
  ct.c1 = a;
  for (int k = 0; k < N; ++k) {
    Big v = big_neg(big_add(as[k], e[k]));
    v = big_add(v, big_mul_u64(c.Delta, m[k]));
    ct.c0[k] = mod_Q(c, v);
  }
  ct_to_rns(c, ct, ct_out);
  return 0;
}

// Decryption: m = round(t [c0 + c1 s]_Q / Q) mod t, then batch decoding.
// noise_bits (optional): invariant-noise budget log2(Q) - 1 - log2 max|[t x]_Q|.
int orc_decrypt(void* h, const int8_t* s, const uint64_t* ct_in, uint32_t* slots_out, double* noise_bits) {
  Ctx& c = *(Ctx*)h;
  Ct ct = ct_from_rns(c, ct_in);
  Poly x = phase(c, ct, s);
  std::vector<uint64_t> m(c.N);
  double worst = -INFINITY;
  for (int k = 0; k < c.N; ++k) {
    Big w = round_t_over_Q(c, x[k]);
    m[k] = big_mod_u64(w, c.t);
    Big y = center_Q(c, mod_Q(c, big_mul_u64(x[k], c.t)));
    worst = std::max(worst, big_log2(y));
  }
#if ORC_MUTANT == 14
  if (noise_bits) *noise_bits = big_log2(c.Q) - worst;
#else
  if (noise_bits) *noise_bits = big_log2(c.Q) - 1.0 - worst;
#endif
  decode_poly(c, m.data(), slots_out);
  return 0;
}

int orc_sub(void* h, const uint64_t* x, const uint64_t* y, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  ct_to_rns(c, ct_sub(c, ct_from_rns(c, x), ct_from_rns(c, y)), out);
  return 0;
}
int orc_sub_const(void* h, const uint64_t* x, uint64_t v, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  ct_to_rns(c, ct_sub_const(c, ct_from_rns(c, x), v), out);
  return 0;
}
int orc_one_minus(void* h, const uint64_t* x, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  ct_to_rns(c, ct_one_minus(c, ct_from_rns(c, x)), out);
  return 0;
}
// general product a * b followed by relinearisation (uses the key from orc_keygen
// or orc_set_relin_key)
int orc_mul_relin(void* h, const uint64_t* a, const uint64_t* b, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk) return -2;
  ct_to_rns(c, ct_mul_relin(c, ct_from_rns(c, a), ct_from_rns(c, b)), out);
  return 0;
}
// The same product for operands at multiplicative depths da and db (the
// product's depth max(da, db) + 1 selects the relinearisation key), e.g. a
// column (depth 0) times a predicate mask (SELECT, Eq. 5).
int orc_mul_relin_depth(void* h, const uint64_t* a, int da, const uint64_t* b, int db, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk) return -2;
  if (da < 0 || db < 0) return -1;
  Ct A = ct_from_rns(c, a), B = ct_from_rns(c, b);
  A.depth = da;
  B.depth = db;
  ct_to_rns(c, ct_mul_relin(c, A, B), out);
  return 0;
}

// EQ: 1 - (x - y)^(2^squarings); y == NULL means x - const_val.
// squarings = 16 gives the paper's predicate for p = 65537.
int orc_eq(void* h, const uint64_t* x, const uint64_t* y, uint64_t const_val, int squarings, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk) return -2;
  Ct d = ct_from_rns(c, x);
  d = y ? ct_sub(c, d, ct_from_rns(c, y)) : ct_sub_const(c, d, const_val);
#if ORC_MUTANT == 8
  --squarings;
#endif
  for (int r = 0; r < squarings; ++r) d = ct_mul_relin(c, d, d);
  ct_to_rns(c, ct_one_minus(c, d), out);
  return 0;
}

// EQ against a plaintext with one constant per slot: d = x - (Delta m, 0) with
// m = encode(cslots) (textbook plaintext subtraction), then the squarings and
// "1 -".  With every slot equal to c this is the broadcast form x - c.
int orc_eq_plain(void* h, const uint64_t* x, const uint32_t* cslots, int squarings, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk) return -2;
  std::vector<uint64_t> m(c.N);
  encode_slots(c, cslots, m.data());
  Ct d = ct_from_rns(c, x);
  for (int k = 0; k < c.N; ++k) d.c0[k] = mod_Q(c, big_sub(d.c0[k], big_mul_u64(c.Delta, m[k])));
  for (int r = 0; r < squarings; ++r) d = ct_mul_relin(c, d, d);
  ct_to_rns(c, ct_one_minus(c, d), out);
  return 0;
}

// ---------------------------------------------------------------------------
// LT comparison (Eq. 4): LT(x, y) = sum_{a = -(p-1)/2}^{-1} (1 - (x - y - a)^(p-1)).
// As a polynomial in z = x - y over F_p (binomial coefficients C(p-1, k) = (-1)^k):
//   f(z) = sum_{k=1}^{p-1} c_k z^k,  c_k = -sum_{a in A} a^(p-1-k),  A = {-1, ..., -(p-1)/2},
// so c_k = sum_{b=1}^{(p-1)/2} b^(p-1-k) for odd k, c_k = 0 for even k < p-1, and
// c_{p-1} = -(p-1)/2.  With w = z^2:  f(z) = z h(w) - ((p-1)/2) w^((p-1)/2),
// h(w) = sum_m c_{2m+1} w^m.
// ---------------------------------------------------------------------------
static std::vector<uint32_t> lt_odd_coefficients(uint64_t p) {
  // h_m = c_{2m+1} = sum_{b=1}^{(p-1)/2} b^(p-2-2m) mod p, m < (p-1)/2 (plain power sums)
  const uint64_t half = (p - 1) / 2;
  std::vector<uint64_t> acc(half, 0);
  for (uint64_t b = 1; b <= half; ++b) {
    const uint64_t b2inv = invmod(b * b % p, p);  // b^(p-2-2m) = b^(p-2) * (b^-2)^m
#if ORC_MUTANT == 9
    uint64_t v = 1;  // b^(p-1)
#else
    uint64_t v = invmod(b, p);                    // b^(p-2)
#endif
    for (uint64_t m = 0; m < half; ++m) {
      acc[m] += v;
      v = v * b2inv % p;
    }
    if ((b & 1023) == 0)
      for (uint64_t m = 0; m < half; ++m) acc[m] %= p;
  }
  std::vector<uint32_t> h(half);
  for (uint64_t m = 0; m < half; ++m) h[m] = (uint32_t)(acc[m] % p);
  return h;
}

// c * ct for an integer c in [0, t), coefficient-wise mod Q
static Ct ct_scale(const Ctx& c, const Ct& a, uint64_t k) {
  Ct r;
  r.depth = a.depth;
  r.c0.resize(c.N);
  r.c1.resize(c.N);
  for (int j = 0; j < c.N; ++j) {
    r.c0[j] = mod_Q(c, big_mul_u64(a.c0[j], k));
    r.c1[j] = mod_Q(c, big_mul_u64(a.c1[j], k));
  }
  return r;
}
static Ct ct_add(const Ctx& c, const Ct& a, const Ct& b) {
  Ct r;
  r.depth = std::max(a.depth, b.depth);
  r.c0.resize(c.N);
  r.c1.resize(c.N);
  for (int j = 0; j < c.N; ++j) {
    r.c0[j] = mod_Q(c, big_add(a.c0[j], b.c0[j]));
    r.c1[j] = mod_Q(c, big_add(a.c1[j], b.c1[j]));
  }
  return r;
}
// (Delta k, 0): the encryption-free plaintext constant k
static Ct ct_constant(const Ctx& c, uint64_t k) {
  Ct r;
  r.c0.assign(c.N, big_zero());
  r.c1.assign(c.N, big_zero());
  r.c0[0] = mod_Q(c, big_mul_u64(c.Delta, k % c.t));
  return r;
}

// sum_i coef[i] * cts[i] + (Delta coef0, 0), evaluated on residues: Z_Q is
// isomorphic to prod Z_{q_i}, so scalar multiply-accumulate is exact per prime.
static Ct ct_linear(const Ctx& c, const std::vector<const Ct*>& cts, const std::vector<uint64_t>& coef, uint64_t coef0) {
  const size_t W = (size_t)2 * c.L * c.N;
  std::vector<unsigned __int128> acc(W, 0);
  std::vector<uint64_t> buf(W);
  for (size_t i = 0; i < cts.size(); ++i) {
    if (coef[i] == 0) continue;
    ct_to_rns(c, *cts[i], buf.data());
    for (size_t w = 0; w < W; ++w) acc[w] += (unsigned __int128)buf[w] * coef[i];
  }
  for (int i = 0; i < c.L; ++i)
    for (int comp = 0; comp < 2; ++comp)
      for (int j = 0; j < c.N; ++j) {
        size_t w = ((size_t)comp * c.L + i) * c.N + j;
        buf[w] = (uint64_t)(acc[w] % c.q[i]);
      }
  Ct r = ct_from_rns(c, buf.data());
  for (const Ct* x : cts) r.depth = std::max(r.depth, x->depth);
  return ct_add(c, r, ct_constant(c, coef0));
}

// The evaluation schedule of f(z) (both the oracle and the CUDA library follow
// it).  Every power is the product of its largest power-of-two part and the
// rest, so the power e sits at depth ceil(log2 e) above its base:
//   w = z z;  B_1 = w;  B_i = B_{i/2}^2 (i a power of 2) or B_{2^k} B_{i-2^k}
//   (2^k < i < 2^(k+1)), i < 256;  depth(B_i) = 1 + ceil(log2 i) <= 9;
//   G_1 = B_128^2 (= w^256, depth 9);  G_j likewise from G_{2^k} and G_{j-2^k},
//   j <= 128;  depth(G_j) = 9 + ceil(log2 j) <= 16;
//   H_j = Delta h_{256 j} + sum_{i=1}^{255} h_{256 j + i} B_i   (j < 128, depth 9);
//   h = H_0 + sum_{j=1}^{127} H_j G_j (depth 17);   out = z h - ((p-1)/2) G_128 (depth 18).
// 511 multiplications in all.
static int top_pow2(int i) {  // largest power of two <= i (i >= 1)
  int k = 1;
  while (2 * k <= i) k *= 2;
  return k;
}
static Ct lt_eval(const Ctx& c, const Ct& z, const std::vector<uint32_t>& hc) {
  const int BS = 256, GS = 128;
  Ct w = ct_mul_relin(c, z, z);
  std::vector<Ct> B(BS), G(GS + 1);
  B[1] = w;
  for (int i = 2; i < BS; ++i) {
    const int k = top_pow2(i);
    B[i] = (k == i) ? ct_mul_relin(c, B[i / 2], B[i / 2]) : ct_mul_relin(c, B[k], B[i - k]);
  }
#if ORC_MUTANT == 13
  G[1] = B[128];
#else
  G[1] = ct_mul_relin(c, B[128], B[128]);
#endif
  for (int j = 2; j <= GS; ++j) {
    const int k = top_pow2(j);
    G[j] = (k == j) ? ct_mul_relin(c, G[j / 2], G[j / 2]) : ct_mul_relin(c, G[k], G[j - k]);
  }
  std::vector<const Ct*> ptrs;
  for (int i = 1; i < BS; ++i) ptrs.push_back(&B[i]);
  Ct h;
  for (int j = 0; j < GS; ++j) {
    std::vector<uint64_t> coef(BS - 1);
    for (int i = 1; i < BS; ++i) coef[i - 1] = hc[(size_t)BS * j + i];
    Ct Hj = ct_linear(c, ptrs, coef, hc[(size_t)BS * j]);
    h = (j == 0) ? Hj : ct_add(c, h, ct_mul_relin(c, Hj, G[j]));
  }
  Ct g = ct_mul_relin(c, z, h);
  return ct_add(c, g, ct_scale(c, G[GS], c.t - (c.t - 1) / 2));  // - ((p-1)/2) w^((p-1)/2)
}

extern "C" {
// h_m = c_{2m+1} of the LT polynomial, m < (t-1)/2 (t = 65537: 32768 words)
static const std::vector<uint32_t>& lt_coeffs(Ctx& c) {
  if (c.lt_h.empty()) c.lt_h = lt_odd_coefficients(c.t);
  return c.lt_h;
}
int orc_lt_coefficients(void* h, uint32_t* out) {
  Ctx& c = *(Ctx*)h;
  const std::vector<uint32_t>& v = lt_coeffs(c);
  std::copy(v.begin(), v.end(), out);
  return 0;
}
// linear combination of n ciphertexts (residue layout [n][2][L][N]) with
// coefficients coef[i] < t plus the constant (Delta coef0, 0)
int orc_linear(void* h, const uint64_t* cts, int n, const uint64_t* coef, uint64_t coef0, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  const size_t W = (size_t)2 * c.L * c.N;
  std::vector<Ct> v(n);
  std::vector<const Ct*> p(n);
  std::vector<uint64_t> k(coef, coef + n);
  for (int i = 0; i < n; ++i) {
    v[i] = ct_from_rns(c, cts + i * W);
    p[i] = &v[i];
  }
  ct_to_rns(c, ct_linear(c, p, k, coef0), out);
  return 0;
}
// LT(x, y) = [x - y in {-(t-1)/2 .. -1}] by the schedule above (t = 65537)
// v - x for a plaintext constant v: (Delta v - c0, -c1) mod Q
static Ct ct_const_minus(const Ctx& c, const Ct& x, uint64_t v) {
  Ct r;
  r.depth = x.depth;
  r.c0.resize(c.N);
  r.c1.resize(c.N);
  for (int j = 0; j < c.N; ++j) {
    r.c0[j] = mod_Q(c, big_neg(x.c0[j]));
    r.c1[j] = mod_Q(c, big_neg(x.c1[j]));
  }
  r.c0[0] = mod_Q(c, big_add(r.c0[0], big_mul_u64(c.Delta, v)));
  return r;
}

// BETWEEN (Sec. 4.2.2): the product of the two comparisons x >= lo and x <= hi.
// With a = LT(x, lo) = f(x - lo) and b = LT(hi, x) = f(hi - x), f the
// comparison polynomial of Eq. 4 (valid while x, lo, hi lie in [0, (p-1)/2]),
// BETWEEN = (1 - a)(1 - b), one multiplication with relinearisation after the
// two comparisons (depth 19).  Empty ranges (lo > hi) are rejected.
int orc_between(void* h, const uint64_t* x, uint64_t lo, uint64_t hi, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk) return -2;
  if (c.t != 65537 || lo >= c.t || hi >= c.t || lo > hi) return -1;
  const std::vector<uint32_t>& hc = lt_coeffs(c);
  Ct X = ct_from_rns(c, x);
  Ct below = lt_eval(c, ct_sub_const(c, X, lo), hc);    // [x < lo]
  Ct above = lt_eval(c, ct_const_minus(c, X, hi), hc);  // [hi < x]
#if ORC_MUTANT == 12
  ct_to_rns(c, ct_mul_relin(c, below, ct_one_minus(c, above)), out);
#else
  ct_to_rns(c, ct_mul_relin(c, ct_one_minus(c, below), ct_one_minus(c, above)), out);  // (1 - a)(1 - b)
#endif
  return 0;
}

int orc_lt(void* h, const uint64_t* x, const uint64_t* y, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk) return -2;
  if (c.t != 65537) return -1;
  const std::vector<uint32_t>& hc = lt_coeffs(c);
  Ct z = ct_sub(c, ct_from_rns(c, x), ct_from_rns(c, y));
  ct_to_rns(c, lt_eval(c, z, hc), out);
  return 0;
}
}  // extern "C"

// Squarings only (no difference, no "1 -"): for noise-depth tests.
int orc_square_chain(void* h, const uint64_t* x, int squarings, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk) return -2;
  Ct d = ct_from_rns(c, x);
  for (int r = 0; r < squarings; ++r) d = ct_mul_relin(c, d, d);
  ct_to_rns(c, d, out);
  return 0;
}

// The textbook scale-and-round alone, for tiny-N brute-force pins:
// given a ciphertext pair a, b, write round(t d_j / Q) mod Q for j = 0, 1, 2
// (residue layout [3][L][N]) without relinearisation.
int orc_tensor_round(void* h, const uint64_t* a_in, const uint64_t* b_in, uint64_t* out3) {
  Ctx& c = *(Ctx*)h;
  int N = c.N;
  Ct a = ct_from_rns(c, a_in), b = ct_from_rns(c, b_in);
  Poly a0(N), a1(N), b0(N), b1(N);
  for (int j = 0; j < N; ++j) {
    a0[j] = center_Q(c, a.c0[j]);
    a1[j] = center_Q(c, a.c1[j]);
    b0[j] = center_Q(c, b.c0[j]);
    b1[j] = center_Q(c, b.c1[j]);
  }
  std::vector<Poly> d = tensor_exact(c, a0, a1, b0, b1);
  for (int k = 0; k < 3; ++k) {
    for (int j = 0; j < N; ++j) d[k][j] = mod_Q(c, round_t_over_Q(c, d[k][j]));
    poly_to_rns(c, d[k], out3 + (size_t)k * c.L * N);
  }
  return 0;
}

// Relinearisation alone on (d0, d1, d2) given as residues [3][L][N].
int orc_relin(void* h, const uint64_t* d3, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.have_rk) return -2;
  size_t s = (size_t)c.L * c.N;
  Poly d0 = poly_from_rns(c, d3), d1 = poly_from_rns(c, d3 + s), d2 = poly_from_rns(c, d3 + 2 * s);
  ct_to_rns(c, relinearize(c, d0, d1, d2, 1), out);  // a product of fresh ciphertexts
  return 0;
}

// ---------------------------------------------------------------------------
// Rotations and the rotate-and-add reduction behind COUNT and SUM (Sec. 4.2.2:
// rotate, add, and double the rotation amount until every slot holds the sum).
// The N slots form two rows of N/2 under the Galois group {+-3^k} mod 2N: g =
// 3^(2^i) rotates each row by 2^i, g = 2N - 1 exchanges the rows.  The
// reduction applies the row rotations by N/4, N/8, ..., 1 (largest first, as in
// the paper's worked example), then the row exchange: log2 N steps in all.
// ---------------------------------------------------------------------------

// Galois key for element g (odd, < 2N) from the secret s: source tau_g(s).
// gk_out (may be null): uint64 [D][2][L+1][N] residues mod q_0..q_{L-1}, P.
int orc_galois_keygen(void* h, uint64_t seed, const int8_t* s_in, uint64_t g, uint64_t* gk_out) {
  Ctx& c = *(Ctx*)h;
  if (g % 2 == 0 || g >= 2 * (uint64_t)c.N) return -1;
  Poly s = secret_poly(c, s_in);
  Poly sg = automorph(c, s, g, nullptr);
  make_ks_key(c, seed, s, sg, DOM_A_GK, DOM_E_GK, (uint32_t)(g << 5), c.dp, c.gk[g], gk_out);
  return 0;
}

// tau_g applied to both components (no key switching).
int orc_automorphism(void* h, const uint64_t* x, uint64_t g, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (g % 2 == 0 || g >= 2 * (uint64_t)c.N) return -1;
  ct_to_rns(c, ct_automorph(c, ct_from_rns(c, x), g), out);
  return 0;
}

int orc_rotate(void* h, const uint64_t* x, uint64_t g, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  if (!c.gk.count(g)) return -2;
  ct_to_rns(c, ct_rotate(c, ct_from_rns(c, x), g), out);
  return 0;
}

// ct <- ct + rotate(ct, g) for the first `row_steps` row rotations (by N/4, ...,
// of the full logN - 1), then, if `swap`, the row exchange.
int orc_rotate_sum(void* h, const uint64_t* x, int row_steps, int swap, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  const uint64_t twoN = 2 * (uint64_t)c.N;
  if (row_steps < 0 || row_steps > c.logn - 1) return -1;
  Ct a = ct_from_rns(c, x);
  for (int st = 0; st < row_steps; ++st) {
    const int i = c.logn - 2 - st;
    const uint64_t g = powmod(3, (uint64_t)1 << i, twoN);
    if (!c.gk.count(g)) return -2;
    a = ct_add(c, a, ct_rotate(c, a, g));
  }
#if ORC_MUTANT == 11
  swap = 0;
#endif
  if (swap) {
    if (!c.gk.count(twoN - 1)) return -2;
    a = ct_add(c, a, ct_rotate(c, a, twoN - 1));
  }
  ct_to_rns(c, a, out);
  return 0;
}

// ---------------------------------------------------------------------------
// Plaintext multiplication and Extract + Broadcast (JOIN, Sec. 4.2.2).
// ---------------------------------------------------------------------------

// ct * m for a plaintext polynomial m (coefficients mod t, taken as centred
// representatives in (-t/2, t/2]): (c0 m, c1 m) mod Q, exact negacyclic
// products.  It decrypts to the slot-wise product of the two plaintexts.
int orc_mul_plain(void* h, const uint64_t* x, const uint64_t* m, uint64_t* out) {
  Ctx& c = *(Ctx*)h;
  Poly mp(c.N);
  for (int j = 0; j < c.N; ++j) {
    if (m[j] >= c.t) return -1;
    mp[j] = m[j] > c.t / 2 ? big_neg(big_u64(c.t - m[j])) : big_u64(m[j]);
  }
  Ct a = ct_from_rns(c, x), r;
  r.c0 = poly_mul_exact(c, a.c0, mp);
  r.c1 = poly_mul_exact(c, a.c1, mp);
  for (int j = 0; j < c.N; ++j) {
    r.c0[j] = mod_Q(c, r.c0[j]);
    r.c1[j] = mod_Q(c, r.c1[j]);
  }
  ct_to_rns(c, r, out);
  return 0;
}

}  // extern "C"
