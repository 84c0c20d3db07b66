// Host-side parameter logic of libhp: prime search, the constant block for the
// exact RNS conversions, and the static depth estimate.
#include <math.h>
#include <algorithm>
#include <vector>
#include <stdio.h>
#include <string.h>

#include "hp_defs.h"

namespace hp {

typedef unsigned __int128 u128;

uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)(((u128)a * b) % m); }

uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m, x = a % m;
  for (; e; e >>= 1) {
    if (e & 1) r = h_mulmod(r, x, m);
    x = h_mulmod(x, x, m);
  }
  return r;
}

uint64_t h_invmod(uint64_t a, uint64_t m) { return h_powmod(a, m - 2, m); }

uint64_t h_shoup(uint64_t w, uint64_t p) { return (uint64_t)(((u128)w << 64) / p); }

// Miller-Rabin with the seven bases of Jaeschke/Sinclair, deterministic below 2^64.
bool is_prime(uint64_t n) {
  if (n < 4) return n >= 2;
  if (n % 2 == 0 || n % 3 == 0) return false;
  uint64_t d = n - 1;
  int r = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++r;
  }
  static const uint64_t bases[7] = {2, 325, 9375, 28178, 450775, 9780504, 1795265022};
  for (uint64_t b : bases) {
    uint64_t a = b % n;
    if (a == 0) continue;
    uint64_t x = h_powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int i = 1; i < r && witness; ++i) {
      x = h_mulmod(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

int find_primes(int bits, int count, const uint64_t* exclude, int nexclude, uint64_t* out) {
  const uint64_t step = 1ULL << 16;
  int found = 0;
  for (uint64_t c = ((1ULL << bits) - 1) / step * step + 1; c > step && found < count; c -= step) {
    if (c >= (1ULL << bits)) continue;
    bool skip = false;
    for (int i = 0; i < nexclude; ++i) skip |= exclude[i] == c;
    if (!skip && is_prime(c)) out[found++] = c;
  }
  return found;
}

uint64_t h_qnr(uint64_t p) {
  for (uint64_t g = 2;; ++g)
    if (h_powmod(g, (p - 1) / 2, p) == p - 1) return g;
}

// -p^{-1} mod 2^64 by Newton iteration (p odd)
static uint64_t neg_inv64(uint64_t p) {
  uint64_t x = p;  // correct to 3 bits
  for (int i = 0; i < 6; ++i) x *= 2 - p * x;
  return (uint64_t)0 - x;
}

// prod of the moduli in `ms` (skipping index `skip`) reduced mod m
static uint64_t prod_mod(const uint64_t* ms, int n, int skip, uint64_t m) {
  uint64_t r = 1 % m;
  for (int i = 0; i < n; ++i)
    if (i != skip) r = h_mulmod(r, ms[i] % m, m);
  return r;
}

// x 2^64 mod p
static uint64_t to_mont(uint64_t x, uint64_t p) { return (uint64_t)(((u128)(x % p) << 64) % p); }

// floor(2^128 / p) for odd p > 2^54, as (hi, lo)
static void recip128(uint64_t p, uint64_t* hi, uint64_t* lo) {
  u128 all = ~(u128)0;  // 2^128 - 1; p odd never divides 2^128
  u128 r = all / p;
  *hi = (uint64_t)(r >> 64);
  *lo = (uint64_t)r;
}

int build_consts(const uint64_t* q, uint64_t P, uint64_t t, Consts* C, char* err, int errlen) {
  memset(C, 0, sizeof(Consts));
  for (int i = 0; i < L; ++i) {
    if (!is_prime(q[i]) || q[i] >= (1ULL << 55) || q[i] % 65536 != 1) {
      snprintf(err, errlen, "q[%d] = %llu is not a prime < 2^55 congruent to 1 mod 2^16", i, (unsigned long long)q[i]);
      return -1;
    }
    for (int j = 0; j < i; ++j)
      if (q[j] == q[i]) {
        snprintf(err, errlen, "duplicate data prime");
        return -1;
      }
  }
  if (!is_prime(P) || P >= (1ULL << 56) || P % 65536 != 1) {
    snprintf(err, errlen, "P is not a prime < 2^56 congruent to 1 mod 2^16");
    return -1;
  }
  if (t != 65537) {
    snprintf(err, errlen, "plaintext modulus must be 65537");
    return -6;
  }
  // auxiliary base: the largest primes below 2^55 (= 1 mod 2^16) not used by Q or P
  uint64_t excl[L + 1];
  for (int i = 0; i < L; ++i) excl[i] = q[i];
  excl[L] = P;
  uint64_t b[K];
  if (find_primes(55, K, excl, L + 1, b) != K) {
    snprintf(err, errlen, "auxiliary prime search failed");
    return -1;
  }
  // digit reductions use one conditional subtraction (max q < 2 min q, P > max q),
  // the mod-down reduces residues mod P with two (P < 4 min q)
  uint64_t lo = q[0], hi = q[0];
  for (int i = 0; i < L; ++i) lo = q[i] < lo ? q[i] : lo, hi = q[i] > hi ? q[i] : hi;
  if (hi >= 2 * lo || P <= hi || P >= 4 * lo || lo < (1ULL << 54)) {
    snprintf(err, errlen, "primes must satisfy 2^54 <= q_i, max q < 2 min q < P < 4 min q");
    return -1;
  }
  // B must exceed t N_max Q by a margin: log2 B > log2 Q + 17 + 15 + 20
  double lq = 0, lb = 0;
  for (int i = 0; i < L; ++i) lq += log2((double)q[i]);
  for (int k = 0; k < K; ++k) lb += log2((double)b[k]);
  if (lb < lq + 52) {
    snprintf(err, errlen, "auxiliary base too small");
    return -1;
  }

  uint64_t all[NPRIME];
  for (int i = 0; i < L; ++i) all[i] = q[i];
  for (int k = 0; k < K; ++k) all[L + k] = b[k];
  all[ID_P] = P;
  all[ID_T] = t;
  for (int i = 0; i < NPRIME; ++i) {
    C->p[i] = all[i];
    C->pinv[i] = neg_inv64(all[i]);
    C->r2[i] = h_mulmod(to_mont(1, all[i]), to_mont(1, all[i]), all[i]);  // 2^128 mod p
    C->pbar[i] = ~0ull / all[i];
  }
  // Q -> B
  for (int i = 0; i < L; ++i) {
    uint64_t qh = prod_mod(q, L, i, q[i]);
    C->qhatinv[i] = h_invmod(qh, q[i]);
    C->qhatinv_s[i] = h_shoup(C->qhatinv[i], q[i]);
    C->qhat[i] = qh;
    C->qhat_s[i] = h_shoup(qh, q[i]);
    recip128(q[i], &C->om_hi[i], &C->om_lo[i]);
    for (int k = 0; k < K; ++k) C->MQB[i][k] = to_mont(prod_mod(q, L, i, b[k]), b[k]);
  }
  for (int k = 0; k < K; ++k) {
    uint64_t Qb = prod_mod(q, L, -1, b[k]);
    C->QmodB[k] = Qb;
    C->negQB[k] = to_mont((b[k] - Qb) % b[k], b[k]);
    // B -> Q
    uint64_t bh = prod_mod(b, K, k, b[k]);
    C->QBinv[k] = h_mulmod(h_invmod(Qb, b[k]), h_invmod(bh, b[k]), b[k]);
    C->QBinv_s[k] = h_shoup(C->QBinv[k], b[k]);
    recip128(b[k], &C->omb_hi[k], &C->omb_lo[k]);
    for (int i = 0; i < L; ++i) C->MBQ[k][i] = to_mont(prod_mod(b, K, k, q[i]), q[i]);
  }
  for (int i = 0; i < L; ++i) {
    uint64_t Bq = prod_mod(b, K, -1, q[i]);
    C->negBQ[i] = to_mont((q[i] - Bq) % q[i], q[i]);
  }
  // Garner digits of (Q-1)/2: residue mod q_i is (q_i - 1)/2
  uint64_t dig[L];
  for (int i = 0; i < L; ++i) {
    for (int j = 0; j < L; ++j) {
      C->mrc_inv[j][i] = j < i ? h_invmod(q[j] % q[i], q[i]) : 0;
      C->mrc_inv_s[j][i] = j < i ? h_shoup(C->mrc_inv[j][i], q[i]) : 0;
    }
  }
  for (int i = 0; i < L; ++i) {
    uint64_t x = (q[i] - 1) / 2;
    for (int j = 0; j < i; ++j) {
      uint64_t d = dig[j] % q[i];
      x = x >= d ? x - d : x + q[i] - d;
      x = h_mulmod(x, C->mrc_inv[j][i], q[i]);
    }
    dig[i] = x;
    C->half_digit[i] = x;
  }
  // mod-down and plaintext constants
  uint64_t Qt = prod_mod(q, L, -1, t);
  uint64_t tinvq, rt = Qt;  // Q = t Delta + rt
  for (int i = 0; i < L; ++i) {
    C->Pinv[i] = h_invmod(P % q[i], q[i]);
    C->Pinv_s[i] = h_shoup(C->Pinv[i], q[i]);
    C->r32[i] = (uint64_t)(((unsigned __int128)1 << 32) % q[i]);
    C->r32_s[i] = h_shoup(C->r32[i], q[i]);
    C->Pmodq[i] = P % q[i];
    tinvq = h_invmod(t, q[i]);
    C->delta[i] = h_mulmod((q[i] - rt % q[i]) % q[i], tinvq, q[i]);  // (Q - rt)/t mod q_i
    C->delta_s[i] = h_shoup(C->delta[i], q[i]);
    C->tqhatinv[i] = h_mulmod(t, C->qhatinv[i], q[i]);
    C->tqhatinv_s[i] = h_shoup(C->tqhatinv[i], q[i]);
    C->MQt[i] = to_mont(prod_mod(q, L, i, t), t);
  }
  for (int k = 0; k < K; ++k) {
    C->r32b[k] = (uint64_t)(((unsigned __int128)1 << 32) % b[k]);
    C->r32b_s[k] = h_shoup(C->r32b[k], b[k]);
  }
  // mixed-radix recombination constants [q_ga ... q_ga+m-1]_{p_j} for both groupings
  for (int j = 0; j < NKS; ++j) {
    const uint64_t pj = j < L ? q[j] : P;
    for (int a = 0; a < NDIG; ++a) {
      uint64_t c = 1;
      for (int m = 1; m < DIGIT_PRIMES; ++m) {
        c = h_mulmod(c, q[DIGIT_PRIMES * a + m - 1] % pj, pj);
        C->digm3[m - 1][a][j] = c;
        C->digm3_s[m - 1][a][j] = h_shoup(c, pj);
      }
    }
    for (int a = 0; a < NDIG5; ++a) {
      uint64_t c = 1;
      for (int m = 1; m < DIGIT_PRIMES5; ++m) {
        c = h_mulmod(c, q[DIGIT_PRIMES5 * a + m - 1] % pj, pj);
        C->digm5[m - 1][a][j] = c;
        C->digm5_s[m - 1][a][j] = h_shoup(c, pj);
      }
    }
    for (int a = 0; a < NDIG2; ++a) {
      uint64_t c = 1;
      const int base = COARSE_DIGIT_PRIMES * a, g = std::min(COARSE_DIGIT_PRIMES, L - base);
      for (int m = 1; m < COARSE_DIGIT_PRIMES; ++m) {
        if (m < g) c = h_mulmod(c, q[base + m - 1] % pj, pj);
        C->digm8[m - 1][a][j] = m < g ? c : 0;
        C->digm8_s[m - 1][a][j] = m < g ? h_shoup(c, pj) : 0;
      }
    }
  }
  C->negQt = to_mont((t - Qt) % t, t);
  // 28-bit limb splits of the conversion matrices (device multiply-accumulate)
  const uint64_t M28 = (1ULL << 28) - 1;
  for (int i = 0; i < L; ++i)
    for (int k = 0; k < K; ++k) {
      C->MQB_l[i][k] = (uint32_t)(C->MQB[i][k] & M28);
      C->MQB_h[i][k] = (uint32_t)(C->MQB[i][k] >> 28);
      C->MBQ_l[k][i] = (uint32_t)(C->MBQ[k][i] & M28);
      C->MBQ_h[k][i] = (uint32_t)(C->MBQ[k][i] >> 28);
    }
  for (int k = 0; k < K; ++k) {
    C->negQB_l[k] = (uint32_t)(C->negQB[k] & M28);
    C->negQB_h[k] = (uint32_t)(C->negQB[k] >> 28);
  }
  for (int i = 0; i < L; ++i) {
    C->negBQ_l[i] = (uint32_t)(C->negBQ[i] & M28);
    C->negBQ_h[i] = (uint32_t)(C->negBQ[i] >> 28);
  }
  C->Qinv_t = h_invmod(Qt, t);
  return 0;
}

// Odd coefficients h_m = c_{2m+1} (m < 32768) of the LT polynomial over F_65537:
// c_k = sum_{b=1}^{32768} b^(p-1-k) for odd k.  All power sums S(e) = sum_{b<=32768}
// b^e come from one cyclic transform of length p - 1 = 2^16 with root g = 3 (a
// generator of F_p^*): writing b = g^u, S(e) = sum_u [g^u <= 32768] (g^e)^u.
int lt_coefficients(uint32_t* out) {
  const uint64_t p = 65537, n = 65536, g = 3;
  std::vector<uint64_t> a(n, 0);
  uint64_t x = 1;
  for (uint64_t u = 0; u < n; ++u) {
    a[u] = x <= (p - 1) / 2 ? 1 : 0;
    x = x * g % p;
  }
  for (uint64_t i = 1, j = 0; i < n; ++i) {  // bit-reversal permutation
    uint64_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (uint64_t len = 2; len <= n; len <<= 1) {  // DIT butterflies, root of order len = g^(n/len)
    const uint64_t wl = h_powmod(g, n / len, p);
    for (uint64_t st = 0; st < n; st += len) {
      uint64_t w = 1;
      for (uint64_t k = 0; k < len / 2; ++k) {
        const uint64_t u = a[st + k], v = a[st + k + len / 2] * w % p;
        a[st + k] = (u + v) % p;
        a[st + k + len / 2] = (u + p - v) % p;
        w = w * wl % p;
      }
    }
  }
  for (uint64_t m = 0; m < (p - 1) / 2; ++m) out[m] = (uint32_t)a[(p - 2 - 2 * m) % n];
  return 0;
}

// f16 bit pattern of an integer below 2048 (exact: at most 11 significant bits)
// f16 bit pattern of an integer v < 2^16 that f16 holds exactly (v < 2048, or
// v with no bits below its eleven leading ones)
static uint16_t f16_of_int(uint32_t v) {
  if (v == 0) return 0;
  const int e = 31 - __builtin_clz(v);  // v = 1.m 2^e
  const uint32_t m = e <= 10 ? v << (10 - e) : v >> (e - 10);
  return (uint16_t)(((uint32_t)(e + 15) << 10) | (m & 0x3FFu));
}
static int tc_cm_host(int r, int k) { return ((r >> 3) * (TC_K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

// limb l (8 bits) of floor(2^(64 + 8a) / m), the fixed-point weight of limb a
// of a residue mod m in sum_i y_i / m_i (m > 2^54, a < 7: the value is < 2^58)
static uint32_t fix_limb(uint64_t m, int a, int l) {
  const u128 c = ((u128)1 << (64 + 8 * a)) / m;
  return (uint32_t)(c >> (8 * l)) & 255u;
}

void build_tc_tables(const Consts& C, uint16_t* ops, uint64_t* tabs) {
  const uint64_t* q = C.p;
  const uint64_t* b = C.p + L;
  uint16_t* B1L = ops + TCT_B1L;
  uint16_t* B1S = ops + TCT_B1S;
  uint16_t* B2 = ops + TCT_B2;
  memset(ops, 0, sizeof(uint16_t) * TCT_OPS);
  for (int k = 0; k < K; ++k)
    for (int i = 0; i < L; ++i) {
      uint64_t c = prod_mod(q, L, i, b[k]);          // [Q/q_i]_{b_k}
      uint64_t cs = h_mulmod(c, C.QBinv[k], b[k]);  // times [Q^{-1} (B/b_k)^{-1}]_{b_k}
      for (int a = 0; a < 7; ++a, c = h_mulmod(c, 256, b[k]), cs = h_mulmod(cs, 256, b[k]))
        for (int l = 0; l < 7; ++l) {
          B1L[tc_cm_host(8 * k + l, 8 * i + a)] = f16_of_int((uint32_t)(c >> (8 * l)) & 255);
          B1S[tc_cm_host(8 * k + l, 8 * i + a)] = f16_of_int((uint32_t)(cs >> (8 * l)) & 255);
        }
    }
  for (int l = 0; l < 8; ++l)  // the fixed-point sum of y_i / q_i in column 8l + 7
    for (int i = 0; i < L; ++i)
      for (int a = 0; a < 7; ++a) {
        B1L[tc_cm_host(8 * l + 7, 8 * i + a)] = f16_of_int(fix_limb(q[i], a, l));
        B1S[tc_cm_host(8 * l + 7, 8 * i + a)] = f16_of_int(fix_limb(q[i], a, l));
      }
  for (int i = 0; i < L; ++i)
    for (int k = 0; k < K; ++k) {
      uint64_t c = prod_mod(b, K, k, q[i]);  // [B/b_k]_{q_i}
      for (int a = 0; a < 7; ++a, c = h_mulmod(c, 256, q[i]))
        for (int l = 0; l < 7; ++l) B2[tc_cm_host(8 * i + l, 8 * k + a)] = f16_of_int((uint32_t)(c >> (8 * l)) & 255);
    }
  for (int l = 0; l < 8; ++l)  // the fixed-point sum of y_k / b_k in columns 120 .. 127
    for (int k = 0; k < K; ++k)
      for (int a = 0; a < 7; ++a) B2[tc_cm_host(8 * L + l, 8 * k + a)] = f16_of_int(fix_limb(b[k], a, l));
  for (int n = 0; n < TC_ROWS; ++n)  // the bias columns: 2^23 added to every accumulator word
    for (int c = 0; c < 2; ++c) {
      B1L[tc_cm_host(n, TC_BIAS1[c])] = f16_of_int(2048);
      B1S[tc_cm_host(n, TC_BIAS1[c])] = f16_of_int(2048);
      B2[tc_cm_host(n, TC_BIAS2[c])] = f16_of_int(2048);
    }
  uint64_t* T1 = tabs + TCT_T1;
  uint64_t* T1S = tabs + TCT_T1S;
  uint64_t* T2 = tabs + TCT_T2;
  for (int v = 0; v < 16; ++v)
    for (int k = 0; k < 16; ++k) {
      const uint64_t Qb = prod_mod(q, L, -1, b[k]);
      T1[v * 16 + k] = (b[k] - h_mulmod((uint64_t)v, Qb, b[k])) % b[k];
      T1S[v * 16 + k] = h_mulmod(T1[v * 16 + k], C.QBinv[k], b[k]);
    }
  for (int v = 0; v <= 2 * K; ++v)
    for (int i = 0; i < 16; ++i) {
      if (i >= L) {
        T2[v * 16 + i] = 0;
        continue;
      }
      const uint64_t Bq = prod_mod(b, K, -1, q[i]);
      T2[v * 16 + i] = (q[i] - h_mulmod((uint64_t)v, Bq, q[i])) % q[i];
    }
}

// ---- invariant-noise budget model --------------------------------------------
// Budgets in bits, log2(Q / (2 |v|)) for the invariant noise v.  The model:
//   fresh          log Q - log t - log N - 8 (a fresh encryption, |e| <= 21)
//   per level      log t + log N + 1 (a product multiplies the noise by about t N)
//   key switching  a product relinearised with digits of g data primes adds
//                  noise |digit| sqrt(N) 2^6 / P, so its budget is at most
//                  (log Q - log t) - (log |digit| + log N / 2 + 6 - log P)
// B(d) = min(B(d-1) - per level, key-switching bound of the key used at depth d):
// the three-prime key's bound (about 686 bits at N = 32768; the five-prime
// key's about 576, the two-digit key's about 410) is what costs budget when a
// level uses it while the product's own budget is still above it; the
// per-prime key's lies above the fresh budget.  Every constant sits on the conservative side of the oracle's
// measured budgets (per level 27.6 bits measured at N = 4096, 30.3 at N = 32768).
struct NoiseModel {
  double fresh, per_level, ks3, ks1, ks8;  // ks3: the cap of the handle's main grouping (3 or 5 primes)
  int fine_depth, coarse_from;
  // the cap of the key that relinearises a product at depth d
  double cap(int d) const { return d <= fine_depth ? ks1 : (coarse_from > 0 && d >= coarse_from ? ks8 : ks3); }
};
// the largest digit, in bits, of digits of dp consecutive data primes
static double digit_bits(const uint64_t* q, int nq, int dp) {
  double best = 0;
  for (int a = 0; a * dp < nq; ++a) {
    double g = 0;
    for (int i = a * dp; i < nq && i < (a + 1) * dp; ++i) g += log2((double)q[i]);
    best = best > g ? best : g;
  }
  return best;
}
static NoiseModel noise_model(int log_n, const uint64_t* q, int nq, uint64_t P, uint64_t t, int dp, int fine_depth,
                              int coarse_from) {
  double lq = 0;
  for (int i = 0; i < nq; ++i) lq += log2((double)q[i]);
  const double lt = log2((double)t), lp = log2((double)P);
  auto ks_cap = [&](int g) { return (lq - lt) - (digit_bits(q, nq, g) + 0.5 * log_n + 6.0 - lp); };
  NoiseModel m;
  m.fresh = lq - lt - log_n - 8.0;
  m.per_level = lt + log_n + 1.0;
  m.ks3 = ks_cap(dp);
  m.ks1 = ks_cap(1);
  m.ks8 = ks_cap(COARSE_DIGIT_PRIMES);
  m.fine_depth = fine_depth;
  m.coarse_from = coarse_from;
  return m;
}
// budget after a chain of products whose d-th lies at depth d (d = 1 .. depth)
static double chain_budget(const NoiseModel& m, int depth) {
  double b = m.fresh;
  for (int d = 1; d <= depth; ++d) b = std::min(b - m.per_level, m.cap(d));
  return b;
}

double budget_estimate(int log_n, const uint64_t* q, int nq, uint64_t P, uint64_t t, int dp, int fine_depth,
                       int coarse_from, int op, int in_depth, double in_bits) {
  const NoiseModel m = noise_model(log_n, q, nq, P, t, dp, fine_depth, coarse_from);
  // a product of a fresh operand with one of budget `bits` lying at depth `d`
  auto product = [&](double bits, int d) { return std::min(std::min(bits, m.fresh) - m.per_level, m.cap(d)); };
  // LT: the giant-step sum adds 128 products of depth <= 17 (7 bits), the
  // scalar combinations before them scale the baby-step noise by < 2^24, which
  // stays below the giant powers' (at least 7 levels deeper)
  const double lt = chain_budget(m, 18) - 8.0;
  switch (op) {
    case BUDGET_EQ: return chain_budget(m, 16);
    case BUDGET_SELECT: return product(chain_budget(m, 16), 17);
    case BUDGET_SQUARE: return chain_budget(m, 1);
    case BUDGET_LT: return lt;
    case BUDGET_BETWEEN: return product(lt, 19) - 1.0;  // two LT results, each at budget lt
    case BUDGET_PRODUCT: return product(in_bits, in_depth + 1);
    case BUDGET_ROTATE_SUM: return std::min(in_bits - log_n - 1.0, m.ks3);  // N slots summed
    default: return -1e9;
  }
}

int supported_depth(int log_n, const uint64_t* q, int nq, uint64_t P, uint64_t t) {
  double lq = 0;
  for (int i = 0; i < nq; ++i) lq += log2((double)q[i]);
  double lt = log2((double)t);
  // fresh invariant-noise budget and the per-squaring cost, both on the
  // conservative side of the oracle's measured budgets (e.g. 793 bits fresh,
  // about 31 bits per squaring at N = 32768)
  double fresh = lq - lt - log_n - 8.0;
  double per = lt + log_n + 2.0;
  if (fresh <= 0) return 0;
  // key switching adds |digit| sqrt(N) 2^4 / P at every level; it bounds the
  // budget left after the first squaring (digits: groups of DIGIT_PRIMES primes)
  double dbits = 0;
  for (int a = 0; a * DIGIT_PRIMES < nq; ++a) {
    double g = 0;
    for (int i = a * DIGIT_PRIMES; i < nq && i < (a + 1) * DIGIT_PRIMES; ++i) g += log2((double)q[i]);
    dbits = dbits > g ? dbits : g;
  }
  double b1 = fresh - per;
  const double ks = (lq - lt) - (dbits + 0.5 * log_n + 4.0 - log2((double)P));
  if (ks < b1) b1 = ks;
  if (b1 <= 1.0) return 0;
  return 1 + (int)floor((b1 - 1.0) / per);
}

}  // namespace hp
