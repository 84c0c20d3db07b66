// Shared definitions of libhp (host and device): RNS bases and the constant
// block that the kernels read from __constant__ memory.
//
// Prime ids (one numbering for every table):
//   0 .. L-1        data primes q_i            (Q = prod q_i)
//   L .. L+K-1      auxiliary primes b_k       (B = prod b_k), exact tensor base
//   L+K             special prime P            (relinearisation)
//   L+K+1           plaintext modulus t = 65537
#pragma once
#include <stdint.h>

namespace hp {

constexpr int L = 15;              // data primes (paper Sec. 5.1: log QP = 881 with P)
constexpr int K = 16;              // auxiliary base: B > t N Q covers |round(t d / Q)| < B / 2
constexpr int NQB = L + K;         // primes of the extended base Q u B
constexpr int ID_P = L + K;        // 31
constexpr int ID_T = L + K + 1;    // 32
constexpr int NPRIME = L + K + 2;  // 33
constexpr int NKS = L + 1;         // key-switching targets: q_0..q_{L-1}, P
constexpr int DIGIT_PRIMES = 3;    // default data primes per key-switching digit (relinearisation, rotations)
constexpr int NDIG = L / DIGIT_PRIMES;  // its digits: digit a = [d]_{q_3a q_3a+1 q_3a+2}
static_assert(L % DIGIT_PRIMES == 0, "digits are whole groups of data primes");
// The other grouping a handle may choose (ks_digit_primes = 5): three digits
// [d]_{q_5a ... q_5a+4}, fewer key-switching transforms for more key-switching noise.
constexpr int DIGIT_PRIMES5 = 5, NDIG5 = L / DIGIT_PRIMES5;
static_assert(L % DIGIT_PRIMES5 == 0, "digits are whole groups of data primes");
// The per-prime relinearisation key (digit i = [d]_{q_i}) used for products at
// output depth <= the handle's ks_fine_depth; its digits draw Philox with
// object index FINE_OBJ + i.
constexpr int NDIG_FINE = L;
constexpr uint32_t FINE_OBJ = 16;
// The two-digit relinearisation key (digits [d]_{q_0 ... q_7} and
// [d]_{q_8 ... q_14}) used for products at output depth >= the handle's
// ks_coarse_from (0 = never); its digits draw Philox with object index
// COARSE_OBJ + a.  Digit a covers data primes 8a .. min(L, 8a + 8) - 1.
constexpr int COARSE_DIGIT_PRIMES = 8, NDIG2 = 2;
constexpr uint32_t COARSE_OBJ = 48;
static_assert(L > COARSE_DIGIT_PRIMES && L <= NDIG2 * COARSE_DIGIT_PRIMES, "two digits, the second shorter");
constexpr int LOGN_MIN = 12, LOGN_MAX = 15;

// Constants for the exact RNS base conversions, relinearisation and the
// client-side helpers.  All residues are canonical; "(s)" entries are the
// Shoup companions floor(w 2^64 / p) of the preceding constant.
struct Consts {
  uint64_t p[NPRIME];     // moduli by id
  uint64_t pinv[NPRIME];  // -p^{-1} mod 2^64 (Montgomery)
  uint64_t r2[NPRIME];    // 2^128 mod p (to enter Montgomery form)
  uint64_t pbar[NPRIME];  // floor(2^64 / p): Shoup companion of 1 (full reduction of any word)
  // exact centred conversion Q -> B
  uint64_t qhatinv[L], qhatinv_s[L];  // [(Q/q_i)^{-1}]_{q_i}
  uint64_t qhat[L], qhat_s[L];        // [Q/q_i]_{q_i} (rebuilds residues from y_i in the fallback)
  uint64_t om_hi[L], om_lo[L];        // floor(2^128 / q_i) split in 64-bit halves
  uint64_t MQB[L][K];                 // [(Q/q_i) 2^64]_{b_k}
  uint64_t negQB[K];                  // [-Q 2^64]_{b_k}
  uint32_t MQB_l[L][K], MQB_h[L][K];  // MQB in 28-bit limbs: low 28 bits, the rest
  uint32_t negQB_l[K], negQB_h[K];
  uint64_t QmodB[K];                  // [Q]_{b_k}
  // exact centred conversion B -> Q
  uint64_t QBinv[K], QBinv_s[K];  // [Q^{-1} (B/b_k)^{-1}]_{b_k}
  uint64_t omb_hi[K], omb_lo[K];  // floor(2^128 / b_k)
  uint64_t MBQ[K][L];             // [(B/b_k) 2^64]_{q_i}
  uint64_t negBQ[L];              // [-B 2^64]_{q_i}
  uint32_t MBQ_l[K][L], MBQ_h[K][L];  // MBQ in 28-bit limbs
  uint32_t negBQ_l[L], negBQ_h[L];
  // mixed-radix (Garner) comparison with (Q-1)/2, the exact fallback
  uint64_t mrc_inv[L][L], mrc_inv_s[L][L];  // [q_j^{-1}]_{q_i} for j < i
  uint64_t half_digit[L];                   // mixed-radix digits of (Q-1)/2
  // relinearisation mod-down
  uint64_t Pinv[L], Pinv_s[L];  // [P^{-1}]_{q_i}
  uint64_t r32[L], r32_s[L];    // [2^32]_{q_i} (reduction of split 64-bit sums)
  // plaintext side
  uint64_t delta[L], delta_s[L];          // [floor(Q/t)]_{q_i}
  uint64_t tqhatinv[L], tqhatinv_s[L];    // [t (Q/q_i)^{-1}]_{q_i}   (decryption)
  uint64_t MQt[L];                        // [(Q/q_i) 2^64]_t
  uint64_t negQt;                         // [-Q 2^64]_t
  uint64_t Qinv_t;                        // [Q^{-1}]_t
  uint64_t Pmodq[L];                      // [P]_{q_i}   (key generation)
  // key-switching digits of g primes in mixed radix (Garner, with the inverses
  // mrc_inv): digit a = t_0 + q_ga t_1 + q_ga q_ga+1 t_2 + ... with t_0 = [d]_{q_ga};
  // their recombination modulo a target prime p_j uses [q_ga ... q_ga+m-1]_{p_j}:
  uint64_t digm3[2][NDIG][NKS], digm3_s[2][NDIG][NKS];    // g = 3, m = 1, 2 (index m - 1)
  uint64_t digm5[4][NDIG5][NKS], digm5_s[4][NDIG5][NKS];  // g = 5, m = 1 .. 4
  uint64_t digm8[COARSE_DIGIT_PRIMES - 1][NDIG2][NKS];    // the two-digit key's groups, m = 1 .. 7 (6 for the second)
  uint64_t digm8_s[COARSE_DIGIT_PRIMES - 1][NDIG2][NKS];
  uint64_t r32b[K], r32b_s[K];                  // [2^32]_{b_k}
};

// Host side: build the constant block for (q, P, t) with the auxiliary primes
// chosen by the library.  Returns 0 on success, negative HP_ERR_* otherwise.
int build_consts(const uint64_t* q, uint64_t P, uint64_t t, Consts* out, char* err, int errlen);

// Largest `count` primes below 2^bits with p = 1 mod 2^16, descending, skipping
// the values in `exclude`.  Returns the number found.
int find_primes(int bits, int count, const uint64_t* exclude, int nexclude, uint64_t* out);
bool is_prime(uint64_t n);

// Smallest g with g^((p-1)/2) = -1 mod p; psi = g^((p-1)/2N) is then a
// primitive 2N-th root of unity.
uint64_t h_qnr(uint64_t p);
uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t m);
uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t m);
uint64_t h_invmod(uint64_t a, uint64_t m);
uint64_t h_shoup(uint64_t w, uint64_t p);

// Tables of the tensor-core base conversions (8-bit limbs, f16 operands), all
// [128][128] f16 bit patterns in the no-swizzle K-major core-matrix layout:
//   B1L (lift):   row 8k+b (k < K, b < 7), column 8i+a (i < L, a < 7):
//                 limb b of [2^(8a) (Q/q_i)]_{b_k};
//   B1S (scale-and-round): the same entries times [Q^{-1} (B/b_k)^{-1}]_{b_k}, so
//                 that the product is the B residue already multiplied by it;
//   both also:    row 8l+7 (l < 8), column 8i+a: limb l of floor(2^(64+8a) / q_i),
//                 whose column sums give sum_i y_i / q_i in 64-bit fixed point;
//   B2:           row 8i+b (i < L, b < 7), column 8k+a (k < K, a < 7):
//                 limb b of [2^(8a) (B/b_k)]_{q_i}; row 120+l: limb l of
//                 floor(2^(64+8a) / b_k) (the fixed-point sum of y_k / b_k).
//   Bias columns: 2048 in every row of columns TC_BIAS1 (B1L, B1S: 120, 121,
//                 where the A operand's unused residue slot 15 holds 2048, 2048)
//                 and TC_BIAS2 (B2: 7, 15, the zero eighth columns of residues
//                 0 and 1, where A holds 2048): every accumulator word receives
//                 2 x 2048 x 2048 = 2^23, so it holds the f32 value 2^23 + D with
//                 D < 2^23 in its low 23 bits.
// Correction tables (uint64):
//   T1 [16][16]:  [-v Q]_{b_k} for v < 16 (k < K);  T1S: the same times [Q^{-1} (B/b_k)^{-1}]_{b_k}
//   T2 [33][16]:  [-v B]_{q_i} for v <= 2K (i < L; column 15 unused): the B -> Q
//                 operand's residues lie in [0, 2 b_k), so its centring count is at most 2K
constexpr int TC_ROWS = 128, TC_K = 128, TC_T1 = 16 * 16, TC_T2 = 33 * 16;
constexpr int TC_BIAS1[2] = {120, 121}, TC_BIAS2[2] = {7, 15};
static_assert(TC_T2 == (2 * K + 1) * 16 && L < TC_K / 8 && K == TC_K / 8, "table and slot sizes");
constexpr int TC_OPER = TC_ROWS * TC_K;                       // f16 elements of one operand
constexpr int TCT_B1L = 0, TCT_B1S = TC_OPER, TCT_B2 = 2 * TC_OPER, TCT_OPS = 3 * TC_OPER;  // in f16 elements
constexpr int TCT_T1 = 0, TCT_T1S = TC_T1, TCT_T2 = 2 * TC_T1, TCT_TABS = 2 * TC_T1 + TC_T2;  // in words
void build_tc_tables(const Consts& C, uint16_t* ops, uint64_t* tabs);

// LT polynomial's odd coefficients (32768 words), see hp_host.cpp.
int lt_coefficients(uint32_t* out);

// Static noise estimate: how many successive squarings (each relinearised)
// the parameters support with a positive invariant-noise budget, from the
// heuristic growth bound (fresh budget log Q - log t - log N - 8 bits, log t +
// log N + 2 bits per squaring, the key-switching noise bounding the budget
// after the first), below the oracle's measured budgets.  Used by hp_create.
int supported_depth(int log_n, const uint64_t* q, int nq, uint64_t P, uint64_t t);

// Static estimate of the invariant-noise budget (bits) left in the result of
// one of the operations below on fresh inputs (BUDGET_PRODUCT: a fresh column
// times an operand of budget in_bits at depth in_depth; BUDGET_ROTATE_SUM: the
// rotate-and-add reduction of an operand of budget in_bits).  Operations refuse
// to run when it is below BUDGET_MARGIN.  Values match hp_budget_op in hp.h.
enum { BUDGET_EQ = 0, BUDGET_SELECT = 1, BUDGET_SQUARE = 2, BUDGET_LT = 3, BUDGET_BETWEEN = 4, BUDGET_PRODUCT = 5,
       BUDGET_ROTATE_SUM = 6 };
constexpr double BUDGET_MARGIN = 10.0;
double budget_estimate(int log_n, const uint64_t* q, int nq, uint64_t P, uint64_t t, int dp, int fine_depth,
                       int coarse_from, int op, int in_depth, double in_bits);

}  // namespace hp
