// Device arithmetic of libhp: 64-bit modular operations on 32-bit integer
// ALUs, Philox4x32-10, and the exact centred RNS base conversions.
#pragma once
#include <stdint.h>

#include "hp_defs.h"

#define HPD __device__ __forceinline__

namespace hp {

// Constant block of the RNS conversions (defined here: libhp.cu is the only
// translation unit with device code).
__constant__ Consts cK;

// ---------------------------------------------------------------------------
// modular arithmetic (all moduli < 2^56)
// ---------------------------------------------------------------------------
HPD uint64_t csub(uint64_t x, uint64_t p) { return x >= p ? x - p : x; }

// Shoup multiplication by a constant w < p with wp = floor(w 2^64 / p):
// for any a < 2^64 the result a w - floor(a wp / 2^64) p lies in [0, 2p).
HPD uint64_t mul_shoup_lazy(uint64_t a, uint64_t w, uint64_t wp, uint64_t p) {
  uint64_t qh = __umul64hi(a, wp);
  return a * w - qh * p;
}
HPD uint64_t mul_shoup(uint64_t a, uint64_t w, uint64_t wp, uint64_t p) {
  return csub(mul_shoup_lazy(a, w, wp, p), p);
}
// The same product with the quotient from three 32-bit partial products
// (ah wh + hi(ah wl) + hi(al wh), the low partial product and two carries
// dropped: at most 2 below floor(a wp / 2^64)), so the result lies in [0, 4p)
// for any a < 2^64.
HPD uint64_t mul_shoup_q3(uint64_t a, uint64_t w, uint64_t wp, uint64_t p) {
  const uint32_t al = (uint32_t)a, ah = (uint32_t)(a >> 32), wl = (uint32_t)wp, wh = (uint32_t)(wp >> 32);
  const uint64_t q = (uint64_t)ah * wh + __umulhi(ah, wl) + __umulhi(al, wh);
  return a * w - q * p;
}

// 128-bit accumulator for lazy multiply-accumulate
struct Acc {
  uint64_t lo, hi;
};
HPD void acc_zero(Acc& a) { a.lo = 0; a.hi = 0; }
HPD void acc_mac(Acc& a, uint64_t x, uint64_t y) {
  uint64_t lo = x * y, hi = __umul64hi(x, y);
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(lo), "l"(hi));
}
// Montgomery reduction: for x < p 2^64 returns x 2^-64 mod p in [0, 2p).
// m = x_lo (-p^-1) mod 2^64 makes x + m p divisible by 2^64; the low words
// cancel, carrying exactly when x_lo != 0.
HPD uint64_t redc_lazy(const Acc& x, uint64_t p, uint64_t pinv) {
  uint64_t m = x.lo * pinv;
  return x.hi + __umul64hi(m, p) + (x.lo != 0 ? 1 : 0);
}
HPD uint64_t redc(const Acc& x, uint64_t p, uint64_t pinv) { return csub(redc_lazy(x, p, pinv), p); }
// a b 2^-64 mod p for a, b < p, in [0, 2p)
HPD uint64_t mont_mul_lazy(uint64_t a, uint64_t b, uint64_t p, uint64_t pinv) {
  Acc x;
  x.lo = a * b;
  x.hi = __umul64hi(a, b);
  return redc_lazy(x, p, pinv);
}
// Multiply-accumulate of 56-bit operands in 28-bit limbs: y = yh 2^28 + yl,
// m = mh 2^28 + ml; a0 += yl ml, a1 += yl mh + yh ml, a2 += yh mh, each a
// single 32x32+64 multiply-add.  Up to 17 terms stay below 2^61 per word.
struct Acc3 {
  uint64_t a0, a1, a2;
};
HPD void acc3_zero(Acc3& a) { a.a0 = a.a1 = a.a2 = 0; }
HPD void acc3_mac(Acc3& a, uint32_t yl, uint32_t yh, uint32_t ml, uint32_t mh) {
  a.a0 += (uint64_t)yl * ml;
  a.a1 += (uint64_t)yl * mh;
  a.a1 += (uint64_t)yh * ml;
  a.a2 += (uint64_t)yh * mh;
}
// a0 + a1 2^28 + a2 2^56 as a 128-bit value
HPD Acc acc3_fold(const Acc3& a) {
  Acc r;
  const uint64_t t = a.a1 << 28, u = a.a2 << 56;
  uint64_t lo = a.a0 + t;
  uint64_t c = lo < t ? 1 : 0;
  lo += u;
  c += lo < u ? 1 : 0;
  r.lo = lo;
  r.hi = (a.a1 >> 36) + (a.a2 >> 8) + c;
  return r;
}
HPD uint32_t lo28(uint64_t y) { return (uint32_t)(y & 0xFFFFFFFull); }
HPD uint32_t hi28(uint64_t y) { return (uint32_t)(y >> 28); }

HPD uint64_t add_mod(uint64_t a, uint64_t b, uint64_t p) { return csub(a + b, p); }
HPD uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t p) { return a >= b ? a - b : a + p - b; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): two 32x32->64 products
// per round, ten rounds, Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
HPD uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}
// Galois keys draw with object index (g << 5) | digit for Galois element g.
enum { DOM_S = 1, DOM_E_ENC = 2, DOM_A_ENC = 3, DOM_E_RK = 4, DOM_A_RK = 5, DOM_E_GK = 6, DOM_A_GK = 7 };
HPD int draw_ternary(uint4 w) { return (int)(((uint64_t)w.x * 3u) >> 32) - 1; }
HPD int draw_cbd21(uint4 w) { return __popc(w.x & 0x1FFFFFu) - __popc(w.y & 0x1FFFFFu); }
// floor(r m / 2^128) for the 128-bit r = w.w:w.z:w.y:w.x
HPD uint64_t draw_uniform(uint4 w, uint64_t m) {
  uint64_t lo = ((uint64_t)w.y << 32) | w.x, hi = ((uint64_t)w.w << 32) | w.z;
  uint64_t a_hi = __umul64hi(lo, m);
  uint64_t b_lo = hi * m, b_hi = __umul64hi(hi, m);
  uint64_t s = b_lo + a_hi;
  return b_hi + (s < b_lo ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Exact centred base conversion.
//
// Input residues x_i of X in [0, Q).  With y_i = [x_i (Q/q_i)^{-1}]_{q_i},
//   sum_i y_i (Q/q_i) = X + Q floor(S),  S = sum_i y_i / q_i,  frac(S) = X / Q.
// The centred representative is X~ = sum_i y_i (Q/q_i) - v Q with
// v = floor(S + 1/2) (no tie: Q is odd).  v is estimated with 64-bit fixed
// point, f_i = floor(y_i floor(2^128/q_i) / 2^64) underestimates y_i 2^64/q_i by
// less than 2, so the true S 2^64 lies in [F, F + 2L).  When that window does
// not decide v (frac(S) within 2L 2^-64 of 1/2, probability ~2^-59 per
// coefficient), v = floor(S) + [X > (Q-1)/2] is decided exactly by comparing
// mixed-radix digits.
// ---------------------------------------------------------------------------
struct Fix {
  uint64_t lo;
  uint32_t hi;
};
HPD void fix_add(Fix& F, uint64_t f) {
  F.lo += f;
  F.hi += (F.lo < f) ? 1u : 0u;
}
// fixed-point term floor(y floor(2^128/m) / 2^64)
HPD uint64_t fix_term(uint64_t y, uint64_t om_hi, uint64_t om_lo) { return y * om_hi + __umul64hi(y, om_lo); }

// Returns v if the window [F, F + width) decides floor(S + 1/2), else -1.
HPD int fix_round(const Fix& F, uint64_t width) {
  uint64_t a = F.lo + 0x8000000000000000ull;
  uint32_t va = F.hi + (a < F.lo ? 1u : 0u);
  uint64_t b = a + width;
  uint32_t vb = va + (b < a ? 1u : 0u);
  return va == vb ? (int)va : -1;
}

// [X > (Q-1)/2] for X given by residues x[i * stride] (i < L), by Garner
// mixed-radix digits.  Reads the residues from memory so that callers keep
// their working arrays in registers.
__device__ __noinline__ int greater_than_half(const uint64_t* x, size_t stride) {
  uint64_t a[L];
  for (int i = 0; i < L; ++i) {
    uint64_t p = cK.p[i];
    uint64_t v = x[(size_t)i * stride];
    for (int j = 0; j < i; ++j) {
      uint64_t d = csub(a[j], p);  // a_j < q_j < 2 q_i
      v = sub_mod(v, d, p);
      v = mul_shoup(v, cK.mrc_inv[j][i], cK.mrc_inv_s[j][i], p);
    }
    a[i] = v;
  }
  for (int i = L - 1; i >= 0; --i) {
    if (a[i] != cK.half_digit[i]) return a[i] > cK.half_digit[i] ? 1 : 0;
  }
  return 0;  // X == (Q-1)/2
}

// v = floor(S + 1/2) for a lift whose fixed-point sum is F and whose lifted
// value has residues x[i * stride] in memory (read only on the exact path).
HPD int lift_v_mem(const Fix& F, const uint64_t* x, size_t stride) {
  int v = fix_round(F, 2 * L);
  if (v < 0) v = (int)F.hi + greater_than_half(x, stride);
  return v;
}

// Same, for a lift whose residues are only known through y_i: the exact path
// rebuilds r_i = [y_i (Q/q_i)]_{q_i} into a local array (client helpers only).
__device__ __noinline__ int lift_v_from_y(const uint64_t* y, uint32_t Fhi) {
  uint64_t r[L];
  for (int i = 0; i < L; ++i) r[i] = mul_shoup(y[i], cK.qhat[i], cK.qhat_s[i], cK.p[i]);
  return (int)Fhi + greater_than_half(r, 1);
}

}  // namespace hp
