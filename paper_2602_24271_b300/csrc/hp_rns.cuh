// Element-wise RNS kernels of one squaring + relinearisation (textbook FV,
// bit-exact):
//   k_lift        (x - y) or x, centred-lifted exactly from Q to Q u B
//   k_tensor      d0 = a0^2, d1 = 2 a0 a1, d2 = a1^2 (NTT domain, Montgomery)
//   k_scale_round w = round(t d / Q) mod Q, exactly, via r = [t d]_Q lifted to B
//   k_ks_mac      u_j = sum_i digit_i rk_{i,j} (NTT domain, 128-bit lazy sums)
//   k_moddown     c += round(u / P) mod Q  (optionally fused with "1 -")
#pragma once
#include "hp_device.cuh"

namespace hp {

constexpr int EW_THREADS = 256;

// status bits written by kernels (never expected; checked by the host)
enum { ST_BQ_WINDOW = 1, ST_TC_TIMEOUT = 2 };  // device status bits

// Difference modes of the first lift (row a1).  LIFT_SUB_PT subtracts
// (Delta m, 0) for a plaintext polynomial m per ciphertext (sub: [nct][N],
// coefficients < t): the packed form of x = c with per-slot constants.
// LIFT_SUB_CONSTS subtracts (Delta c_b, 0) with one constant per ciphertext
// (sub: uint64 [nct], values < t): the fan-out of one column against many
// constants (GROUP BY, IN).
enum { LIFT_COPY = 0, LIFT_SUB_CT = 1, LIFT_SUB_CONST = 2, LIFT_SUB_PT = 3, LIFT_SUB_CONSTS = 4 };

// One thread per (ciphertext b, component c, coefficient n).
// src, sub: [nct][2][L][N]; ext: [nct][2][NQB][N].
__global__ void __launch_bounds__(EW_THREADS) k_lift(const uint64_t* __restrict__ src, const uint64_t* __restrict__ sub,
                                                     uint64_t const_val, int mode, uint64_t* __restrict__ ext, int logN,
                                                     int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * 2 * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t bc = gid >> logN;  // b * 2 + c
  const int comp = (int)(bc & 1);
  const uint64_t* x = src + bc * L * N + n;
  uint64_t* o = ext + bc * NQB * N + n;
  uint64_t y[L];
  Fix F = {0, 0};
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const uint64_t p = cK.p[i];
    uint64_t v = x[(size_t)i * N];
    if (mode == LIFT_SUB_CT) {
      v = sub_mod(v, sub[bc * L * N + (size_t)i * N + n], p);
    } else if (mode == LIFT_SUB_CONST && comp == 0 && n == 0) {
      v = sub_mod(v, mul_shoup(const_val, cK.delta[i], cK.delta_s[i], p), p);
    } else if (mode == LIFT_SUB_PT && comp == 0) {
      v = sub_mod(v, mul_shoup(sub[(bc >> 1) * N + n], cK.delta[i], cK.delta_s[i], p), p);
    } else if (mode == LIFT_SUB_CONSTS && comp == 0 && n == 0) {
      v = sub_mod(v, mul_shoup(sub[bc >> 1], cK.delta[i], cK.delta_s[i], p), p);
    }
    o[(size_t)i * N] = v;
    y[i] = mul_shoup(v, cK.qhatinv[i], cK.qhatinv_s[i], p);
    fix_add(F, fix_term(y[i], cK.om_hi[i], cK.om_lo[i]));
  }
  const uint32_t v = (uint32_t)lift_v_mem(F, o, N);  // exact path re-reads the residues written above
  uint32_t yl[L], yh[L];
#pragma unroll
  for (int i = 0; i < L; ++i) yl[i] = lo28(y[i]), yh[i] = hi28(y[i]);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t b = cK.p[L + k];
    Acc3 a;
    acc3_zero(a);
#pragma unroll
    for (int i = 0; i < L; ++i) acc3_mac(a, yl[i], yh[i], cK.MQB_l[i][k], cK.MQB_h[i][k]);
    acc3_mac(a, v, 0, cK.negQB_l[k], cK.negQB_h[k]);
    o[(size_t)(L + k) * N] = redc(acc3_fold(a), b, cK.pinv[L + k]);
  }
}

// One thread per (b, prime index pi in Q u B, n).  ext values in [0, 8p) (NTT
// domain), so every product is below 64 p^2 < p 2^64 as Montgomery reduction
// requires.  dprod: [nct][3][NQB][N], values a b 2^-64 in [0, 2p).
__global__ void __launch_bounds__(EW_THREADS) k_tensor_sq(const uint64_t* __restrict__ ext, uint64_t* __restrict__ dprod,
                                                          int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * NQB * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t bp = gid >> logN;
  const int pi = (int)(bp % NQB);
  const size_t b = bp / NQB;
  const uint64_t p = cK.p[pi], pinv = cK.pinv[pi], p2 = 2 * p;
  const uint64_t a0 = ext[((b * 2 + 0) * NQB + pi) * N + n];
  const uint64_t a1 = ext[((b * 2 + 1) * NQB + pi) * N + n];
  uint64_t d1 = 2 * mont_mul_lazy(a0, a1, p, pinv);
  dprod[((b * 3 + 0) * NQB + pi) * N + n] = mont_mul_lazy(a0, a0, p, pinv);
  dprod[((b * 3 + 1) * NQB + pi) * N + n] = d1 >= p2 ? d1 - p2 : d1;
  dprod[((b * 3 + 2) * NQB + pi) * N + n] = mont_mul_lazy(a1, a1, p, pinv);
}

// General tensor of ciphertexts a and b (SELECT): d1 = a0 b1 + a1 b0.
__global__ void __launch_bounds__(EW_THREADS) k_tensor_gen(const uint64_t* __restrict__ ea, const uint64_t* __restrict__ eb,
                                                           uint64_t* __restrict__ dprod, int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * NQB * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t bp = gid >> logN;
  const int pi = (int)(bp % NQB);
  const size_t b = bp / NQB;
  const uint64_t p = cK.p[pi], pinv = cK.pinv[pi];
  const uint64_t a0 = ea[((b * 2 + 0) * NQB + pi) * N + n], a1 = ea[((b * 2 + 1) * NQB + pi) * N + n];
  const uint64_t b0 = eb[((b * 2 + 0) * NQB + pi) * N + n], b1 = eb[((b * 2 + 1) * NQB + pi) * N + n];
  Acc x;
  acc_zero(x);
  acc_mac(x, a0, b1);
  acc_mac(x, a1, b0);
  dprod[((b * 3 + 0) * NQB + pi) * N + n] = mont_mul_lazy(a0, b0, p, pinv);
  dprod[((b * 3 + 1) * NQB + pi) * N + n] = redc_lazy(x, p, pinv);
  dprod[((b * 3 + 2) * NQB + pi) * N + n] = mont_mul_lazy(a1, b1, p, pinv);
}

// A key-switching digit of G primes from a coefficient's residues r[m] mod
// q_{base+m} (m < G): the digit [d]_{q_base ... q_base+G-1} = t_0 + q_base t_1 +
// q_base q_base+1 t_2 + ... is kept as its mixed-radix form (t_0, ..., t_{G-1}),
// t_0 = r_0 and t_m = (((r_m - t_0) q_base^{-1} - t_1) q_base+1^{-1} - ...) q_base+m-1^{-1}
// mod q_base+m (Garner).  Data primes lie within a factor 2 of each other, so a
// canonical t_k < q_k < 2 q_m: each step takes v + 2 q_m - t_k (positive, below
// 6 q_m for v < 4 q_m) times the inverse with the three-partial-product Shoup
// quotient (result in [0, 4 q_m)); two conditional subtractions make t_m
// canonical at the end.
template <int G>
HPD void digit_mixed_radix(uint64_t (&r)[G], int base) {
#pragma unroll
  for (int m = 1; m < G; ++m) {
    const int im = base + m;
    const uint64_t qm = cK.p[im];
    uint64_t v = r[m];
#pragma unroll
    for (int k = 0; k < m; ++k)
      v = mul_shoup_q3(v + 2 * qm - r[k], cK.mrc_inv[base + k][im], cK.mrc_inv_s[base + k][im], qm);
    r[m] = csub(csub(v, 2 * qm), qm);
  }
}

// One thread per (b, j in {0,1,2}, n).  dprod holds t d (coefficient domain,
// canonical) in Q u B.  Writes w = round(t d / Q) mod q_i to w3[b][j][i][n].
//
// r = [t d]_Q is lifted exactly (centred) to B; then w = (t d - r) / Q is an
// exact integer with |w| <= t N Q / 2 + 1 < B / 2^24, known mod B as
// (t d - r) Q^{-1}; its centred conversion B -> Q needs no fallback because
// w / B is within 2^-24 of an integer, far from 1/2.
__global__ void __launch_bounds__(EW_THREADS) k_scale_round(const uint64_t* __restrict__ dprod, uint64_t* __restrict__ w3,
                                                            int* __restrict__ status, int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * 3 * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t bj = gid >> logN;  // b * 3 + j
  const uint64_t* d = dprod + bj * NQB * N + n;
  uint64_t y[L];
  Fix F = {0, 0};
#pragma unroll
  for (int i = 0; i < L; ++i) {
    y[i] = mul_shoup(d[(size_t)i * N], cK.qhatinv[i], cK.qhatinv_s[i], cK.p[i]);
    fix_add(F, fix_term(y[i], cK.om_hi[i], cK.om_lo[i]));
  }
  const uint32_t v = (uint32_t)lift_v_mem(F, d, N);  // lifted value r = [t d]_Q has residues d_i
  uint32_t yl[L], yh[L];
#pragma unroll
  for (int i = 0; i < L; ++i) yl[i] = lo28(y[i]), yh[i] = hi28(y[i]);
  uint64_t yb[K];
  Fix G = {0, 0};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t b = cK.p[L + k];
    Acc3 a;
    acc3_zero(a);
#pragma unroll
    for (int i = 0; i < L; ++i) acc3_mac(a, yl[i], yh[i], cK.MQB_l[i][k], cK.MQB_h[i][k]);
    acc3_mac(a, v, 0, cK.negQB_l[k], cK.negQB_h[k]);
    const uint64_t r = redc(acc3_fold(a), b, cK.pinv[L + k]);
    const uint64_t z = sub_mod(d[(size_t)(L + k) * N], r, b);
    yb[k] = mul_shoup(z, cK.QBinv[k], cK.QBinv_s[k], b);
    fix_add(G, fix_term(yb[k], cK.omb_hi[k], cK.omb_lo[k]));
  }
  int vb = fix_round(G, 2 * K);
  if (vb < 0) {  // cannot happen for |w| < B / 2^24; recorded for the host
    atomicOr(status, ST_BQ_WINDOW);
    vb = (int)G.hi;
  }
  uint64_t* o = w3 + bj * L * N + n;
  uint32_t bl[K], bh[K];
#pragma unroll
  for (int k = 0; k < K; ++k) bl[k] = lo28(yb[k]), bh[k] = hi28(yb[k]);
  const bool digits = (bj % 3) == 2;  // d2 is stored as key-switching digits (uniform per warp)
#pragma unroll
  for (int g = 0; g < NDIG; ++g) {
    uint64_t r[DIGIT_PRIMES];
#pragma unroll
    for (int e = 0; e < DIGIT_PRIMES; ++e) {
      const int i = g * DIGIT_PRIMES + e;
      const uint64_t p = cK.p[i];
      Acc3 a;
      acc3_zero(a);
#pragma unroll
      for (int k = 0; k < K; ++k) acc3_mac(a, bl[k], bh[k], cK.MBQ_l[k][i], cK.MBQ_h[k][i]);
      acc3_mac(a, (uint32_t)vb, 0, cK.negBQ_l[i], cK.negBQ_h[i]);
      r[e] = redc(acc3_fold(a), p, cK.pinv[i]);
    }
    if (digits) digit_mixed_radix<DIGIT_PRIMES>(r, g * DIGIT_PRIMES);
#pragma unroll
    for (int e = 0; e < DIGIT_PRIMES; ++e) o[(size_t)(g * DIGIT_PRIMES + e) * N] = r[e];
  }
}

HPD int ks_id(int j) { return j < L ? j : ID_P; }

// One thread per (target j, n), looping over the tile's ciphertexts so that
// each key word is read once per launch.  rk: [ND][2][NKS][N], NTT domain,
// Montgomery form (canonical); digits in [0, 8p): sums < ND 8 p^2 < p 2^64
// for ND <= 15.  ksin: [nct][ND][NKS][N]; ksout: [nct][2][NKS][N] in [0, 2p).
// ND = NDIG (three-prime digits) or NDIG_FINE (per-prime digits).
template <int ND>
__global__ void __launch_bounds__(EW_THREADS) k_ks_mac(const uint64_t* __restrict__ ksin, const uint64_t* __restrict__ rk,
                                                       uint64_t* __restrict__ ksout, int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)NKS * N) return;
  const int n = (int)(gid & (N - 1));
  const int j = (int)(gid >> logN);
  const int id = ks_id(j);
  const uint64_t p = cK.p[id], pinv = cK.pinv[id];
  uint64_t k0[ND], k1[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    k0[i] = rk[((size_t)(i * 2 + 0) * NKS + j) * N + n];
    k1[i] = rk[((size_t)(i * 2 + 1) * NKS + j) * N + n];
  }
  for (int b = 0; b < nct; ++b) {
    Acc a0, a1;
    acc_zero(a0);
    acc_zero(a1);
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      const uint64_t d = ksin[(((size_t)b * ND + i) * NKS + j) * N + n];
      acc_mac(a0, d, k0[i]);
      acc_mac(a1, d, k1[i]);
    }
    ksout[(((size_t)b * 2 + 0) * NKS + j) * N + n] = redc_lazy(a0, p, pinv);
    ksout[(((size_t)b * 2 + 1) * NKS + j) * N + n] = redc_lazy(a1, p, pinv);
  }
}

// x mod q for x < 4q
HPD uint64_t red4(uint64_t x, uint64_t q) {
  x = x >= 2 * q ? x - 2 * q : x;
  return csub(x, q);
}

// One thread per (b, comp, i, n):
//   out = w + (u_i - [u_P]) P^{-1} mod q_i,   [u_P] the centred residue mod P.
// one_minus: additionally out <- (Delta - out) for comp 0 at n = 0, -out otherwise.
__global__ void __launch_bounds__(EW_THREADS) k_moddown(const uint64_t* __restrict__ ksout, const uint64_t* __restrict__ w3,
                                                        uint64_t* __restrict__ out, int one_minus, int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * 2 * L * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t bci = gid >> logN;
  const int i = (int)(bci % L);
  const size_t bc = bci / L;
  const int comp = (int)(bc & 1);
  const size_t b = bc >> 1;
  const uint64_t q = cK.p[i], P = cK.p[ID_P];
  const uint64_t uP = ksout[(bc * NKS + L) * N + n];
  const uint64_t ui = ksout[(bc * NKS + i) * N + n];
  uint64_t diff;
  if (uP <= (P - 1) / 2) {
    diff = sub_mod(ui, red4(uP, q), q);
  } else {
    diff = add_mod(ui, red4(P - uP, q), q);
  }
  uint64_t ks = mul_shoup(diff, cK.Pinv[i], cK.Pinv_s[i], q);
  uint64_t w = w3[((b * 3 + comp) * L + i) * N + n];
  uint64_t r = add_mod(w, ks, q);
  if (one_minus) {
    r = sub_mod(0, r, q);
    if (comp == 0 && n == 0) r = add_mod(r, cK.delta[i], q);
  }
  out[gid] = r;
}

// Plaintext slots of a tile of slot-packed instances: slot j of ciphertext
// ct0 + c gets the constant of the instance whose global slot range
// [start, start + len) contains (ct0 + c) N + j, or 0.  Instances sorted by
// start, non-overlapping.  M: [nct][N] (input of the encoding transform).
__global__ void k_pack_slots(const uint64_t* __restrict__ start, const uint32_t* __restrict__ len,
                             const uint64_t* __restrict__ cval, int n_inst, uint64_t ct0, uint64_t* __restrict__ M,
                             int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * N) return;
  const uint64_t g = (ct0 << logN) + gid;
  int lo = 0, hi = n_inst - 1, f = -1;  // last instance with start <= g
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= g) {
      f = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  M[gid] = (f >= 0 && g < start[f] + len[f]) ? cval[f] : 0;
}

// ---- ciphertext-level linear operations (LT comparison) -----------------------
// Word w of an array of ciphertexts [b][2][L][N] lives mod q_{(w >> logN) % L}.
HPD int prime_of_word(size_t w, int logN) { return (int)((w >> logN) % L); }

// out = a - b (or a + b)
__global__ void k_ct_addsub(const uint64_t* __restrict__ a, const uint64_t* __restrict__ b, uint64_t* __restrict__ out,
                            int subtract, int logN, size_t nwords) {
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwords) return;
  const uint64_t q = cK.p[prime_of_word(w, logN)];
  out[w] = subtract ? sub_mod(a[w], b[w], q) : add_mod(a[w], b[w], q);
}

// out = x - (Delta v, 0), or (Delta v, 0) - x when `from_const` (BETWEEN's
// differences against plaintext bounds); v < t
__global__ void k_ct_const_diff(const uint64_t* __restrict__ x, uint64_t v, int from_const, uint64_t* __restrict__ out,
                                int logN, size_t nwords) {
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwords) return;
  const size_t poly = w >> logN;
  const int i = (int)(poly % L), comp = (int)((poly / L) & 1);
  const uint64_t q = cK.p[i];
  uint64_t r = x[w];
  if (comp == 0 && (w & ((1u << logN) - 1)) == 0) r = sub_mod(r, mul_shoup(v, cK.delta[i], cK.delta_s[i], q), q);
  out[w] = from_const ? sub_mod(0, r, q) : r;
}

// out += a (IN accumulation of one tile of masks into the running sum; out
// and a are distinct buffers, out is read and written in place)
__global__ void k_ct_acc(uint64_t* out, const uint64_t* __restrict__ a, int logN, size_t nwords) {
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwords) return;
  const uint64_t q = cK.p[prime_of_word(w, logN)];
  out[w] = add_mod(out[w], a[w], q);
}

// out = sum_k M[k] over n_const arrays of nwords words each (Eq. 6 sum of the
// GROUP BY masks in one pass: every mask is read once)
__global__ void k_ct_sum(const uint64_t* __restrict__ M, int n_const, uint64_t* __restrict__ out, int logN,
                         size_t nwords) {
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwords) return;
  const uint64_t q = cK.p[prime_of_word(w, logN)];
  uint64_t acc = 0;
  for (int k = 0; k < n_const; ++k) acc = add_mod(acc, M[(size_t)k * nwords + w], q);
  out[w] = acc;
}

// out[o] = sum of the ciphertexts x[o G .. min(n_ct, (o + 1) G)) (mod Q, word by
// word; G = group).  out may alias x when G = 1 (each word is read, then written
// by the same thread).
__global__ void k_ct_group_sum(const uint64_t* x, size_t n_ct, size_t group, uint64_t* out, int logN, size_t W,
                               size_t n_out) {
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= n_out * W) return;
  const size_t o = gid / W, w = gid - o * W;
  const uint64_t q = cK.p[prime_of_word(w, logN)];
  const size_t c0 = o * group, c1 = c0 + group < n_ct ? c0 + group : n_ct;
  uint64_t acc = 0;
  for (size_t c = c0; c < c1; ++c) acc = add_mod(acc, x[c * W + w], q);
  out[gid] = acc;
}

// Galois automorphism tau_g (rotation of the slots), gathered per output
// coefficient: tau_g(a)_n = a_j with j = n g^{-1} mod 2N when j < N, else
// -a_{j - N}.  One thread per (b, digit g, n), covering the digit's G primes;
// writes the key-switching input
//   w3[b][0] = (acc ? c0 : 0) + tau_g(c0),  w3[b][1] = acc ? c1 : 0,
//   w3[b][2] = tau_g(c1) as key-switching digits of G primes (switched from
//   tau_g(s) to s), and, with res, res[b] = tau_g(c1)'s residues (the digits'
//   values modulo their own primes, read by the digit transform),
// so the mod-down that follows yields ct + rotate(ct) (acc) or rotate(ct).
template <int G>
__global__ void k_automorph(const uint64_t* __restrict__ x, uint64_t* __restrict__ w3, uint64_t* __restrict__ res,
                            uint32_t ginv, int acc, int logN, int nct) {
  constexpr int ND = L / G;
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * ND * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t bg = gid >> logN;
  const int g = (int)(bg % ND);
  const size_t b = bg / ND;
  const uint32_t j = (uint32_t)(((uint64_t)n * ginv) & (2 * (uint64_t)N - 1));
  const uint32_t src = j < (uint32_t)N ? j : j - N;
  uint64_t r[G];
#pragma unroll
  for (int e = 0; e < G; ++e) {
    const int i = g * G + e;
    const uint64_t q = cK.p[i];
    const uint64_t* x0 = x + ((b * 2 + 0) * L + i) * N;
    const uint64_t* x1 = x + ((b * 2 + 1) * L + i) * N;
    uint64_t t0 = x0[src], t1 = x1[src];
    if (j >= (uint32_t)N) {
      t0 = sub_mod(0, t0, q);
      t1 = sub_mod(0, t1, q);
    }
    uint64_t* o = w3 + (b * 3 * L + i) * N + n;
    o[0] = acc ? add_mod(x0[n], t0, q) : t0;
    o[(size_t)L * N] = acc ? x1[n] : 0;
    if (res) res[(b * L + i) * N + n] = t1;
    r[e] = t1;
  }
  digit_mixed_radix<G>(r, g * G);
#pragma unroll
  for (int e = 0; e < G; ++e) w3[((b * 3 + 2) * L + g * G + e) * N + n] = r[e];
}

// ---- Extract (JOIN, Sec. 4.2.2): product with a plaintext unit vector --------------
// Slot-domain unit vectors of rows r0 .. r0 + nct - 1: M[c][j] = [j == (r0 + c) mod N]
// (input of the encoding transform).
__global__ void k_unit_slots(uint64_t* __restrict__ M, uint64_t r0, int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * N) return;
  const size_t c = gid >> logN;
  const uint64_t j = gid & (N - 1);
  M[gid] = j == ((r0 + c) & (N - 1)) ? 1 : 0;
}

// Plaintext polynomials (coefficients < t) to the data primes with centred
// representatives in (-t/2, t/2]: Mq[c][i][n].
__global__ void k_plain_to_q(const uint64_t* __restrict__ M, uint64_t* __restrict__ Mq, int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * L * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t ci = gid >> logN;
  const int i = (int)(ci % L);
  const size_t c = ci / L;
  const uint64_t v = M[c * N + n], t = cK.p[ID_T];
  Mq[gid] = v > t / 2 ? cK.p[i] - (t - v) : v;
}

// X[c][comp][i] <- X[c][comp][i] * Mq[c][i] 2^-64 (NTT domain, Montgomery; the
// inverse transform's scaling restores the factor)
__global__ void k_mul_plain_ntt(uint64_t* __restrict__ X, const uint64_t* __restrict__ Mq, int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * 2 * L * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t bci = gid >> logN;
  const int i = (int)(bci % L);
  const size_t c = bci / (2 * L);
  X[gid] = mont_mul_lazy(X[gid], Mq[(c * L + i) * N + n], cK.p[i], cK.pinv[i]);
}

// out = g + k G  for a small integer k (Shoup companions per prime passed by value)
struct ScalarK {
  uint64_t k[L], ks[L];
};
__global__ void k_ct_axpy(const uint64_t* __restrict__ g, const uint64_t* __restrict__ G, uint64_t* __restrict__ out,
                          ScalarK sk, int logN, size_t nwords) {
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwords) return;
  const int i = prime_of_word(w, logN);
  const uint64_t q = cK.p[i];
  out[w] = add_mod(g[w], mul_shoup(G[w], sk.k[i], sk.ks[i], q), q);
}

// Eight inner sums of the baby-step / giant-step evaluation at once:
//   out_jj = (Delta coef[256 (j0+jj)], 0) + sum_{i=1}^{255} coef[256 (j0+jj) + i] B_i,  jj < 8.
// B: [255][bw] (bw = words of one tile of ciphertexts), out: [8][bw].  Each
// coefficient is < 2^17 and each word < 2^56, split in 32-bit halves: the two
// 64-bit sums of 255 terms stay below 2^57.
constexpr int LT_J = 8;
__global__ void __launch_bounds__(EW_THREADS) k_lt_inner(const uint64_t* __restrict__ B, const uint32_t* __restrict__ coef,
                                                         int j0, uint64_t* __restrict__ out, int logN, size_t bw) {
  const size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= bw) return;
  uint64_t lo[LT_J], hi[LT_J];
#pragma unroll
  for (int jj = 0; jj < LT_J; ++jj) lo[jj] = hi[jj] = 0;
  const uint32_t* c = coef + (size_t)256 * j0;
  for (int i = 1; i < 256; ++i) {
    const uint64_t v = B[(size_t)(i - 1) * bw + w];
    const uint32_t vl = (uint32_t)v, vh = (uint32_t)(v >> 32);
#pragma unroll
    for (int jj = 0; jj < LT_J; ++jj) {
      const uint32_t k = __ldg(c + 256 * jj + i);
      lo[jj] += (uint64_t)vl * k;
      hi[jj] += (uint64_t)vh * k;
    }
  }
  const int ip = prime_of_word(w, logN);
  const uint64_t q = cK.p[ip], pbar = cK.pbar[ip];
  const bool const_slot = ((w >> logN) / L) % 2 == 0 && (w & ((1 << logN) - 1)) == 0;  // c0, coefficient 0
#pragma unroll
  for (int jj = 0; jj < LT_J; ++jj) {
    uint64_t r = mul_shoup(hi[jj], cK.r32[ip], cK.r32_s[ip], q);  // hi 2^32 mod q
    uint64_t t = lo[jj] - __umul64hi(lo[jj], pbar) * q;             // lo mod q, in [0, 2q)
    r = csub(csub(r + t, q), q);
    if (const_slot) r = add_mod(r, mul_shoup(c[256 * jj], cK.delta[ip], cK.delta_s[ip], q), q);
    out[(size_t)jj * bw + w] = r;
  }
}

// "1 -" alone: out = (Delta - c0, -c1).  One thread per word of [nct][2][L][N].
__global__ void __launch_bounds__(EW_THREADS) k_one_minus(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                          int logN, int nct) {
  const int N = 1 << logN;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * 2 * L * N) return;
  const int n = (int)(gid & (N - 1));
  const size_t bci = gid >> logN;
  const int i = (int)(bci % L);
  const int comp = (int)((bci / L) & 1);
  const uint64_t q = cK.p[i];
  uint64_t r = sub_mod(0, in[gid], q);
  if (comp == 0 && n == 0) r = add_mod(r, cK.delta[i], q);
  out[gid] = r;
}

}  // namespace hp
