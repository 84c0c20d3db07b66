// Negacyclic NTT over 64-bit primes, batched over many polynomials.
//
// Forward (Cooley-Tukey, natural -> bit-reversed order), stage s = 0..logN-1:
//   t = N >> (s+1); for every j with bit (j / t) even:
//     (a_j, a_{j+t}) <- (a_j + W a_{j+t}, a_j - W a_{j+t}),  W = psi^{brv(2^s + j / 2t)}
// so that output position j holds m(psi^(2 brv(j) + 1)).  The inverse
// (Gentleman-Sande) undoes the stages in reverse order with psi^{-brv(.)} and
// scales by N^{-1} (times a per-launch constant).
//
// Decomposition: N = R x C (j = r C + k).  Stages s < logR pair elements of
// one column, stages s >= logR elements of one row.  Each pass is one kernel
// over a 2048-word tile; every thread keeps 16 residues in registers and runs
// 4 stages as a radix-16 block (index arithmetic once per element, one twiddle
// load per butterfly group), then the tile is exchanged once through shared
// memory for the remaining stages of the pass.
//
// Twiddle tables.  Entry j of a prime's table holds psi^{brv(j)} (inverse:
// psi^{-brv(j)}) and its Shoup companion; stage s reads entries [2^s, 2^{s+1}).
// The stages of the row pass's second half (s = LOGR + 4 + l, 0 <= l < LOGC - 4)
// give every thread its own twiddles: row `row`, column group g < 16 and
// butterfly group g' < 2^l need entry 2^s + row 2^{4+l} + g 2^l + g'.  Those
// entries are stored transposed within each row's range, at
// 2^s + row 2^{4+l} + g' 16 + g, so that the threads of a row (consecutive g)
// read consecutive entries.  Entries of the earlier stages keep their order.
//
// Ranges.  The twiddle product uses a Shoup quotient from three 32-bit partial
// products, which is at most 2 below the exact one, so W Y mod p is returned
// in [0, 4p) for any 64-bit Y.  Forward (CT) butterflies then need no
// correction at all: (X + V, X - V + 4p) grows the bound by 4p per stage, at
// most 61p < 2^62 after 15 stages for every prime here (p < 2^56); the last
// forward pass brings it to [0, 8p) with conditional subtractions of 32p,
// 16p, 8p: every consumer of the forward transform (Montgomery products and
// multiply-accumulates, whose sums stay below p 2^64) accepts that range.
// Inverse (GS) butterflies keep every value in [0, 4p): (X + Y) - 4p when
// >= 4p, and W (X - Y + 4p) in [0, 4p).  The integer multiplier (FMA-heavy
// pipe) is the bottleneck on this GPU, so range control uses only
// compare/subtract (ALU pipe) instructions.
#pragma once
#include "hp_device.cuh"

namespace hp {

constexpr int NTT_TILE = 2048;
constexpr int NTT_THREADS = 128;  // 2048 words / 16 per thread

// Which prime each polynomial of a batch uses: polynomial index p has
// position r = p % period; id = (r == period-1 && last_id >= 0) ? last_id : base + r.
struct PolyMap {
  int period, base, last_id;
  HPD int id(int p) const {
    int r = p % period;
    return (r == period - 1 && last_id >= 0) ? last_id : base + r;
  }
};

struct NttTabs {
  const ulonglong2* tw;   // [NPRIME][N] (psi^{brv(j)}, Shoup companion)
  const ulonglong2* itw;  // [NPRIME][N] (psi^{-brv(j)}, Shoup companion)
  // [NSCALE][NPRIME][4]: the output scale c and c W1 (W1 = psi^{-brv(1)}, the
  // twiddle of the last inverse stage), each with its Shoup companion
  const uint64_t* scale;
};
// c = N^{-1}; t N^{-1} 2^64; N^{-1} 2^64; N^{-1} P^{-1} (data primes, mod-down);
// t N^{-1} 2^64 times the first factor of each base conversion of the
// tensor-core scale-and-round ([(Q/q_i)^{-1}]_{q_i}, [Q^{-1} (B/b_k)^{-1}]_{b_k})
enum { SCALE_NINV = 0, SCALE_T_NINV_R = 1, SCALE_NINV_R = 2, SCALE_NINV_PINV = 3, SCALE_T_NINV_R_CONV = 4, NSCALE = 5 };

// Optional fused load of the forward column pass: polynomial (b, g, j) of the
// key-switching batch is digit g of ciphertext b reduced modulo target prime
// j.  A digit of G = dp primes (3 or 5) is stored in mixed radix as
// (t_0, ..., t_{G-1}) in w3[b][2][Gg .. Gg+G-1] and recombined as
// t_0 + sum_{m >= 1} [q_Gg ... q_Gg+m-1]_{p_j} t_m mod p_j (the terms whose
// constant contains p_j itself vanish); the two-digit key's digits are the
// same with G = 8 for data primes 0..7 and G = 7 for 8..14; a per-prime digit (dp = 1) is the
// residue w3[b][2][g] < q_g, which one conditional subtraction reduces modulo
// any target (q_g < 2 p_j).
// A digit's value modulo one of its own primes is the residue of d2 itself: with
// res (d2's residues, [b][L][N]) those targets are read from there instead of
// being recombined.
struct DigitSrc {
  const uint64_t* w3;  // nullptr: the pass transforms `data` in place
  int dp;              // data primes per digit: 1, 3, 5 or COARSE_DIGIT_PRIMES (the two-digit key)
  const uint64_t* res = nullptr;  // d2's residues, or nullptr
};

// ---- modular helpers for the transform ------------------------------------------
struct PForm {
  uint64_t p, np;  // p and 2^64 - p
};
HPD PForm pform(int id) {
  PForm f;
  f.p = cK.p[id];
  f.np = 0 - f.p;
  return f;
}
// W Y mod p in [0, 4p) for any 64-bit Y; wp = floor(W 2^64 / p).
// q = yh wh + hi(yh wl) + hi(yl wh) drops the low partial product and two
// carries, so floor(Y wp / 2^64) - 2 <= q <= floor(Y wp / 2^64);
// Y W - q p = Y W + q (2^64 - p) is then evaluated mod 2^64.
HPD uint64_t mul_shoup4(uint64_t y, uint64_t w, uint64_t wp, const PForm& f) {
  const uint32_t yl = (uint32_t)y, yh = (uint32_t)(y >> 32);
  const uint32_t wl = (uint32_t)wp, wh = (uint32_t)(wp >> 32);
  const uint64_t q = (uint64_t)yh * wh + __umulhi(yh, wl) + __umulhi(yl, wh);
  return y * w + q * f.np;
}
// x in [0, 64p) -> [0, 8p) by conditional subtractions (no multiplications)
HPD uint64_t red64to8(uint64_t x, uint64_t p) {
  x = csub(x, 32 * p);
  x = csub(x, 16 * p);
  return csub(x, 8 * p);
}

// Digit (t_0, ..., t_{G-1}) modulo target p for the 16 rows rb + u RB of one
// column (offset col), with the NT terms m = 1 .. NT:
// t_0 < 2p (primes within a factor 2) plus NT Shoup products in [0, 4p), so the
// sum lies below (2 + 4 NT) p and conditional subtractions of 16p .. p (those
// below the bound) bring it to [0, p).
template <int NT, int G, int LOGR, int LOGC>
HPD void digit_terms(uint64_t (&x)[16], const uint64_t* __restrict__ src, int rb, int col, const uint64_t (&c)[G - 1],
                     const uint64_t (&cs)[G - 1], const PForm& f) {
  constexpr int N = 1 << (LOGR + LOGC), C = 1 << LOGC, RB = 1 << (LOGR - 4);
  const uint64_t p = f.p;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const size_t off = (size_t)(rb + u * RB) * C + col;
    uint64_t v = src[off];
#pragma unroll
    for (int m = 1; m <= NT; ++m) v += mul_shoup4(src[(size_t)m * N + off], c[m - 1], cs[m - 1], f);
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1)
      if (k < 2 + 4 * NT) v = csub(v, k * p);
    x[u] = v;
  }
}

// Polynomial (b, g, j) of a key-switching batch of G-prime digits: digit g of
// ciphertext b reduced modulo target prime j.  For a target outside the digit's
// group every term counts; at offset o inside it the terms m > o vanish (their
// constant is a multiple of p_j), and at o = 0 the value is t_0 itself, already
// canonical.
template <int G, int LOGR, int LOGC>
HPD void load_digit(uint64_t (&x)[16], const uint64_t* __restrict__ w3, const uint64_t* __restrict__ res, int poly,
                    int rb, int col, const PForm& f) {
  constexpr int N = 1 << (LOGR + LOGC), C = 1 << LOGC, RB = 1 << (LOGR - 4), ND = L / G;
  const int b = poly / (ND * NKS), g = (poly / NKS) % ND, j = poly % NKS;
  const uint64_t* src = w3 + ((size_t)(b * 3 + 2) * L + g * G) * N;
  const int o = j - G * g;  // offset of the target inside the digit's group
  if (o == 0 || (res && o > 0 && o < G)) {  // t_0, or the stored residue modulo the digit's own prime j
    const uint64_t* r = o == 0 ? src : res + ((size_t)b * L + j) * N;
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = r[(size_t)(rb + u * RB) * C + col];
    return;
  }
  uint64_t c[G - 1], cs[G - 1];
#pragma unroll
  for (int m = 1; m < G; ++m) {
    c[m - 1] = G == 3 ? cK.digm3[m - 1][g][j] : cK.digm5[m - 1][g][j];
    cs[m - 1] = G == 3 ? cK.digm3_s[m - 1][g][j] : cK.digm5_s[m - 1][g][j];
  }
  const int nt = (o > 0 && o < G) ? o : G - 1;
  if (nt == G - 1) return digit_terms<G - 1, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
  if (nt == 1) return digit_terms<1, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
  if constexpr (G > 3) {
    if (nt == 2) return digit_terms<2, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
    if (nt == 3) return digit_terms<3, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
  }
}

// Polynomial (b, a, j) of a key-switching batch of the two-digit key: digit a
// (data primes 8a .. 8a + 7, the second digit one prime shorter) of ciphertext
// b reduced modulo target prime j, as load_digit.
template <int LOGR, int LOGC>
HPD void load_digit2(uint64_t (&x)[16], const uint64_t* __restrict__ w3, const uint64_t* __restrict__ res, int poly,
                     int rb, int col, const PForm& f) {
  constexpr int N = 1 << (LOGR + LOGC), C = 1 << LOGC, RB = 1 << (LOGR - 4), G = COARSE_DIGIT_PRIMES;
  const int b = poly / (NDIG2 * NKS), a = (poly / NKS) % NDIG2, j = poly % NKS;
  const int base = G * a, g = a == 0 ? G : L - G;  // primes in this digit
  const uint64_t* src = w3 + ((size_t)(b * 3 + 2) * L + base) * N;
  const int o = j - base;
  if (o == 0 || (res && o > 0 && o < g)) {  // t_0, or the stored residue modulo the digit's own prime j
    const uint64_t* r = o == 0 ? src : res + ((size_t)b * L + j) * N;
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = r[(size_t)(rb + u * RB) * C + col];
    return;
  }
  uint64_t c[G - 1], cs[G - 1];
#pragma unroll
  for (int m = 1; m < G; ++m) {
    c[m - 1] = cK.digm8[m - 1][a][j];
    cs[m - 1] = cK.digm8_s[m - 1][a][j];
  }
  const int nt = (o > 0 && o < g) ? o : g - 1;
  switch (nt) {
    case 1: return digit_terms<1, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
    case 2: return digit_terms<2, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
    case 3: return digit_terms<3, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
    case 4: return digit_terms<4, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
    case 5: return digit_terms<5, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
    case 6: return digit_terms<6, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
    default: return digit_terms<7, G, LOGR, LOGC>(x, src, rb, col, c, cs, f);
  }
}

// ---- register blocks --------------------------------------------------------
// x[u] holds a_{base + (u << (logN - s0 - A))}, u < 2^A; base has zero bits in
// the u positions.  Runs forward stages s0 .. s0 + A - 1 in registers.
template <int A>
HPD void fwd_block(uint64_t (&x)[1 << A], uint32_t base, int s0, int logN, const ulonglong2* __restrict__ tw,
                   const PForm& f) {
  const uint64_t p4 = 4 * f.p;
#pragma unroll
  for (int l = 0; l < A; ++l) {
    const int s = s0 + l;
    const uint32_t tb = (1u << s) + (base >> (logN - s));
#pragma unroll
    for (int g = 0; g < (1 << l); ++g) {
      const ulonglong2 W = __ldg(tw + tb + g);
#pragma unroll
      for (int o = 0; o < (1 << (A - l - 1)); ++o) {
        const int u = (g << (A - l)) + o, v = u + (1 << (A - l - 1));
        const uint64_t X = x[u];
        const uint64_t V = mul_shoup4(x[v], W.x, W.y, f);
        x[u] = X + V;
        x[v] = X - V + p4;
      }
    }
  }
}

// The same stages for the second half of the row pass (s0 = logR + 4): the
// elements are 2^A consecutive columns of group `grp` of row `row`, and the
// twiddles come from the transposed layout described above.
template <int A>
HPD void fwd_block_tr(uint64_t (&x)[1 << A], uint32_t row, uint32_t grp, int s0, const ulonglong2* __restrict__ tw,
                      const PForm& f) {
  const uint64_t p4 = 4 * f.p;
#pragma unroll
  for (int l = 0; l < A; ++l) {
    const uint32_t tb = (1u << (s0 + l)) + (row << (4 + l)) + grp;
#pragma unroll
    for (int g = 0; g < (1 << l); ++g) {
      const ulonglong2 W = __ldg(tw + tb + (g << 4));
#pragma unroll
      for (int o = 0; o < (1 << (A - l - 1)); ++o) {
        const int u = (g << (A - l)) + o, v = u + (1 << (A - l - 1));
        const uint64_t X = x[u];
        const uint64_t V = mul_shoup4(x[v], W.x, W.y, f);
        x[u] = X + V;
        x[v] = X - V + p4;
      }
    }
  }
}

// Inverse stages s0 + A - 1 .. s0 on the same element set; values in [0, 4p).
template <int A>
HPD void inv_block(uint64_t (&x)[1 << A], uint32_t base, int s0, int logN, const ulonglong2* __restrict__ itw,
                   const PForm& f) {
  const uint64_t p4 = 4 * f.p;
#pragma unroll
  for (int l = A - 1; l >= 0; --l) {
    const int s = s0 + l;
    const uint32_t tb = (1u << s) + (base >> (logN - s));
#pragma unroll
    for (int g = 0; g < (1 << l); ++g) {
      const ulonglong2 W = __ldg(itw + tb + g);
#pragma unroll
      for (int o = 0; o < (1 << (A - l - 1)); ++o) {
        const int u = (g << (A - l)) + o, v = u + (1 << (A - l - 1));
        const uint64_t X = x[u], Y = x[v];
        x[u] = csub(X + Y, p4);
        x[v] = mul_shoup4(X - Y + p4, W.x, W.y, f);
      }
    }
  }
}

// inv_block for the second half of the row pass (transposed twiddles, as fwd_block_tr)
template <int A>
HPD void inv_block_tr(uint64_t (&x)[1 << A], uint32_t row, uint32_t grp, int s0, const ulonglong2* __restrict__ itw,
                      const PForm& f) {
  const uint64_t p4 = 4 * f.p;
#pragma unroll
  for (int l = A - 1; l >= 0; --l) {
    const uint32_t tb = (1u << (s0 + l)) + (row << (4 + l)) + grp;
#pragma unroll
    for (int g = 0; g < (1 << l); ++g) {
      const ulonglong2 W = __ldg(itw + tb + (g << 4));
#pragma unroll
      for (int o = 0; o < (1 << (A - l - 1)); ++o) {
        const int u = (g << (A - l)) + o, v = u + (1 << (A - l - 1));
        const uint64_t X = x[u], Y = x[v];
        x[u] = csub(X + Y, p4);
        x[v] = mul_shoup4(X - Y + p4, W.x, W.y, f);
      }
    }
  }
}

// Inverse stages A - 1 .. 0 of the column pass (s0 = 0) with the output scale
// c folded into stage 0, whose single twiddle is W1: (X + Y, W1 (X - Y)) becomes
// (c (X + Y), c W1 (X - Y)); sc = (c, Shoup, c W1, Shoup).  Values in [0, 4p).
template <int A>
HPD void inv_block_scaled(uint64_t (&x)[1 << A], uint32_t base, int logN, const ulonglong2* __restrict__ itw,
                          const PForm& f, const uint64_t* __restrict__ sc) {
  const uint64_t p4 = 4 * f.p;
#pragma unroll
  for (int l = A - 1; l >= 1; --l) {
    const uint32_t tb = (1u << l) + (base >> (logN - l));
#pragma unroll
    for (int g = 0; g < (1 << l); ++g) {
      const ulonglong2 W = __ldg(itw + tb + g);
#pragma unroll
      for (int o = 0; o < (1 << (A - l - 1)); ++o) {
        const int u = (g << (A - l)) + o, v = u + (1 << (A - l - 1));
        const uint64_t X = x[u], Y = x[v];
        x[u] = csub(X + Y, p4);
        x[v] = mul_shoup4(X - Y + p4, W.x, W.y, f);
      }
    }
  }
  const uint64_t c = __ldg(sc), cs = __ldg(sc + 1), cw = __ldg(sc + 2), cws = __ldg(sc + 3);
#pragma unroll
  for (int u = 0; u < (1 << (A - 1)); ++u) {
    const int v = u + (1 << (A - 1));
    const uint64_t X = x[u], Y = x[v];
    x[u] = mul_shoup4(X + Y, c, cs, f);
    x[v] = mul_shoup4(X - Y + p4, cw, cws, f);
  }
}

// ---- forward, columns (stages 0 .. LOGR-1) -------------------------------------
// Block: COLS = 2048 / R adjacent columns.  Step A: thread (k, rb) holds rows
// rb + 16-stride (stages 0..3); step B: groups of 2^(LOGR-4) consecutive rows.
// DG selects the input: 0 the polynomials of `data` (in place), 1, 3 or 5 a
// key-switching batch built from dig.w3 in digits of that many data primes,
// COARSE_DIGIT_PRIMES the two-digit key's batch.
template <int LOGR, int LOGC, int DG>
__global__ void __launch_bounds__(NTT_THREADS, DG == COARSE_DIGIT_PRIMES ? 6 : 7) k_ntt_fwd_cols(uint64_t* __restrict__ data, PolyMap map, NttTabs T,
                                                                 DigitSrc dig) {
  constexpr int logN = LOGR + LOGC, N = 1 << logN, C = 1 << LOGC;
  constexpr int COLS = NTT_TILE >> LOGR, A2 = LOGR - 4, RB = 1 << (LOGR - 4);
  __shared__ uint64_t s[NTT_TILE];
  const int t = threadIdx.x, k = t % COLS, rb = t / COLS;
  const int poly = blockIdx.y, k0 = blockIdx.x * COLS;
  const int id = map.id(poly);
  const PForm f = pform(id);
  const uint64_t p = f.p;
  const ulonglong2* tw = T.tw + (size_t)id * N;
  uint64_t* a = data + (size_t)poly * N;
  uint64_t x[16];
  if constexpr (DG == 1) {  // per-prime digits: poly = (b * L + g) * NKS + j
    const int b = poly / (NDIG_FINE * NKS), g = (poly / NKS) % NDIG_FINE;
    const uint64_t* src = dig.w3 + ((size_t)(b * 3 + 2) * L + g) * N;
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = csub(src[(size_t)(rb + u * RB) * C + k0 + k], p);
  } else if constexpr (DG == COARSE_DIGIT_PRIMES) {  // the two-digit key: poly = (b * NDIG2 + a) * NKS + j
    load_digit2<LOGR, LOGC>(x, dig.w3, dig.res, poly, rb, k0 + k, f);
  } else if constexpr (DG > 1) {  // digits of DG primes: poly = (b * (L / DG) + g) * NKS + j
    load_digit<DG, LOGR, LOGC>(x, dig.w3, dig.res, poly, rb, k0 + k, f);
  } else {
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = a[(size_t)(rb + u * RB) * C + k0 + k];
  }
  fwd_block<4>(x, (uint32_t)(rb * C + k0 + k), 0, logN, tw, f);
#pragma unroll
  for (int u = 0; u < 16; ++u) s[(rb + u * RB) * COLS + k] = x[u];
  __syncthreads();
#pragma unroll
  for (int m = 0; m < (16 >> A2); ++m) {
    const int g = rb + m * RB;  // group of 2^A2 consecutive rows, g < 16
    uint64_t y[1 << A2];
#pragma unroll
    for (int u = 0; u < (1 << A2); ++u) y[u] = s[((g << A2) + u) * COLS + k];
    fwd_block<A2>(y, (uint32_t)(((g << A2) * C) + k0 + k), 4, logN, tw, f);
#pragma unroll
    for (int u = 0; u < (1 << A2); ++u) a[(size_t)((g << A2) + u) * C + k0 + k] = y[u];
  }
}

// ---- forward, rows (stages LOGR .. logN-1); output in [0, 8p) ----------------------
// Block: ROWS = 2048 / C rows; padded shared rows (one word per 16) avoid bank
// conflicts of the contiguous groups of step B.
template <int LOGR, int LOGC>
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_fwd_rows(uint64_t* __restrict__ data, PolyMap map, NttTabs T) {
  constexpr int logN = LOGR + LOGC, N = 1 << logN, C = 1 << LOGC;
  constexpr int ROWS = NTT_TILE >> LOGC, TPR = C / 16, B2 = LOGC - 4, PADC = C + C / 16;
  __shared__ uint64_t s[ROWS * PADC];
  const int t = threadIdx.x, r = t / TPR, kb = t % TPR;
  const int poly = blockIdx.y, row0 = blockIdx.x * ROWS, row = row0 + r;
  const int id = map.id(poly);
  const PForm f = pform(id);
  const uint64_t p = f.p;
  const ulonglong2* tw = T.tw + (size_t)id * N;
  uint64_t* a = data + (size_t)poly * N;
  uint64_t x[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) x[u] = a[(size_t)row * C + kb + u * TPR];
  fwd_block<4>(x, (uint32_t)(row * C + kb), LOGR, logN, tw, f);
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int kk = kb + u * TPR;
    s[r * PADC + kk + (kk >> 4)] = x[u];
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < (16 / TPR); ++m) {
    const int g = kb + m * TPR;  // group of 2^B2 consecutive columns, g < 16
    uint64_t y[1 << B2];
#pragma unroll
    for (int u = 0; u < (1 << B2); ++u) {
      const int kk = (g << B2) + u;
      y[u] = s[r * PADC + kk + (kk >> 4)];
    }
    fwd_block_tr<B2>(y, (uint32_t)row, (uint32_t)g, LOGR + 4, tw, f);
#pragma unroll
    for (int u = 0; u < (1 << B2); ++u) {
      const int kk = (g << B2) + u;
      s[r * PADC + kk + (kk >> 4)] = red64to8(y[u], p);
    }
  }
  __syncthreads();
  uint64_t* dst = a + (size_t)row0 * C;
#pragma unroll
  for (int u = 0; u < NTT_TILE / NTT_THREADS; ++u) {
    const int e = t + u * NTT_THREADS, rr = e / C, kk = e % C;
    dst[e] = s[rr * PADC + kk + (kk >> 4)];
  }
}

// ---- forward rows of both components + squaring tensor ----------------------------
// The row pass of k_ntt_fwd_rows on components 0 and 1 of one ciphertext's
// lifted polynomial for one prime (blockIdx.y = b * NQB + pi), followed by the
// squaring tensor of k_tensor_sq on the two finished tiles:
//   d0 = a0 a0 2^-64, d1 = 2 a0 a1 2^-64 (reduced to [0, 2p)), d2 = a1 a1 2^-64.
// ext: [nct][2][NQB][N] after the column pass; dprod: [nct][3][NQB][N].
template <int LOGR, int LOGC>
__global__ void __launch_bounds__(NTT_THREADS, 6) k_ntt_fwd_rows_sq(const uint64_t* __restrict__ ext,
                                                                 uint64_t* __restrict__ dprod, NttTabs T) {
  constexpr int logN = LOGR + LOGC, N = 1 << logN, C = 1 << LOGC;
  constexpr int ROWS = NTT_TILE >> LOGC, TPR = C / 16, B2 = LOGC - 4, PADC = C + C / 16;
  __shared__ uint64_t s[ROWS * PADC];   // exchange, then component 1's result
  __shared__ uint64_t s0[ROWS * PADC];  // component 0's result
  const int t = threadIdx.x, r = t / TPR, kb = t % TPR;
  const int bp = blockIdx.y, pi = bp % NQB, row0 = blockIdx.x * ROWS, row = row0 + r;
  const size_t b = bp / NQB;
  const PForm f = pform(pi);
  const uint64_t p = f.p, pinv = cK.pinv[pi];
  const ulonglong2* tw = T.tw + (size_t)pi * N;
#pragma unroll 1
  for (int comp = 0; comp < 2; ++comp) {
    const uint64_t* a = ext + ((b * 2 + comp) * NQB + pi) * N;
    uint64_t* res = comp ? s : s0;
    uint64_t x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = a[(size_t)row * C + kb + u * TPR];
    fwd_block<4>(x, (uint32_t)(row * C + kb), LOGR, logN, tw, f);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int kk = kb + u * TPR;
      s[r * PADC + kk + (kk >> 4)] = x[u];
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < (16 / TPR); ++m) {
      const int g = kb + m * TPR;
      uint64_t y[1 << B2];
#pragma unroll
      for (int u = 0; u < (1 << B2); ++u) {
        const int kk = (g << B2) + u;
        y[u] = s[r * PADC + kk + (kk >> 4)];
      }
      fwd_block_tr<B2>(y, (uint32_t)row, (uint32_t)g, LOGR + 4, tw, f);
#pragma unroll
      for (int u = 0; u < (1 << B2); ++u) {
        const int kk = (g << B2) + u;
        res[r * PADC + kk + (kk >> 4)] = red64to8(y[u], p);
      }
    }
    __syncthreads();
  }
  const uint64_t p2 = 2 * p;
  uint64_t* d0 = dprod + ((b * 3 + 0) * NQB + pi) * N + (size_t)row0 * C;
  uint64_t* d1 = d0 + (size_t)NQB * N;
  uint64_t* d2 = d1 + (size_t)NQB * N;
#pragma unroll
  for (int u = 0; u < NTT_TILE / NTT_THREADS; ++u) {
    const int e = t + u * NTT_THREADS, rr = e / C, kk = e % C, si = rr * PADC + kk + (kk >> 4);
    const uint64_t a0 = s0[si], a1 = s[si];
    const uint64_t m01 = 2 * mont_mul_lazy(a0, a1, p, pinv);
    d0[e] = mont_mul_lazy(a0, a0, p, pinv);
    d1[e] = m01 >= p2 ? m01 - p2 : m01;
    d2[e] = mont_mul_lazy(a1, a1, p, pinv);
  }
}

// ---- inverse, rows (stages logN-1 .. LOGR); input in [0, 2p) --------------------
template <int LOGR, int LOGC>
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_inv_rows(uint64_t* __restrict__ data, PolyMap map, NttTabs T) {
  constexpr int logN = LOGR + LOGC, N = 1 << logN, C = 1 << LOGC;
  constexpr int ROWS = NTT_TILE >> LOGC, TPR = C / 16, B2 = LOGC - 4, PADC = C + C / 16;
  __shared__ uint64_t s[ROWS * PADC];
  const int t = threadIdx.x, r = t / TPR, kb = t % TPR;
  const int poly = blockIdx.y, row0 = blockIdx.x * ROWS, row = row0 + r;
  const int id = map.id(poly);
  const PForm f = pform(id);
  const ulonglong2* itw = T.itw + (size_t)id * N;
  uint64_t* a = data + (size_t)poly * N;
  {  // the tile is contiguous: all 16 loads of a thread in flight, then the padded stores
    const uint64_t* src = a + (size_t)row0 * C;
    uint64_t v[NTT_TILE / NTT_THREADS];
#pragma unroll
    for (int u = 0; u < NTT_TILE / NTT_THREADS; ++u) v[u] = src[t + u * NTT_THREADS];
#pragma unroll
    for (int u = 0; u < NTT_TILE / NTT_THREADS; ++u) {
      const int e = t + u * NTT_THREADS, rr = e / C, kk = e % C;
      s[rr * PADC + kk + (kk >> 4)] = v[u];
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < (16 / TPR); ++m) {
    const int g = kb + m * TPR;
    uint64_t y[1 << B2];
#pragma unroll
    for (int u = 0; u < (1 << B2); ++u) {
      const int kk = (g << B2) + u;
      y[u] = s[r * PADC + kk + (kk >> 4)];
    }
    inv_block_tr<B2>(y, (uint32_t)row, (uint32_t)g, LOGR + 4, itw, f);
#pragma unroll
    for (int u = 0; u < (1 << B2); ++u) {
      const int kk = (g << B2) + u;
      s[r * PADC + kk + (kk >> 4)] = y[u];
    }
  }
  __syncthreads();
  uint64_t x[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int kk = kb + u * TPR;
    x[u] = s[r * PADC + kk + (kk >> 4)];
  }
  inv_block<4>(x, (uint32_t)(row * C + kb), LOGR, logN, itw, f);
#pragma unroll
  for (int u = 0; u < 16; ++u) a[(size_t)row * C + kb + u * TPR] = x[u];
}

// ---- inverse, columns (stages LOGR-1 .. 0) and scaling; canonical output --------
// Optional fused key-switching mod-down (MD = true): block y transforms the
// key-switching sum u_i of (ciphertext-component bc = y / L, data prime
// i = y % L), polynomial bc NKS + i of `data`, whose special-prime
// polynomial u_P (bc NKS + L) is already transformed, and writes
//   out[bc][i] = w3[b][c][i] + (u_i - [u_P]) P^{-1} mod q_i   ([u_P] centred),
// or its "1 -" form, instead of u_i.  Otherwise (MD = false) block y
// transforms polynomial y pstride + poff in place.
struct ModDown {
  const uint64_t* w3;  // [nct][3][L][N]: (d0, d1) to add to
  uint64_t* out;       // [nct][2][L][N]
  int one_minus;
  int pstride, poff;
};
// Bounds: 8 blocks per SM (64 registers, 12 B of spills) for the plain pass, 7
// for the mod-down form (72 registers; 8 would spill 104 B).
template <int LOGR, int LOGC, bool MD>
__global__ void __launch_bounds__(NTT_THREADS, MD ? 7 : 8) k_ntt_inv_cols(uint64_t* __restrict__ data, PolyMap map, NttTabs T,
                                                              int scale_mode, ModDown md) {
  constexpr int logN = LOGR + LOGC, N = 1 << logN, C = 1 << LOGC;
  constexpr int COLS = NTT_TILE >> LOGR, A2 = LOGR - 4, RB = 1 << (LOGR - 4);
  __shared__ uint64_t s[NTT_TILE];
  const int t = threadIdx.x, k = t % COLS, rb = t / COLS;
  const int y0 = blockIdx.y, k0 = blockIdx.x * COLS;
  const int poly = MD ? (y0 / L) * NKS + (y0 % L) : y0 * md.pstride + md.poff;
  const int id = map.id(poly);
  const PForm f = pform(id);
  const uint64_t p = f.p;
  const ulonglong2* itw = T.itw + (size_t)id * N;
  uint64_t* a = data + (size_t)poly * N;
  if (MD) {  // the epilogue's operands into L2 while the transform runs
    const size_t bc = (size_t)(y0 / L);
    const int i = y0 % L, comp = (int)(bc & 1);
    const uint64_t* uP = data + (bc * NKS + L) * N;
    const uint64_t* wv = md.w3 + (((bc >> 1) * 3 + comp) * L + i) * N;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int n = (rb + u * RB) * C + k0 + k;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(uP + n));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(wv + n));
    }
  }
#pragma unroll
  for (int m = 0; m < (16 >> A2); ++m) {
    const int g = rb + m * RB;
    uint64_t y[1 << A2];
#pragma unroll
    for (int u = 0; u < (1 << A2); ++u) y[u] = a[(size_t)((g << A2) + u) * C + k0 + k];
    inv_block<A2>(y, (uint32_t)(((g << A2) * C) + k0 + k), 4, logN, itw, f);
#pragma unroll
    for (int u = 0; u < (1 << A2); ++u) s[((g << A2) + u) * COLS + k] = y[u];
  }
  __syncthreads();
  uint64_t x[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) x[u] = s[(rb + u * RB) * COLS + k];
  // scaled by c (MD: N^{-1} P^{-1}, so that x holds u_i P^{-1})
  inv_block_scaled<4>(x, (uint32_t)(rb * C + k0 + k), logN, itw, f,
                      T.scale + ((size_t)(MD ? SCALE_NINV_PINV : scale_mode) * NPRIME + id) * 4);
  if (!MD) {
#pragma unroll
    for (int u = 0; u < 16; ++u) a[(size_t)(rb + u * RB) * C + k0 + k] = csub(csub(x[u], 2 * p), p);
  } else {
    const size_t bc = (size_t)(y0 / L);
    const int i = y0 % L, comp = (int)(bc & 1);
    const uint64_t P = cK.p[ID_P];
    const uint64_t* uP = data + (bc * NKS + L) * N;
    const uint64_t* wv = md.w3 + (((bc >> 1) * 3 + comp) * L + i) * N;
    uint64_t* o = md.out + (bc * L + i) * N;
    const uint64_t pinv = cK.Pinv[i], pinv_s = cK.Pinv_s[i];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int n = (rb + u * RB) * C + k0 + k;
      const uint64_t up = uP[n];
      const bool low = up <= (P - 1) / 2;  // [u_P] = up or up - P
      // m = |[u_P]| P^{-1} in [0, 4p); x[u] = u_i P^{-1} in [0, 4p), wv < p:
      // x + wv + (4p - m or m) < 9p, four conditional subtractions to [0, p)
      const uint64_t m = mul_shoup4(low ? up : P - up, pinv, pinv_s, f);
      uint64_t r = x[u] + wv[n] + (low ? 4 * p - m : m);
      r = csub(csub(csub(csub(r, 8 * p), 4 * p), 2 * p), p);
      if (md.one_minus) {
        r = sub_mod(0, r, p);
        if (comp == 0 && n == 0) r = add_mod(r, cK.delta[i], p);
      }
      o[n] = r;
    }
  }
}

}  // namespace hp
