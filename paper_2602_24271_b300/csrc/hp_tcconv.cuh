// Exact scale-and-round with the base conversions on the tensor cores.
//
// The two RNS base conversions of round(t d / Q) (Q -> B for r = [t d]_Q and
// B -> Q for w = (t d - r) / Q, see k_scale_round) are dense contractions of
// every coefficient's residue vector with a fixed matrix: 15 x 16 and 16 x 15
// products of 55-bit numbers.  Here each residue y is split into seven 8-bit
// limbs y^(a) and the matrix entries are pre-multiplied by 2^(8a), so that
//   sum_i y_i c_ik = sum_{i,a} y_i^(a) [2^(8a) c_ik]_{b_k}   (mod b_k)
// and every [2^(8a) c_ik] is itself split into limbs.  One f16 MMA
// (tcgen05.mma, M = 128 coefficients, N = 128 = 16 primes x 8 limb columns,
// K = 128 = 16 residues x 8 columns, the eighth zero) then gives, per
// coefficient and prime, the seven limb sums D_l = sum y^(a) c^(l)
// < 112 * 255^2 < 2^23: exact in the f32 accumulator.  Two bias columns
// (2048 x 2048 each, in K columns the residues leave free) add 2^23 to every
// accumulator word, so each holds 2^23 + D_l < 2^24 exactly and D_l is its low
// 23 bits.  The value sum_l D_l 2^(8l) < 2^72 is reduced modulo the prime on
// the CUDA cores.
//
// The eighth column of each prime's block is free, and the centring sums go
// there: column 8l + 7 (l < 8) of the Q -> B product holds
// E_l = sum_{i,a} y_i^(a) [floor(2^(64+8a) / q_i)]^(l), limb l of the fixed-point
// weight of y_i^(a) in S = sum_i y_i / q_i, so that sum_l E_l 2^(8l) lies within
// 15 * 7 * 255 < 2^15 below S 2^64 (each weight truncated by less than 1); the
// B -> Q product holds the same for sum_k y_k / b_k in columns 120 .. 127.  The
// rounding decisions v = floor(S + 1/2) are read from there, and an undecided
// window (probability about 2^-49) falls back to the exact mixed-radix
// comparison, as in k_lift.
//
// The inputs come from the inverse transform with its output scale extended
// (SCALE_T_NINV_R_CONV): the Q residues arrive as y_i = [t d (Q/q_i)^{-1}]_{q_i}
// and the B residues as [t d Q^{-1} (B/b_k)^{-1}]_{b_k}; the Q -> B operand and
// its correction table carry the factor [Q^{-1} (B/b_k)^{-1}]_{b_k} too, so
// y_k of w = (t d - r) / Q in B is one modular subtraction.  The outputs are
// bit-identical to k_scale_round's.
#pragma once
#include <cuda_fp16.h>

#include "hp_rns.cuh"
#include "hp_tc.cuh"

namespace hp {

constexpr int SRT_GROUPS = 4;                    // tiles of 128 coefficients in flight per CTA
constexpr int SRT_THREADS = 128 * SRT_GROUPS;    // one thread per coefficient
constexpr int SRT_OPER = TC_OPER;                // f16 elements of one operand tile
constexpr size_t SRT_SMEM = (size_t)(2 + SRT_GROUPS) * SRT_OPER * 2 + (TC_T1 + TC_T2) * 8 + SRT_GROUPS * 8 + 32;
constexpr uint64_t FIX_WINDOW = 1ull << 15;       // the fixed-point sums' window (units of 2^-64)

HPD void named_sync(int id, int count) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory"); }

// 32 TMEM lanes x 1 column
HPD uint32_t tc_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
  return r;
}

// 32 TMEM lanes x 8 consecutive 32-bit columns
HPD void tc_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}

// 32 TMEM lanes x 32 (resp. 64) consecutive 32-bit columns
HPD void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr)
               : "memory");
}
HPD void tc_ld64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
               : "r"(taddr)
               : "memory");
}

// Row `m` of an operand tile: residue i occupies columns 8 i .. 8 i + 7, its
// seven 8-bit limbs as f16 and a zero; columns of residues i >= R are zero.
// Two limbs at a time: a byte permute builds the f16 pair (1024 + u, 1024 + v)
// (bit patterns 0x64uu, 0x64vv), and one packed subtraction of 1024 leaves
// the exact f16 values u, v.  The bias columns hold 2048 (f16 0x6800): for
// R = 15 the first two columns of the free slot 15 (columns 120, 121), for
// R = 16 the eighth columns of residues 0 and 1 (columns 7, 15).
HPD uint32_t limb_pair(uint32_t w, uint32_t sel) {
  const uint32_t biased = __byte_perm(w, 0x64006400u, sel);
  const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&biased), __float2half2_rn(1024.0f));
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <int R>
HPD void put_limb_row(uint16_t* tile, int m, const uint64_t (&y)[R]) {
  static_assert(R == TC_K / 8 - 1 || R == TC_K / 8, "bias columns: a free slot 15 (R = 15) or residues 0, 1 (R = 16)");
#pragma unroll
  for (int i = 0; i < TC_K / 8; ++i) {
    uint4 v = make_uint4(0, 0, 0, 0);
    if (i < R) {
      const uint32_t lo = (uint32_t)y[i], hi = (uint32_t)(y[i] >> 32);
      v.x = limb_pair(lo, 0x7150u);  // bytes 0, 1
      v.y = limb_pair(lo, 0x7352u);  // bytes 2, 3
      v.z = limb_pair(hi, 0x7150u);  // bytes 4, 5
      v.w = limb_pair(hi, 0x7452u);  // byte 6 and 0 (the constant's zero byte)
      if (R == TC_K / 8 && i < 2) v.w |= 0x68000000u;  // column 8 i + 7: 2048
    } else if (i == TC_K / 8 - 1) {
      v.x = 0x68006800u;  // columns 120, 121: 2048
    }
    *(uint4*)(tile + tc_cm(m, 8 * i, TC_K)) = v;
  }
}

// D < 2^23 from an accumulator word holding the f32 value 2^23 + D (the bias)
HPD uint32_t acc_int(uint32_t bits) { return bits & 0x7FFFFFu; }

// The fixed-point sum sum_l E_l 2^(8l) (< 2^80) of eight accumulator words
// holding exact integers E_l < 2^23, as a Fix (64 low bits, the rest above):
// with the 32-bit pairs A = E_0 + 2^8 E_1, B = E_2 + 2^8 E_3, C = E_4 + 2^8 E_5,
// D = E_6 + 2^8 E_7 it is lo + 2^32 hi, lo = A + 2^16 B, hi = C + 2^16 D.
HPD Fix fix_from_limbs(const uint32_t* e) {
  const uint32_t A = acc_int(e[0]) + (acc_int(e[1]) << 8), B = acc_int(e[2]) + (acc_int(e[3]) << 8),
                 C = acc_int(e[4]) + (acc_int(e[5]) << 8), D = acc_int(e[6]) + (acc_int(e[7]) << 8);
  const uint64_t lo = (uint64_t)B * 65536u + A, hi = (uint64_t)D * 65536u + C;  // each < 2^49
  Fix F;
  F.lo = lo + (hi << 32);
  F.hi = (uint32_t)(hi >> 32) + (F.lo < lo ? 1u : 0u);
  return F;
}

// Exact centring decision v of the Q -> B conversion when the fixed-point
// window does not decide it: the residues [t d]_{q_i} = y_i [Q/q_i]_{q_i} are
// rebuilt from the y_i in memory (stride N) and compared with (Q-1)/2.
__device__ __noinline__ int lift_v_y_mem(const uint64_t* y, size_t stride, uint32_t Fhi) {
  uint64_t r[L];
  for (int i = 0; i < L; ++i) r[i] = mul_shoup(y[(size_t)i * stride], cK.qhat[i], cK.qhat_s[i], cK.p[i]);
  return (int)Fhi + greater_than_half(r, 1);
}

// sum_l D_l 2^(8l) + corr mod p in [0, 2p), for the limb sums D_0..D_6 of one
// prime; c32 = [2^32]_p (Shoup pair).  With the 32-bit pairs
// A = D_0 + 2^8 D_1, B = D_2 + 2^8 D_3, C = D_4 + 2^8 D_5 (each < 2^32, D_l < 2^23)
// the sum is lo + 2^32 hi, lo = A + 2^16 B < 2^49 < p, hi = C + 2^16 D_6 < 2^40;
// 2^32 hi reduces to [0, 2p), corr < p: below 4p before the one subtraction
// of 2p.  r points at the prime's 8 accumulator columns (constant offsets into
// a register array).
HPD uint64_t limb_sum_mod2(const uint32_t* r, uint64_t corr, uint64_t p, uint64_t c32, uint64_t c32s) {
  const uint32_t A = acc_int(r[0]) + (acc_int(r[1]) << 8), B = acc_int(r[2]) + (acc_int(r[3]) << 8),
                 C = acc_int(r[4]) + (acc_int(r[5]) << 8);
  const uint64_t lo = (uint64_t)B * 65536u + A, hi = (uint64_t)acc_int(r[6]) * 65536u + C;
  return csub(lo + mul_shoup_lazy(hi, c32, c32s, p) + corr, 2 * p);
}
// the same, reduced to [0, p)
HPD uint64_t limb_sum_mod(const uint32_t* r, uint64_t corr, uint64_t p, uint64_t c32, uint64_t c32s) {
  return csub(limb_sum_mod2(r, corr, p, c32, c32s), p);
}

// One key-switching digit of d2 (data primes base .. base + G - 1) of one
// coefficient: its residues to rr (if not null), its mixed-radix form to o.
template <int G>
HPD void digit_group_out(const uint64_t (&out)[L], int base, uint64_t* __restrict__ o, uint64_t* __restrict__ rr,
                         int N) {
  uint64_t r[G];
#pragma unroll
  for (int e = 0; e < G; ++e) r[e] = out[base + e];
  if (rr) {
#pragma unroll
    for (int e = 0; e < G; ++e) rr[(size_t)(base + e) * N] = r[e];
  }
  digit_mixed_radix<G>(r, base);
#pragma unroll
  for (int e = 0; e < G; ++e) o[(size_t)(base + e) * N] = r[e];
}

// Persistent: SRT_GROUPS groups of four warps, each taking tiles of 128
// consecutive coefficients (one per thread) of the nct x 3 coefficient
// polynomials.  ops / tabs: the operand and correction tables of
// build_tc_tables (B1S, B2; T1S, T2).  d2 is written as key-switching digits
// of dp primes in mixed radix (dp = 3 or 5; COARSE_DIGIT_PRIMES: the two-digit
// key's digits of 8 and 7 primes), or as plain residues (dp = 1: the per-prime
// digits); with `res` (not null) its residues also go to res[b][i][n], where the
// digit transform reads a digit's value modulo its own primes.
__global__ void __launch_bounds__(SRT_THREADS, 1)
    k_scale_round_tc(const uint64_t* __restrict__ dprod, uint64_t* __restrict__ w3, int* __restrict__ status,
                     const uint16_t* __restrict__ ops, const uint64_t* __restrict__ tabs, int logN, int nct, int dp,
                     uint64_t* __restrict__ res) {
  extern __shared__ __align__(1024) uint8_t srt_smem[];
  uint16_t* B1s = (uint16_t*)srt_smem;  // B1S
  uint16_t* B2s = B1s + SRT_OPER;       // B2
  uint16_t* As = B2s + SRT_OPER;        // SRT_GROUPS tiles
  uint64_t* T1s = (uint64_t*)(As + SRT_GROUPS * SRT_OPER);  // T1S
  uint64_t* T2s = T1s + TC_T1;
  uint64_t* mbar = T2s + TC_T2;
  uint32_t* tslot = (uint32_t*)(mbar + SRT_GROUPS);
  uint32_t* okf = tslot + 1;  // per group: the last MMA batch completed
  const int N = 1 << logN, t = threadIdx.x, warp = t >> 5, g = warp >> 2, m = t & 127;
  {  // constant operands and tables, once per CTA
    const uint4* src = (const uint4*)(ops + TCT_B1S);  // B1S and B2 are adjacent
    uint4* dst = (uint4*)srt_smem;
    for (int e = t; e < 2 * SRT_OPER / 8; e += SRT_THREADS) dst[e] = src[e];
    for (int e = t; e < TC_T1; e += SRT_THREADS) T1s[e] = tabs[TCT_T1S + e];
    for (int e = t; e < TC_T2; e += SRT_THREADS) T2s[e] = tabs[TCT_T2 + e];
  }
  if (t < SRT_GROUPS) mbar_init(mbar + t, 1);
  fence_async_smem();
  if (warp == 0) tc_alloc(tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + (uint32_t)(g * 128) + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t tcol = *tslot + (uint32_t)(g * 128);
  uint16_t* A = As + g * SRT_OPER;
  const uint32_t idesc = tc_idesc_f16(128, 128, 0);
  const uint32_t a_addr = smem_u32(A), b1_addr = smem_u32(B1s), b2_addr = smem_u32(B2s);
  const size_t ntiles = ((size_t)nct * 3) << (logN - 7);
  uint32_t phase = 0;
  for (size_t tile = (size_t)blockIdx.x * SRT_GROUPS + g; tile < ntiles; tile += (size_t)gridDim.x * SRT_GROUPS) {
    const size_t gid = (tile << 7) + m;
    const int n = (int)(gid & (N - 1));
    const size_t bj = gid >> logN;
    const uint64_t* d = dprod + bj * NQB * N + n;
    // ---- r = [t d]_Q to B: y_i = [t d (Q/q_i)^{-1}]_{q_i} straight from the transform ----
    {
      uint64_t y[L];
#pragma unroll
      for (int i = 0; i < L; ++i) y[i] = d[(size_t)i * N];
      put_limb_row<L>(A, m, y);
    }
    fence_async_smem();
    uint64_t dB[K];  // [t d Q^{-1} (B/b_k)^{-1}]_{b_k}, loaded while the MMA runs
#pragma unroll
    for (int k = 0; k < K; ++k) dB[k] = d[(size_t)(L + k) * N];
    tc_fence_before();
    named_sync(1 + g, 128);  // A written; every lane has read the previous tile's D
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < TC_K / 16; ++ks)
        tc_mma_f16(tcol, tc_desc(a_addr + ks * 256, 128, TC_K * 16), tc_desc(b1_addr + ks * 256, 128, TC_K * 16),
                   idesc, ks > 0);
      tc_commit(mbar + g);
      okf[g] = mbar_wait(mbar + g, phase, 1u << 22) ? 1u : 0u;  // one bounded waiter per group
    }
    named_sync(1 + g, 128);
    if (!okf[g]) {  // uniform in the group: leave the loop, free TMEM below
      if (m == 0) atomicOr(status, ST_TC_TIMEOUT);
      break;
    }
    phase ^= 1;
    tc_fence_after();
    // the centring decision v = floor(S + 1/2), S = sum_i y_i / q_i, from columns 8l + 7
    int v;
    {
      uint32_t e[8];
#pragma unroll
      for (int l = 0; l < 8; ++l) e[l] = tc_ld1(tmem + 8 * l + 7);
      tc_wait_ld();
      const Fix F = fix_from_limbs(e);
      v = fix_round(F, FIX_WINDOW);
      if (v < 0) v = lift_v_y_mem(d, N, F.hi);
    }
    // ---- y_k of w = (t d - r) Q^{-1} in B: one subtraction per prime ----
    uint64_t yb[K];
#pragma unroll
    for (int kb = 0; kb < K / 4; ++kb) {  // four primes (32 columns) per TMEM load
      uint32_t r32[32];
      tc_ld32(tmem + 32 * kb, r32);
      tc_wait_ld();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int k = kb * 4 + kk;
        const uint64_t b = cK.p[L + k];
        // [0, 2p) is enough here: yb only feeds the B -> Q operand (2p < 2^56, seven limbs),
        // whose sums are congruent and whose centring sum uses the same yb
        const uint64_t x = limb_sum_mod2(r32 + 8 * kk, T1s[v * 16 + k], b, cK.r32b[k], cK.r32b_s[k]);
        yb[k] = dB[k] + (dB[k] < x ? 2 * b : 0) - x;
      }
    }
    put_limb_row<K>(A, m, yb);  // the first MMA has finished with A
    fence_async_smem();
    tc_fence_before();
    named_sync(1 + g, 128);  // A written; every lane has read D
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < TC_K / 16; ++ks)
        tc_mma_f16(tcol, tc_desc(a_addr + ks * 256, 128, TC_K * 16), tc_desc(b2_addr + ks * 256, 128, TC_K * 16),
                   idesc, ks > 0);
      tc_commit(mbar + g);
      okf[g] = mbar_wait(mbar + g, phase, 1u << 22) ? 1u : 0u;  // one bounded waiter per group
    }
    named_sync(1 + g, 128);
    if (!okf[g]) {  // uniform in the group: leave the loop, free TMEM below
      if (m == 0) atomicOr(status, ST_TC_TIMEOUT);
      break;
    }
    phase ^= 1;
    tc_fence_after();
    // the centring decision vb of the B -> Q conversion, from columns 120 .. 127
    int vb;
    {
      uint32_t e[8];
      tc_ld8(tmem + 8 * L, e);
      tc_wait_ld();
      const Fix G = fix_from_limbs(e);
      vb = fix_round(G, FIX_WINDOW);
      if (vb < 0) {  // cannot happen for |w| < B / 2^24; recorded for the host
        atomicOr(status, ST_BQ_WINDOW);
        vb = (int)G.hi;
      }
    }
    // ---- w mod q_i (B -> Q), stored; d2 as key-switching digits ----
    uint64_t* o = w3 + bj * L * N + n;
    uint64_t out[L];
#pragma unroll
    for (int ib = 0; ib < 4; ++ib) {  // four primes (32 columns) per TMEM load
      uint32_t r32[32];
      tc_ld32(tmem + 32 * ib, r32);
      tc_wait_ld();
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) {
        const int i = ib * 4 + ii;
        if (i < L) out[i] = limb_sum_mod(r32 + 8 * ii, T2s[vb * 16 + i], cK.p[i], cK.r32[i], cK.r32_s[i]);
      }
    }
    if ((bj % 3) == 2 && dp != 1) {  // d2 as key-switching digits (and, with res, its residues)
      uint64_t* rr = res ? res + (bj / 3) * L * N + n : nullptr;
      if (dp == DIGIT_PRIMES) {
#pragma unroll
        for (int gq = 0; gq < NDIG; ++gq) digit_group_out<DIGIT_PRIMES>(out, DIGIT_PRIMES * gq, o, rr, N);
      } else if (dp == DIGIT_PRIMES5) {
#pragma unroll
        for (int gq = 0; gq < NDIG5; ++gq) digit_group_out<DIGIT_PRIMES5>(out, DIGIT_PRIMES5 * gq, o, rr, N);
      } else {  // the two-digit key: 8 + 7 primes
        digit_group_out<COARSE_DIGIT_PRIMES>(out, 0, o, rr, N);
        digit_group_out<L - COARSE_DIGIT_PRIMES>(out, COARSE_DIGIT_PRIMES, o, rr, N);
      }
    } else {
#pragma unroll
      for (int i = 0; i < L; ++i) o[(size_t)i * N] = out[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(*tslot, 512);
}

// ---- exact centred lift Q -> B (k_lift) with the conversion on the tensor cores ----
// Same first-lift modes and residue outputs as k_lift; the auxiliary residues
// come from one f16 MMA per 128-coefficient tile with the operand B1L (the plain
// Q -> B conversion) and the correction table T1, the centring decision from the
// same MMA's fixed-point columns.
constexpr size_t LFT_SMEM = (size_t)(1 + SRT_GROUPS) * SRT_OPER * 2 + TC_T1 * 8 + SRT_GROUPS * 8 + 32;

// the input residues of coefficient `m` of a lift tile (and the subtrahend's, for LIFT_SUB_CT)
template <bool SUBCT>
HPD void lift_tile_load(const uint64_t* __restrict__ src, const uint64_t* __restrict__ sub, size_t tile, int m, int logN,
                        uint64_t (&xv)[L], uint64_t (&sv)[SUBCT ? L : 1]) {
  const int N = 1 << logN;
  const size_t gid = (tile << 7) + m, bc = gid >> logN;
  const size_t off = bc * L * N + (gid & (N - 1));
#pragma unroll
  for (int i = 0; i < L; ++i) xv[i] = src[off + (size_t)i * N];
  if (SUBCT) {
#pragma unroll
    for (int i = 0; i < L; ++i) sv[i] = sub[off + (size_t)i * N];
  }
}

// SUBCT: mode LIFT_SUB_CT (a second ciphertext is read per coefficient); the
// other modes read at most one plaintext word, so their prefetch holds half the
// registers.
template <bool SUBCT>
__global__ void __launch_bounds__(SRT_THREADS, 1)
    k_lift_tc(const uint64_t* __restrict__ src, const uint64_t* __restrict__ sub, uint64_t const_val, int mode,
              uint64_t* __restrict__ ext, int* __restrict__ status, const uint16_t* __restrict__ ops,
              const uint64_t* __restrict__ tabs, int logN, int nct) {
  extern __shared__ __align__(1024) uint8_t lft_smem[];
  uint16_t* B1s = (uint16_t*)lft_smem;
  uint16_t* As = B1s + SRT_OPER;
  uint64_t* T1s = (uint64_t*)(As + SRT_GROUPS * SRT_OPER);
  uint64_t* mbar = T1s + TC_T1;
  uint32_t* tslot = (uint32_t*)(mbar + SRT_GROUPS);
  uint32_t* okf = tslot + 1;
  const int N = 1 << logN, t = threadIdx.x, warp = t >> 5, g = warp >> 2, m = t & 127;
  {
    const uint4* bsrc = (const uint4*)(ops + TCT_B1L);
    uint4* dst = (uint4*)lft_smem;
    for (int e = t; e < SRT_OPER / 8; e += SRT_THREADS) dst[e] = bsrc[e];
    for (int e = t; e < TC_T1; e += SRT_THREADS) T1s[e] = tabs[TCT_T1 + e];
  }
  if (t < SRT_GROUPS) mbar_init(mbar + t, 1);
  fence_async_smem();
  if (warp == 0) tc_alloc(tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + (uint32_t)(g * 128) + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t tcol = *tslot + (uint32_t)(g * 128);
  uint16_t* A = As + g * SRT_OPER;
  const uint32_t idesc = tc_idesc_f16(128, 128, 0);
  const uint32_t a_addr = smem_u32(A), b1_addr = smem_u32(B1s);
  const size_t ntiles = ((size_t)nct * 2) << (logN - 7), stride = (size_t)gridDim.x * SRT_GROUPS;
  uint32_t phase = 0;
  uint64_t xv[L], sv[SUBCT ? L : 1];  // this tile's inputs; the next tile's are loaded during the MMA
  size_t tile = (size_t)blockIdx.x * SRT_GROUPS + g;
  if (tile < ntiles) lift_tile_load<SUBCT>(src, sub, tile, m, logN, xv, sv);
  for (; tile < ntiles; tile += stride) {
    const size_t gid = (tile << 7) + m;
    const int n = (int)(gid & (N - 1));
    const size_t bc = gid >> logN;  // b * 2 + c
    const int comp = (int)(bc & 1);
    uint64_t* o = ext + bc * NQB * N + n;
    uint64_t y[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
      const uint64_t p = cK.p[i];
      uint64_t v = xv[i];
      if (SUBCT) {
        v = sub_mod(v, sv[SUBCT ? i : 0], p);
      } else if (mode == LIFT_SUB_CONST && comp == 0 && n == 0) {
        v = sub_mod(v, mul_shoup(const_val, cK.delta[i], cK.delta_s[i], p), p);
      } else if (mode == LIFT_SUB_PT && comp == 0) {
        v = sub_mod(v, mul_shoup(sub[(bc >> 1) * N + n], cK.delta[i], cK.delta_s[i], p), p);
      } else if (mode == LIFT_SUB_CONSTS && comp == 0 && n == 0) {
        v = sub_mod(v, mul_shoup(sub[bc >> 1], cK.delta[i], cK.delta_s[i], p), p);
      }
      o[(size_t)i * N] = v;
      y[i] = mul_shoup(v, cK.qhatinv[i], cK.qhatinv_s[i], p);
    }
    put_limb_row<L>(A, m, y);
    fence_async_smem();
    if (tile + stride < ntiles) lift_tile_load<SUBCT>(src, sub, tile + stride, m, logN, xv, sv);
    tc_fence_before();
    named_sync(1 + g, 128);  // A written; every lane has read the previous tile's D
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < TC_K / 16; ++ks)
        tc_mma_f16(tcol, tc_desc(a_addr + ks * 256, 128, TC_K * 16), tc_desc(b1_addr + ks * 256, 128, TC_K * 16),
                   idesc, ks > 0);
      tc_commit(mbar + g);
      okf[g] = mbar_wait(mbar + g, phase, 1u << 22) ? 1u : 0u;
    }
    named_sync(1 + g, 128);
    if (!okf[g]) {
      if (m == 0) atomicOr(status, ST_TC_TIMEOUT);
      break;
    }
    phase ^= 1;
    tc_fence_after();
    int v;  // floor(S + 1/2), S = sum_i y_i / q_i, from the fixed-point columns 8l + 7
    {
      uint32_t e[8];
#pragma unroll
      for (int l = 0; l < 8; ++l) e[l] = tc_ld1(tmem + 8 * l + 7);
      tc_wait_ld();
      const Fix F = fix_from_limbs(e);
      v = fix_round(F, FIX_WINDOW);
      if (v < 0) v = (int)F.hi + greater_than_half(o, N);  // exact: the residues written above
    }
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {  // four primes (32 columns) per TMEM load
      uint32_t r32[32];
      tc_ld32(tmem + 32 * kb, r32);
      tc_wait_ld();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int k = kb * 4 + kk;
        o[(size_t)(L + k) * N] = limb_sum_mod(r32 + 8 * kk, T1s[v * 16 + k], cK.p[L + k], cK.r32b[k], cK.r32b_s[k]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(*tslot, 512);
}

}  // namespace hp
