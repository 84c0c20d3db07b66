// Peak probes for the ALU roofline: the same 64-bit Shoup butterfly and the
// same 128-bit multiply-accumulate that the kernels use, on register-resident
// data only (no memory traffic), over a grid that fills every SM.
#pragma once
#include "hp_ntt.cuh"

namespace hp {

constexpr int PROBE_CHAINS = 8;

// Each thread runs PROBE_CHAINS independent butterfly chains for `iters` rounds.
__global__ void __launch_bounds__(256) k_probe_butterfly(uint64_t* sink, int iters, uint64_t p, uint64_t w,
                                                         uint64_t wp) {
  uint64_t X[PROBE_CHAINS], Y[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) {
    X[c] = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % p;
    Y[c] = (threadIdx.x * 15485863u + c * 32452843u) % p;
  }
  const uint64_t p4 = 4 * p;
  PForm f;
  f.p = p;
  f.np = 0 - p;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) {  // the forward transform's butterfly
      const uint64_t x = X[c];  // wraps mod 2^64 over many rounds: only the instruction stream matters here
      const uint64_t v = mul_shoup4(Y[c], w, wp, f);
      X[c] = x + v;
      Y[c] = x - v + p4;
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) acc ^= X[c] ^ Y[c];
  if (acc == 0x123456789ull) sink[0] = acc;  // keeps the chains live
}

// The same forward butterfly on 32-bit words for a prime p < 2^30 (a narrower
// residue word than the library's 55-bit primes): Shoup's product W Y - q p with
// q = floor(Y W' / 2^32), W' = floor(W 2^32 / p), is three 32-bit multiplies
// (low W Y, high Y W', low q p) and lies in [0, 2p); the lazy range grows by 2p
// per stage as in the 64-bit form.  Measures what a 32-bit residue basis would
// buy per multiplier slot; no kernel of the library uses it.
__global__ void __launch_bounds__(256) k_probe_butterfly32(uint64_t* sink, int iters, uint32_t p, uint32_t w,
                                                           uint32_t wp) {
  uint32_t X[PROBE_CHAINS], Y[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) {
    X[c] = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % p;
    Y[c] = (threadIdx.x * 15485863u + c * 32452843u) % p;
  }
  const uint32_t p2 = 2 * p;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) {
      const uint32_t x = X[c];  // wraps mod 2^32 over many rounds: only the instruction stream matters here
      const uint32_t q = __umulhi(Y[c], wp);
      const uint32_t v = Y[c] * w - q * p;
      X[c] = x + v;
      Y[c] = x - v + p2;
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) acc ^= X[c] ^ Y[c];
  if (acc == 0x12345679u) sink[0] = acc;  // keeps the chains live
}

// The base conversions' multiply-accumulate: 56-bit operands in 28-bit limbs,
// three 64-bit accumulators (four 32x32+64 multiply-adds per MAC).
__global__ void __launch_bounds__(256) k_probe_mac(uint64_t* sink, int iters, uint64_t p, uint64_t pinv) {
  uint32_t yl[PROBE_CHAINS], yh[PROBE_CHAINS];
  Acc3 acc[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) {
    const uint64_t y = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % p;
    yl[c] = lo28(y);
    yh[c] = hi28(y);
    acc3_zero(acc[c]);
  }
  for (int it = 0; it < iters; ++it) {
    const uint32_t ml = (uint32_t)it & 0xFFFFFFF, mh = (uint32_t)(it * 7) & 0x7FFFFFF;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) acc3_mac(acc[c], yl[c], yh[c], ml, mh);
  }
  uint64_t r = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) r ^= redc_lazy(acc3_fold(acc[c]), p, pinv);
  if (r == 0x123456789ull) sink[0] = r;
}

}  // namespace hp
