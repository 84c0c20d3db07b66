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
