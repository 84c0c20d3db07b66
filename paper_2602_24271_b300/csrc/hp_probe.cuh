// Peak probes for the ALU roofline: the same 64-bit Shoup butterfly and the
// same 128-bit multiply-accumulate that the kernels use, on register-resident
// data only (no memory traffic), over a grid that fills every SM.
#pragma once
#include "hp_device.cuh"

namespace hp {

constexpr int PROBE_CHAINS = 8;

// Each thread runs PROBE_CHAINS independent butterfly chains for `iters` rounds.
__global__ void __launch_bounds__(256) k_probe_butterfly(uint64_t* sink, int iters, uint64_t p, uint64_t w,
                                                         uint64_t wp) {
  uint64_t X[PROBE_CHAINS], Y[PROBE_CHAINS];
  const uint64_t p2 = 2 * p;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) {
    X[c] = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % p;
    Y[c] = (threadIdx.x * 15485863u + c * 32452843u) % p;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) {
      uint64_t x = X[c] >= p2 ? X[c] - p2 : X[c];
      uint64_t v = mul_shoup_lazy(Y[c], w, wp, p);
      X[c] = x + v;
      Y[c] = x - v + p2;
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) acc ^= X[c] ^ Y[c];
  if (acc == 0x123456789ull) sink[0] = acc;  // keeps the chains live
}

// 128-bit lazy multiply-accumulate (base conversion / key switching inner loop).
__global__ void __launch_bounds__(256) k_probe_mac(uint64_t* sink, int iters, uint64_t p, uint64_t pinv) {
  uint64_t a[PROBE_CHAINS];
  Acc acc[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) {
    a[c] = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % p;
    acc_zero(acc[c]);
  }
  const uint64_t m = p - 12345;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) acc_mac(acc[c], a[c], m - it);
  }
  uint64_t r = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) r ^= redc_lazy(acc[c], p, pinv);
  if (r == 0x123456789ull) sink[0] = r;
}

}  // namespace hp
