// Fifth-generation tensor core (tcgen05) helpers in inline PTX: shared-memory
// matrix descriptors, tensor-memory (TMEM) allocation, MMA issue and commit to
// an mbarrier, TMEM loads.  Used for the exact integer contractions of the RNS
// base conversions: residues split into 8-bit limbs are f16 values, products
// of two limbs (< 2^16) and sums of up to 128 of them (< 2^23) are exact in the
// f32 accumulator.
#pragma once
#include <stdint.h>

#include "hp_device.cuh"

namespace hp {

HPD uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor without swizzling for a K-major operand
// stored as core matrices of 8 rows x 16 bytes (8 f16), each core matrix 128
// contiguous bytes: lbo = byte step between core matrices along K, sbo = byte
// step between 8-row groups along M (or N).  Bits 46-47 hold the descriptor
// version (1); base offset, stride mode and layout type (0 = no swizzle) are 0.
HPD uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: f32 accumulator (bits 4-5 = 1), A and B
// both f16 (bits 7-9, 10-12 = 0) or both bf16 (= 1), both K-major (bits 15, 16
// = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
HPD constexpr uint32_t tc_idesc_f16(int M, int N, int bf16 = 0) {
  return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation of `ncols` columns (a power of two >= 32) by one whole warp;
// the TMEM address is written to `slot` in shared memory.
HPD void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
HPD void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] x B[smem]^T, one thread issues
HPD void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on `mbar` once every MMA issued so far by this thread has completed
HPD void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
HPD void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
HPD void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core
HPD void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

HPD void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
// Wait for the phase with parity `parity` to complete: at most `limit` polls
// (each poll may itself suspend for a bounded, implementation-defined time).
HPD bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 32 TMEM lanes (the warp's quarter) x 16 consecutive 32-bit columns: thread i
// of the warp receives lane (base lane + i), columns c .. c + 15.
HPD void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
HPD void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Offset (in f16 elements) of element (row r, column k) of a K-major operand
// with `kdim` columns in the core-matrix layout above.
HPD int tc_cm(int r, int k, int kdim) { return ((r >> 3) * (kdim >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

// ---- probe: one CTA computes D = A B^T for f16 or bf16 operands holding integers ----
// A: [128][112], B: [n][112] (row-major 16-bit patterns), D: [128][n] f32; n a
// multiple of 16 in [16, 256]; bf16 selects the operand type.  Checks the
// descriptor encodings and the exactness of the f32 accumulation of limb
// products on the hardware.
constexpr int TCP_M = 128, TCP_K = 112;
// With issue = 0 no MMA is issued and nothing arrives on the mbarrier: the
// bounded wait (`polls` polls) expires, the status word records it and the
// kernel frees its TMEM and returns (the failure path, exercised without a fault).
__global__ void __launch_bounds__(128) k_tc_probe(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B,
                                                  float* __restrict__ D, int n, int bf16, int issue, uint32_t polls,
                                                  int* status) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  uint16_t* As = (uint16_t*)tsm;
  uint16_t* Bs = As + TCP_M * TCP_K;
  uint64_t* mbar = (uint64_t*)(Bs + 256 * TCP_K);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5;
  for (int e = t; e < TCP_M * TCP_K; e += 128) As[tc_cm(e / TCP_K, e % TCP_K, TCP_K)] = A[e];
  for (int e = t; e < n * TCP_K; e += 128) Bs[tc_cm(e / TCP_K, e % TCP_K, TCP_K)] = B[e];
  if (t == 0) mbar_init(mbar, 1);
  fence_async_smem();
  if (warp == 0) tc_alloc(tslot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  if (t == 0 && issue) {
    const uint32_t idesc = tc_idesc_f16(TCP_M, n, bf16);
    for (int ks = 0; ks < TCP_K / 16; ++ks) {
      const uint64_t ad = tc_desc(smem_u32(As) + ks * 256, 128, (TCP_K / 8) * 128);
      const uint64_t bd = tc_desc(smem_u32(Bs) + ks * 256, 128, (TCP_K / 8) * 128);
      tc_mma_f16(tbase, ad, bd, idesc, ks > 0);
    }
    tc_commit(mbar);
  }
  __syncwarp();
  const bool ok = mbar_wait(mbar, 0, polls);
  if (!ok) atomicOr(status, 1);
  tc_fence_after();
  if (ok) {
    for (int c = 0; c < n; c += 16) {
      uint32_t r[16];
      tc_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
      tc_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) D[(size_t)t * n + c + j] = __uint_as_float(r[j]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tbase, 256);
}

}  // namespace hp
