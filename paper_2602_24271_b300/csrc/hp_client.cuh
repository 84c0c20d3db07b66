// Client-side helper kernels (key generation, encryption, decryption) used by
// tests and by the benchmark's input generation.  Randomness: Philox4x32-10
// with counter (coefficient k, prime index j, object index, domain).
#pragma once
#include "hp_device.cuh"

namespace hp {

// s[k] = floor(3 w0 / 2^32) - 1
__global__ void k_sample_secret(int8_t* s, uint64_t seed, int N) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) s[k] = (int8_t)draw_ternary(philox((uint32_t)k, 0u, 0u, DOM_S, seed));
}

// out[j][k] = s_k mod p_{map(j)} for j < nprimes (PolyMap layout, one poly per prime)
__global__ void k_secret_to_primes(const int8_t* s, uint64_t* out, int nprimes, int id_base, int last_id, int N) {
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nprimes * N) return;
  int k = (int)(gid % N), j = (int)(gid / N);
  int id = (j == nprimes - 1 && last_id >= 0) ? last_id : id_base + j;
  int v = s[k];
  uint64_t p = cK.p[id];
  out[gid] = v < 0 ? p - 1 : (uint64_t)v;
}

// c[g] = a[g] b[g mod period_b] 2^-64 mod p  (Montgomery product; polys of N words,
// prime of poly g from the PolyMap of a)
__global__ void k_pointwise_mont(const uint64_t* a, const uint64_t* b, uint64_t* c, int period_b, int period,
                                 int id_base, int last_id, size_t npoly, int logN) {
  const int N = 1 << logN;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= npoly * N) return;
  size_t poly = gid >> logN;
  int n = (int)(gid & (N - 1));
  int r = (int)(poly % period);
  int id = (r == period - 1 && last_id >= 0) ? last_id : id_base + r;
  uint64_t bb = b[(size_t)(poly % period_b) * N + n];
  c[gid] = mont_mul_lazy(a[gid], bb, cK.p[id], cK.pinv[id]);
}

// tau_g(s) for the ternary secret: coefficient k moves to k g mod 2N, and to
// -X^(e - N) when k g mod 2N = e >= N.
__global__ void k_secret_automorph(const int8_t* s, int8_t* out, uint32_t g, int logN) {
  const int N = 1 << logN;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const uint32_t e = (uint32_t)(((uint64_t)k * g) & (2 * (uint64_t)N - 1));
  if (e < (uint32_t)N) {
    out[e] = s[k];
  } else {
    out[e - N] = (int8_t)(-s[k]);
  }
}

// Key-switching key with nd digits of dp data primes each (relinearisation:
// source s^2, domains A_RK / E_RK, object i for the three-prime key and
// FINE_OBJ + i for the per-prime key; Galois element g: source tau_g(s),
// domains A_GK / E_GK, object (g << 5) | i), part 1: a_{i,j,k} (uniform mod p_j)
// into both the output rk[i][1][j][k] and a work copy A[i][j][k].
__global__ void k_rk_sample_a(uint64_t* rk, uint64_t* A, uint64_t seed, int logN, uint32_t dom, uint32_t obj_base,
                              int nd) {
  const int N = 1 << logN;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nd * NKS * N) return;
  int k = (int)(gid & (N - 1));
  size_t ij = gid >> logN;
  int j = (int)(ij % NKS), i = (int)(ij / NKS);
  int id = j < L ? j : ID_P;
  uint64_t a = draw_uniform(philox((uint32_t)k, (uint32_t)j, obj_base | (uint32_t)i, dom, seed), cK.p[id]);
  A[gid] = a;
  rk[(((size_t)i * 2 + 1) * NKS + j) * N + k] = a;
}

// part 2: rk[i][0][j][k] = -(a s + e) + [q_j in digit i] [P]_{q_j} src  mod p_j, with
// AS = a s and S2 = the source secret in coefficient domain (canonical).
__global__ void k_rk_finish(uint64_t* rk, const uint64_t* AS, const uint64_t* S2, uint64_t seed, int logN,
                            uint32_t dom, uint32_t obj_base, int nd, int dp) {
  const int N = 1 << logN;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nd * NKS * N) return;
  int k = (int)(gid & (N - 1));
  size_t ij = gid >> logN;
  int j = (int)(ij % NKS), i = (int)(ij / NKS);
  int id = j < L ? j : ID_P;
  uint64_t p = cK.p[id];
  int e = draw_cbd21(philox((uint32_t)k, 0u, obj_base | (uint32_t)i, dom, seed));
  uint64_t em = e < 0 ? p - (uint64_t)(-e) : (uint64_t)e;
  uint64_t v = sub_mod(0, add_mod(AS[gid], em, p), p);
  if (j < L && j / dp == i) {  // g_i = 1 mod the digit's primes, 0 mod the others and P
    uint64_t s2 = S2[(size_t)j * N + k];
    uint64_t t = (uint64_t)(((unsigned __int128)s2 * cK.Pmodq[j]) % p);
    v = add_mod(v, t, p);
  }
  rk[(((size_t)i * 2 + 0) * NKS + j) * N + k] = v;
}

// Encryption, part 1: a for ciphertext c (object index idx0 + c) into ct[c][1]
// and a work copy A[c][j]; slots (< t) into the plaintext work M[c] for the
// encoding transform.
__global__ void k_enc_sample(uint64_t* ct, uint64_t* A, const uint32_t* slots, uint64_t* M, uint64_t seed,
                             uint32_t idx0, int logN, int nct) {
  const int N = 1 << logN;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * L * N) return;
  int k = (int)(gid & (N - 1));
  size_t cj = gid >> logN;
  int j = (int)(cj % L);
  size_t c = cj / L;
  uint64_t a = draw_uniform(philox((uint32_t)k, (uint32_t)j, (uint32_t)(idx0 + c), DOM_A_ENC, seed), cK.p[j]);
  A[gid] = a;
  ct[((c * 2 + 1) * L + j) * N + k] = a;
  if (j == 0) M[c * N + k] = slots[c * N + k];
}

// part 2: c0 = -(a s + e) + [Delta]_{q_j} m  mod q_j
__global__ void k_enc_finish(uint64_t* ct, const uint64_t* AS, const uint64_t* M, uint64_t seed, uint32_t idx0,
                             int logN, int nct) {
  const int N = 1 << logN;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * L * N) return;
  int k = (int)(gid & (N - 1));
  size_t cj = gid >> logN;
  int j = (int)(cj % L);
  size_t c = cj / L;
  uint64_t p = cK.p[j];
  int e = draw_cbd21(philox((uint32_t)k, 0u, (uint32_t)(idx0 + c), DOM_E_ENC, seed));
  uint64_t em = e < 0 ? p - (uint64_t)(-e) : (uint64_t)e;
  uint64_t v = sub_mod(0, add_mod(AS[gid], em, p), p);
  v = add_mod(v, mul_shoup(M[c * N + k], cK.delta[j], cK.delta_s[j], p), p);
  ct[((c * 2 + 0) * L + j) * N + k] = v;
}

// Decryption: X = [c0 + c1 s]_Q given C1S = c1 s (coefficient domain); the
// plaintext coefficient is m = round(t X / Q) mod t = -[t X]_Q Q^{-1} mod t,
// where [t X]_Q (centred) is lifted exactly to the modulus t.  Writes m into M.
__global__ void k_dec_round(const uint64_t* ct, const uint64_t* C1S, uint64_t* M, int logN, int nct) {
  const int N = 1 << logN;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (size_t)nct * N) return;
  int k = (int)(gid & (N - 1));
  size_t c = gid >> logN;
  uint64_t y[L];
  Fix F = {0, 0};
#pragma unroll
  for (int i = 0; i < L; ++i) {
    uint64_t p = cK.p[i];
    uint64_t x = add_mod(ct[((c * 2 + 0) * L + i) * N + k], C1S[(c * L + i) * N + k], p);
    y[i] = mul_shoup(x, cK.tqhatinv[i], cK.tqhatinv_s[i], p);  // [t x (Q/q_i)^{-1}]
    fix_add(F, fix_term(y[i], cK.om_hi[i], cK.om_lo[i]));
  }
  int vi = fix_round(F, 2 * L);
  uint64_t v = (uint64_t)(vi >= 0 ? vi : lift_v_from_y(y, F.hi));
  Acc acc;
  acc_zero(acc);
#pragma unroll
  for (int i = 0; i < L; ++i) acc_mac(acc, y[i], cK.MQt[i]);
  acc_mac(acc, v, cK.negQt);
  const uint64_t t = cK.p[ID_T];
  uint64_t r = redc(acc, t, cK.pinv[ID_T]);  // [t X]_Q centred, mod t
  uint64_t m = (uint64_t)(((unsigned __int128)sub_mod(0, r, t) * cK.Qinv_t) % t);
  M[gid] = m;
}

// decoded slots: forward-transform output (in [0, 8t)) reduced mod t
__global__ void k_u64_to_u32(const uint64_t* in, uint32_t* out, size_t n) {
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid < n) out[gid] = (uint32_t)(in[gid] % cK.p[ID_T]);
}

// Montgomery form of the relinearisation key after its forward transform:
// x -> x 2^64 mod p = REDC(x (2^128 mod p)).
__global__ void k_to_mont(uint64_t* a, int period, int id_base, int last_id, size_t npoly, int logN) {
  const int N = 1 << logN;
  size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= npoly * N) return;
  size_t poly = gid >> logN;
  int r = (int)(poly % period);
  int id = (r == period - 1 && last_id >= 0) ? last_id : id_base + r;
  uint64_t p = cK.p[id];
  a[gid] = csub(mont_mul_lazy(a[gid], cK.r2[id], p, cK.pinv[id]), p);
}

}  // namespace hp
