// libhp: C ABI, handle management and the per-tile pipeline of the equality
// predicate EQ(x, y) = 1 - (x - y)^(p-1) (16 squarings + relinearisation).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hp.h"
#include "hp_client.cuh"
#include "hp_defs.h"
#include "hp_device.cuh"
#include "hp_ntt.cuh"
#include "hp_probe.cuh"
#include "hp_rns.cuh"
#include "hp_tc.cuh"
#include "hp_tcconv.cuh"

using namespace hp;

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct hp_handle {
  int logn = 0, N = 0, logR = 0;
  uint64_t q[L] = {}, P = 0, t = 0;
  uint32_t max_depth = 0;
  Consts C;
  int device = 0;
  // transform tables [NPRIME][N] and scaling constants [NSCALE][NPRIME][4]
  ulonglong2 *tw = nullptr, *itw = nullptr;  // (value, Shoup) pairs
  uint64_t* scale = nullptr;
  // key-switching digits of the relinearisation and Galois keys: dp primes
  // each (3 or 5), nd = L / dp of them
  int dp = DIGIT_PRIMES, nd = NDIG;
  // relinearisation key, NTT domain, Montgomery form: [nd][2][NKS][N]
  uint64_t* rkm = nullptr;
  bool have_rk = false;
  // products at output depth <= fine_depth are relinearised with the per-prime
  // key rkm1 ([NDIG_FINE][2][NKS][N], same form), allocated when fine_depth > 0
  uint32_t fine_depth = 0;
  uint64_t* rkm1 = nullptr;
  bool have_rk1 = false;
  // products at output depth >= coarse_from (> 0) are relinearised with the
  // two-digit key rkm2 ([NDIG2][2][NKS][N], same form), allocated when set
  uint32_t coarse_from = 0;
  uint64_t* rkm2 = nullptr;
  bool have_rk2 = false;
  // workspace for one pipeline tile of `tile` ciphertexts
  size_t tile = 0;
  uint64_t *ext = nullptr, *ext2 = nullptr, *dprod = nullptr, *w3 = nullptr, *ksin = nullptr, *ksout = nullptr,
           *ctbuf = nullptr, *maskbuf = nullptr;
  uint64_t* d2res = nullptr;  // [tile][L][N]: d2's residues (the digits' values modulo their own primes)
  // staging for host-memory calls and graph-replayed tiles: x, y, out, and the
  // plaintext polynomials of packed per-instance constants ([tile][N])
  uint64_t *stx = nullptr, *sty = nullptr, *sto = nullptr, *stm = nullptr;
  // second staging set and copy streams for overlapped host-memory calls
  uint64_t *stx2 = nullptr, *sty2 = nullptr, *sto2 = nullptr;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  size_t run_tile = 0;  // tile used by hp_run / hp_run_batched (autotuned, <= tile; 0 = tile)
  // CUDA graphs of the whole per-tile launch sequence, keyed by (first-lift mode, tile size)
  // The first node of a tile's sequence is the first lift (reads x and y or the
  // plaintext polynomials), the last the inverse column pass that writes out:
  // hp_run_batched points those two at each tile's ciphertexts before the launch.
  struct GraphEntry {
    int mode, b;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaGraphNode_t first, last;
    uint64_t kernels;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap = nullptr;
  // LT comparison: baby-step (255), giant-step (128), inner-sum (8) and four
  // temporary ciphertext arrays per tile, and one lifted, transformed operand
  // shared by consecutive products, allocated on the first LT call
  uint64_t* ltws = nullptr;
  size_t lt_tile = 0;
  uint32_t* lt_coef = nullptr;  // 32768 odd coefficients of the LT polynomial
  // Galois keys of the rotate-and-add reduction (one per element of
  // galois_elements, same layout and form as rkm), allocated on first use
  uint64_t* gkm = nullptr;
  bool have_gk = false;
  // tensor-core conversion operands and correction tables (build_tc_tables), SM count
  uint16_t* tct = nullptr;
  uint64_t* tctab = nullptr;
  int sms = 0;
  int* status = nullptr;  // device status word (ST_* bits)
  uint64_t launches = 0;
  std::string err;
  // opt-in per-kernel-class timing (CUDA events on the launching stream)
  uint32_t prof_mask = 0;
  struct Rec {
    int cls;
    cudaEvent_t e0, e1;
    double work;
  };
  std::vector<Rec> prof;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
};

// kernel classes for hp_profile_* (work unit in brackets)
enum {
  PK_NTT_FWD_COLS = 0,  // [butterflies]
  PK_NTT_FWD_ROWS = 1,  // [butterflies]
  PK_NTT_INV_ROWS = 2,  // [butterflies]
  PK_NTT_INV_COLS = 3,  // [butterflies]
  PK_LIFT = 4,          // [coefficients lifted]
  PK_TENSOR = 5,        // [residue products]
  PK_SCALE_ROUND = 6,   // [coefficients rounded]
  PK_AUTOMORPH = 7,     // [words written]
  PK_KS_MAC = 8,        // [multiply-accumulates]
  PK_MODDOWN = 9,       // [words]
  PK_COUNT = 10
};

static cudaEvent_t prof_event(hp_handle* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}
struct ProfScope {
  hp_handle* h;
  int cls;
  cudaStream_t s;
  double work;
  cudaEvent_t e0 = nullptr;
  ProfScope(hp_handle* h_, int cls_, cudaStream_t s_, double work_) : h(h_), cls(cls_), s(s_), work(work_) {
    if (h->prof_mask & (1u << cls)) {
      e0 = prof_event(h);
      cudaEventRecord(e0, s);
    }
  }
  ~ProfScope() {
    if (e0) {
      cudaEvent_t e1 = prof_event(h);
      cudaEventRecord(e1, s);
      h->prof.push_back({cls, e0, e1, work});
    }
  }
};

static std::string g_create_err;
extern "C" int hp_check_status(hp_handle* h);

#define HP_FAIL(h, code, ...)                                  \
  do {                                                         \
    char _b[512];                                              \
    snprintf(_b, sizeof(_b), __VA_ARGS__);                     \
    if (h) (h)->err = _b; else g_create_err = _b;              \
    return code;                                               \
  } while (0)

#define CU(h, call)                                                                  \
  do {                                                                               \
    cudaError_t _e = (call);                                                         \
    if (_e != cudaSuccess) HP_FAIL(h, HP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
  } while (0)

static inline size_t words_ct(const hp_handle* h) { return (size_t)2 * L * h->N; }

// per-ciphertext workspace words (nd: key-switching digits of the finest key used)
static size_t ws_words_per_ct(int N, int nd) {
  return (size_t)N * (2 * NQB      // ext
                      + 2 * NQB    // ext2 (SELECT operand)
                      + 3 * NQB    // dprod
                      + 3 * L      // w3
                      + L          // d2res
                      + nd * NKS   // ksin
                      + 2 * NKS    // ksout
                      + 2 * L      // ctbuf
                      + 2 * L      // maskbuf
                      + 6 * 2 * L  // two staging sets x, y, out
                      + 1          // staging plaintext polynomials
                     );
}

static inline unsigned ew_blocks(size_t n) { return (unsigned)((n + EW_THREADS - 1) / EW_THREADS); }

static NttTabs tabs(const hp_handle* h) {
  NttTabs T;
  T.tw = h->tw;
  T.itw = h->itw;
  T.scale = h->scale;
  return T;
}

static const PolyMap MAP_QB = {NQB, 0, -1};  // [.][NQB][N]: ids 0..30
static const PolyMap MAP_KS = {NKS, 0, ID_P}; // [.][NKS][N]: q_0..q_14, P
static const PolyMap MAP_Q = {L, 0, -1};      // [.][L][N]
static const PolyMap MAP_T = {1, ID_T, -1};   // plaintext modulus

template <int LR, int LC>
static void ntt_fwd_t(hp_handle* h, uint64_t* data, size_t npoly, PolyMap m, DigitSrc dig, cudaStream_t s) {
  const dim3 gc((1u << LC) / (NTT_TILE >> LR), (unsigned)npoly), gr((1u << LR) / (NTT_TILE >> LC), (unsigned)npoly);
  const double half = (double)npoly * (h->N / 2);
  {
    ProfScope ps(h, PK_NTT_FWD_COLS, s, half * LR);
    if (!dig.w3)
      k_ntt_fwd_cols<LR, LC, 0><<<gc, NTT_THREADS, 0, s>>>(data, m, tabs(h), dig);
    else if (dig.dp == 1)
      k_ntt_fwd_cols<LR, LC, 1><<<gc, NTT_THREADS, 0, s>>>(data, m, tabs(h), dig);
    else if (dig.dp == DIGIT_PRIMES5)
      k_ntt_fwd_cols<LR, LC, DIGIT_PRIMES5><<<gc, NTT_THREADS, 0, s>>>(data, m, tabs(h), dig);
    else if (dig.dp == COARSE_DIGIT_PRIMES)
      k_ntt_fwd_cols<LR, LC, COARSE_DIGIT_PRIMES><<<gc, NTT_THREADS, 0, s>>>(data, m, tabs(h), dig);
    else
      k_ntt_fwd_cols<LR, LC, DIGIT_PRIMES><<<gc, NTT_THREADS, 0, s>>>(data, m, tabs(h), dig);
  }
  {
    ProfScope ps(h, PK_NTT_FWD_ROWS, s, half * LC);
    k_ntt_fwd_rows<LR, LC><<<gr, NTT_THREADS, 0, s>>>(data, m, tabs(h));
  }
  h->launches += 2;
}

// Forward transform of the lifted squaring operand (nct x 2 x NQB polynomials)
// with the squaring tensor fused into the row pass: ext -> dprod.
template <int LR, int LC>
static void ntt_fwd_sq_t(hp_handle* h, uint64_t* ext, uint64_t* dprod, int nct, cudaStream_t s) {
  const size_t npoly = (size_t)nct * 2 * NQB;
  const dim3 gc((1u << LC) / (NTT_TILE >> LR), (unsigned)npoly),
      gr((1u << LR) / (NTT_TILE >> LC), (unsigned)(nct * NQB));
  const double half = (double)npoly * (h->N / 2);
  DigitSrc d;
  d.w3 = nullptr;
  d.dp = DIGIT_PRIMES;
  {
    ProfScope ps(h, PK_NTT_FWD_COLS, s, half * LR);
    k_ntt_fwd_cols<LR, LC, 0><<<gc, NTT_THREADS, 0, s>>>(ext, MAP_QB, tabs(h), d);
  }
  {
    ProfScope ps(h, PK_NTT_FWD_ROWS, s, half * LC);
    k_ntt_fwd_rows_sq<LR, LC><<<gr, NTT_THREADS, 0, s>>>(ext, dprod, tabs(h));
  }
  h->launches += 2;
}

template <int LR, int LC>
static void ntt_inv_t(hp_handle* h, uint64_t* data, size_t npoly, PolyMap m, int scale_mode, cudaStream_t s) {
  const dim3 gc((1u << LC) / (NTT_TILE >> LR), (unsigned)npoly), gr((1u << LR) / (NTT_TILE >> LC), (unsigned)npoly);
  const double half = (double)npoly * (h->N / 2);
  {
    ProfScope ps(h, PK_NTT_INV_ROWS, s, half * LC);
    k_ntt_inv_rows<LR, LC><<<gr, NTT_THREADS, 0, s>>>(data, m, tabs(h));
  }
  {
    ProfScope ps(h, PK_NTT_INV_COLS, s, half * LR);
    ModDown md = {nullptr, nullptr, 0, 1, 0};
    k_ntt_inv_cols<LR, LC, false><<<gc, NTT_THREADS, 0, s>>>(data, m, tabs(h), scale_mode, md);
  }
  h->launches += 2;
}

// Inverse transform of the key-switching sums (nct x 2 x NKS polynomials) with
// the mod-down fused into the column pass of the data primes: the special
// prime's polynomials first, then out[bc][i] = w3 + round(u / P) (or "1 -").
template <int LR, int LC>
static void ntt_inv_moddown_t(hp_handle* h, uint64_t* ksout, int nct, uint64_t* out, int one_minus, cudaStream_t s) {
  const size_t npoly = (size_t)nct * 2 * NKS;
  const unsigned cx = (1u << LC) / (NTT_TILE >> LR);
  const dim3 gr((1u << LR) / (NTT_TILE >> LC), (unsigned)npoly);
  const double half = (double)(h->N / 2);
  {
    ProfScope ps(h, PK_NTT_INV_ROWS, s, half * npoly * LC);
    k_ntt_inv_rows<LR, LC><<<gr, NTT_THREADS, 0, s>>>(ksout, MAP_KS, tabs(h));
  }
  {
    ProfScope ps(h, PK_NTT_INV_COLS, s, half * npoly * LR);
    ModDown mp = {nullptr, nullptr, 0, NKS, L};  // polynomials bc NKS + L: the special prime
    k_ntt_inv_cols<LR, LC, false><<<dim3(cx, (unsigned)(nct * 2)), NTT_THREADS, 0, s>>>(ksout, MAP_KS, tabs(h),
                                                                                        SCALE_NINV, mp);
    ModDown md = {h->w3, out, one_minus, 0, 0};
    k_ntt_inv_cols<LR, LC, true><<<dim3(cx, (unsigned)(nct * 2 * L)), NTT_THREADS, 0, s>>>(ksout, MAP_KS, tabs(h),
                                                                                           SCALE_NINV, md);
  }
  h->launches += 3;
}
static void ntt_inv_moddown(hp_handle* h, uint64_t* ksout, int nct, uint64_t* out, int one_minus, cudaStream_t s) {
  switch (h->logn) {
    case 12: ntt_inv_moddown_t<6, 6>(h, ksout, nct, out, one_minus, s); break;
    case 13: ntt_inv_moddown_t<6, 7>(h, ksout, nct, out, one_minus, s); break;
    case 14: ntt_inv_moddown_t<7, 7>(h, ksout, nct, out, one_minus, s); break;
    default: ntt_inv_moddown_t<7, 8>(h, ksout, nct, out, one_minus, s); break;
  }
}

// N = R x C with log R = floor(log N / 2)
static void ntt_fwd(hp_handle* h, uint64_t* data, size_t npoly, PolyMap m, cudaStream_t s,
                    const uint64_t* digits = nullptr, int dp = DIGIT_PRIMES, const uint64_t* res = nullptr) {
  if (npoly == 0) return;
  DigitSrc d;
  d.res = res;
  d.w3 = digits;
  d.dp = dp;
  switch (h->logn) {
    case 12: ntt_fwd_t<6, 6>(h, data, npoly, m, d, s); break;
    case 13: ntt_fwd_t<6, 7>(h, data, npoly, m, d, s); break;
    case 14: ntt_fwd_t<7, 7>(h, data, npoly, m, d, s); break;
    default: ntt_fwd_t<7, 8>(h, data, npoly, m, d, s); break;
  }
}

static void ntt_fwd_sq(hp_handle* h, uint64_t* ext, uint64_t* dprod, int nct, cudaStream_t s) {
  switch (h->logn) {
    case 12: ntt_fwd_sq_t<6, 6>(h, ext, dprod, nct, s); break;
    case 13: ntt_fwd_sq_t<6, 7>(h, ext, dprod, nct, s); break;
    case 14: ntt_fwd_sq_t<7, 7>(h, ext, dprod, nct, s); break;
    default: ntt_fwd_sq_t<7, 8>(h, ext, dprod, nct, s); break;
  }
}

static void ntt_inv(hp_handle* h, uint64_t* data, size_t npoly, PolyMap m, int scale_mode, cudaStream_t s) {
  if (npoly == 0) return;
  switch (h->logn) {
    case 12: ntt_inv_t<6, 6>(h, data, npoly, m, scale_mode, s); break;
    case 13: ntt_inv_t<6, 7>(h, data, npoly, m, scale_mode, s); break;
    case 14: ntt_inv_t<7, 7>(h, data, npoly, m, scale_mode, s); break;
    default: ntt_inv_t<7, 8>(h, data, npoly, m, scale_mode, s); break;
  }
}

// ---------------------------------------------------------------------------
// one squaring (or general product) + relinearisation on a tile of b
// ciphertexts whose extended-base transforms are in h->ext (and h->ext2); the
// product lies at multiplicative depth `depth`, which selects the key:
// per-prime digits up to the handle's fine depth, the two-digit key from its
// coarse depth on, digits of the handle's grouping (three or five primes) between
// ---------------------------------------------------------------------------
// The key-switching multiply-accumulate for keys of nd digits (2, 3, 5 or 15).
static void ks_mac(hp_handle* h, const uint64_t* rk, int nd, int b, cudaStream_t s) {
  const unsigned grid = ew_blocks((size_t)NKS * h->N);
  ProfScope ps(h, PK_KS_MAC, s, 2.0 * b * nd * NKS * h->N);
  if (nd == NDIG_FINE)
    k_ks_mac<NDIG_FINE><<<grid, EW_THREADS, 0, s>>>(h->ksin, rk, h->ksout, h->logn, b);
  else if (nd == NDIG5)
    k_ks_mac<NDIG5><<<grid, EW_THREADS, 0, s>>>(h->ksin, rk, h->ksout, h->logn, b);
  else if (nd == NDIG2)
    k_ks_mac<NDIG2><<<grid, EW_THREADS, 0, s>>>(h->ksin, rk, h->ksout, h->logn, b);
  else
    k_ks_mac<NDIG><<<grid, EW_THREADS, 0, s>>>(h->ksin, rk, h->ksout, h->logn, b);
  h->launches += 1;
}

// With `ea` (general products only) the first operand's lifted, transformed
// form is taken from there instead of h->ext.
static void mul_relin_tail(hp_handle* h, int b, bool general, uint64_t* out, int one_minus, cudaStream_t s,
                           int depth, const uint64_t* ea = nullptr) {
  const int N = h->N, logN = h->logn;
  const bool fine = depth <= (int)h->fine_depth;
  const bool coarse = !fine && h->coarse_from > 0 && depth >= (int)h->coarse_from;
  const int nd = fine ? NDIG_FINE : (coarse ? NDIG2 : h->nd), dp = fine ? 1 : (coarse ? COARSE_DIGIT_PRIMES : h->dp);
  const uint64_t* rk = fine ? h->rkm1 : (coarse ? h->rkm2 : h->rkm);
  if (general) {  // SELECT: general product
    if (!ea) {
      ntt_fwd(h, h->ext, (size_t)b * 2 * NQB, MAP_QB, s);
      ea = h->ext;
    }
    ntt_fwd(h, h->ext2, (size_t)b * 2 * NQB, MAP_QB, s);
    ProfScope ps(h, PK_TENSOR, s, 4.0 * b * NQB * N);
    k_tensor_gen<<<ew_blocks((size_t)b * NQB * N), EW_THREADS, 0, s>>>(ea, h->ext2, h->dprod, logN, b);
    h->launches += 1;
  } else {  // squaring: the tensor is fused into the forward row pass
    ntt_fwd_sq(h, h->ext, h->dprod, b, s);
  }
  ntt_inv(h, h->dprod, (size_t)b * 3 * NQB, MAP_QB, SCALE_T_NINV_R_CONV, s);
  {
    ProfScope ps(h, PK_SCALE_ROUND, s, 3.0 * b * N);
    const size_t tiles = ((size_t)b * 3 * N) >> 7, ctas = (tiles + SRT_GROUPS - 1) / SRT_GROUPS;
    k_scale_round_tc<<<(unsigned)std::min<size_t>(ctas, (size_t)h->sms), SRT_THREADS, SRT_SMEM, s>>>(
        h->dprod, h->w3, h->status, h->tct, h->tctab, logN, b, dp, h->d2res);
  }
  h->launches += 1;
  // key switching: the digits [d2]_{Q_a} (dp data primes each, stored in
  // mixed radix by the scale-and-round, or one prime each) reduced mod every
  // target prime p_j in the first transform pass, key multiply-accumulate,
  // inverse transform, mod-down
  ntt_fwd(h, h->ksin, (size_t)b * nd * NKS, MAP_KS, s, h->w3, dp, h->d2res);
  ks_mac(h, rk, nd, b, s);
  ntt_inv_moddown(h, h->ksout, b, out, one_minus, s);
}

static void lift(hp_handle* h, const uint64_t* src, const uint64_t* sub, uint64_t cval, int mode, uint64_t* ext, int b,
                 cudaStream_t s) {
  ProfScope ps(h, PK_LIFT, s, 2.0 * b * h->N);
  const size_t tiles = ((size_t)b * 2 * h->N) >> 7, ctas = (tiles + SRT_GROUPS - 1) / SRT_GROUPS;
  const unsigned grid = (unsigned)std::min<size_t>(ctas, (size_t)h->sms);
  if (mode == LIFT_SUB_CT)
    k_lift_tc<true><<<grid, SRT_THREADS, LFT_SMEM, s>>>(src, sub, cval, mode, ext, h->status, h->tct, h->tctab,
                                                          h->logn, b);
  else
    k_lift_tc<false><<<grid, SRT_THREADS, LFT_SMEM, s>>>(src, sub, cval, mode, ext, h->status, h->tct, h->tctab,
                                                           h->logn, b);
  h->launches += 1;
}

// The whole hot path for one tile of b device-resident ciphertexts; the first
// lift applies row a1 in mode `lmode` (sub = y for LIFT_SUB_CT, the plaintext
// polynomials for LIFT_SUB_PT).
static void run_tile_mode(hp_handle* h, int op, int lmode, const uint64_t* x, const uint64_t* sub, const uint64_t* y,
                          uint64_t cval, uint64_t* out, int b, cudaStream_t s) {
  if (op == HP_SQUARE) {  // the input is taken as fresh: the square lies at depth 1
    lift(h, x, nullptr, 0, LIFT_COPY, h->ext, b, s);
    mul_relin_tail(h, b, false, out, 0, s, 1);
    return;
  }
  // a1: difference, fused into the first lift
  lift(h, x, sub, cval, lmode, h->ext, b, s);
  // a2: 16 squarings; a3: "1 -" fused into the last mod-down
  for (int it = 0; it < 16; ++it) {
    if (it > 0) lift(h, h->ctbuf, nullptr, 0, LIFT_COPY, h->ext, b, s);
    const bool last = it == 15;
    uint64_t* dst = !last ? h->ctbuf : (op == HP_SELECT ? h->maskbuf : out);
    mul_relin_tail(h, b, false, dst, last ? 1 : 0, s, it + 1);
  }
  if (op == HP_SELECT) {  // a4: column * mask (depth 17)
    lift(h, h->maskbuf, nullptr, 0, LIFT_COPY, h->ext, b, s);
    lift(h, y, nullptr, 0, LIFT_COPY, h->ext2, b, s);
    mul_relin_tail(h, b, true, out, 0, s, 17);
  }
}

static void run_tile(hp_handle* h, int op, const uint64_t* x, const uint64_t* y, uint64_t cval, uint64_t* out, int b,
                     cudaStream_t s) {
  const int lmode = op == HP_EQ_CT_CT ? LIFT_SUB_CT : LIFT_SUB_CONST;
  run_tile_mode(h, op, lmode, x, op == HP_EQ_CT_CT ? y : nullptr, y, cval, out, b, s);
}

// ---------------------------------------------------------------------------
// LT comparison (Eq. 4) on a tile of b ciphertext pairs: f(z) = z h(w) -
// 32768 w^32768 with z = x - y, w = z^2, evaluated by a baby-step /
// giant-step schedule in which every power is the product of its largest
// power-of-two part and the rest (511 multiplications, depth 18):
//   B_1 = w, B_i = B_{i/2}^2 (i = 2^k) or B_{2^k} B_{i-2^k} (2^k < i < 2^(k+1)), i < 256;
//   G_1 = B_128^2, G_j likewise from G_{2^k} and G_{j-2^k}, j <= 128;
//   H_j = (Delta h_{256j}, 0) + sum_i h_{256j+i} B_i;  h = H_0 + sum_{j>=1} H_j G_j.
// B_i then lies at depth 1 + ceil(log2 i) <= 9 and G_j at 9 + ceil(log2 j) <= 16.
// ---------------------------------------------------------------------------
static int top_pow2(int i) {  // largest power of two <= i (i >= 1)
  int k = 1;
  while (2 * k <= i) k *= 2;
  return k;
}
static int ceil_log2(int i) {  // i >= 1
  int e = 0;
  while ((1 << e) < i) ++e;
  return e;
}
// a^2 (resp. a c) relinearised, the product at multiplicative depth `depth`
static void hsquare(hp_handle* h, const uint64_t* a, uint64_t* out, int b, cudaStream_t s, int depth) {
  lift(h, a, nullptr, 0, LIFT_COPY, h->ext, b, s);
  mul_relin_tail(h, b, false, out, 0, s, depth);
}
static void hmul(hp_handle* h, const uint64_t* a, const uint64_t* c, uint64_t* out, int b, cudaStream_t s,
                 int depth) {
  lift(h, a, nullptr, 0, LIFT_COPY, h->ext, b, s);
  lift(h, c, nullptr, 0, LIFT_COPY, h->ext2, b, s);
  mul_relin_tail(h, b, true, out, 0, s, depth);
}
// a's lift, transformed, into ea: the shared operand of the products that follow
static void lift_ntt(hp_handle* h, const uint64_t* a, uint64_t* ea, int b, cudaStream_t s) {
  lift(h, a, nullptr, 0, LIFT_COPY, ea, b, s);
  ntt_fwd(h, ea, (size_t)b * 2 * NQB, MAP_QB, s);
}
// a c relinearised for an operand a already in ea (lift_ntt)
static void hmul_ntt(hp_handle* h, const uint64_t* ea, const uint64_t* c, uint64_t* out, int b, cudaStream_t s,
                     int depth) {
  lift(h, c, nullptr, 0, LIFT_COPY, h->ext2, b, s);
  mul_relin_tail(h, b, true, out, 0, s, depth, ea);
}
static void ct_addsub(hp_handle* h, const uint64_t* a, const uint64_t* c, uint64_t* out, int subtract, int b,
                      cudaStream_t s) {
  const size_t nw = (size_t)b * words_ct(h);
  k_ct_addsub<<<ew_blocks(nw), EW_THREADS, 0, s>>>(a, c, out, subtract, h->logn, nw);
  h->launches += 1;
}

// LT workspace of a tile: B_1 .. B_255, G_1 .. G_128, 8 inner sums, then the
// ciphertext arrays z (the difference), acc, tmp and r (BETWEEN's first result),
// then ea: the lifted, transformed B_{2^k} (G_{2^k}) that the products
// B_{2^k} B_{i - 2^k} (G_{2^k} G_{j - 2^k}) of one k share
struct LtWs {
  uint64_t *Bp, *Gp, *Hp, *z, *acc, *tmp, *r, *ea;
};
static LtWs lt_ws(hp_handle* h) {
  const size_t T = h->lt_tile * words_ct(h);
  LtWs w;
  w.Bp = h->ltws;
  w.Gp = w.Bp + 255 * T;
  w.Hp = w.Gp + 128 * T;
  w.z = w.Hp + LT_J * T;
  w.acc = w.z + T;
  w.tmp = w.acc + T;
  w.r = w.tmp + T;
  w.ea = w.r + T;
  return w;
}

// f(z) of Eq. 4 for the tile's differences already in the workspace's z.
static void run_lt_z(hp_handle* h, uint64_t* out, int b, cudaStream_t s) {
  const size_t W = words_ct(h), bw = (size_t)b * W, T = h->lt_tile * W;
  const LtWs ws = lt_ws(h);
  uint64_t *Bp = ws.Bp, *Gp = ws.Gp, *Hp = ws.Hp, *z = ws.z, *acc = ws.acc, *tmp = ws.tmp;
  auto B = [&](int i) { return Bp + (size_t)(i - 1) * T; };
  auto G = [&](int j) { return Gp + (size_t)(j - 1) * T; };
  // depths: B_i at 1 + ceil(log2 i), G_j at 9 + ceil(log2 j)
  // the shared factor B_{2^k} (G_{2^k}) is lifted and transformed once per k
  hsquare(h, z, B(1), b, s, 1);
  for (int i = 2; i < 256; ++i) {
    const int k = top_pow2(i), d = 1 + ceil_log2(i);
    if (k == i) {
      hsquare(h, B(i / 2), B(i), b, s, d);
    } else {
      if (i == k + 1) lift_ntt(h, B(k), ws.ea, b, s);
      hmul_ntt(h, ws.ea, B(i - k), B(i), b, s, d);
    }
  }
  hsquare(h, B(128), G(1), b, s, 9);
  for (int j = 2; j <= 128; ++j) {
    const int k = top_pow2(j), d = 9 + ceil_log2(j);
    if (k == j) {
      hsquare(h, G(j / 2), G(j), b, s, d);
    } else {
      if (j == k + 1) lift_ntt(h, G(k), ws.ea, b, s);
      hmul_ntt(h, ws.ea, G(j - k), G(j), b, s, d);
    }
  }
  // The inner-sum kernel reads B as [255][bw]; with a partial tile (b < lt_tile)
  // the arrays keep their stride T, so compact them is unnecessary: pass bw = T
  // and ignore the unused tail words.
  for (int j0 = 0; j0 < 128; j0 += LT_J) {
    k_lt_inner<<<ew_blocks(T), EW_THREADS, 0, s>>>(Bp, h->lt_coef, j0, Hp, h->logn, T);
    h->launches += 1;
    for (int jj = 0; jj < LT_J; ++jj) {
      const int j = j0 + jj;
      if (j == 0) {
        cudaMemcpyAsync(acc, Hp, bw * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
      } else {
        hmul(h, Hp + (size_t)jj * T, G(j), tmp, b, s, 10 + ceil_log2(j));
        ct_addsub(h, acc, tmp, acc, 0, b, s);
      }
    }
  }
  hmul(h, z, acc, tmp, b, s, 18);
  ScalarK sk;  // out = tmp - 32768 G_128 = tmp + (t - 32768) G_128
  for (int i = 0; i < L; ++i) {
    sk.k[i] = (h->t - (h->t - 1) / 2) % h->q[i];
    sk.ks[i] = h_shoup(sk.k[i], h->q[i]);
  }
  k_ct_axpy<<<ew_blocks(bw), EW_THREADS, 0, s>>>(tmp, G(128), out, sk, h->logn, bw);
  h->launches += 1;
}

static void run_lt_tile(hp_handle* h, const uint64_t* x, const uint64_t* y, uint64_t* out, int b, cudaStream_t s) {
  ct_addsub(h, x, y, lt_ws(h).z, 1, b, s);
  run_lt_z(h, out, b, s);
}

// BETWEEN on a tile: (1 - f(x - lo)) (1 - f(hi - x)) = [lo <= x <= hi], the
// product of the two comparisons (depth 19).
static void run_between_tile(hp_handle* h, const uint64_t* x, uint64_t lo, uint64_t hi, uint64_t* out, int b,
                             cudaStream_t s) {
  const LtWs ws = lt_ws(h);
  const size_t bw = (size_t)b * words_ct(h);
  k_ct_const_diff<<<ew_blocks(bw), EW_THREADS, 0, s>>>(x, lo, 0, ws.z, h->logn, bw);
  h->launches += 1;
  run_lt_z(h, ws.r, b, s);  // a = [x < lo]
  k_ct_const_diff<<<ew_blocks(bw), EW_THREADS, 0, s>>>(x, hi, 1, ws.z, h->logn, bw);
  h->launches += 1;
  run_lt_z(h, out, b, s);  // b = [hi < x]
  k_one_minus<<<ew_blocks(bw), EW_THREADS, 0, s>>>(ws.r, ws.acc, h->logn, b);
  k_one_minus<<<ew_blocks(bw), EW_THREADS, 0, s>>>(out, ws.tmp, h->logn, b);
  h->launches += 2;
  hmul(h, ws.acc, ws.tmp, out, b, s, 19);
}

static int lt_prepare(hp_handle* h) {
  if (h->ltws) return HP_OK;
  h->lt_tile = h->tile < 8 ? h->tile : 8;
  const size_t words = (size_t)(255 + 128 + LT_J + 4) * h->lt_tile * words_ct(h) + h->lt_tile * 2 * NQB * h->N;
  if (cudaMalloc(&h->ltws, words * sizeof(uint64_t)) != cudaSuccess) {
    cudaGetLastError();
    h->ltws = nullptr;
    HP_FAIL(h, HP_ERR_OOM, "LT workspace (%zu MB) allocation failed", (words * 8) >> 20);
  }
  std::vector<uint32_t> coef(32768);
  lt_coefficients(coef.data());
  CU(h, cudaMalloc(&h->lt_coef, coef.size() * sizeof(uint32_t)));
  CU(h, cudaMemcpy(h->lt_coef, coef.data(), coef.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  return HP_OK;
}

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
static int brv(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// Operands and correction tables of the tensor-core scale-and-round, and the
// kernel's shared-memory limit.
static int build_tc(hp_handle* h) {
  std::vector<uint16_t> ops(TCT_OPS);
  std::vector<uint64_t> tabs(TCT_TABS);
  build_tc_tables(h->C, ops.data(), tabs.data());
  CU(h, cudaMalloc((void**)&h->tct, ops.size() * sizeof(uint16_t)));
  CU(h, cudaMemcpy(h->tct, ops.data(), ops.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
  CU(h, cudaMalloc((void**)&h->tctab, tabs.size() * sizeof(uint64_t)));
  CU(h, cudaMemcpy(h->tctab, tabs.data(), tabs.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
  CU(h, cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device));
  CU(h, cudaFuncSetAttribute(k_scale_round_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SRT_SMEM));
  CU(h, cudaFuncSetAttribute(k_lift_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LFT_SMEM));
  CU(h, cudaFuncSetAttribute(k_lift_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LFT_SMEM));
  return HP_OK;
}

// Position of twiddle entry j in the device table: entries of the stages
// s >= logR + 4 (the second half of the row pass) are transposed within each
// row's range of 2^{4+l} entries, l = s - logR - 4: entry 2^s + row 2^{4+l} +
// g 2^l + g' (column group g < 16, butterfly group g' < 2^l) is stored at
// 2^s + row 2^{4+l} + g' 16 + g, the order in which a row's threads read them.
static size_t row_pass_twiddle_pos(size_t j, int logR) {
  if (j < ((size_t)1 << (logR + 4))) return j;
  int s = 0;
  while ((j >> (s + 1)) != 0) ++s;
  const int l = s - logR - 4;
  const size_t off = j - ((size_t)1 << s), row = off >> (4 + l), w = off & (((size_t)1 << (4 + l)) - 1);
  const size_t g = w >> l, gp = w & (((size_t)1 << l) - 1);
  return ((size_t)1 << s) + (row << (4 + l)) + (gp << 4) + g;
}

static int build_tables(hp_handle* h) {
  const int N = h->N;
  std::vector<ulonglong2> tw((size_t)NPRIME * N), itw(tw.size());
  std::vector<uint64_t> sc((size_t)NSCALE * NPRIME * 4);
  std::vector<uint64_t> pw(N), ipw(N);
  for (int id = 0; id < NPRIME; ++id) {
    const uint64_t p = h->C.p[id];
    const uint64_t psi = h_powmod(h_qnr(p), (p - 1) / (2 * (uint64_t)N), p);
    const uint64_t ipsi = h_invmod(psi, p);
    pw[0] = ipw[0] = 1;
    for (int e = 1; e < N; ++e) {
      pw[e] = h_mulmod(pw[e - 1], psi, p);
      ipw[e] = h_mulmod(ipw[e - 1], ipsi, p);
    }
    for (int j = 0; j < N; ++j) {
      size_t o = (size_t)id * N + row_pass_twiddle_pos(j, h->logR);
      const uint64_t w = pw[brv(j, h->logn)], iw = ipw[brv(j, h->logn)];
      tw[o] = make_ulonglong2(w, h_shoup(w, p));
      itw[o] = make_ulonglong2(iw, h_shoup(iw, p));
    }
    const uint64_t ninv = h_invmod((uint64_t)N % p, p);
    const uint64_t r64 = (uint64_t)(((unsigned __int128)1 << 64) % p);
    // N^{-1} P^{-1} is used for the data primes only (the mod-down)
    const uint64_t tnr = h_mulmod(h_mulmod(h->t % p, ninv, p), r64, p);
    // SCALE_T_NINV_R_CONV: the scale-and-round's inputs already multiplied by
    // [(Q/q_i)^{-1}]_{q_i} (data primes) or [Q^{-1} (B/b_k)^{-1}]_{b_k} (auxiliary primes)
    const uint64_t conv = id < L ? h->C.qhatinv[id] : (id < L + K ? h->C.QBinv[id - L] : 1);
    const uint64_t vals[NSCALE] = {ninv, tnr, h_mulmod(ninv, r64, p),
                                   id < L ? h_mulmod(ninv, h->C.Pinv[id], p) : ninv, h_mulmod(tnr, conv, p)};
    const uint64_t w1 = ipw[brv(1, h->logn)];  // the last inverse stage's twiddle
    for (int m = 0; m < NSCALE; ++m) {
      const uint64_t cw = h_mulmod(vals[m], w1, p);
      uint64_t* e = &sc[((size_t)m * NPRIME + id) * 4];
      e[0] = vals[m];
      e[1] = h_shoup(vals[m], p);
      e[2] = cw;
      e[3] = h_shoup(cw, p);
    }
  }
  size_t tb = tw.size() * sizeof(ulonglong2);
  CU(h, cudaMalloc(&h->tw, tb));
  CU(h, cudaMalloc(&h->itw, tb));
  CU(h, cudaMalloc(&h->scale, sc.size() * sizeof(uint64_t)));
  CU(h, cudaMemcpy(h->tw, tw.data(), tb, cudaMemcpyHostToDevice));
  CU(h, cudaMemcpy(h->itw, itw.data(), tb, cudaMemcpyHostToDevice));
  CU(h, cudaMemcpy(h->scale, sc.data(), sc.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
  return HP_OK;
}

// Process-wide tables shared by all handles (per-device constants, the
// autotune cache, the allocation-free scratch addresses) are read and written
// under this mutex, so handles may be created and tuned from several threads.
static std::mutex g_tables_mu;

// The constant block lives in __constant__ memory, one per device; handles on
// the same device must agree on (q, P, t).
static bool g_loaded[64];
static Consts g_consts[64];

static int load_consts(hp_handle* h) {
  std::lock_guard<std::mutex> lock(g_tables_mu);
  if (h->device < 0 || h->device >= 64) HP_FAIL(h, HP_ERR_UNSUPPORTED, "device index out of range");
  if (g_loaded[h->device]) {
    if (memcmp(&g_consts[h->device], &h->C, sizeof(Consts)) != 0)
      HP_FAIL(h, HP_ERR_UNSUPPORTED, "a handle with different primes already uses this device");
    return HP_OK;
  }
  CU(h, cudaMemcpyToSymbol(cK, &h->C, sizeof(Consts)));
  g_consts[h->device] = h->C;
  g_loaded[h->device] = true;
  return HP_OK;
}

static void free_all(hp_handle* h) {
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  for (auto& g : h->graphs) {
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
  }
  h->graphs.clear();
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->h2d) cudaStreamDestroy(h->h2d);
  if (h->d2h) cudaStreamDestroy(h->d2h);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_in[i]) cudaEventDestroy(h->ev_in[i]);
    if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
    if (h->ev_out[i]) cudaEventDestroy(h->ev_out[i]);
  }
  void* ptrs[] = {h->tw, h->itw, h->scale, h->rkm, h->rkm1, h->rkm2, h->ext, h->ext2, h->dprod, h->w3, h->d2res,
                  h->ksin, h->ksout, h->ctbuf, h->maskbuf, h->stx, h->sty, h->sto, h->stm,
                  h->stx2, h->sty2, h->sto2, h->ltws, h->lt_coef, h->gkm, h->tct, h->tctab};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->status) cudaFree(h->status);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int hp_default_params(uint32_t Lreq, uint64_t* q_out, uint64_t* P_out, uint64_t* t_out) {
  if (!q_out || !P_out || !t_out || Lreq == 0 || Lreq > (uint32_t)L) return HP_ERR_ARG;
  uint64_t q[L];
  if (find_primes(55, (int)Lreq, nullptr, 0, q) != (int)Lreq) return HP_ERR_UNSUPPORTED;
  uint64_t P;
  if (find_primes(56, 1, nullptr, 0, &P) != 1) return HP_ERR_UNSUPPORTED;
  for (uint32_t i = 0; i < Lreq; ++i) q_out[i] = q[i];
  *P_out = P;
  *t_out = 65537;
  return HP_OK;
}

int hp_create(const hp_params* prm, const uint64_t* relin_key, size_t max_tile_ct, hp_handle** out) {
  hp_handle* h0 = nullptr;
  if (!prm || !out || !prm->q) HP_FAIL(h0, HP_ERR_ARG, "null argument");
  *out = nullptr;
  if (prm->log_n < LOGN_MIN || prm->log_n > LOGN_MAX)
    HP_FAIL(h0, HP_ERR_UNSUPPORTED, "log_n must be in [%d, %d]", LOGN_MIN, LOGN_MAX);
  if (prm->L != (uint32_t)L) HP_FAIL(h0, HP_ERR_UNSUPPORTED, "L must be %d", L);
  hp_handle* h = new hp_handle();
  h->logn = (int)prm->log_n;
  h->N = 1 << h->logn;
  h->logR = h->logn / 2;
  memcpy(h->q, prm->q, sizeof(h->q));
  h->P = prm->P;
  h->t = prm->t;
  h->max_depth = prm->max_depth;
  h->fine_depth = prm->ks_fine_depth;
  if (prm->ks_digit_primes != 0 && prm->ks_digit_primes != DIGIT_PRIMES && prm->ks_digit_primes != DIGIT_PRIMES5) {
    g_create_err = "ks_digit_primes must be 0 (default 3), 3 or 5";
    delete h;
    return HP_ERR_UNSUPPORTED;
  }
  h->dp = prm->ks_digit_primes ? (int)prm->ks_digit_primes : DIGIT_PRIMES;
  h->nd = L / h->dp;
  if (prm->ks_coarse_from != 0 && prm->ks_coarse_from <= prm->ks_fine_depth) {
    g_create_err = "ks_coarse_from must be 0 or above ks_fine_depth";
    delete h;
    return HP_ERR_ARG;
  }
  h->coarse_from = prm->ks_coarse_from;
  char eb[256] = {0};
  int rc = build_consts(h->q, h->P, h->t, &h->C, eb, sizeof(eb));
  if (rc != 0) {
    g_create_err = eb;
    delete h;
    return rc == -6 ? HP_ERR_UNSUPPORTED : HP_ERR_ARG;
  }
  int depth = supported_depth(h->logn, h->q, L, h->P, h->t);
  if ((int)prm->max_depth > depth) {
    char b[128];
    snprintf(b, sizeof(b), "max_depth %u exceeds the estimated supported depth %d", prm->max_depth, depth);
    g_create_err = b;
    delete h;
    return HP_ERR_DEPTH;
  }
  auto fail = [&](int code) {
    g_create_err = h->err;
    free_all(h);
    delete h;
    return code;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    h->err = "no CUDA device";
    return fail(HP_ERR_CUDA);
  }
  if ((rc = load_consts(h)) != HP_OK) return fail(rc);

  if ((rc = build_tables(h)) != HP_OK) return fail(rc);
  if ((rc = build_tc(h)) != HP_OK) return fail(rc);
  const int nd_ws = h->fine_depth > 0 ? NDIG_FINE : h->nd;
  size_t per = ws_words_per_ct(h->N, nd_ws) * sizeof(uint64_t);
  // default: about 22 GB of workspace, i.e. the largest tile (128 ciphertexts at N = 32768)
  h->tile = max_tile_ct ? max_tile_ct : (size_t)(((size_t)22 << 30) / per);
  if (h->tile < 1) h->tile = 1;
  if (h->tile > 128) h->tile = 128;
  const size_t T = h->tile, N = h->N;
  struct {
    uint64_t** p;
    size_t words;
  } allocs[] = {{&h->ext, T * 2 * NQB * N},  {&h->ext2, T * 2 * NQB * N}, {&h->dprod, T * 3 * NQB * N},
                {&h->w3, T * 3 * L * N},     {&h->ksin, T * nd_ws * NKS * N}, {&h->ksout, T * 2 * NKS * N},
                {&h->d2res, T * L * N},
                {&h->ctbuf, T * 2 * L * N},  {&h->maskbuf, T * 2 * L * N}, {&h->stx, T * 2 * L * N},
                {&h->sty, T * 2 * L * N},    {&h->sto, T * 2 * L * N},    {&h->stm, T * N},
                {&h->stx2, T * 2 * L * N},   {&h->sty2, T * 2 * L * N},   {&h->sto2, T * 2 * L * N},
                {&h->rkm, (size_t)h->nd * 2 * NKS * N},
                {&h->rkm1, h->fine_depth > 0 ? (size_t)NDIG_FINE * 2 * NKS * N : 0},
                {&h->rkm2, h->coarse_from > 0 ? (size_t)NDIG2 * 2 * NKS * N : 0}};
  for (auto& a : allocs) {
    if (a.words == 0) continue;
    if (cudaMalloc(a.p, a.words * sizeof(uint64_t)) != cudaSuccess) {
      h->err = "device allocation failed for the workspace";
      return fail(HP_ERR_OOM);
    }
  }
  // staging starts zeroed (the autotuner times tiles on it)
  if (cudaMemset(h->stx, 0, T * 2 * L * N * 8) != cudaSuccess || cudaMemset(h->sty, 0, T * 2 * L * N * 8) != cudaSuccess) {
    h->err = "workspace initialisation failed";
    return fail(HP_ERR_CUDA);
  }
  if (cudaMalloc(&h->status, sizeof(int)) != cudaSuccess || cudaMemset(h->status, 0, sizeof(int)) != cudaSuccess) {
    h->err = "status word allocation failed";
    return fail(HP_ERR_OOM);
  }
  if (relin_key) {
    if ((rc = hp_set_relin_key(h, relin_key)) != HP_OK) return fail(rc);
  }
  *out = h;
  return HP_OK;
}

// A key of nd digits in coefficient form (device) into dst in the form the
// key-switching multiply-accumulate reads: NTT domain, Montgomery form.
static int install_ks_key(hp_handle* h, uint64_t* dst, const uint64_t* key, int nd, cudaStream_t s) {
  const size_t words = (size_t)nd * 2 * NKS * h->N;
  CU(h, cudaMemcpyAsync(dst, key, words * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  ntt_fwd(h, dst, (size_t)nd * 2 * NKS, MAP_KS, s);
  k_to_mont<<<ew_blocks(words), EW_THREADS, 0, s>>>(dst, NKS, 0, ID_P, (size_t)nd * 2 * NKS, h->logn);
  CU(h, cudaGetLastError());
  return HP_OK;
}

int hp_set_relin_key(hp_handle* h, const uint64_t* rk) {
  if (!h) return HP_ERR_ARG;
  if (!rk) HP_FAIL(h, HP_ERR_ARG, "null relinearisation key");
  if (int rc = install_ks_key(h, h->rkm, rk, h->nd, 0)) return rc;
  CU(h, cudaDeviceSynchronize());
  h->have_rk = true;
  return HP_OK;
}

int hp_set_relin_key_fine(hp_handle* h, const uint64_t* rk) {
  if (!h) return HP_ERR_ARG;
  if (!rk) HP_FAIL(h, HP_ERR_ARG, "null per-prime relinearisation key");
  if (!h->rkm1) HP_FAIL(h, HP_ERR_STATE, "the handle was created with ks_fine_depth = 0");
  if (int rc = install_ks_key(h, h->rkm1, rk, NDIG_FINE, 0)) return rc;
  CU(h, cudaDeviceSynchronize());
  h->have_rk1 = true;
  return HP_OK;
}

int hp_set_relin_key_coarse(hp_handle* h, const uint64_t* rk) {
  if (!h) return HP_ERR_ARG;
  if (!rk) HP_FAIL(h, HP_ERR_ARG, "null two-digit relinearisation key");
  if (!h->rkm2) HP_FAIL(h, HP_ERR_STATE, "the handle was created with ks_coarse_from = 0");
  if (int rc = install_ks_key(h, h->rkm2, rk, NDIG2, 0)) return rc;
  CU(h, cudaDeviceSynchronize());
  h->have_rk2 = true;
  return HP_OK;
}

// Every relinearisation key the handle's products may use is installed.
static bool keys_ready(const hp_handle* h) {
  return h->have_rk && (h->fine_depth == 0 || h->have_rk1) && (h->coarse_from == 0 || h->have_rk2);
}

// The static budget estimate of `op` on this handle's parameters.
static double budget_of(const hp_handle* h, int op, int in_depth = 0, double in_bits = 0) {
  return budget_estimate(h->logn, h->q, L, h->P, h->t, h->dp, (int)h->fine_depth, (int)h->coarse_from, op, in_depth,
                         in_bits);
}
#define HP_NEED_BUDGET(h, op, what)                                                                        \
  do {                                                                                                     \
    const double bud_ = budget_of(h, op);                                                                  \
    if (bud_ < BUDGET_MARGIN)                                                                              \
      HP_FAIL(h, HP_ERR_DEPTH, "%s: estimated noise budget %.1f bits is below the %.0f-bit margin", what,  \
              bud_, BUDGET_MARGIN);                                                                        \
  } while (0)

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int hp_run(hp_handle* h, int op, const uint64_t* x, const uint64_t* y, uint64_t cval, uint64_t* out, size_t n_ct,
           void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (op < HP_EQ_CT_CT || op > HP_LT) HP_FAIL(h, HP_ERR_ARG, "unknown op %d", op);
  if (n_ct == 0) return HP_OK;
  if (!x || !out) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if ((op == HP_EQ_CT_CT || op == HP_SELECT || op == HP_LT) && !y) HP_FAIL(h, HP_ERR_ARG, "op needs ct_y");
  if ((op == HP_EQ_CT_CONST || op == HP_SELECT) && cval >= h->t) HP_FAIL(h, HP_ERR_ARG, "const_val must be < t");
  if (!keys_ready(h)) HP_FAIL(h, HP_ERR_STATE, "relinearisation key not set");
  HP_NEED_BUDGET(h, op == HP_SQUARE ? BUDGET_SQUARE : (op == HP_SELECT ? BUDGET_SELECT : (op == HP_LT ? BUDGET_LT : BUDGET_EQ)),
                 "hp_run");
  if (((uintptr_t)x | (uintptr_t)out | (uintptr_t)y) & 15) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t W = words_ct(h);
  const bool dev = is_device_ptr(x);
  if (dev != is_device_ptr(out) || ((op == HP_EQ_CT_CT || op == HP_SELECT || op == HP_LT) && dev != is_device_ptr(y)))
    HP_FAIL(h, HP_ERR_ARG, "ciphertext arguments must all be device memory or all host memory");
  if (op == HP_LT) {
    if (!dev) HP_FAIL(h, HP_ERR_UNSUPPORTED, "HP_LT takes device memory");
    int rc = lt_prepare(h);
    if (rc != HP_OK) return rc;
    for (size_t c0 = 0; c0 < n_ct; c0 += h->lt_tile) {
      const int b = (int)((n_ct - c0 < h->lt_tile) ? n_ct - c0 : h->lt_tile);
      const size_t off = c0 * W;
      run_lt_tile(h, x + off, y + off, out + off, b, s);
      CU(h, cudaGetLastError());
    }
    return HP_OK;
  }
  const size_t TT = h->run_tile ? h->run_tile : h->tile;
  if (dev) {
    for (size_t c0 = 0; c0 < n_ct; c0 += TT) {
      const int b = (int)((n_ct - c0 < TT) ? n_ct - c0 : TT);
      const size_t off = c0 * W;
      run_tile(h, op, x + off, y ? y + off : nullptr, cval, out + off, b, s);
      CU(h, cudaGetLastError());
    }
    return HP_OK;
  }
  // Host memory: two staging sets; tile k copies in on the h2d stream, computes
  // on the caller's stream, copies out on the d2h stream, so that with pinned
  // buffers the copies of tiles k-1 / k+1 overlap the compute of tile k.
  if (!h->h2d) {
    CU(h, cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking));
    CU(h, cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      CU(h, cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming));
      CU(h, cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming));
      CU(h, cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming));
    }
  }
  uint64_t* SX[2] = {h->stx, h->stx2};
  uint64_t* SY[2] = {h->sty, h->sty2};
  uint64_t* SO[2] = {h->sto, h->sto2};
  const bool two = op == HP_EQ_CT_CT || op == HP_SELECT;
  CU(h, cudaEventRecord(h->ev_done[0], s));  // staging free (orders after earlier work on s)
  CU(h, cudaEventRecord(h->ev_done[1], s));
  CU(h, cudaEventRecord(h->ev_out[0], s));
  CU(h, cudaEventRecord(h->ev_out[1], s));
  size_t k = 0;
  for (size_t c0 = 0; c0 < n_ct; c0 += TT, ++k) {
    const int i = (int)(k & 1);
    const int b = (int)((n_ct - c0 < TT) ? n_ct - c0 : TT);
    const size_t off = c0 * W, bytes = (size_t)b * W * sizeof(uint64_t);
    CU(h, cudaStreamWaitEvent(h->h2d, h->ev_done[i], 0));  // inputs of tile k-2 consumed
    CU(h, cudaMemcpyAsync(SX[i], x + off, bytes, cudaMemcpyHostToDevice, h->h2d));
    if (two) CU(h, cudaMemcpyAsync(SY[i], y + off, bytes, cudaMemcpyHostToDevice, h->h2d));
    CU(h, cudaEventRecord(h->ev_in[i], h->h2d));
    CU(h, cudaStreamWaitEvent(s, h->ev_in[i], 0));
    CU(h, cudaStreamWaitEvent(s, h->ev_out[i], 0));  // outputs of tile k-2 copied out
    run_tile(h, op, SX[i], SY[i], cval, SO[i], b, s);
    CU(h, cudaEventRecord(h->ev_done[i], s));
    CU(h, cudaStreamWaitEvent(h->d2h, h->ev_done[i], 0));
    CU(h, cudaMemcpyAsync(out + off, SO[i], bytes, cudaMemcpyDeviceToHost, h->d2h));
    CU(h, cudaEventRecord(h->ev_out[i], h->d2h));
    CU(h, cudaGetLastError());
  }
  CU(h, cudaStreamSynchronize(h->d2h));
  CU(h, cudaStreamSynchronize(s));
  return HP_OK;
}

// Graph of one tile's launch sequence (captured once per (mode, tile size) on
// an internal stream on the staging buffers, replayed on the caller's stream
// with its first and last kernels pointed at the tile's own ciphertexts).
enum { GM_CTCT = 0, GM_PT = 1 };
static const void* moddown_kernel(int logn) {
  switch (logn) {
    case 12: return (const void*)k_ntt_inv_cols<6, 6, true>;
    case 13: return (const void*)k_ntt_inv_cols<6, 7, true>;
    case 14: return (const void*)k_ntt_inv_cols<7, 7, true>;
    default: return (const void*)k_ntt_inv_cols<7, 8, true>;
  }
}
static int tile_graph(hp_handle* h, int mode, int b, hp_handle::GraphEntry** entry) {
  for (auto& g : h->graphs)
    if (g.mode == mode && g.b == b) {
      *entry = &g;
      return HP_OK;
    }
  if (!h->cap) CU(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  const uint32_t saved_mask = h->prof_mask;
  const uint64_t saved_launches = h->launches;
  h->prof_mask = 0;  // no timing events inside graphs
  h->launches = 0;
  CU(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  if (mode == GM_CTCT)
    run_tile_mode(h, HP_EQ_CT_CT, LIFT_SUB_CT, h->stx, h->sty, nullptr, 0, h->sto, b, h->cap);
  else
    run_tile_mode(h, HP_EQ_CT_CONST, LIFT_SUB_PT, h->stx, h->stm, nullptr, 0, h->sto, b, h->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap, &g);
  h->prof_mask = saved_mask;
  const uint64_t nk = h->launches;
  h->launches = saved_launches;
  if (e != cudaSuccess) HP_FAIL(h, HP_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  // the sequence is a chain of kernel nodes: its root is the first lift, its
  // only node without dependents the final inverse column pass
  size_t n = 0;
  CU(h, cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CU(h, cudaGraphGetNodes(g, nodes.data(), &n));
  cudaGraphNode_t first = nullptr, last = nullptr;
  for (cudaGraphNode_t nd : nodes) {
    size_t deps = 0, outs = 0;
    CU(h, cudaGraphNodeGetDependencies(nd, nullptr, nullptr, &deps));
    CU(h, cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &outs));
    if (deps == 0) first = nd;
    if (outs == 0) last = nd;
  }
  cudaKernelNodeParams pf, pl;
  if (!first || !last || cudaGraphKernelNodeGetParams(first, &pf) != cudaSuccess ||
      cudaGraphKernelNodeGetParams(last, &pl) != cudaSuccess ||
      pf.func != (mode == GM_CTCT ? (void*)k_lift_tc<true> : (void*)k_lift_tc<false>) ||
      pl.func != moddown_kernel(h->logn)) {
    cudaGraphDestroy(g);
    HP_FAIL(h, HP_ERR_CUDA, "captured tile sequence does not start with the lift and end with the mod-down");
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    HP_FAIL(h, HP_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  h->graphs.push_back({mode, b, g, ex, first, last, nk});
  *entry = &h->graphs.back();
  return HP_OK;
}

// Number of parameters of a kernel, from its signature.
extern "C++" {
template <typename... A>
constexpr int kernel_arity(void (*)(A...)) {
  return (int)sizeof...(A);
}
}
constexpr int LIFT_ARGS = kernel_arity(k_lift_tc<true>);          // (src, sub, ...): src first, sub second
constexpr int MODDOWN_ARGS = kernel_arity(k_ntt_inv_cols<7, 8, true>);  // (..., ModDown md): md last
static_assert(LIFT_ARGS == kernel_arity(k_lift_tc<false>), "both lift forms take the same arguments");
static_assert(MODDOWN_ARGS == 5, "the mod-down pass takes (data, map, tables, scale mode, mod-down)");

// Point the tile graph's first lift at x (and y for EQ ct-ct) and its final
// pass at out: the other arguments keep their captured values.
static int tile_graph_bind(hp_handle* h, hp_handle::GraphEntry* g, const uint64_t* x, const uint64_t* y, uint64_t* out) {
  cudaKernelNodeParams p;
  CU(h, cudaGraphKernelNodeGetParams(g->first, &p));
  void* args[LIFT_ARGS];
  for (int i = 0; i < LIFT_ARGS; ++i) args[i] = p.kernelParams[i];
  const uint64_t* src = x;
  const uint64_t* sub = y;
  args[0] = &src;
  if (g->mode == GM_CTCT) args[1] = &sub;
  p.kernelParams = args;
  CU(h, cudaGraphExecKernelNodeSetParams(g->exec, g->first, &p));
  CU(h, cudaGraphKernelNodeGetParams(g->last, &p));
  void* largs[MODDOWN_ARGS];
  for (int i = 0; i < MODDOWN_ARGS; ++i) largs[i] = p.kernelParams[i];
  ModDown md = *(const ModDown*)p.kernelParams[MODDOWN_ARGS - 1];
  md.out = out;
  largs[MODDOWN_ARGS - 1] = &md;
  p.kernelParams = largs;
  CU(h, cudaGraphExecKernelNodeSetParams(g->exec, g->last, &p));
  return HP_OK;
}

int hp_run_batched(hp_handle* h, int op, const hp_instance* inst, size_t n_inst, const uint64_t* x, const uint64_t* y,
                   uint64_t* out, size_t n_ct_total, void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (op != HP_EQ_CT_CT && op != HP_EQ_CT_CONST) HP_FAIL(h, HP_ERR_ARG, "batched op must be EQ_CT_CT or EQ_CT_CONST");
  if (n_ct_total == 0) return HP_OK;
  if (!inst || n_inst == 0) HP_FAIL(h, HP_ERR_ARG, "no instances");
  if (!x || !out || (op == HP_EQ_CT_CT && !y)) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if (!keys_ready(h)) HP_FAIL(h, HP_ERR_STATE, "relinearisation key not set");
  if (!is_device_ptr(x) || !is_device_ptr(out) || (op == HP_EQ_CT_CT && !is_device_ptr(y)))
    HP_FAIL(h, HP_ERR_ARG, "batched ciphertext arrays must be device memory");
  if (((uintptr_t)x | (uintptr_t)out | (uintptr_t)y) & 15) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  // validate the descriptors: ranges inside the batch, every ciphertext covered,
  // slot ranges inside their ciphertexts and pairwise disjoint
  const uint64_t N = (uint64_t)h->N;
  std::vector<size_t> order(n_inst);
  std::vector<uint64_t> start(n_inst);
  std::vector<uint8_t> covered(n_ct_total, 0);
  for (size_t i = 0; i < n_inst; ++i) {
    const hp_instance& d = inst[i];
    if (d.n_ct == 0 || d.ct_offset + d.n_ct > n_ct_total) HP_FAIL(h, HP_ERR_ARG, "instance %zu: ciphertext range outside the batch", i);
    if (d.slot_offset >= N || d.slot_offset + (uint64_t)d.n_slots > (uint64_t)d.n_ct * N)
      HP_FAIL(h, HP_ERR_ARG, "instance %zu: slot range outside its ciphertexts", i);
    if (op == HP_EQ_CT_CONST && d.const_val >= h->t) HP_FAIL(h, HP_ERR_ARG, "instance %zu: const_val must be < t", i);
    for (uint64_t c = d.ct_offset; c < d.ct_offset + d.n_ct; ++c) covered[c] = 1;
    start[i] = d.ct_offset * N + d.slot_offset;
    order[i] = i;
  }
  for (size_t c = 0; c < n_ct_total; ++c)
    if (!covered[c]) HP_FAIL(h, HP_ERR_ARG, "ciphertext %zu is not covered by any instance", c);
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return start[a] < start[b]; });
  std::vector<uint64_t> st(n_inst), cv(n_inst);
  std::vector<uint32_t> ln(n_inst);
  for (size_t k = 0; k < n_inst; ++k) {
    st[k] = start[order[k]];
    ln[k] = inst[order[k]].n_slots;
    cv[k] = inst[order[k]].const_val;
    if (k > 0 && st[k] < st[k - 1] + ln[k - 1]) HP_FAIL(h, HP_ERR_ARG, "instances overlap in slot space");
  }
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t *d_st = nullptr, *d_cv = nullptr;
  uint32_t* d_ln = nullptr;
  if (op == HP_EQ_CT_CONST) {
    CU(h, cudaMallocAsync((void**)&d_st, n_inst * 8, s));
    CU(h, cudaMallocAsync((void**)&d_cv, n_inst * 8, s));
    CU(h, cudaMallocAsync((void**)&d_ln, n_inst * 4, s));
    CU(h, cudaMemcpyAsync(d_st, st.data(), n_inst * 8, cudaMemcpyHostToDevice, s));
    CU(h, cudaMemcpyAsync(d_cv, cv.data(), n_inst * 8, cudaMemcpyHostToDevice, s));
    CU(h, cudaMemcpyAsync(d_ln, ln.data(), n_inst * 4, cudaMemcpyHostToDevice, s));
  }
  const size_t W = words_ct(h), TT = h->run_tile ? h->run_tile : h->tile;
  uint64_t total = 0;
  int rc = HP_OK;
  for (size_t c0 = 0; c0 < n_ct_total && rc == HP_OK; c0 += TT) {
    const int b = (int)((n_ct_total - c0 < TT) ? n_ct_total - c0 : TT);
    const size_t off = c0 * W;
    hp_handle::GraphEntry* g = nullptr;
    rc = tile_graph(h, op == HP_EQ_CT_CT ? GM_CTCT : GM_PT, b, &g);
    if (rc != HP_OK) break;
    if (op == HP_EQ_CT_CONST) {  // per-slot constants of this tile, encoded (slots -> plaintext polynomial)
      k_pack_slots<<<ew_blocks((size_t)b * N), EW_THREADS, 0, s>>>(d_st, d_ln, d_cv, (int)n_inst, c0, h->stm, h->logn,
                                                                    b);
      ntt_inv(h, h->stm, b, MAP_T, SCALE_NINV, s);
      total += 3;
    }
    rc = tile_graph_bind(h, g, x + off, op == HP_EQ_CT_CT ? y + off : nullptr, out + off);
    if (rc != HP_OK) break;
    CU(h, cudaGraphLaunch(g->exec, s));
    total += g->kernels;
  }
  if (d_st) {
    cudaFreeAsync(d_st, s);
    cudaFreeAsync(d_cv, s);
    cudaFreeAsync(d_ln, s);
  }
  h->launches = total;
  if (rc != HP_OK) return rc;
  CU(h, cudaGetLastError());
  return HP_OK;
}

// Tile-size autotuner: times the EQ launch sequence for candidate tile sizes on
// the handle's own staging buffers (the path is data-oblivious, so timings do
// not depend on the data) and keeps the largest tile within 1 % of the fastest
// per ciphertext.  Results are cached per (ring degree, device, workspace
// tile) for the process.
struct TuneKey {
  int logn, device;
  size_t maxtile, best;
};
static std::vector<TuneKey> g_tune;

int hp_autotune(hp_handle* h, size_t* best_tile) {
  if (!h) return HP_ERR_ARG;
  if (!keys_ready(h)) HP_FAIL(h, HP_ERR_STATE, "relinearisation key not set");
  {
    std::lock_guard<std::mutex> lock(g_tables_mu);
    for (auto& k : g_tune)
      if (k.logn == h->logn && k.device == h->device && k.maxtile == h->tile) {
        h->run_tile = k.best;
        if (best_tile) *best_tile = k.best;
        return HP_OK;
      }
  }
  const size_t cand[] = {1, 2, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128};
  cudaEvent_t e0, e1;
  CU(h, cudaEventCreate(&e0));
  CU(h, cudaEventCreate(&e1));
  const uint32_t saved_mask = h->prof_mask;
  h->prof_mask = 0;
  std::vector<size_t> cs;
  for (size_t c : cand)
    if (c < h->tile) cs.push_back(c);
  cs.push_back(h->tile);
  // per candidate: one warm-up pass, then the fastest of three timed passes
  // (per ciphertext); the choice is the largest tile within 1 % of the fastest,
  // so that run-to-run jitter between nearly equal tiles does not flip it
  std::vector<double> per(cs.size(), 1e30);
  for (size_t k = 0; k < cs.size(); ++k) {
    const size_t T = cs[k];
    run_tile(h, HP_EQ_CT_CT, h->stx, h->sty, 0, h->sto, (int)T, 0);
    for (int r = 0; r < 3; ++r) {
      CU(h, cudaEventRecord(e0, 0));
      run_tile(h, HP_EQ_CT_CT, h->stx, h->sty, 0, h->sto, (int)T, 0);
      CU(h, cudaEventRecord(e1, 0));
      CU(h, cudaEventSynchronize(e1));
      float ms = 0;
      CU(h, cudaEventElapsedTime(&ms, e0, e1));
      per[k] = std::min(per[k], (double)ms / T);
    }
  }
  const double best = *std::min_element(per.begin(), per.end());
  size_t bt = cs[0];
  for (size_t k = 0; k < cs.size(); ++k)
    if (per[k] <= best * 1.01) bt = cs[k];
  h->prof_mask = saved_mask;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CU(h, hp_check_status(h) == HP_OK ? cudaSuccess : cudaErrorUnknown);
  h->run_tile = bt;
  {
    std::lock_guard<std::mutex> lock(g_tables_mu);
    g_tune.push_back({h->logn, h->device, h->tile, bt});
  }
  if (best_tile) *best_tile = bt;
  return HP_OK;
}

// ---------------------------------------------------------------------------
// Fan-out of one column against many constants: GROUP BY masks EQ(x, c_k)
// (Sec. 4.2.2) and IN(x, S) = sum_k EQ(x, c_k) (Eq. 6).  The n_const * n_ct
// chains (item = k * n_ct + c) are independent and run in tiles; each tile
// gathers its x ciphertexts into staging and its first lift subtracts one
// constant per ciphertext.  Ciphertext addition is exact mod Q, so the sum
// equals the paper's divide-and-conquer addition for any order: with masks
// kept it is one pass over all masks, otherwise each tile's masks are added
// into the running sum and only one tile of masks is ever stored.
// ---------------------------------------------------------------------------
int hp_eq_fanout(hp_handle* h, const uint64_t* x, size_t n_ct, const uint64_t* consts, size_t n_const,
                 uint64_t* masks, uint64_t* in_out, void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (n_ct == 0 || n_const == 0) return HP_OK;
  if (!x || !consts || (!masks && !in_out)) HP_FAIL(h, HP_ERR_ARG, "null argument");
  if (n_const > (1u << 20)) HP_FAIL(h, HP_ERR_ARG, "at most 2^20 constants");
  if (!keys_ready(h)) HP_FAIL(h, HP_ERR_STATE, "relinearisation key not set");
  HP_NEED_BUDGET(h, BUDGET_EQ, "hp_eq_fanout");
  for (size_t k = 0; k < n_const; ++k)
    if (consts[k] >= h->t) HP_FAIL(h, HP_ERR_ARG, "constant %zu must be < t", k);
  if (!is_device_ptr(x) || (masks && !is_device_ptr(masks)) || (in_out && !is_device_ptr(in_out)))
    HP_FAIL(h, HP_ERR_ARG, "fan-out arrays must be device memory");
  if (((uintptr_t)x | (uintptr_t)masks | (uintptr_t)in_out) & 15) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t W = words_ct(h), TT = h->run_tile ? h->run_tile : h->tile, items = n_const * n_ct;
  std::vector<uint64_t> hc(items);
  for (size_t it = 0; it < items; ++it) hc[it] = consts[it / n_ct];
  uint64_t* dconst = nullptr;
  CU(h, cudaMallocAsync((void**)&dconst, items * sizeof(uint64_t), s));
  CU(h, cudaMemcpyAsync(dconst, hc.data(), items * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  if (in_out && !masks) CU(h, cudaMemsetAsync(in_out, 0, n_ct * W * sizeof(uint64_t), s));
  for (size_t i0 = 0; i0 < items; i0 += TT) {
    const int b = (int)((items - i0 < TT) ? items - i0 : TT);
    for (int u = 0; u < b; ++u)
      CU(h, cudaMemcpyAsync(h->stx + (size_t)u * W, x + ((i0 + u) % n_ct) * W, W * sizeof(uint64_t),
                            cudaMemcpyDeviceToDevice, s));
    uint64_t* dst = masks ? masks + i0 * W : h->sto;
    run_tile_mode(h, HP_EQ_CT_CONST, LIFT_SUB_CONSTS, h->stx, dconst + i0, nullptr, 0, dst, b, s);
    if (!masks) {  // add each run of consecutive c into the running sum
      for (int u = 0; u < b;) {
        const size_t c = (i0 + u) % n_ct;
        const int run = (int)std::min<size_t>(b - u, n_ct - c);
        const size_t nw = (size_t)run * W;
        k_ct_acc<<<ew_blocks(nw), EW_THREADS, 0, s>>>(in_out + c * W, h->sto + (size_t)u * W, h->logn, nw);
        h->launches += 1;
        u += run;
      }
    }
    CU(h, cudaGetLastError());
  }
  if (masks && in_out) {
    const size_t nw = n_ct * W;
    k_ct_sum<<<ew_blocks(nw), EW_THREADS, 0, s>>>(masks, (int)n_const, in_out, h->logn, nw);
    h->launches += 1;
  }
  cudaFreeAsync(dconst, s);
  CU(h, cudaGetLastError());
  return HP_OK;
}

// ---------------------------------------------------------------------------
// Rotations and the rotate-and-add reduction of COUNT and SUM (Sec. 4.2.2).
// The Galois group {+-3^k} mod 2N splits the slots into two rows of N/2:
// g = 3^(2^i) rotates each row by 2^i, g = 2N - 1 exchanges the rows.  The
// reduction rotates by N/4, N/8, ..., 1 (largest first, as in the paper's
// doubling pattern) and then exchanges the rows: log2 N steps, one Galois key
// each.
// ---------------------------------------------------------------------------
static void galois_elements(int logn, uint64_t* g) {
  const uint64_t twoN = 2ull << logn;
  int k = 0;
  for (int i = logn - 2; i >= 0; --i) {
    uint64_t v = 1, b = 3;
    for (uint64_t e = 1ull << i; e; e >>= 1, b = b * b % twoN)
      if (e & 1) v = v * b % twoN;
    g[k++] = v;
  }
  g[k] = twoN - 1;
}

// g^{-1} mod 2N for odd g by Newton's iteration x <- x (2 - g x), which doubles
// the number of correct low bits (g g = 1 mod 8 gives 3 to start).
static uint32_t inverse_mod_2n(uint64_t g, int logn) {
  uint64_t x = g;
  for (int it = 0; it < 5; ++it) x = x * (2 - g * x);
  return (uint32_t)(x & ((2ull << logn) - 1));
}

int hp_galois_elements(int logn, uint64_t* g_out) {
  if (logn < 3 || logn > 16 || !g_out) return HP_ERR_ARG;
  galois_elements(logn, g_out);
  return HP_OK;
}

static size_t key_words(const hp_handle* h) { return (size_t)h->nd * 2 * NKS * h->N; }

static int install_galois_key(hp_handle* h, int st, const uint64_t* gk, cudaStream_t s) {
  const size_t kw = key_words(h);
  uint64_t* dst = h->gkm + (size_t)st * kw;
  CU(h, cudaMemcpyAsync(dst, gk, kw * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  ntt_fwd(h, dst, (size_t)h->nd * 2 * NKS, MAP_KS, s);
  k_to_mont<<<ew_blocks(kw), EW_THREADS, 0, s>>>(dst, NKS, 0, ID_P, (size_t)h->nd * 2 * NKS, h->logn);
  CU(h, cudaGetLastError());
  return HP_OK;
}

static int alloc_gkm(hp_handle* h) {
  if (!h->gkm) CU(h, cudaMalloc((void**)&h->gkm, (size_t)h->logn * key_words(h) * sizeof(uint64_t)));
  return HP_OK;
}

int hp_set_galois_keys(hp_handle* h, const uint64_t* gk) {
  if (!h) return HP_ERR_ARG;
  if (!gk) HP_FAIL(h, HP_ERR_ARG, "null Galois keys");
  if (!is_device_ptr(gk)) HP_FAIL(h, HP_ERR_ARG, "Galois keys must be device memory");
  if (int rc = alloc_gkm(h)) return rc;
  for (int st = 0; st < h->logn; ++st)
    if (int rc = install_galois_key(h, st, gk + (size_t)st * key_words(h), 0)) return rc;
  CU(h, cudaDeviceSynchronize());
  h->have_gk = true;
  return HP_OK;
}

int hp_galois_keygen(hp_handle* h, uint64_t seed, const int8_t* sk, uint64_t* gk, void* stream) {
  if (!h) return HP_ERR_ARG;
  if (!sk) HP_FAIL(h, HP_ERR_ARG, "null secret key");
  if (!is_device_ptr(sk) || (gk && !is_device_ptr(gk))) HP_FAIL(h, HP_ERR_ARG, "keys must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = h->N, logN = h->logn;
  const size_t kw = key_words(h);
  if (int rc = alloc_gkm(h)) return rc;
  uint64_t g[16];
  galois_elements(logN, g);
  uint64_t *S = nullptr, *S2 = nullptr, *A = nullptr, *K = nullptr;
  int8_t* ts = nullptr;
  CU(h, cudaMalloc(&S, (size_t)NKS * N * 8));
  CU(h, cudaMalloc(&S2, (size_t)NKS * N * 8));
  CU(h, cudaMalloc(&A, (size_t)h->nd * NKS * N * 8));
  CU(h, cudaMalloc(&ts, N));
  if (!gk) CU(h, cudaMalloc(&K, kw * 8));
  k_secret_to_primes<<<ew_blocks((size_t)NKS * N), EW_THREADS, 0, s>>>(sk, S, NKS, 0, ID_P, N);
  ntt_fwd(h, S, NKS, MAP_KS, s);
  for (int st = 0; st < logN; ++st) {
    uint64_t* key = gk ? gk + (size_t)st * kw : K;
    const uint32_t obj = (uint32_t)(g[st] << 5);
    k_secret_automorph<<<ew_blocks(N), EW_THREADS, 0, s>>>(sk, ts, (uint32_t)g[st], logN);
    k_secret_to_primes<<<ew_blocks((size_t)NKS * N), EW_THREADS, 0, s>>>(ts, S2, NKS, 0, ID_P, N);
    const int nd = h->nd;
    k_rk_sample_a<<<ew_blocks((size_t)nd * NKS * N), EW_THREADS, 0, s>>>(key, A, seed, logN, DOM_A_GK, obj, nd);
    ntt_fwd(h, A, (size_t)nd * NKS, MAP_KS, s);
    k_pointwise_mont<<<ew_blocks((size_t)nd * NKS * N), EW_THREADS, 0, s>>>(A, S, A, NKS, NKS, 0, ID_P,
                                                                        (size_t)nd * NKS, logN);
    ntt_inv(h, A, (size_t)nd * NKS, MAP_KS, SCALE_NINV_R, s);
    k_rk_finish<<<ew_blocks((size_t)nd * NKS * N), EW_THREADS, 0, s>>>(key, A, S2, seed, logN, DOM_E_GK, obj, nd,
                                                                       h->dp);
    if (int rc = install_galois_key(h, st, key, s)) return rc;
  }
  CU(h, cudaGetLastError());
  CU(h, cudaStreamSynchronize(s));
  cudaFree(S);
  cudaFree(S2);
  cudaFree(A);
  cudaFree(ts);
  if (K) cudaFree(K);
  h->have_gk = true;
  return HP_OK;
}

// ct <- ct + rotate(ct, g_st) in place on a tile of b ciphertexts.
static void rotate_add_tile(hp_handle* h, uint64_t* ct, int b, int st, uint32_t ginv, cudaStream_t s) {
  const int N = h->N, logN = h->logn;
  {
    ProfScope ps(h, PK_AUTOMORPH, s, 3.0 * b * L * N);
    if (h->dp == DIGIT_PRIMES5)
      k_automorph<DIGIT_PRIMES5><<<ew_blocks((size_t)b * NDIG5 * N), EW_THREADS, 0, s>>>(ct, h->w3, h->d2res, ginv, 1,
                                                                                         logN, b);
    else
      k_automorph<DIGIT_PRIMES><<<ew_blocks((size_t)b * NDIG * N), EW_THREADS, 0, s>>>(ct, h->w3, h->d2res, ginv, 1,
                                                                                       logN, b);
  }
  h->launches += 1;
  ntt_fwd(h, h->ksin, (size_t)b * h->nd * NKS, MAP_KS, s, h->w3, h->dp, h->d2res);
  ks_mac(h, h->gkm + (size_t)st * key_words(h), h->nd, b, s);
  ntt_inv_moddown(h, h->ksout, b, ct, 0, s);
}

int hp_ct_sum(hp_handle* h, const uint64_t* x, size_t n_ct, size_t group, uint64_t* out, void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (group == 0) HP_FAIL(h, HP_ERR_ARG, "group must be >= 1");
  if (n_ct == 0) return HP_OK;
  if (!x || !out) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if (!is_device_ptr(x) || !is_device_ptr(out)) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be device memory");
  const size_t W = words_ct(h), n_out = (n_ct + group - 1) / group;
  if (group > 1 && out < x + n_ct * W && x < out + n_out * W)
    HP_FAIL(h, HP_ERR_ARG, "out overlaps x (allowed only in place with group = 1)");
  k_ct_group_sum<<<ew_blocks(n_out * W), EW_THREADS, 0, (cudaStream_t)stream>>>(x, n_ct, group, out, h->logn, W, n_out);
  h->launches = 1;
  CU(h, cudaGetLastError());
  return HP_OK;
}

// The reduction on n ciphertexts in place, in tiles.
static void rotate_sum_inplace(hp_handle* h, uint64_t* ct, size_t n, cudaStream_t s) {
  uint64_t g[16];
  galois_elements(h->logn, g);
  const size_t W = words_ct(h), TT = h->run_tile ? h->run_tile : h->tile;
  for (size_t o0 = 0; o0 < n; o0 += TT) {
    const int b = (int)((n - o0 < TT) ? n - o0 : TT);
    for (int st = 0; st < h->logn; ++st) rotate_add_tile(h, ct + o0 * W, b, st, inverse_mod_2n(g[st], h->logn), s);
  }
}

int hp_rotate_sum(hp_handle* h, const uint64_t* x, size_t n_ct, size_t group, uint64_t* out, void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (group == 0) HP_FAIL(h, HP_ERR_ARG, "group must be >= 1");
  if (n_ct == 0) return HP_OK;
  if (!x || !out) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if (!h->have_gk) HP_FAIL(h, HP_ERR_STATE, "Galois keys not set");
  if (!is_device_ptr(x) || !is_device_ptr(out)) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be device memory");
  if (((uintptr_t)x | (uintptr_t)out) & 15) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  const size_t W = words_ct(h), n_out = (n_ct + group - 1) / group;
  if (group > 1 && out < x + n_ct * W && x < out + n_out * W)
    HP_FAIL(h, HP_ERR_ARG, "out overlaps x (allowed only in place with group = 1)");
  cudaStream_t s = (cudaStream_t)stream;
  if (!(group == 1 && out == x)) {
    k_ct_group_sum<<<ew_blocks(n_out * W), EW_THREADS, 0, s>>>(x, n_ct, group, out, h->logn, W, n_out);
    h->launches += 1;
  }
  rotate_sum_inplace(h, out, n_out, s);
  CU(h, cudaGetLastError());
  return HP_OK;
}

// ---------------------------------------------------------------------------
// JOIN by Extract + Broadcast (Sec. 4.2.2).  Extract keeps one slot of a
// ciphertext (product with the plaintext unit vector of that slot), Broadcast
// spreads it to every slot (the rotate-and-add reduction).  The equi-join
// masks the A table with EQ(A.key, Broadcast(B.key[r])) per B row r and sums
// mask x Broadcast(B.attr[r]) over r.
// ---------------------------------------------------------------------------
// out[c] = Broadcast(Extract(column, r0 + c)) for c < b (b <= tile); Mt, Mq:
// temporaries of b N and b L N words.
static int extract_broadcast_tile(hp_handle* h, const uint64_t* column, size_t r0, int b, uint64_t* out, uint64_t* Mt,
                                  uint64_t* Mq, cudaStream_t s) {
  const size_t W = words_ct(h), N = h->N;
  const int logN = h->logn;
  for (int c = 0; c < b; ++c)
    CU(h, cudaMemcpyAsync(out + c * W, column + ((r0 + c) / N) * W, W * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  k_unit_slots<<<ew_blocks((size_t)b * N), EW_THREADS, 0, s>>>(Mt, r0, logN, b);
  ntt_inv(h, Mt, b, MAP_T, SCALE_NINV, s);  // encoding: slots are the transform of m
  k_plain_to_q<<<ew_blocks((size_t)b * L * N), EW_THREADS, 0, s>>>(Mt, Mq, logN, b);
  ntt_fwd(h, Mq, (size_t)b * L, MAP_Q, s);
  ntt_fwd(h, out, (size_t)b * 2 * L, MAP_Q, s);
  k_mul_plain_ntt<<<ew_blocks((size_t)b * 2 * L * N), EW_THREADS, 0, s>>>(out, Mq, logN, b);
  ntt_inv(h, out, (size_t)b * 2 * L, MAP_Q, SCALE_NINV_R, s);
  h->launches += 3;
  rotate_sum_inplace(h, out, b, s);
  return HP_OK;
}

static int extract_broadcast(hp_handle* h, const uint64_t* column, size_t row0, size_t n_rows, uint64_t* out,
                             cudaStream_t s) {
  const size_t W = words_ct(h), TT = h->run_tile ? h->run_tile : h->tile;
  uint64_t *Mt = nullptr, *Mq = nullptr;
  CU(h, cudaMallocAsync((void**)&Mt, TT * h->N * sizeof(uint64_t), s));
  CU(h, cudaMallocAsync((void**)&Mq, TT * L * h->N * sizeof(uint64_t), s));
  for (size_t r = 0; r < n_rows; r += TT) {
    const int b = (int)((n_rows - r < TT) ? n_rows - r : TT);
    if (int rc = extract_broadcast_tile(h, column, row0 + r, b, out + r * W, Mt, Mq, s)) return rc;
  }
  cudaFreeAsync(Mt, s);
  cudaFreeAsync(Mq, s);
  CU(h, cudaGetLastError());
  return HP_OK;
}

int hp_extract_broadcast(hp_handle* h, const uint64_t* column, size_t n_ct, size_t row0, size_t n_rows, uint64_t* out,
                         void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (n_rows == 0) return HP_OK;
  if (!column || !out) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if (!h->have_gk) HP_FAIL(h, HP_ERR_STATE, "Galois keys not set");
  if (row0 + n_rows > n_ct * (size_t)h->N) HP_FAIL(h, HP_ERR_ARG, "rows beyond the column");
  if (!is_device_ptr(column) || !is_device_ptr(out)) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be device memory");
  if (((uintptr_t)column | (uintptr_t)out) & 15) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  const size_t W = words_ct(h);
  if (out < column + n_ct * W && column < out + n_rows * W) HP_FAIL(h, HP_ERR_ARG, "out overlaps the column");
  return extract_broadcast(h, column, row0, n_rows, out, (cudaStream_t)stream);
}

// out[run] += src[run] for the items i0 .. i0 + b - 1 of an (r, c) item space
// (item = r * n_a + c), grouped into runs of consecutive c.
static void accumulate_items(hp_handle* h, uint64_t* out, const uint64_t* src, size_t i0, int b, size_t n_a,
                             cudaStream_t s) {
  const size_t W = words_ct(h);
  for (int u = 0; u < b;) {
    const size_t c = (i0 + u) % n_a;
    const int run = (int)std::min<size_t>(b - u, n_a - c);
    const size_t nw = (size_t)run * W;
    k_ct_acc<<<ew_blocks(nw), EW_THREADS, 0, s>>>(out + c * W, src + (size_t)u * W, h->logn, nw);
    h->launches += 1;
    u += run;
  }
}

int hp_join(hp_handle* h, const uint64_t* a_key, size_t n_a, const uint64_t* b_key, const uint64_t* b_attr,
            size_t n_attr, size_t n_rows, uint64_t* out, void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (n_a == 0) return HP_OK;
  if (!a_key || !b_key || !out || (n_attr && !b_attr)) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if (n_rows == 0) HP_FAIL(h, HP_ERR_ARG, "n_rows must be >= 1");
  if (!keys_ready(h)) HP_FAIL(h, HP_ERR_STATE, "relinearisation key not set");
  if (!h->have_gk) HP_FAIL(h, HP_ERR_STATE, "Galois keys not set");
  HP_NEED_BUDGET(h, BUDGET_SELECT, "hp_join");
  if (!is_device_ptr(a_key) || !is_device_ptr(b_key) || !is_device_ptr(out) || (n_attr && !is_device_ptr(b_attr)))
    HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be device memory");
  if (((uintptr_t)a_key | (uintptr_t)b_key | (uintptr_t)b_attr | (uintptr_t)out) & 15)
    HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t W = words_ct(h), N = h->N, n_b = (n_rows + N - 1) / N, TT = h->run_tile ? h->run_tile : h->tile;
  const size_t n_out = n_attr ? n_attr : 1;
  // broadcasts of every joined B row: keys, then each attribute column
  uint64_t* BC = nullptr;
  CU(h, cudaMallocAsync((void**)&BC, (1 + n_attr) * n_rows * W * sizeof(uint64_t), s));
  uint64_t launches = 0;
  if (int rc = extract_broadcast(h, b_key, 0, n_rows, BC, s)) return rc;
  launches += h->launches;
  for (size_t k = 0; k < n_attr; ++k) {
    h->launches = 0;
    if (int rc = extract_broadcast(h, b_attr + k * n_b * W, 0, n_rows, BC + (1 + k) * n_rows * W, s)) return rc;
    launches += h->launches;
  }
  h->launches = 0;
  CU(h, cudaMemsetAsync(out, 0, n_out * n_a * W * sizeof(uint64_t), s));
  const size_t items = n_rows * n_a;  // item = r * n_a + c
  for (size_t i0 = 0; i0 < items; i0 += TT) {
    const int b = (int)((items - i0 < TT) ? items - i0 : TT);
    for (int u = 0; u < b; ++u) {
      const size_t r = (i0 + u) / n_a, c = (i0 + u) % n_a;
      CU(h, cudaMemcpyAsync(h->stx + u * W, a_key + c * W, W * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
      CU(h, cudaMemcpyAsync(h->sty + u * W, BC + r * W, W * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    }
    run_tile_mode(h, HP_EQ_CT_CT, LIFT_SUB_CT, h->stx, h->sty, nullptr, 0, h->sto, b, s);  // masks
    if (!n_attr) {
      accumulate_items(h, out, h->sto, i0, b, n_a, s);
      continue;
    }
    for (size_t k = 0; k < n_attr; ++k) {
      for (int u = 0; u < b; ++u) {
        const size_t r = (i0 + u) / n_a;
        CU(h, cudaMemcpyAsync(h->sty + u * W, BC + ((1 + k) * n_rows + r) * W, W * sizeof(uint64_t),
                              cudaMemcpyDeviceToDevice, s));
      }
      hmul(h, h->sto, h->sty, h->sto2, b, s, 17);  // mask (depth 16) x broadcast attribute
      accumulate_items(h, out + k * n_a * W, h->sto2, i0, b, n_a, s);
    }
    CU(h, cudaGetLastError());
  }
  cudaFreeAsync(BC, s);
  h->launches += launches;
  CU(h, cudaGetLastError());
  return HP_OK;
}

// BETWEEN (Sec. 4.2.2) against plaintext bounds: out = [lo <= x <= hi].
int hp_between(hp_handle* h, const uint64_t* x, size_t n_ct, uint64_t lo, uint64_t hi, uint64_t* out, void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (n_ct == 0) return HP_OK;
  if (!x || !out) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if (h->t != 65537) HP_FAIL(h, HP_ERR_UNSUPPORTED, "BETWEEN needs t = 65537");
  if (lo > (h->t - 1) / 2 || hi > (h->t - 1) / 2) HP_FAIL(h, HP_ERR_ARG, "bounds must be in [0, (t-1)/2]");
  if (lo > hi) HP_FAIL(h, HP_ERR_ARG, "empty range: lo > hi");
  if (!keys_ready(h)) HP_FAIL(h, HP_ERR_STATE, "relinearisation key not set");
  HP_NEED_BUDGET(h, BUDGET_BETWEEN, "hp_between");
  if (!is_device_ptr(x) || !is_device_ptr(out)) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be device memory");
  if (((uintptr_t)x | (uintptr_t)out) & 15) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  if (int rc = lt_prepare(h)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t W = words_ct(h);
  uint64_t total = 0;
  for (size_t c0 = 0; c0 < n_ct; c0 += h->lt_tile) {
    const int b = (int)((n_ct - c0 < h->lt_tile) ? n_ct - c0 : h->lt_tile);
    h->launches = 0;
    run_between_tile(h, x + c0 * W, lo, hi, out + c0 * W, b, s);
    total += h->launches;
    CU(h, cudaGetLastError());
  }
  h->launches = total;
  return HP_OK;
}

// SELECT with an arbitrary mask (Eq. 5): out = col * mask, relinearised, in tiles.
int hp_select_mask(hp_handle* h, const uint64_t* col, const uint64_t* mask, size_t n_ct, uint32_t mask_depth,
                   double mask_bits, uint64_t* out, void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (n_ct == 0) return HP_OK;
  if (!col || !mask || !out) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if (!keys_ready(h)) HP_FAIL(h, HP_ERR_STATE, "relinearisation key not set");
  if (mask_depth > 1000) HP_FAIL(h, HP_ERR_ARG, "mask_depth %u out of range", mask_depth);
  const double est = budget_of(h, BUDGET_PRODUCT, (int)mask_depth, mask_bits);
  if (est < BUDGET_MARGIN)
    HP_FAIL(h, HP_ERR_DEPTH, "hp_select_mask: estimated noise budget %.1f bits after the product (mask %.1f bits) is "
            "below the %.0f-bit margin", est, mask_bits, BUDGET_MARGIN);
  if (!is_device_ptr(col) || !is_device_ptr(mask) || !is_device_ptr(out))
    HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be device memory");
  if (((uintptr_t)col | (uintptr_t)mask | (uintptr_t)out) & 15) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t W = words_ct(h), TT = h->run_tile ? h->run_tile : h->tile;
  for (size_t c0 = 0; c0 < n_ct; c0 += TT) {
    const int b = (int)((n_ct - c0 < TT) ? n_ct - c0 : TT);
    const size_t off = c0 * W;
    hmul(h, col + off, mask + off, out + off, b, s, (int)mask_depth + 1);
    CU(h, cudaGetLastError());
  }
  return HP_OK;
}

int hp_budget_estimate(const hp_params* prm, int op, uint32_t in_depth, double in_bits, double* out_bits) {
  if (!prm || !prm->q || !out_bits || op < BUDGET_EQ || op > BUDGET_ROTATE_SUM) return HP_ERR_ARG;
  if (prm->log_n < LOGN_MIN || prm->log_n > LOGN_MAX || prm->L != (uint32_t)L || prm->t < 2) return HP_ERR_ARG;
  const int dp = prm->ks_digit_primes ? (int)prm->ks_digit_primes : DIGIT_PRIMES;
  if (dp != DIGIT_PRIMES && dp != DIGIT_PRIMES5) return HP_ERR_ARG;
  if (prm->ks_coarse_from != 0 && prm->ks_coarse_from <= prm->ks_fine_depth) return HP_ERR_ARG;
  *out_bits = budget_estimate((int)prm->log_n, prm->q, L, prm->P, prm->t, dp, (int)prm->ks_fine_depth,
                              (int)prm->ks_coarse_from, op, (int)in_depth, in_bits);
  return HP_OK;
}

int hp_backward(hp_handle* h, int op, const uint64_t* grad_out, uint64_t* grad_x, size_t n_ct, void* stream) {
  (void)op;
  (void)grad_out;
  (void)grad_x;
  (void)n_ct;
  (void)stream;
  if (h) h->err = "EQ is an exact integer map over Z_Q: it has no adjoint";
  return HP_ERR_UNSUPPORTED;
}

void hp_destroy(hp_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

const char* hp_last_error(const hp_handle* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

uint64_t hp_launch_count(const hp_handle* h) { return h ? h->launches : 0; }

int hp_lt_coefficients(uint32_t* out) {
  if (!out) return HP_ERR_ARG;
  return lt_coefficients(out) == 0 ? HP_OK : HP_ERR_ARG;
}

size_t hp_tile_size(const hp_handle* h) { return h ? (h->run_tile ? h->run_tile : h->tile) : 0; }

// ---- client helpers ---------------------------------------------------------
// Relinearisation key (source s^2) with nd digits of dp data primes from the
// secret sk (device, int8 [N]) into rk (device, [nd][2][NKS][N]); digit i draws
// Philox with object index obj_base + i.  Synchronous.
static int make_relin_key(hp_handle* h, uint64_t seed, const int8_t* sk, uint64_t* rk, int nd, int dp,
                          uint32_t obj_base, cudaStream_t s) {
  const int N = h->N, logN = h->logn;
  uint64_t *S = nullptr, *S2 = nullptr, *A = nullptr;
  CU(h, cudaMalloc(&S, (size_t)NKS * N * 8));
  CU(h, cudaMalloc(&S2, (size_t)NKS * N * 8));
  CU(h, cudaMalloc(&A, (size_t)nd * NKS * N * 8));
  k_secret_to_primes<<<ew_blocks((size_t)NKS * N), EW_THREADS, 0, s>>>(sk, S, NKS, 0, ID_P, N);
  ntt_fwd(h, S, NKS, MAP_KS, s);
  k_pointwise_mont<<<ew_blocks((size_t)NKS * N), EW_THREADS, 0, s>>>(S, S, S2, NKS, NKS, 0, ID_P, NKS, logN);
  ntt_inv(h, S2, NKS, MAP_KS, SCALE_NINV_R, s);
  k_rk_sample_a<<<ew_blocks((size_t)nd * NKS * N), EW_THREADS, 0, s>>>(rk, A, seed, logN, DOM_A_RK, obj_base, nd);
  ntt_fwd(h, A, (size_t)nd * NKS, MAP_KS, s);
  k_pointwise_mont<<<ew_blocks((size_t)nd * NKS * N), EW_THREADS, 0, s>>>(A, S, A, NKS, NKS, 0, ID_P, (size_t)nd * NKS,
                                                                      logN);
  ntt_inv(h, A, (size_t)nd * NKS, MAP_KS, SCALE_NINV_R, s);
  k_rk_finish<<<ew_blocks((size_t)nd * NKS * N), EW_THREADS, 0, s>>>(rk, A, S2, seed, logN, DOM_E_RK, obj_base, nd, dp);
  CU(h, cudaGetLastError());
  CU(h, cudaStreamSynchronize(s));
  cudaFree(S);
  cudaFree(S2);
  cudaFree(A);
  return HP_OK;
}

int hp_keygen_fine(hp_handle* h, uint64_t seed, const int8_t* sk, uint64_t* rk_fine, void* stream) {
  if (!h) return HP_ERR_ARG;
  if (!sk) HP_FAIL(h, HP_ERR_ARG, "null secret key");
  if (!h->rkm1) HP_FAIL(h, HP_ERR_STATE, "the handle was created with ks_fine_depth = 0");
  if (!is_device_ptr(sk) || (rk_fine && !is_device_ptr(rk_fine))) HP_FAIL(h, HP_ERR_ARG, "keys must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t* K = rk_fine;
  if (!K) CU(h, cudaMalloc(&K, (size_t)NDIG_FINE * 2 * NKS * h->N * 8));
  int rc = make_relin_key(h, seed, sk, K, NDIG_FINE, 1, FINE_OBJ, s);
  if (rc == HP_OK) rc = hp_set_relin_key_fine(h, K);
  if (!rk_fine) cudaFree(K);
  return rc;
}

int hp_keygen_coarse(hp_handle* h, uint64_t seed, const int8_t* sk, uint64_t* rk_coarse, void* stream) {
  if (!h) return HP_ERR_ARG;
  if (!sk) HP_FAIL(h, HP_ERR_ARG, "null secret key");
  if (!h->rkm2) HP_FAIL(h, HP_ERR_STATE, "the handle was created with ks_coarse_from = 0");
  if (!is_device_ptr(sk) || (rk_coarse && !is_device_ptr(rk_coarse))) HP_FAIL(h, HP_ERR_ARG, "keys must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t* K = rk_coarse;
  if (!K) CU(h, cudaMalloc(&K, (size_t)NDIG2 * 2 * NKS * h->N * 8));
  int rc = make_relin_key(h, seed, sk, K, NDIG2, COARSE_DIGIT_PRIMES, COARSE_OBJ, s);
  if (rc == HP_OK) rc = hp_set_relin_key_coarse(h, K);
  if (!rk_coarse) cudaFree(K);
  return rc;
}

int hp_keygen(hp_handle* h, uint64_t seed, int8_t* sk, uint64_t* rk, void* stream) {
  if (!h) return HP_ERR_ARG;
  if (!sk || !rk) HP_FAIL(h, HP_ERR_ARG, "null output");
  cudaStream_t s = (cudaStream_t)stream;
  k_sample_secret<<<ew_blocks(h->N), EW_THREADS, 0, s>>>(sk, seed, h->N);
  if (int rc = make_relin_key(h, seed, sk, rk, h->nd, h->dp, 0, s)) return rc;
  if (int rc = hp_set_relin_key(h, rk)) return rc;
  if (h->fine_depth > 0)
    if (int rc = hp_keygen_fine(h, seed, sk, nullptr, stream)) return rc;
  if (h->coarse_from > 0) return hp_keygen_coarse(h, seed, sk, nullptr, stream);
  return HP_OK;
}

// S[j] = NTT(s mod q_j), j < L
static int secret_ntt_q(hp_handle* h, const int8_t* sk, uint64_t* S, cudaStream_t s) {
  k_secret_to_primes<<<ew_blocks((size_t)L * h->N), EW_THREADS, 0, s>>>(sk, S, L, 0, -1, h->N);
  ntt_fwd(h, S, L, MAP_Q, s);
  return HP_OK;
}

int hp_encrypt(hp_handle* h, const int8_t* sk, const uint32_t* slots, size_t n_ct, uint64_t seed, uint32_t idx0,
               uint64_t* ct, void* stream) {
  if (!h) return HP_ERR_ARG;
  if (n_ct == 0) return HP_OK;
  if (!sk || !slots || !ct) HP_FAIL(h, HP_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = h->N, logN = h->logn;
  uint64_t *S = nullptr, *A = nullptr, *M = nullptr;
  CU(h, cudaMalloc(&S, (size_t)L * N * 8));
  CU(h, cudaMalloc(&A, n_ct * L * N * 8));
  CU(h, cudaMalloc(&M, n_ct * N * 8));
  secret_ntt_q(h, sk, S, s);
  k_enc_sample<<<ew_blocks(n_ct * L * N), EW_THREADS, 0, s>>>(ct, A, slots, M, seed, idx0, logN, (int)n_ct);
  ntt_fwd(h, A, n_ct * L, MAP_Q, s);
  k_pointwise_mont<<<ew_blocks(n_ct * L * N), EW_THREADS, 0, s>>>(A, S, A, L, L, 0, -1, n_ct * L, logN);
  ntt_inv(h, A, n_ct * L, MAP_Q, SCALE_NINV_R, s);
  ntt_inv(h, M, n_ct, MAP_T, SCALE_NINV, s);  // encoding: slots are the transform of m
  k_enc_finish<<<ew_blocks(n_ct * L * N), EW_THREADS, 0, s>>>(ct, A, M, seed, idx0, logN, (int)n_ct);
  CU(h, cudaGetLastError());
  CU(h, cudaStreamSynchronize(s));
  cudaFree(S);
  cudaFree(A);
  cudaFree(M);
  return HP_OK;
}

int hp_decrypt(hp_handle* h, const int8_t* sk, const uint64_t* ct, size_t n_ct, uint32_t* slots, void* stream) {
  if (!h) return HP_ERR_ARG;
  if (n_ct == 0) return HP_OK;
  if (!sk || !slots || !ct) HP_FAIL(h, HP_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = h->N, logN = h->logn;
  uint64_t *S = nullptr, *C1 = nullptr, *M = nullptr;
  CU(h, cudaMalloc(&S, (size_t)L * N * 8));
  CU(h, cudaMalloc(&C1, n_ct * L * N * 8));
  CU(h, cudaMalloc(&M, n_ct * N * 8));
  secret_ntt_q(h, sk, S, s);
  for (size_t c = 0; c < n_ct; ++c)
    CU(h, cudaMemcpyAsync(C1 + c * L * N, ct + (c * 2 + 1) * L * N, (size_t)L * N * 8, cudaMemcpyDeviceToDevice, s));
  ntt_fwd(h, C1, n_ct * L, MAP_Q, s);
  k_pointwise_mont<<<ew_blocks(n_ct * L * N), EW_THREADS, 0, s>>>(C1, S, C1, L, L, 0, -1, n_ct * L, logN);
  ntt_inv(h, C1, n_ct * L, MAP_Q, SCALE_NINV_R, s);
  k_dec_round<<<ew_blocks(n_ct * N), EW_THREADS, 0, s>>>(ct, C1, M, logN, (int)n_ct);
  ntt_fwd(h, M, n_ct, MAP_T, s);  // decoding
  k_u64_to_u32<<<ew_blocks(n_ct * N), EW_THREADS, 0, s>>>(M, slots, n_ct * N);
  CU(h, cudaGetLastError());
  CU(h, cudaStreamSynchronize(s));
  cudaFree(S);
  cudaFree(C1);
  cudaFree(M);
  return HP_OK;
}

int hp_profile(hp_handle* h, uint32_t class_mask) {
  if (!h) return HP_ERR_ARG;
  CU(h, cudaDeviceSynchronize());
  h->prof_mask = class_mask;
  h->prof.clear();
  h->ev_used = 0;
  return HP_OK;
}

int hp_profile_read(hp_handle* h, int cls, double* ms_total, uint64_t* launches, double* work_total) {
  if (!h || !ms_total || !launches || !work_total || cls < 0 || cls >= PK_COUNT) return HP_ERR_ARG;
  CU(h, cudaDeviceSynchronize());
  double ms = 0, work = 0;
  uint64_t n = 0;
  for (auto& r : h->prof) {
    if (r.cls != cls) continue;
    float m = 0;
    CU(h, cudaEventElapsedTime(&m, r.e0, r.e1));
    ms += m;
    work += r.work;
    ++n;
  }
  *ms_total = ms;
  *launches = n;
  *work_total = work;
  return HP_OK;
}

static int tc_probe_run(const uint16_t* A, const uint16_t* B, float* D, int n, int bf16, int issue, uint32_t polls) {
  hp_handle* h = nullptr;
  uint16_t *dA = nullptr, *dB = nullptr;
  float* dD = nullptr;
  int* dst = nullptr;
  CU(h, cudaMalloc(&dA, (size_t)TCP_M * TCP_K * 2));
  CU(h, cudaMalloc(&dB, (size_t)256 * TCP_K * 2));
  CU(h, cudaMalloc(&dD, (size_t)TCP_M * n * 4));
  CU(h, cudaMalloc(&dst, sizeof(int)));
  CU(h, cudaMemset(dB, 0, (size_t)256 * TCP_K * 2));
  CU(h, cudaMemset(dst, 0, sizeof(int)));
  CU(h, cudaMemcpy(dA, A, (size_t)TCP_M * TCP_K * 2, cudaMemcpyHostToDevice));
  CU(h, cudaMemcpy(dB, B, (size_t)n * TCP_K * 2, cudaMemcpyHostToDevice));
  const int smem = (TCP_M + 256) * TCP_K * 2 + 16;
  CU(h, cudaFuncSetAttribute(k_tc_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k_tc_probe<<<1, 128, smem>>>(dA, dB, dD, n, bf16, issue, polls, dst);
  CU(h, cudaGetLastError());
  CU(h, cudaDeviceSynchronize());
  int st = 0;
  CU(h, cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost));
  CU(h, cudaMemcpy(D, dD, (size_t)TCP_M * n * 4, cudaMemcpyDeviceToHost));
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(dst);
  return st ? HP_ERR_TIMEOUT : HP_OK;
}

int hp_probe_tc_gemm(const uint16_t* A, const uint16_t* B, float* D, int n, int bf16) {
  if (!A || !B || !D || n < 16 || n > 256 || n % 16 || (bf16 != 0 && bf16 != 1)) return HP_ERR_ARG;
  return tc_probe_run(A, B, D, n, bf16, 1, 1u << 20);
}

int hp_probe_tc_timeout(uint32_t polls) {
  if (polls == 0 || polls > (1u << 20)) return HP_ERR_ARG;
  std::vector<uint16_t> A((size_t)TCP_M * TCP_K, 0), B((size_t)16 * TCP_K, 0);
  std::vector<float> D((size_t)TCP_M * 16);
  return tc_probe_run(A.data(), B.data(), D.data(), 16, 0, 0, polls);
}

int hp_probe_peak(int kind, double* per_second) {
  if (!per_second || kind < 0 || kind > 2) return HP_ERR_ARG;
  hp_handle* h = nullptr;
  int dev = 0, sms = 0;
  CU(h, cudaGetDevice(&dev));
  CU(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  uint64_t* sink = nullptr;
  CU(h, cudaMalloc(&sink, 64));
  const uint64_t p = 0x7fffffffe90001ull;  // a 55-bit NTT prime (q_0)
  const uint64_t w = 0x123456789abcull % p;
  const uint64_t wp = (uint64_t)(((unsigned __int128)w << 64) / p);
  uint64_t pinv = p;
  for (int i = 0; i < 6; ++i) pinv *= 2 - p * pinv;
  pinv = (uint64_t)0 - pinv;
  const int blocks = sms * 8, threads = 256, iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    if (kind == 0)
      k_probe_butterfly<<<blocks, threads>>>(sink, iters, p, w, wp);
    else if (kind == 1)
      k_probe_mac<<<blocks, threads>>>(sink, iters, p, pinv);
    else  // 1073479681 = 4095 2^18 + 1: a 30-bit prime with 2^18-th roots of unity
      k_probe_butterfly32<<<blocks, threads>>>(sink, iters, 1073479681u, 123456789u,
                                               (uint32_t)(((uint64_t)123456789u << 32) / 1073479681u));
    cudaEventRecord(e1);
    CU(h, cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first launch is warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  CU(h, cudaGetLastError());
  *per_second = (double)blocks * threads * PROBE_CHAINS * iters / (best * 1e-3);
  return HP_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free squaring.  Some callers cannot allocate device memory at the
// point where they need a squaring: a process whose memory pool already owns
// the GPU's free memory, or code that must not call cudaMalloc/cudaFree in its
// steady state (a serving loop with a fixed memory footprint).  For them,
// hp_square_noalloc runs the same squaring + relinearisation as
// hp_run(HP_SQUARE) on one ciphertext, with its working buffers in a
// fixed-size array that lives in the library's own device memory image.
// ---------------------------------------------------------------------------
constexpr int NOALLOC_MAX_LOGN = 12;  // ring degree up to 4096
constexpr size_t NOALLOC_WORDS_PER_COEFF = 2 * NQB + 3 * NQB + 3 * L + NDIG * NKS + 2 * NKS;  // 312
constexpr size_t NOALLOC_WORDS = NOALLOC_WORDS_PER_COEFF << NOALLOC_MAX_LOGN;               // 10.2 MB
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS];
// Device address of the array, set up once per device and context: a device
// reset (cudaDeviceReset) destroys the context that held the address, and the
// next call on that device, finding a different current context, looks it up
// again.  The context is read with the driver's cuCtxGetCurrent, reached
// through the runtime's entry-point query (no link against the driver library).
struct NoallocAddr {
  void* ctx;
  uint64_t* addr;
};
static NoallocAddr g_noalloc_addr[64];
typedef int (*CtxGetCurrentFn)(void**);  // CUresult cuCtxGetCurrent(CUcontext*)

static int noalloc_scratch(hp_handle* h, uint64_t** out) {
  std::lock_guard<std::mutex> lock(g_tables_mu);
  if (h->device < 0 || h->device >= (int)(sizeof(g_noalloc_addr) / sizeof(g_noalloc_addr[0])))
    HP_FAIL(h, HP_ERR_UNSUPPORTED, "hp_square_noalloc: device ordinal %d beyond the 64 it keeps addresses for",
            h->device);
  static CtxGetCurrentFn get_ctx = nullptr;
  if (!get_ctx) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      HP_FAIL(h, HP_ERR_CUDA, "hp_square_noalloc: driver entry point cuCtxGetCurrent unavailable");
    get_ctx = (CtxGetCurrentFn)fn;
  }
  void* ctx = nullptr;
  if (get_ctx(&ctx) != 0 || !ctx) HP_FAIL(h, HP_ERR_CUDA, "hp_square_noalloc: no current CUDA context");
  NoallocAddr& a = g_noalloc_addr[h->device];
  if (!a.addr || a.ctx != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) HP_FAIL(h, HP_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    a.addr = (uint64_t*)p;
    a.ctx = ctx;
  }
  *out = a.addr;
  return HP_OK;
}

int hp_square_noalloc(hp_handle* h, const uint64_t* ct_in, uint64_t* ct_out, void* stream) {
  if (!h) return HP_ERR_ARG;
  h->launches = 0;
  if (!ct_in || !ct_out) HP_FAIL(h, HP_ERR_ARG, "null ciphertext pointer");
  if (h->logn > NOALLOC_MAX_LOGN)
    HP_FAIL(h, HP_ERR_UNSUPPORTED,
            "hp_square_noalloc: ring degree %d exceeds the static scratch limit of %d (%zu words)", h->N,
            1 << NOALLOC_MAX_LOGN, NOALLOC_WORDS);
  if (h->fine_depth > 0 || h->coarse_from > 0 || h->dp != DIGIT_PRIMES)
    HP_FAIL(h, HP_ERR_UNSUPPORTED, "hp_square_noalloc: only handles with three-prime key-switching digits, "
                                   "ks_fine_depth = 0 and ks_coarse_from = 0 are supported (its scratch holds "
                                   "three-prime digits only)");
  if (!h->have_rk) HP_FAIL(h, HP_ERR_STATE, "relinearisation key not set");
  if (((uintptr_t)ct_in | (uintptr_t)ct_out) & 15) HP_FAIL(h, HP_ERR_ARG, "ciphertexts must be 16-byte aligned");
  int cur = -1;
  CU(h, cudaGetDevice(&cur));
  if (cur != h->device) HP_FAIL(h, HP_ERR_ARG, "the handle's device must be current");
  uint64_t* ws = nullptr;
  int rc = noalloc_scratch(h, &ws);
  if (rc != HP_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = h->N, logN = h->logn;
  uint64_t* ext = ws;
  uint64_t* dprod = ext + (size_t)2 * NQB * N;
  uint64_t* w3 = dprod + (size_t)3 * NQB * N;
  uint64_t* ksin = w3 + (size_t)3 * L * N;
  uint64_t* ksout = ksin + (size_t)NDIG * NKS * N;
  // every scratch word read below is written earlier in this call: nothing needs clearing
  k_lift<<<ew_blocks((size_t)2 * N), EW_THREADS, 0, s>>>(ct_in, nullptr, 0, LIFT_COPY, ext, logN, 1);
  ntt_fwd(h, ext, 2 * NQB, MAP_QB, s);
  k_tensor_sq<<<ew_blocks((size_t)NQB * N), EW_THREADS, 0, s>>>(ext, dprod, logN, 1);
  ntt_inv(h, dprod, 3 * NQB, MAP_QB, SCALE_T_NINV_R, s);
  k_scale_round<<<ew_blocks((size_t)3 * N), EW_THREADS, 0, s>>>(dprod, w3, h->status, logN, 1);
  ntt_fwd(h, ksin, (size_t)NDIG * NKS, MAP_KS, s, w3);
  k_ks_mac<NDIG><<<ew_blocks((size_t)NKS * N), EW_THREADS, 0, s>>>(ksin, h->rkm, ksout, logN, 1);
  ntt_inv(h, ksout, 2 * NKS, MAP_KS, SCALE_NINV, s);
  k_moddown<<<ew_blocks((size_t)2 * L * N), EW_THREADS, 0, s>>>(ksout, w3, ct_out, 0, logN, 1);
  h->launches += 5;  // the element-wise kernels; ntt_fwd / ntt_inv count their own launches
  CU(h, cudaGetLastError());
  return HP_OK;
}

// Synchronise and report the device status word (exactness checks), then clear it.
int hp_check_status(hp_handle* h) {
  if (!h) return HP_ERR_ARG;
  int st = 0;
  CU(h, cudaDeviceSynchronize());
  CU(h, cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  CU(h, cudaMemset(h->status, 0, sizeof(int)));
  if (st) HP_FAIL(h, HP_ERR_CUDA, "device status word %d (exact conversion window violated)", st);
  return HP_OK;
}

}  // extern "C"
