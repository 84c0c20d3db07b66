// Negacyclic NTT over 64-bit primes, batched over many polynomials.
//
// Forward (Cooley-Tukey, natural -> bit-reversed order), stage s = 0..logN-1:
//   t = N >> (s+1); for every j with bit (j / t) even:
//     (a_j, a_{j+t}) <- (a_j + W a_{j+t}, a_j - W a_{j+t}),  W = psi^{brv(2^s + j / 2t)}
// so that output position j holds m(psi^(2 brv(j) + 1)).  The inverse
// (Gentleman-Sande) undoes the stages in reverse order with psi^{-brv(.)} and
// scales by N^{-1} (times a per-launch constant).
//
// N = R x C (R = 2^logR rows, C = 2^logC columns, element j = r C + k).  Stages
// s < logR pair elements of the same column; stages s >= logR pair elements of
// the same row.  Each pass loads one 2048-word tile into shared memory, runs
// its stages with one barrier per stage, and writes the tile back.  Lazy
// ranges (Harvey): forward values stay in [0, 4p), inverse values in [0, 2p);
// the last pass of each direction returns canonical residues.
#pragma once
#include "hp_device.cuh"

namespace hp {

constexpr int NTT_TILE = 2048;
constexpr int NTT_THREADS = 256;

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
  const uint64_t* tw;    // [NPRIME][N] psi^{brv(j)}
  const uint64_t* tws;   // Shoup companions
  const uint64_t* itw;   // [NPRIME][N] psi^{-brv(j)}
  const uint64_t* itws;  // Shoup companions
  const uint64_t* scale; // [NSCALE][NPRIME][2] (value, Shoup)
};
enum { SCALE_NINV = 0, SCALE_T_NINV_R = 1, SCALE_NINV_R = 2, NSCALE = 3 };

// ---- forward, columns (stages 0 .. logR-1) ----
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_fwd_cols(uint64_t* data, PolyMap map, NttTabs T, int logN,
                                                              int logR) {
  __shared__ uint64_t s[NTT_TILE];
  const int N = 1 << logN, logC = logN - logR;
  const int logCOLS = 11 - logR;  // NTT_TILE = 2^11 = R * COLS
  const int COLS = 1 << logCOLS;
  const int poly = blockIdx.y, k0 = blockIdx.x << logCOLS;
  const int id = map.id(poly);
  const uint64_t p = cK.p[id], p2 = 2 * p;
  uint64_t* a = data + (size_t)poly * N;
  const uint64_t* tw = T.tw + (size_t)id * N;
  const uint64_t* tws = T.tws + (size_t)id * N;
  for (int e = threadIdx.x; e < NTT_TILE; e += NTT_THREADS) {
    int r = e >> logCOLS, c = e & (COLS - 1);
    s[e] = a[((size_t)r << logC) + k0 + c];
  }
  __syncthreads();
  for (int st = 0; st < logR; ++st) {
    const int logt = logR - st - 1;  // pair distance in rows
    for (int b = threadIdx.x; b < NTT_TILE / 2; b += NTT_THREADS) {
      int c = b & (COLS - 1), bb = b >> logCOLS;
      int g = bb >> logt, o = bb & ((1 << logt) - 1);
      int r = (g << (logt + 1)) + o;
      int ti = (1 << st) + g;
      uint64_t W = tw[ti], Wp = tws[ti];
      int i0 = (r << logCOLS) + c, i1 = i0 + (1 << (logt + logCOLS));
      uint64_t X = s[i0], Y = s[i1];
      X = X >= p2 ? X - p2 : X;
      uint64_t V = mul_shoup_lazy(Y, W, Wp, p);
      s[i0] = X + V;
      s[i1] = X - V + p2;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NTT_TILE; e += NTT_THREADS) {
    int r = e >> logCOLS, c = e & (COLS - 1);
    a[((size_t)r << logC) + k0 + c] = s[e];
  }
}

// ---- forward, rows (stages logR .. logN-1); canonical output ----
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_fwd_rows(uint64_t* data, PolyMap map, NttTabs T, int logN,
                                                              int logR) {
  __shared__ uint64_t s[NTT_TILE];
  const int N = 1 << logN, logC = logN - logR;
  const int logROWS = 11 - logC;
  const int poly = blockIdx.y, row0 = blockIdx.x << logROWS;
  const int id = map.id(poly);
  const uint64_t p = cK.p[id], p2 = 2 * p;
  uint64_t* a = data + (size_t)poly * N + ((size_t)row0 << logC);
  const uint64_t* tw = T.tw + (size_t)id * N;
  const uint64_t* tws = T.tws + (size_t)id * N;
  for (int e = threadIdx.x; e < NTT_TILE; e += NTT_THREADS) s[e] = a[e];
  __syncthreads();
  for (int st = logR; st < logN; ++st) {
    const int logt = logN - st - 1;  // pair distance in elements (< C)
    for (int b = threadIdx.x; b < NTT_TILE / 2; b += NTT_THREADS) {
      int rr = b >> (logC - 1), bb = b & ((1 << (logC - 1)) - 1);
      int g = bb >> logt, o = bb & ((1 << logt) - 1);
      int k = (g << (logt + 1)) + o;
      int ti = (1 << st) + (((row0 + rr) << (logC - logt - 1)) + g);
      uint64_t W = tw[ti], Wp = tws[ti];
      int i0 = (rr << logC) + k, i1 = i0 + (1 << logt);
      uint64_t X = s[i0], Y = s[i1];
      X = X >= p2 ? X - p2 : X;
      uint64_t V = mul_shoup_lazy(Y, W, Wp, p);
      s[i0] = X + V;
      s[i1] = X - V + p2;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NTT_TILE; e += NTT_THREADS) {
    uint64_t x = s[e];
    x = x >= p2 ? x - p2 : x;
    a[e] = csub(x, p);
  }
}

// ---- inverse, rows (stages logN-1 .. logR); input in [0, 2p) ----
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_inv_rows(uint64_t* data, PolyMap map, NttTabs T, int logN,
                                                              int logR) {
  __shared__ uint64_t s[NTT_TILE];
  const int N = 1 << logN, logC = logN - logR;
  const int logROWS = 11 - logC;
  const int poly = blockIdx.y, row0 = blockIdx.x << logROWS;
  const int id = map.id(poly);
  const uint64_t p = cK.p[id], p2 = 2 * p;
  uint64_t* a = data + (size_t)poly * N + ((size_t)row0 << logC);
  const uint64_t* tw = T.itw + (size_t)id * N;
  const uint64_t* tws = T.itws + (size_t)id * N;
  for (int e = threadIdx.x; e < NTT_TILE; e += NTT_THREADS) s[e] = a[e];
  __syncthreads();
  for (int st = logN - 1; st >= logR; --st) {
    const int logt = logN - st - 1;
    for (int b = threadIdx.x; b < NTT_TILE / 2; b += NTT_THREADS) {
      int rr = b >> (logC - 1), bb = b & ((1 << (logC - 1)) - 1);
      int g = bb >> logt, o = bb & ((1 << logt) - 1);
      int k = (g << (logt + 1)) + o;
      int ti = (1 << st) + (((row0 + rr) << (logC - logt - 1)) + g);
      uint64_t W = tw[ti], Wp = tws[ti];
      int i0 = (rr << logC) + k, i1 = i0 + (1 << logt);
      uint64_t X = s[i0], Y = s[i1];
      uint64_t U = X + Y;
      s[i0] = U >= p2 ? U - p2 : U;
      s[i1] = mul_shoup_lazy(X - Y + p2, W, Wp, p);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NTT_TILE; e += NTT_THREADS) a[e] = s[e];
}

// ---- inverse, columns (stages logR-1 .. 0) and scaling; canonical output ----
__global__ void __launch_bounds__(NTT_THREADS) k_ntt_inv_cols(uint64_t* data, PolyMap map, NttTabs T, int logN,
                                                              int logR, int scale_mode) {
  __shared__ uint64_t s[NTT_TILE];
  const int N = 1 << logN, logC = logN - logR;
  const int logCOLS = 11 - logR;
  const int COLS = 1 << logCOLS;
  const int poly = blockIdx.y, k0 = blockIdx.x << logCOLS;
  const int id = map.id(poly);
  const uint64_t p = cK.p[id], p2 = 2 * p;
  uint64_t* a = data + (size_t)poly * N;
  const uint64_t* tw = T.itw + (size_t)id * N;
  const uint64_t* tws = T.itws + (size_t)id * N;
  for (int e = threadIdx.x; e < NTT_TILE; e += NTT_THREADS) {
    int r = e >> logCOLS, c = e & (COLS - 1);
    s[e] = a[((size_t)r << logC) + k0 + c];
  }
  __syncthreads();
  for (int st = logR - 1; st >= 0; --st) {
    const int logt = logR - st - 1;
    for (int b = threadIdx.x; b < NTT_TILE / 2; b += NTT_THREADS) {
      int c = b & (COLS - 1), bb = b >> logCOLS;
      int g = bb >> logt, o = bb & ((1 << logt) - 1);
      int r = (g << (logt + 1)) + o;
      int ti = (1 << st) + g;
      uint64_t W = tw[ti], Wp = tws[ti];
      int i0 = (r << logCOLS) + c, i1 = i0 + (1 << (logt + logCOLS));
      uint64_t X = s[i0], Y = s[i1];
      uint64_t U = X + Y;
      s[i0] = U >= p2 ? U - p2 : U;
      s[i1] = mul_shoup_lazy(X - Y + p2, W, Wp, p);
    }
    __syncthreads();
  }
  const uint64_t* sc = T.scale + ((size_t)scale_mode * NPRIME + id) * 2;
  const uint64_t w = sc[0], wp = sc[1];
  for (int e = threadIdx.x; e < NTT_TILE; e += NTT_THREADS) {
    int r = e >> logCOLS, c = e & (COLS - 1);
    a[((size_t)r << logC) + k0 + c] = mul_shoup(s[e], w, wp, p);
  }
}

}  // namespace hp
