/* libhp — the NSHEDB equality predicate over BFV-packed columns on one GPU.
 *
 * Paper: "NSHEDB: Noise-Sensitive Homomorphic Encrypted Database Query Engine"
 * (arXiv 2602.24271).  The operation is the equality predicate of Sec. 2.1.7,
 * Eq. 3:  EQ(x, y) = 1 - (x - y)^(p-1), evaluated slot-wise on BFV
 * ciphertexts that pack N column values each (Sec. 4.1), with p = 65537 so that
 * exponentiation by squaring (Sec. 4.3.1, Table 3: ceil(log(p-1)) = 16
 * multiplications) is 16 ciphertext squarings, each relinearised.
 *
 * Scheme and parameters (paper Sec. 5.1: N = 32768, log QP = 881, p = 65537):
 *   ring            Z_Q[X] / (X^N + 1), N = 2^log_n, 12 <= log_n <= 15
 *   data modulus    Q = q_0 ... q_{L-1}, L = 15, q_i prime < 2^55, q_i = 1 mod 2^16
 *   special prime   P < 2^56, P = 1 mod 2^16 (relinearisation only)
 *   plaintext       t = p = 65537
 *   multiplication  textbook Fan-Vercauteren: centred lift, exact tensor,
 *                   round(t d / Q) mod Q; key switching (relinearisation,
 *                   rotations) with D = L / G digits, each the residue of d2
 *                   modulo a group of G = ks_digit_primes consecutive data
 *                   primes (3 by default, or 5), and the special prime P;
 *                   products at multiplicative depth up to the handle's
 *                   ks_fine_depth are relinearised with L per-prime digits
 *                   [d2]_{q_i} instead, and products from ks_coarse_from on
 *                   with two digits (q_0..q_7 and q_8..q_14).  Results are
 *                   bit-exact against that integer definition.
 *
 * Memory layouts (all words uint64, residues canonical in [0, prime)):
 *   ciphertext      [2][L][N]        (c0, c1) residues mod q_0..q_{L-1},
 *                                    coefficient domain; n ciphertexts are
 *                                    contiguous: [n][2][L][N]
 *   relin key       [D][2][L+1][N]   rk_a = (rk_a0, rk_a1) for digit a < D = L / ks_digit_primes,
 *                                    residues mod q_0..q_{L-1}, P; coefficient
 *                                    domain
 *   secret key      int8 [N]         coefficients in {-1, 0, 1}
 *   slots           uint32 [N]       plaintext slot values mod t
 *
 * Pointers: "device" arguments must be CUDA device (or managed) memory.  The
 * ciphertext arguments of hp_run may instead be host memory (pageable or
 * pinned); the library then streams them through two device staging sets
 * (copy-in, compute and copy-out of consecutive tiles overlap when the host
 * buffers are pinned) and returns after the last result is back in host memory.
 *
 * Streams: every call is ordered on the caller's `stream` (a cudaStream_t
 * passed as void*, NULL = legacy default stream).  Device-pointer calls are
 * asynchronous and return before the GPU finishes.
 *
 * Errors: 0 = success, negative = HP_ERR_*; hp_last_error(h) returns a
 * description of the last failure on that handle.  On error the output
 * buffers are unspecified.
 *
 * Thread safety: a handle may be used by one host thread at a time.  The
 * library's process-wide tables (per-device constants, the autotune cache, the
 * allocation-free scratch addresses) are guarded by a mutex.
 */
#ifndef LIBHP_HP_H
#define LIBHP_HP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HP_OK 0
#define HP_ERR_ARG (-1)         /* bad argument: null pointer, size, range, alignment */
#define HP_ERR_DEPTH (-2)       /* parameters cannot evaluate the requested depth */
#define HP_ERR_OOM (-3)         /* device allocation failed */
#define HP_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define HP_ERR_TIMEOUT (-5)     /* a bounded device wait expired */
#define HP_ERR_UNSUPPORTED (-6) /* operation or parameter set not supported */
#define HP_ERR_STATE (-7)       /* handle not ready (e.g. no relinearisation key) */

typedef struct hp_handle hp_handle;

/* Scheme parameters.  q points to L host words. */
typedef struct {
  uint32_t log_n;     /* ring degree N = 2^log_n, 12..15 */
  uint32_t L;         /* number of data primes, must be 15 */
  const uint64_t* q;  /* data primes q_0 > q_1 > ... > q_{L-1} */
  uint64_t P;         /* special prime */
  uint64_t t;         /* plaintext modulus, must be 65537 */
  uint32_t max_depth; /* multiplicative depth the caller needs (16 for EQ, 17 with SELECT) */
  uint32_t ks_fine_depth; /* products at multiplicative depth <= this are relinearised with a
                             per-prime key (15 digits [d2]_{q_i}, SEAL's decomposition); deeper
                             ones with the key of ks_digit_primes (or the two-digit key, see
                             ks_coarse_from).  0 = no per-prime key; >= the deepest product =
                             per-prime throughout.  See hp_budget_estimate. */
  uint32_t ks_digit_primes; /* data primes per digit of the relinearisation and Galois keys: 3 (the
                               default, also for 0; D = 5 digits) or 5 (D = 3 digits: 48 instead of
                               80 key-switching transforms per product, for more key-switching noise:
                               EQ then leaves about 114 bits of budget at N = 32768, against 224) */
  uint32_t ks_coarse_from;  /* products at multiplicative depth >= this are relinearised with a
                               two-digit key (digits [d2] mod q_0..q_7 and mod q_8..q_14: 32 key-
                               switching transforms per product).  Its key-switching noise (about
                               2^400 at N = 32768) costs nothing once the product's own noise is
                               larger: the oracle measures the same EQ budget with it from depth 7
                               on (five-prime digits below), 8 bits less from depth 6.  0 = never;
                               otherwise above ks_fine_depth (HP_ERR_ARG).  See hp_budget_estimate. */
} hp_params;

/* Operations of hp_run / hp_run_batched. */
typedef enum {
  HP_EQ_CT_CT = 0,    /* EQ(x, y) = 1 - (x - y)^(p-1), Eq. 3 */
  HP_EQ_CT_CONST = 1, /* EQ(x, c) with c broadcast to every slot */
  HP_SELECT = 2,      /* y * EQ(x, c): the SELECT tail of Eq. 5; ct_y is the column */
  HP_SQUARE = 3,      /* one squaring + relinearisation (building block, for tests) */
  HP_LT = 4           /* LT(x, y) = [x < y], Eq. 4, for x, y in [0, (p-1)/2] (depth 18) */
} hp_op;

/* Fill q_out[0..L) and *P_out with the default primes (largest primes below
 * 2^55, resp. 2^56, congruent to 1 mod 2^16) and *t_out = 65537.
 * Returns HP_ERR_ARG for L outside 1..15 or null pointers. */
int hp_default_params(uint32_t L, uint64_t* q_out, uint64_t* P_out, uint64_t* t_out);

/* Create a handle for `params` on the current CUDA device.  Validates the
 * parameters (primality, congruences, sizes) and the static depth estimate
 * (HP_ERR_DEPTH if max_depth exceeds what the modulus supports).
 * `max_tile_ct` bounds how many ciphertexts are processed per pipeline tile
 * (0 = library default: the tile that fits about 22 GB of workspace, at most
 * 128); device workspace grows linearly with it (165 MB per ciphertext at
 * N = 32768, including two staging sets for overlapped host-memory calls).  `relin_key` may be NULL (set it later
 * with hp_set_relin_key); otherwise it is a device pointer with the layout
 * above.  On success *out owns all device memory it allocated. */
int hp_create(const hp_params* params, const uint64_t* relin_key, size_t max_tile_ct, hp_handle** out);

/* Load (replace) the relinearisation key from device memory (layout above).
 * The handle keeps its own transformed copy; the caller keeps ownership of
 * `relin_key_dev`.  Synchronous with respect to the host. */
int hp_set_relin_key(hp_handle* h, const uint64_t* relin_key_dev);

/* The per-prime relinearisation key of a handle created with ks_fine_depth > 0
 * (HP_ERR_STATE otherwise): digit i = [d2]_{q_i} (i < L), key
 * rk_i = (-(a_i s + e_i) + P g_i s^2, a_i) mod QP with g_i = (Q/q_i) [(Q/q_i)^{-1}]_{q_i};
 * layout [L][2][L+1][N] (residues mod q_0..q_{L-1}, P; coefficient domain).
 *   hp_set_relin_key_fine: install a key made elsewhere (device memory);
 *   hp_keygen_fine: make it from the secret sk (device int8 [N]) and `seed`
 *     (Philox counter (k, j, 16 + i, 5) for a_i, (k, 0, 16 + i, 4) for e_i) and
 *     install it; rk_fine_out (device, optional) receives it.  hp_keygen calls
 *     it itself for such handles.
 * Both synchronous. */
int hp_set_relin_key_fine(hp_handle* h, const uint64_t* rk_fine_dev);
int hp_keygen_fine(hp_handle* h, uint64_t seed, const int8_t* sk, uint64_t* rk_fine_out, void* stream);

/* The two-digit relinearisation key of a handle created with ks_coarse_from > 0
 * (HP_ERR_STATE otherwise): digit a = [d2]_{Q_a}, Q_0 = q_0 ... q_7,
 * Q_1 = q_8 ... q_14, key rk_a = (-(a_a s + e_a) + P g_a s^2, a_a) mod QP with
 * g_a = (Q/Q_a) [(Q/Q_a)^{-1}]_{Q_a}; layout [2][2][L+1][N] (residues mod
 * q_0..q_{L-1}, P; coefficient domain).
 *   hp_set_relin_key_coarse: install a key made elsewhere (device memory);
 *   hp_keygen_coarse: make it from the secret sk (device int8 [N]) and `seed`
 *     (Philox counter (k, j, 48 + a, 5) for a_a, (k, 0, 48 + a, 4) for e_a) and
 *     install it; rk_coarse_out (device, optional) receives it.  hp_keygen
 *     calls it itself for such handles.
 * Both synchronous. */
int hp_set_relin_key_coarse(hp_handle* h, const uint64_t* rk_coarse_dev);
int hp_keygen_coarse(hp_handle* h, uint64_t seed, const int8_t* sk, uint64_t* rk_coarse_out, void* stream);

/* Evaluate `op` on n_ct ciphertexts.
 *   HP_EQ_CT_CT    out[i] = EQ(x[i], y[i])
 *   HP_EQ_CT_CONST out[i] = EQ(x[i], const_val)           (y ignored, may be NULL)
 *   HP_SELECT      out[i] = y[i] * EQ(x[i], const_val)    (depth 17)
 *   HP_SQUARE      out[i] = relin(x[i]^2)                  (y ignored)
 *   HP_LT          out[i] = LT(x[i], y[i]) = [x < y] slot-wise (Eq. 4), valid
 *                  when x - y lies in [-(p-1)/2, (p-1)/2] (inputs below 2^15 + 1);
 *                  the polynomial f(z) = z h(z^2) - ((p-1)/2) z^(p-1) of Eq. 4
 *                  is evaluated by baby steps (255 powers of z^2) and giant
 *                  steps (128 powers of z^512), each power the product of its
 *                  largest power-of-two part and the rest: 511
 *                  multiplications, depth 18 (the products that share a
 *                  power-of-two factor lift and transform it once).
 *                  Device memory only; the first call allocates its workspace
 *                  (about 3.1 GB per ciphertext of the LT tile, tile <= 8 at
 *                  N = 32768).
 * ct_x, ct_y, ct_out: [n_ct][2][L][N]; all device memory, or all host memory
 * (then the call is synchronous).  ct_out may alias ct_x or ct_y.  n_ct = 0
 * is a no-op.  const_val must be < t.  Requires the relinearisation key. */
int hp_run(hp_handle* h, int op, const uint64_t* ct_x, const uint64_t* ct_y, uint64_t const_val, uint64_t* ct_out,
           size_t n_ct, void* stream);

/* One instance of a batched call: its ciphertexts ct_offset .. ct_offset+n_ct-1
 * of the batch arrays, of which the first n_slots slots are meaningful, and the
 * instance's constant (HP_EQ_CT_CONST).  Instances may share a ciphertext when
 * they are slot-packed: then slot_offset gives the first slot of the instance
 * inside ciphertext ct_offset and n_ct must be 1. */
typedef struct {
  uint64_t ct_offset;
  uint32_t n_ct;
  uint32_t slot_offset;
  uint32_t n_slots;
  uint32_t reserved;
  uint64_t const_val;
} hp_instance;

/* Evaluate `op` (HP_EQ_CT_CT or HP_EQ_CT_CONST) for n_inst instances of
 * uneven size in one pass over the union of their ciphertexts: tiles of
 * ciphertexts, each replayed from a CUDA graph of the whole 16-squaring launch
 * sequence (captured once per tile shape and kept in the handle) whose first
 * and last kernels are pointed at the tile's own ciphertexts before each
 * launch, so the ciphertexts are read and written in place (ct_out may alias
 * ct_x).  `inst` is
 * host memory; ct_x / ct_y / ct_out are device arrays of n_ct_total
 * ciphertexts.  Instance i covers global slots [ct_offset N + slot_offset,
 * + n_slots) inside its ciphertexts ct_offset .. ct_offset + n_ct - 1.  For
 * HP_EQ_CT_CONST each instance's constant applies to its own slot range (slots
 * outside every instance compare against 0).  Every ciphertext must belong to
 * at least one instance and slot ranges must not overlap (HP_ERR_ARG).
 * Stream-ordered; the first call per tile shape also captures its graph. */
int hp_run_batched(hp_handle* h, int op, const hp_instance* inst, size_t n_inst, const uint64_t* ct_x,
                   const uint64_t* ct_y, uint64_t* ct_out, size_t n_ct_total, void* stream);

/* Time the EQ launch sequence for candidate tile sizes (up to the handle's
 * workspace tile; per candidate the fastest of three passes after a warm-up
 * pass) and make the largest tile within 1 % of the fastest per ciphertext the
 * tile used by hp_run and hp_run_batched; *best_tile (optional) receives it.  Runs on the
 * handle's own staging buffers (the computation is data-oblivious, so the
 * timing does not depend on the data); cached per (ring degree, device, max
 * tile) for the process.  Synchronous. */
int hp_autotune(hp_handle* h, size_t* best_tile);

/* BETWEEN (Sec. 4.2.2): out[c] = [lo <= x <= hi] slot-wise for plaintext bounds
 * lo <= hi, as the paper's product of the two comparisons,
 * (1 - LT(x, lo)) (1 - LT(hi, x)): two LT evaluations (511 multiplications
 * each, the Eq. 4 polynomial on x - lo and hi - x, see HP_LT) and one product,
 * depth 19.  Exact when x, lo, hi lie in [0, (t-1)/2]; bounds outside that
 * range or lo > hi give HP_ERR_ARG.  x, out: n_ct device ciphertexts; tiles of
 * up to 8 ciphertexts share the LT workspace.  Needs t = 65537 and the
 * relinearisation key.  The result goes on to hp_select_mask with
 * mask_depth 19 and the budget hp_budget_estimate(HP_BUDGET_BETWEEN) gives. */
int hp_between(hp_handle* h, const uint64_t* ct_x, size_t n_ct, uint64_t lo, uint64_t hi, uint64_t* ct_out,
               void* stream);

/* One column against many constants (device memory, n_ct ciphertexts of x,
 * n_const constants in host memory, each < t):
 *   GROUP BY (Sec. 4.2.2): masks[k][c] = EQ(x[c], consts[k])   (masks: [n_const][n_ct] ciphertexts)
 *   IN (Eq. 6):            in_out[c] = sum_k EQ(x[c], consts[k]) = [x in S]
 * Either output may be NULL (not both); with masks == NULL the masks live in
 * stream-ordered temporary memory.  The sum is a balanced addition tree
 * (Sec. 4.3.1); ciphertext addition is exact mod Q, so the result does not
 * depend on the tree shape.  The n_const * n_ct chains run in tiles of the
 * handle's tile size.  IN is the set-membership mask only when the constants
 * are distinct (else it counts multiplicities). */
int hp_eq_fanout(hp_handle* h, const uint64_t* ct_x, size_t n_ct, const uint64_t* consts, size_t n_const,
                 uint64_t* masks, uint64_t* in_out, void* stream);

/* ---- Rotations, COUNT and SUM (Sec. 4.2.2) ----------------------------------
 * COUNT is the rotate-and-add reduction of an EQ mask, SUM that of
 * column x mask (HP_SELECT, Eq. 5): rotate, add, double the rotation, until
 * every slot holds the sum of all slots (mod t).  The slots form two rows of
 * N/2 under the Galois group {+-3^k} mod 2N; the reduction applies the row
 * rotations by N/4, N/8, ..., 1 (Galois elements 3^(2^i) mod 2N, i = logN-2..0)
 * and then the row exchange (2N - 1): logN steps, one Galois key each.
 *
 * hp_galois_elements: the logN elements in that order (g_out: uint64 [logn]).
 *
 * hp_galois_keygen: Galois keys for those elements from the secret sk (device
 * int8 [N], as made by hp_keygen with the same seed convention) and `seed`,
 * installed in the handle.  Key st is the key-switching key from tau_g(s) to
 * s: gk[st][i] = (-(a_i s + e_i) + P g_i tau_g(s), a_i) mod QP with a_i, e_i
 * drawn by Philox with counter (k, j, (g << 5) | i, 7) resp. (k, 0, (g << 5) | i, 6).
 * gk: NULL or device uint64 [logN][D][2][L+1][N] (residues mod q_0..q_{L-1}, P;
 * the relinearisation-key layout per element).  Synchronous.
 *
 * hp_set_galois_keys: install keys made elsewhere (device, layout as above).
 *
 * hp_rotate_sum: out[o] = reduction of sum_{c in group o} x[c] for the groups of
 * `group` consecutive ciphertexts (the last may be shorter): n_out =
 * ceil(n_ct / group) ciphertexts, each holding in every slot the sum mod t of
 * all slots of its group.  The result is exact (and a count or sum of the
 * plain values) while that sum is below t.  out may equal x only when group ==
 * 1 (in place); otherwise they must not overlap.  HP_ERR_STATE without Galois
 * keys.  Device memory, stream-ordered. */
int hp_galois_elements(int logn, uint64_t* g_out);

/* hp_ct_sum: out[o] = sum of the ciphertexts x[o group .. min(n_ct, (o + 1) group))
 * mod Q (n_out = ceil(n_ct / group)); ciphertext addition, which decrypts to the
 * slot-wise sum mod t.  It combines partial aggregates, e.g. the per-GPU results
 * of a SUM after they are gathered (NCCL has no sum mod q).  Aliasing as for
 * hp_rotate_sum.  Device memory, stream-ordered. */
int hp_ct_sum(hp_handle* h, const uint64_t* ct_x, size_t n_ct, size_t group, uint64_t* ct_out, void* stream);
int hp_galois_keygen(hp_handle* h, uint64_t seed, const int8_t* sk, uint64_t* gk, void* stream);
int hp_set_galois_keys(hp_handle* h, const uint64_t* gk);
int hp_rotate_sum(hp_handle* h, const uint64_t* ct_x, size_t n_ct, size_t group, uint64_t* ct_out, void* stream);

/* ---- JOIN by Extract + Broadcast (Sec. 4.2.2) ---------------------------------
 * Rows of a column: row r is slot r % N of ciphertext r / N (slot order of
 * hp_encrypt).  Extract multiplies a ciphertext by the plaintext unit vector of
 * one slot (plaintext coefficients taken centred in (-t/2, t/2]); Broadcast is
 * the rotate-and-add reduction, so every slot ends holding the extracted value.
 *
 * hp_extract_broadcast: out[k] = Broadcast(Extract(column, row0 + k)),
 * k < n_rows; column: n_ct ciphertexts; out must not overlap it.  Needs the
 * Galois keys.
 *
 * hp_join: equi-join A.key = B.key over the first n_rows rows of table B:
 *   kb_r = Broadcast(Extract(b_key, r)),  mask_r[c] = EQ(a_key[c], kb_r),
 *   n_attr > 0:  out[k][c] = sum_r mask_r[c] * Broadcast(Extract(b_attr[k], r))
 *   n_attr = 0:  out[0][c] = sum_r mask_r[c]   (semi-join: number of matches)
 * a_key: n_a ciphertexts; b_key: ceil(n_rows / N) ciphertexts; b_attr:
 * [n_attr][ceil(n_rows / N)] ciphertexts; out: [max(1, n_attr)][n_a]
 * ciphertexts.  With unique B keys (a key-foreign key join) each A row gets
 * the attributes of its matching B row, or 0.  Cost: n_rows * n_a EQ chains
 * plus n_rows * n_a * n_attr products and (1 + n_attr) n_rows broadcasts.
 * Needs the relinearisation and Galois keys; stream-ordered, device memory. */
int hp_extract_broadcast(hp_handle* h, const uint64_t* column, size_t n_ct, size_t row0, size_t n_rows, uint64_t* out,
                         void* stream);
int hp_join(hp_handle* h, const uint64_t* a_key, size_t n_a, const uint64_t* b_key, const uint64_t* b_attr,
            size_t n_attr, size_t n_rows, uint64_t* out, void* stream);

/* ---- noise budget (Sec. 4.3: the planner keeps every query within the depth
 * the parameters allow) -------------------------------------------------------
 * hp_budget_estimate: a static, conservative estimate of the invariant-noise
 * budget in bits (log2(Q / (2 |v|)); decryption is exact while it is positive)
 * left in the result of `op` for the parameters `params` (log_n, q, P, t,
 * ks_fine_depth, ks_digit_primes, ks_coarse_from; no GPU needed):
 *   HP_BUDGET_EQ / _SELECT / _SQUARE / _LT / _BETWEEN   the operation on fresh inputs
 *   HP_BUDGET_PRODUCT      a fresh column times an operand of budget in_bits
 *                          lying at multiplicative depth in_depth (hp_select_mask)
 *   HP_BUDGET_ROTATE_SUM   the rotate-and-add reduction of an operand of budget
 *                          in_bits (COUNT / SUM over all N slots)
 * The model: fresh budget log Q - log t - log N - 8, log t + log N + 1 bits per
 * level, capped after each product by the key-switching noise of the key used;
 * LT pays 8 more bits for its giant-step sum.  It lies below the oracle's
 * measured budgets.  Every operation of this library refuses to run
 * (HP_ERR_DEPTH) when its estimate is below HP_BUDGET_MARGIN bits. */
#define HP_BUDGET_MARGIN 10.0
typedef enum {
  HP_BUDGET_EQ = 0,
  HP_BUDGET_SELECT = 1,
  HP_BUDGET_SQUARE = 2,
  HP_BUDGET_LT = 3,
  HP_BUDGET_BETWEEN = 4,
  HP_BUDGET_PRODUCT = 5,
  HP_BUDGET_ROTATE_SUM = 6
} hp_budget_op;
int hp_budget_estimate(const hp_params* params, int op, uint32_t in_depth, double in_bits, double* out_bits);

/* SELECT (Eq. 5, Sec. 4.2.2) with any predicate mask: out[c] = col[c] * mask[c]
 * for n_ct device ciphertexts, one multiplication with relinearisation.  The
 * mask is an EQ, LT or BETWEEN result (or a product of such: AND), lying at
 * multiplicative depth mask_depth (16 for EQ, 18 for LT, 19 for BETWEEN) with
 * estimated budget mask_bits (hp_budget_estimate of the operation that made
 * it); the column is fresh.  The product lies at depth mask_depth + 1, which
 * selects the relinearisation key as for every product.  HP_ERR_DEPTH when
 * the estimated budget after the product is below HP_BUDGET_MARGIN.  out may
 * alias col or mask.  Stream-ordered; tiles of the handle's tile size. */
int hp_select_mask(hp_handle* h, const uint64_t* col, const uint64_t* mask, size_t n_ct, uint32_t mask_depth,
                   double mask_bits, uint64_t* out, void* stream);

/* Adjoint of hp_run.  The predicate is an exact integer map over Z_Q with no
 * derivative, so this always returns HP_ERR_UNSUPPORTED. */
int hp_backward(hp_handle* h, int op, const uint64_t* grad_out, uint64_t* grad_x, size_t n_ct, void* stream);

/* Free the handle and its device memory (after synchronising its work). */
void hp_destroy(hp_handle* h);

/* Description of the last error on h (or of the last hp_create failure when
 * h is NULL).  Valid until the next call on the same handle. */
const char* hp_last_error(const hp_handle* h);

/* ---- client-side helpers (tests, benchmark input generation) -------------
 * These take the secret key explicitly; the handle never stores it.  All
 * pointers are device memory; calls are stream-ordered. */

/* Secret key s (int8 [N]) and relinearisation key (layout above), drawn with
 * Philox4x32-10 keyed by `seed` with counter (coefficient, prime, object,
 * domain): s ternary floor(3 w0 / 2^32) - 1, errors centred binomial with
 * eta = 21, uniform residues floor(r m / 2^128).  Also loads the key into the
 * handle. */
int hp_keygen(hp_handle* h, uint64_t seed, int8_t* sk_out, uint64_t* relin_key_out, void* stream);

/* Encrypt n_ct slot vectors (uint32 [n_ct][N], values < t): ciphertext i uses
 * Philox object index ct_index0 + i.  ct = (-(a s + e) + Delta m, a). */
int hp_encrypt(hp_handle* h, const int8_t* sk, const uint32_t* slots, size_t n_ct, uint64_t seed, uint32_t ct_index0,
               uint64_t* ct_out, void* stream);

/* Decrypt n_ct ciphertexts: m = round(t [c0 + c1 s]_Q / Q) mod t, then
 * decode to slots (uint32 [n_ct][N]). */
int hp_decrypt(hp_handle* h, const int8_t* sk, const uint64_t* ct, size_t n_ct, uint32_t* slots_out, void* stream);

/* Number of kernel launches issued by the last hp_run / hp_run_batched call on
 * h (for launch accounting). */
uint64_t hp_launch_count(const hp_handle* h);

/* The 32768 odd coefficients h_m = c_{2m+1} of the LT polynomial of Eq. 4 over
 * F_65537 (c_k = sum_{b=1}^{32768} b^(p-1-k)); host computation, no GPU. */
int hp_lt_coefficients(uint32_t* out);

/* Ciphertexts per pipeline tile used by hp_run / hp_run_batched: the
 * autotuned size if hp_autotune ran, else the workspace tile chosen by
 * hp_create (max_tile_ct or the default that fits about 22 GB of workspace). */
size_t hp_tile_size(const hp_handle* h);

/* Synchronise the device and report the exactness status word of h (a
 * window check inside the exact base conversions that cannot fail for valid
 * parameters); HP_OK if clean.  The word is cleared afterwards. */
int hp_check_status(hp_handle* h);

/* ---- allocation-free squaring (no counterpart in the paper) ------------------
 * For callers that cannot allocate device memory when they need the
 * operation -- e.g. a process whose memory pool already holds the GPU's free
 * memory, or a serving loop that must keep a fixed footprint and never call
 * cudaMalloc/cudaFree in its steady state.  Computes exactly what
 * hp_run(h, HP_SQUARE, ct_in, NULL, 0, ct_out, 1, stream) computes (one
 * squaring + relinearisation of ONE ciphertext, bit-identical), but its
 * working buffers live in a fixed array in the library's device memory image
 * (312 words per coefficient for ring degree <= 4096: 10.2 MB, held by every
 * GPU that loads the library until the process exits) instead of the
 * handle's workspace.  It calls no allocation routine.
 *   - ring degree above 4096, or a handle with ks_fine_depth > 0,
 *     ks_digit_primes = 5 or ks_coarse_from > 0 (the array holds three-prime
 *     key-switching digits only): HP_ERR_UNSUPPORTED, nothing launched;
 *   - ct_in / ct_out: device, [2][L][N], 16-byte aligned; ct_out may alias ct_in;
 *   - the handle's device must be current (HP_ERR_ARG otherwise);
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture;
 *     after a device reset (cudaDeviceReset) the next call on that device
 *     finds a new context and looks the address up again, so make it, too,
 *     before any capture;
 *   - all calls share the one array and it keeps the last call's contents;
 *     nothing in it needs to start at zero.  Calls whose GPU work overlaps
 *     (different streams, or several host threads) race on it: order them.
 * Asynchronous on `stream` like hp_run. */
int hp_square_noalloc(hp_handle* h, const uint64_t* ct_in, uint64_t* ct_out, void* stream);

/* ---- measurement -----------------------------------------------------------
 * Per-kernel-class timing with CUDA events recorded on the launching stream
 * around every launch of the classes in `class_mask` (bit c = class c):
 *   0 NTT forward columns   1 NTT forward rows    2 NTT inverse rows
 *   3 NTT inverse columns   4 exact lift          5 tensor
 *   6 scale-and-round       7 digit expansion     8 key-switch MAC
 *   9 mod-down
 * hp_profile() synchronises, clears the records and sets the mask (0 = off).
 * hp_profile_read() synchronises and returns the summed event time, the
 * number of launches and the summed algorithmic work of class `cls` (NTT:
 * butterflies; lift / scale-and-round: coefficients; MAC: multiply-adds;
 * others: words). */
int hp_profile(hp_handle* h, uint32_t class_mask);
int hp_profile_read(hp_handle* h, int cls, double* ms_total, uint64_t* launches, double* work_total);

/* Tensor-core probe (no counterpart in the paper): one CTA computes
 * D = A B^T with tcgen05.mma kind::f16 (accumulator in tensor memory) for
 * A [128][112] and B [n][112] matrices of f16 (bf16 = 0) or bf16 (bf16 = 1)
 * values (host memory, row-major 16-bit patterns),
 * D [128][n] f32 (host), n a multiple of 16 in [16, 256].  Used by the tests to
 * check the operand layout and that sums of products of 8-bit integers are
 * exact.  Synchronous; HP_ERR_TIMEOUT if the MMA did not complete within the
 * kernel's bounded wait. */
int hp_probe_tc_gemm(const uint16_t* A, const uint16_t* B, float* D, int n, int bf16);

/* Failure path of the tensor-core kernels' bounded waits, exercised without a
 * fault (no counterpart in the paper): the probe issues no MMA, so its mbarrier
 * never completes; after `polls` polls (1 .. 2^20) the kernel sets its status
 * word, frees its tensor memory and returns.  Returns HP_ERR_TIMEOUT when the
 * wait expired as intended (the device stays usable), HP_ERR_ARG for a bad
 * count. */
int hp_probe_tc_timeout(uint32_t polls);

/* Register-only peak probe on the current device (no handle needed):
 * kind 0 = the 64-bit Shoup butterfly of the NTT kernels (butterflies/s),
 * kind 1 = the 64x64->128-bit multiply-accumulate of the base conversions and
 * key switching (MACs/s), kind 2 = the same Shoup butterfly on 32-bit words
 * for a 30-bit prime (butterflies/s; no kernel of the library uses it: it
 * measures what a narrower residue word would buy).  Launches 8 blocks of 256
 * threads per SM. */
int hp_probe_peak(int kind, double* per_second);

#ifdef __cplusplus
}
#endif

#endif /* LIBHP_HP_H */
