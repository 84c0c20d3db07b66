"""Textbook-BFV oracle (plain single-threaded C++), wrapped with ctypes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA library never calls it, and it never calls the CUDA library.

The C++ source (``bfv_oracle.cpp``) restates the paper's equality predicate
(Sec. 2.1.7, Eq. 3: EQ(x, y) = 1 - (x - y)^(p-1)), computed by
exponentiation by squaring (Sec. 4.3.1: ceil(log2(p-1)) = 16 multiplications for
p = 65537), over textbook BFV with the parameters of Sec. 5.1 (N = 32768,
log QP = 881, p = 65537).  Every function below states which operation it
exposes; the arithmetic lives in the C++ file.

Array conventions (numpy):
  ciphertext  uint64 [2][L][N]  residues mod q_0..q_{L-1}, coefficient domain
  relin key   uint64 [D][2][L+1][N]  residues mod q_0..q_{L-1}, P; D = ceil(L / dp)
              key-switching digits, each the residue mod a group of dp data primes
              (dp = 3 unless chosen otherwise); the per-prime key of the first
              levels (fine_depth > 0) has D = L
  secret key  int8 [N] in {-1, 0, 1}
  slots       uint32 [N] values mod t
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfv_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i8p = ctypes.POINTER(ctypes.c_int8)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _compile(path: str, flags, force: bool) -> str:
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    os.makedirs(_BUILD, exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", *flags, "-o", tmp, _SRC], check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (no CUDA involved)."""
    return _compile(_LIB_PATH, ["-Wall"], force)


def build_mutant(k: int, force: bool = False) -> str:
    """A separate copy of the oracle with planted mistake number k (1..16, listed
    at the top of bfv_oracle.cpp), for the tests that check that the pins catch
    such mistakes.  Never loaded by anything but those tests."""
    if not 1 <= k <= 16:
        raise ValueError("no planted mistake %d" % k)
    return _compile(os.path.join(_BUILD, "liboracle_mutant%d.so" % k), ["-DORC_MUTANT=%d" % k], force)


_lib = None
_libs = {}


def galois_elements(logn: int):
    """Elements of the rotate-and-add reduction (Sec. 4.2.2), in order: 3^(2^i)
    mod 2N for i = logN-2 .. 0 (row rotations by N/4 .. 1), then 2N - 1 (row
    exchange)."""
    twoN = 2 << logn
    return [pow(3, 1 << i, twoN) for i in range(logn - 2, -1, -1)] + [twoN - 1]


def _load(path=None):
    """The oracle library (built if needed), or the one at `path` (a planted-
    mistake copy from build_mutant)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    if path is not None and path in _libs:
        return _libs[path]
    lib = ctypes.CDLL(build() if path is None else path)
    V = ctypes.c_void_p
    sig = {
        "orc_default_primes": (ctypes.c_int, [ctypes.c_int, _u64p, _u64p]),
        "orc_create": (V, [ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_uint64, ctypes.c_uint64]),
        "orc_destroy": (None, [V]),
        "orc_num_digits": (ctypes.c_int, [V]),
        "orc_export_big": (ctypes.c_int, [V, ctypes.c_int, _u64p, ctypes.c_int]),
        "orc_philox": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u32p]),
        "orc_philox_raw": (None, [_u32p, _u32p, _u32p]),
        "orc_ntt_forward": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, _u64p]),
        "orc_ntt_inverse": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, _u64p]),
        "orc_polymul_small": (ctypes.c_int, [V, _i64p, _i64p, _i64p]),
        "orc_encode": (ctypes.c_int, [V, _u32p, _u64p]),
        "orc_decode": (ctypes.c_int, [V, _u64p, _u32p]),
        "orc_keygen": (ctypes.c_int, [V, ctypes.c_uint64, _i8p, _u64p]),
        "orc_encrypt": (ctypes.c_int, [V, _i8p, _u32p, ctypes.c_uint64, ctypes.c_uint32, _u64p]),
        "orc_decrypt": (ctypes.c_int, [V, _i8p, _u64p, _u32p, ctypes.POINTER(ctypes.c_double)]),
        "orc_sub": (ctypes.c_int, [V, _u64p, _u64p, _u64p]),
        "orc_sub_const": (ctypes.c_int, [V, _u64p, ctypes.c_uint64, _u64p]),
        "orc_one_minus": (ctypes.c_int, [V, _u64p, _u64p]),
        "orc_mul_relin": (ctypes.c_int, [V, _u64p, _u64p, _u64p]),
        "orc_eq": (ctypes.c_int, [V, _u64p, _u64p, ctypes.c_uint64, ctypes.c_int, _u64p]),
        "orc_square_chain": (ctypes.c_int, [V, _u64p, ctypes.c_int, _u64p]),
        "orc_eq_plain": (ctypes.c_int, [V, _u64p, _u32p, ctypes.c_int, _u64p]),
        "orc_lt_coefficients": (ctypes.c_int, [V, _u32p]),
        "orc_linear": (ctypes.c_int, [V, _u64p, ctypes.c_int, _u64p, ctypes.c_uint64, _u64p]),
        "orc_lt": (ctypes.c_int, [V, _u64p, _u64p, _u64p]),
        "orc_tensor_round": (ctypes.c_int, [V, _u64p, _u64p, _u64p]),
        "orc_relin": (ctypes.c_int, [V, _u64p, _u64p]),
        "orc_galois_keygen": (ctypes.c_int, [V, ctypes.c_uint64, _i8p, ctypes.c_uint64, _u64p]),
        "orc_automorphism": (ctypes.c_int, [V, _u64p, ctypes.c_uint64, _u64p]),
        "orc_rotate": (ctypes.c_int, [V, _u64p, ctypes.c_uint64, _u64p]),
        "orc_rotate_sum": (ctypes.c_int, [V, _u64p, ctypes.c_int, ctypes.c_int, _u64p]),
        "orc_mul_plain": (ctypes.c_int, [V, _u64p, _u64p, _u64p]),
        "orc_between": (ctypes.c_int, [V, _u64p, ctypes.c_uint64, ctypes.c_uint64, _u64p]),
        "orc_set_digits": (ctypes.c_int, [V, ctypes.c_int, ctypes.c_int]),
        "orc_fine_key": (ctypes.c_int, [V, _u64p]),
        "orc_set_coarse": (ctypes.c_int, [V, ctypes.c_int]),
        "orc_coarse_key": (ctypes.c_int, [V, _u64p]),
        "orc_mul_relin_depth": (ctypes.c_int, [V, _u64p, ctypes.c_int, _u64p, ctypes.c_int, _u64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    else:
        _libs[path] = lib
    return lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


T_DEFAULT = 65537
L_DEFAULT = 15


def default_primes(L: int = L_DEFAULT):
    """Data primes q_0 > ... > q_{L-1} (largest below 2^55, = 1 mod 2^16) and the
    special prime P (largest below 2^56, = 1 mod 2^16).  log2(Q P) ~ 881 for
    L = 15 (paper Sec. 5.1)."""
    lib = _load()
    q = np.zeros(L, dtype=np.uint64)
    P = np.zeros(1, dtype=np.uint64)
    if lib.orc_default_primes(L, _p(q, ctypes.c_uint64), _p(P, ctypes.c_uint64)) != 0:
        raise RuntimeError("prime search failed")
    return [int(x) for x in q], int(P[0])


def philox(seed: int, k: int, j: int, obj: int, dom: int):
    """Philox4x32-10 output for counter (k, j, obj, dom), key = 64-bit seed."""
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox(seed, k, j, obj, dom, _p(out, ctypes.c_uint32))
    return [int(x) for x in out]


def philox_raw(ctr4, key2):
    ctr = _c(ctr4, np.uint32)
    key = _c(key2, np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox_raw(_p(ctr, ctypes.c_uint32), _p(key, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return [int(x) for x in out]


def ntt_forward(logn: int, m: int, a) -> np.ndarray:
    """Negacyclic transform A_j = sum_k a_k psi^((2j+1)k) mod m (natural order)."""
    x = _c(a, np.uint64).copy()
    _load().orc_ntt_forward(logn, m, _p(x, ctypes.c_uint64))
    return x


def ntt_inverse(logn: int, m: int, a) -> np.ndarray:
    x = _c(a, np.uint64).copy()
    _load().orc_ntt_inverse(logn, m, _p(x, ctypes.c_uint64))
    return x


class Oracle:
    """One BFV parameter set (ring degree 2^logn, data primes q, special prime P,
    plaintext modulus t).  Holds the relinearisation key after keygen().

    Key switching: the relinearisation and Galois keys have digits of `dp`
    consecutive data primes (3 by default); products whose multiplicative depth
    is at most `fine_depth` are relinearised with a second key of one prime per
    digit instead (0 = never), and products at depth `coarse_from` or more with a
    third key of two digits, data primes 0..7 and 8..14 (0 = never).  Depths
    count from fresh ciphertexts (depth 0)."""

    def __init__(self, logn: int, q=None, P=None, t: int = T_DEFAULT, L: int = L_DEFAULT, lib_path=None,
                 dp: int = 3, fine_depth: int = 0, coarse_from: int = 0):
        if q is None:
            q, P = default_primes(L)
        self.lib = _load(lib_path)
        self.logn = logn
        self.N = 1 << logn
        self.q = [int(x) for x in q]
        self.L = len(self.q)
        self.P = int(P)
        self.t = int(t)
        qa = np.array(self.q, dtype=np.uint64)
        self.h = self.lib.orc_create(logn, self.L, _p(qa, ctypes.c_uint64), self.P, self.t)
        if not self.h:
            raise RuntimeError("orc_create failed")
        if self.lib.orc_set_digits(self.h, dp, fine_depth) != 0:
            raise ValueError("digit grouping must be 1..L data primes and fine_depth >= 0")
        if self.lib.orc_set_coarse(self.h, coarse_from) != 0:
            raise ValueError("coarse_from must be 0 or above fine_depth")
        self.dp, self.fine_depth, self.coarse_from = dp, fine_depth, coarse_from
        self.D = self.lib.orc_num_digits(self.h)
        self.s = None
        self.rk = None

    def close(self):
        if self.h:
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- constants ---------------------------------------------------------
    def export_big(self, which: int) -> int:
        buf = np.zeros(40, dtype=np.uint64)
        n = self.lib.orc_export_big(self.h, which, _p(buf, ctypes.c_uint64), 40)
        return sum(int(buf[i]) << (64 * i) for i in range(n))

    @property
    def Q(self) -> int:
        return self.export_big(0)

    @property
    def QP(self) -> int:
        return self.export_big(1)

    @property
    def Delta(self) -> int:
        return self.export_big(2)

    # -- encoding ------------------------------------------------------------
    def encode(self, slots) -> np.ndarray:
        s = _c(slots, np.uint32)
        m = np.zeros(self.N, dtype=np.uint64)
        self.lib.orc_encode(self.h, _p(s, ctypes.c_uint32), _p(m, ctypes.c_uint64))
        return m

    def decode(self, m) -> np.ndarray:
        mm = _c(m, np.uint64)
        s = np.zeros(self.N, dtype=np.uint32)
        self.lib.orc_decode(self.h, _p(mm, ctypes.c_uint64), _p(s, ctypes.c_uint32))
        return s

    def polymul_small(self, a, b) -> np.ndarray:
        A = _c(a, np.int64)
        B = _c(b, np.int64)
        out = np.zeros(self.N, dtype=np.int64)
        if self.lib.orc_polymul_small(self.h, _p(A, ctypes.c_int64), _p(B, ctypes.c_int64), _p(out, ctypes.c_int64)) != 0:
            raise OverflowError("product does not fit int64")
        return out

    # -- keys and encryption ---------------------------------------------------
    def keygen(self, seed: int):
        """Secret key and relinearisation key from `seed` (stored for later ops)."""
        s = np.zeros(self.N, dtype=np.int8)
        rk = np.zeros((self.D, 2, self.L + 1, self.N), dtype=np.uint64)
        self.lib.orc_keygen(self.h, seed, _p(s, ctypes.c_int8), _p(rk, ctypes.c_uint64))
        self.s, self.rk = s, rk
        return s, rk

    def encrypt(self, slots, seed: int, ct_index: int = 0, s=None) -> np.ndarray:
        s = self.s if s is None else _c(s, np.int8)
        sl = _c(slots, np.uint32)
        ct = np.zeros((2, self.L, self.N), dtype=np.uint64)
        self.lib.orc_encrypt(self.h, _p(s, ctypes.c_int8), _p(sl, ctypes.c_uint32), seed, ct_index, _p(ct, ctypes.c_uint64))
        return ct

    def decrypt(self, ct, s=None, with_noise: bool = False):
        s = self.s if s is None else _c(s, np.int8)
        c = _c(ct, np.uint64)
        out = np.zeros(self.N, dtype=np.uint32)
        nb = ctypes.c_double(0.0)
        self.lib.orc_decrypt(self.h, _p(s, ctypes.c_int8), _p(c, ctypes.c_uint64), _p(out, ctypes.c_uint32), ctypes.byref(nb))
        return (out, nb.value) if with_noise else out

    # -- homomorphic operations --------------------------------------------------
    def _ct_out(self, shape=None):
        return np.zeros(shape or (2, self.L, self.N), dtype=np.uint64)

    def sub(self, x, y):
        X, Y, out = _c(x, np.uint64), _c(y, np.uint64), self._ct_out()
        self.lib.orc_sub(self.h, _p(X, ctypes.c_uint64), _p(Y, ctypes.c_uint64), _p(out, ctypes.c_uint64))
        return out

    def sub_const(self, x, v: int):
        X, out = _c(x, np.uint64), self._ct_out()
        self.lib.orc_sub_const(self.h, _p(X, ctypes.c_uint64), v, _p(out, ctypes.c_uint64))
        return out

    def one_minus(self, x):
        X, out = _c(x, np.uint64), self._ct_out()
        self.lib.orc_one_minus(self.h, _p(X, ctypes.c_uint64), _p(out, ctypes.c_uint64))
        return out

    def mul_relin(self, a, b, depth_a: int = 0, depth_b: int = 0):
        """a * b relinearised; the operands lie at multiplicative depths depth_a and
        depth_b (0 = fresh), the product at max(depth_a, depth_b) + 1, which selects
        the relinearisation key."""
        A, B, out = _c(a, np.uint64), _c(b, np.uint64), self._ct_out()
        if depth_a == 0 and depth_b == 0:
            rc = self.lib.orc_mul_relin(self.h, _p(A, ctypes.c_uint64), _p(B, ctypes.c_uint64), _p(out, ctypes.c_uint64))
        else:
            rc = self.lib.orc_mul_relin_depth(self.h, _p(A, ctypes.c_uint64), depth_a, _p(B, ctypes.c_uint64), depth_b,
                                              _p(out, ctypes.c_uint64))
        if rc != 0:
            raise RuntimeError("relinearisation key not set")
        return out

    def fine_key(self) -> np.ndarray:
        """The per-prime relinearisation key (uint64 [L][2][L+1][N]) made by keygen()
        when fine_depth > 0."""
        out = np.zeros((self.L, 2, self.L + 1, self.N), dtype=np.uint64)
        if self.lib.orc_fine_key(self.h, _p(out, ctypes.c_uint64)) != 0:
            raise RuntimeError("no per-prime key (fine_depth = 0)")
        return out

    def coarse_key(self) -> np.ndarray:
        """The two-digit relinearisation key (uint64 [2][2][L+1][N]) made by keygen()
        when coarse_from > 0."""
        out = np.zeros((2, 2, self.L + 1, self.N), dtype=np.uint64)
        if self.lib.orc_coarse_key(self.h, _p(out, ctypes.c_uint64)) != 0:
            raise RuntimeError("no two-digit key (coarse_from = 0)")
        return out

    def eq(self, x, y=None, const_val: int = 0, squarings: int = 16):
        """EQ(x, y) = 1 - (x - y)^(2^squarings); y None => compare with const_val."""
        X, out = _c(x, np.uint64), self._ct_out()
        yp = None
        if y is not None:
            Y = _c(y, np.uint64)
            yp = _p(Y, ctypes.c_uint64)
        if self.lib.orc_eq(self.h, _p(X, ctypes.c_uint64), yp, const_val, squarings, _p(out, ctypes.c_uint64)) != 0:
            raise RuntimeError("relinearisation key not set")
        return out

    def eq_plain(self, x, cslots, squarings: int = 16):
        """EQ(x, c) with one plaintext constant per slot: x - (Delta encode(c), 0),
        the squarings, then "1 -"."""
        X, C, out = _c(x, np.uint64), _c(cslots, np.uint32), self._ct_out()
        if self.lib.orc_eq_plain(self.h, _p(X, ctypes.c_uint64), _p(C, ctypes.c_uint32), squarings,
                                 _p(out, ctypes.c_uint64)) != 0:
            raise RuntimeError("relinearisation key not set")
        return out

    def lt_coefficients(self) -> np.ndarray:
        """h_m = c_{2m+1} of the LT polynomial (Eq. 4), m < (t-1)/2."""
        out = np.zeros((self.t - 1) // 2, dtype=np.uint32)
        self.lib.orc_lt_coefficients(self.h, _p(out, ctypes.c_uint32))
        return out

    def linear(self, cts, coef, coef0: int = 0):
        """sum_i coef[i] cts[i] + (Delta coef0, 0), coefficients < t."""
        C = _c(cts, np.uint64)
        k = _c(coef, np.uint64)
        out = self._ct_out()
        self.lib.orc_linear(self.h, _p(C, ctypes.c_uint64), len(k), _p(k, ctypes.c_uint64), coef0, _p(out, ctypes.c_uint64))
        return out

    def group_by_masks(self, x, consts):
        """GROUP BY masks (Sec. 4.2.2): EQ(x, c_k) for each constant c_k."""
        return np.stack([self.eq(x, None, const_val=int(c)) for c in consts])

    def in_set(self, x, consts, masks=None):
        """IN (Eq. 6): the sum of the EQ masks of x against every constant."""
        m = self.group_by_masks(x, consts) if masks is None else masks
        return self.linear(m, [1] * len(m))

    # -- rotations, COUNT / SUM (Sec. 4.2.2) -----------------------------------------
    def galois_elements(self):
        return galois_elements(self.logn)

    def galois_keygen(self, seed: int, g: int, s=None):
        """Galois key for element g (uint64 [D][2][L+1][N]); kept for rotations."""
        s = self.s if s is None else _c(s, np.int8)
        gk = np.zeros((self.D, 2, self.L + 1, self.N), dtype=np.uint64)
        if self.lib.orc_galois_keygen(self.h, seed, _p(s, ctypes.c_int8), g, _p(gk, ctypes.c_uint64)) != 0:
            raise ValueError("Galois element must be odd and < 2N")
        return gk

    def automorphism(self, x, g: int):
        """tau_g(ct) without key switching (decrypts under tau_g(s))."""
        X, out = _c(x, np.uint64), self._ct_out()
        if self.lib.orc_automorphism(self.h, _p(X, ctypes.c_uint64), g, _p(out, ctypes.c_uint64)) != 0:
            raise ValueError("Galois element must be odd and < 2N")
        return out

    def rotate(self, x, g: int):
        X, out = _c(x, np.uint64), self._ct_out()
        if self.lib.orc_rotate(self.h, _p(X, ctypes.c_uint64), g, _p(out, ctypes.c_uint64)) != 0:
            raise RuntimeError("Galois key for %d not generated" % g)
        return out

    def rotate_sum(self, x, row_steps=None, swap: bool = True):
        """Rotate-and-add reduction: every slot ends with the sum of all slots."""
        rs = self.logn - 1 if row_steps is None else row_steps
        X, out = _c(x, np.uint64), self._ct_out()
        rc = self.lib.orc_rotate_sum(self.h, _p(X, ctypes.c_uint64), rs, int(swap), _p(out, ctypes.c_uint64))
        if rc != 0:
            raise RuntimeError("orc_rotate_sum failed (%d)" % rc)
        return out

    # -- JOIN by Extract + Broadcast (Sec. 4.2.2) ------------------------------------
    def mul_plain(self, x, m):
        """ct * m for a plaintext polynomial m (uint64 [N], coefficients < t)."""
        X, M, out = _c(x, np.uint64), _c(m, np.uint64), self._ct_out()
        if self.lib.orc_mul_plain(self.h, _p(X, ctypes.c_uint64), _p(M, ctypes.c_uint64), _p(out, ctypes.c_uint64)) != 0:
            raise ValueError("plaintext coefficients must be < t")
        return out

    def extract_broadcast(self, column, row: int):
        """Extract row `row` of a column of ciphertexts (slot row % N of ciphertext
        row // N: multiply by the plaintext unit vector of that slot) and broadcast
        it to every slot by the rotate-and-add reduction."""
        unit = np.zeros(self.N, dtype=np.uint32)
        unit[row % self.N] = 1
        return self.rotate_sum(self.mul_plain(column[row // self.N], self.encode(unit)))

    def join(self, a_key, b_key, b_attrs, n_rows: int):
        """Equi-join A.key = B.key over the first n_rows rows of B (Sec. 4.2.2):
        mask_r = EQ(A.key, Broadcast(B.key[r])); with attributes, out[k] =
        sum_r mask_r * Broadcast(B.attr_k[r]); without, out = sum_r mask_r.  A
        mask is an EQ result at depth 16 (Eq. 3), so its product with a
        broadcast attribute lies at depth 17 and is relinearised with the key of
        that depth."""
        kb = [self.extract_broadcast(b_key, r) for r in range(n_rows)]
        vb = [[self.extract_broadcast(col, r) for r in range(n_rows)] for col in b_attrs]
        outs = []
        for a in a_key:
            masks = [self.eq(a, kb[r]) for r in range(n_rows)]
            if not b_attrs:
                outs.append(self.linear(np.stack(masks), [1] * n_rows)[None])
            else:
                outs.append(np.stack([self.linear(np.stack([self.mul_relin(masks[r], vb[k][r], depth_a=16)
                                                            for r in range(n_rows)]),
                                                  [1] * n_rows) for k in range(len(b_attrs))]))
        return np.stack(outs, axis=1)  # [max(1, n_attr)][n_a][2][L][N]

    def lt(self, x, y):
        """LT(x, y) (Eq. 4) by the baby-step / giant-step schedule of the library."""
        X, Y, out = _c(x, np.uint64), _c(y, np.uint64), self._ct_out()
        rc = self.lib.orc_lt(self.h, _p(X, ctypes.c_uint64), _p(Y, ctypes.c_uint64), _p(out, ctypes.c_uint64))
        if rc != 0:
            raise RuntimeError("orc_lt failed (%d)" % rc)
        return out

    def between(self, x, lo: int, hi: int):
        """BETWEEN: (1 - LT(x, lo)) (1 - LT(hi, x)) = [lo <= x <= hi] for constants lo <= hi."""
        X, out = _c(x, np.uint64), self._ct_out()
        rc = self.lib.orc_between(self.h, _p(X, ctypes.c_uint64), lo, hi, _p(out, ctypes.c_uint64))
        if rc != 0:
            raise RuntimeError("orc_between failed (%d)" % rc)
        return out

    def square_chain(self, x, squarings: int):
        X, out = _c(x, np.uint64), self._ct_out()
        if self.lib.orc_square_chain(self.h, _p(X, ctypes.c_uint64), squarings, _p(out, ctypes.c_uint64)) != 0:
            raise RuntimeError("relinearisation key not set")
        return out

    def tensor_round(self, a, b):
        """round(t d_j / Q) mod Q for the tensor (d0, d1, d2) of a and b."""
        A, B = _c(a, np.uint64), _c(b, np.uint64)
        out = np.zeros((3, self.L, self.N), dtype=np.uint64)
        self.lib.orc_tensor_round(self.h, _p(A, ctypes.c_uint64), _p(B, ctypes.c_uint64), _p(out, ctypes.c_uint64))
        return out

    def relin(self, d3):
        D, out = _c(d3, np.uint64), self._ct_out()
        if self.lib.orc_relin(self.h, _p(D, ctypes.c_uint64), _p(out, ctypes.c_uint64)) != 0:
            raise RuntimeError("relinearisation key not set")
        return out


def crt_to_int(residues, moduli) -> int:
    """Plain CRT of one coefficient (Python integers) — a helper for tests."""
    M = 1
    for m in moduli:
        M *= m
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M
