"""ctypes binding of libhp (include/hp.h): argument marshalling only.

Every step of the hot path runs in the CUDA kernels of ``libhp.so``; this
module converts torch tensors / numpy arrays to pointers and return codes to
exceptions.  It fails loudly when the shared library is missing: there is no
CPU fallback.

Tensor conventions: ciphertexts are torch.int64 CUDA tensors of shape
[n, 2, L, N] holding the uint64 residue words bit for bit.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhp.so")

HP_OK = 0
HP_ERR_ARG = -1
HP_ERR_DEPTH = -2
HP_ERR_OOM = -3
HP_ERR_CUDA = -4
HP_ERR_TIMEOUT = -5
HP_ERR_UNSUPPORTED = -6
HP_ERR_STATE = -7
_NAMES = {v: k for k, v in list(globals().items()) if k.startswith("HP_ERR_") or k == "HP_OK"}

HP_EQ_CT_CT = 0
HP_EQ_CT_CONST = 1
HP_SELECT = 2
HP_SQUARE = 3
HP_LT = 4

# hp_budget_op: operations of the static noise-budget estimate
HP_BUDGET_EQ = 0
HP_BUDGET_SELECT = 1
HP_BUDGET_SQUARE = 2
HP_BUDGET_LT = 3
HP_BUDGET_BETWEEN = 4
HP_BUDGET_PRODUCT = 5
HP_BUDGET_ROTATE_SUM = 6
HP_BUDGET_MARGIN = 10.0

L = 15
T = 65537

EXPORTED = [
    "hp_default_params", "hp_create", "hp_set_relin_key", "hp_run", "hp_run_batched", "hp_backward",
    "hp_destroy", "hp_last_error", "hp_keygen", "hp_encrypt", "hp_decrypt", "hp_launch_count",
    "hp_check_status", "hp_profile", "hp_profile_read", "hp_probe_peak", "hp_tile_size",
    "hp_square_noalloc", "hp_autotune", "hp_lt_coefficients", "hp_eq_fanout",
    "hp_galois_elements", "hp_galois_keygen", "hp_set_galois_keys", "hp_rotate_sum",
    "hp_extract_broadcast", "hp_join", "hp_ct_sum", "hp_probe_tc_gemm", "hp_probe_tc_timeout", "hp_between",
    "hp_set_relin_key_fine", "hp_keygen_fine", "hp_budget_estimate", "hp_select_mask",
    "hp_set_relin_key_coarse", "hp_keygen_coarse",
]

PROFILE_CLASSES = ["ntt_fwd_cols", "ntt_fwd_rows", "ntt_inv_rows", "ntt_inv_cols", "lift", "tensor",
                   "scale_round", "automorph", "ks_mac", "moddown"]
KERNEL_OF_CLASS = ["k_ntt_fwd_cols", "k_ntt_fwd_rows(_sq)", "k_ntt_inv_rows", "k_ntt_inv_cols(+mod-down)", "k_lift_tc",
                   "k_tensor_gen",
                   "k_scale_round_tc", "k_automorph", "k_ks_mac", "k_moddown"]


DIGIT_PRIMES = 3  # default data primes per key-switching digit (D = L / 3 digits); 5 is the other choice


class HpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_NAMES.get(code, "HP_ERR"), code, msg))
        self.code = code


class hp_params(ctypes.Structure):
    _fields_ = [
        ("log_n", ctypes.c_uint32),
        ("L", ctypes.c_uint32),
        ("q", ctypes.POINTER(ctypes.c_uint64)),
        ("P", ctypes.c_uint64),
        ("t", ctypes.c_uint64),
        ("max_depth", ctypes.c_uint32),
        ("ks_fine_depth", ctypes.c_uint32),
        ("ks_digit_primes", ctypes.c_uint32),
        ("ks_coarse_from", ctypes.c_uint32),
    ]


class hp_instance(ctypes.Structure):
    _fields_ = [
        ("ct_offset", ctypes.c_uint64),
        ("n_ct", ctypes.c_uint32),
        ("slot_offset", ctypes.c_uint32),
        ("n_slots", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("const_val", ctypes.c_uint64),
    ]


_lib = None


def load():
    """Load libhp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhp.so not built: run paper_2602_24271_b300/build.py (or __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    V, P64, SZ = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t
    H = ctypes.c_void_p
    sig = {
        "hp_default_params": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
        "hp_create": (ctypes.c_int, [ctypes.POINTER(hp_params), P64, SZ, ctypes.POINTER(H)]),
        "hp_set_relin_key": (ctypes.c_int, [H, P64]),
        "hp_run": (ctypes.c_int, [H, ctypes.c_int, P64, P64, ctypes.c_uint64, P64, SZ, V]),
        "hp_run_batched": (ctypes.c_int, [H, ctypes.c_int, ctypes.POINTER(hp_instance), SZ, P64, P64, P64, SZ, V]),
        "hp_backward": (ctypes.c_int, [H, ctypes.c_int, P64, P64, SZ, V]),
        "hp_destroy": (None, [H]),
        "hp_last_error": (ctypes.c_char_p, [H]),
        "hp_keygen": (ctypes.c_int, [H, ctypes.c_uint64, V, P64, V]),
        "hp_encrypt": (ctypes.c_int, [H, V, V, SZ, ctypes.c_uint64, ctypes.c_uint32, P64, V]),
        "hp_decrypt": (ctypes.c_int, [H, V, P64, SZ, V, V]),
        "hp_launch_count": (ctypes.c_uint64, [H]),
        "hp_check_status": (ctypes.c_int, [H]),
        "hp_profile": (ctypes.c_int, [H, ctypes.c_uint32]),
        "hp_profile_read": (ctypes.c_int, [H, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]),
        "hp_probe_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "hp_tile_size": (ctypes.c_size_t, [H]),
        "hp_square_noalloc": (ctypes.c_int, [H, P64, P64, V]),
        "hp_autotune": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_size_t)]),
        "hp_lt_coefficients": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
        "hp_eq_fanout": (ctypes.c_int, [H, P64, SZ, ctypes.POINTER(ctypes.c_uint64), SZ, P64, P64, V]),
        "hp_galois_elements": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
        "hp_galois_keygen": (ctypes.c_int, [H, ctypes.c_uint64, V, P64, V]),
        "hp_set_galois_keys": (ctypes.c_int, [H, P64]),
        "hp_rotate_sum": (ctypes.c_int, [H, P64, SZ, SZ, P64, V]),
        "hp_ct_sum": (ctypes.c_int, [H, P64, SZ, SZ, P64, V]),
        "hp_probe_tc_gemm": (ctypes.c_int, [V, V, V, ctypes.c_int, ctypes.c_int]),
        "hp_probe_tc_timeout": (ctypes.c_int, [ctypes.c_uint32]),
        "hp_between": (ctypes.c_int, [H, P64, SZ, ctypes.c_uint64, ctypes.c_uint64, P64, V]),
        "hp_extract_broadcast": (ctypes.c_int, [H, P64, SZ, SZ, SZ, P64, V]),
        "hp_join": (ctypes.c_int, [H, P64, SZ, P64, P64, SZ, SZ, P64, V]),
        "hp_set_relin_key_fine": (ctypes.c_int, [H, P64]),
        "hp_keygen_fine": (ctypes.c_int, [H, ctypes.c_uint64, V, P64, V]),
        "hp_set_relin_key_coarse": (ctypes.c_int, [H, P64]),
        "hp_keygen_coarse": (ctypes.c_int, [H, ctypes.c_uint64, V, P64, V]),
        "hp_budget_estimate": (ctypes.c_int, [ctypes.POINTER(hp_params), ctypes.c_int, ctypes.c_uint32,
                                              ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
        "hp_select_mask": (ctypes.c_int, [H, P64, P64, SZ, ctypes.c_uint32, ctypes.c_double, P64, V]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, h=None):
    if rc != HP_OK:
        msg = load().hp_last_error(h)
        raise HpError(rc, msg.decode() if msg else "")


def default_params(nq: int = L):
    lib = load()
    q = (ctypes.c_uint64 * nq)()
    P = ctypes.c_uint64()
    t = ctypes.c_uint64()
    _check(lib.hp_default_params(nq, q, ctypes.byref(P), ctypes.byref(t)))
    return [int(x) for x in q], int(P.value), int(t.value)


def _ptr(x) -> int:
    """Device/host address of a torch tensor or numpy array (None -> 0)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _stream(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Context:
    """One libhp handle: parameters, tables, relinearisation key, workspace."""

    def __init__(self, log_n: int, max_tile_ct: int = 0, max_depth: int = 17, q=None, P=None, t=T,
                 ks_fine_depth: int = 0, ks_digit_primes: int = DIGIT_PRIMES, ks_coarse_from: int = 0):
        import torch  # device memory and streams only

        self.torch = torch
        self.lib = load()
        if q is None:
            q, P, t = default_params()
        self.log_n, self.N, self.L = log_n, 1 << log_n, len(q)
        self.D = self.L // ks_digit_primes  # key-switching digits
        self.q, self.P, self.t = list(q), int(P), int(t)
        self._q = (ctypes.c_uint64 * len(q))(*q)
        self.ks_fine_depth, self.ks_digit_primes, self.ks_coarse_from = ks_fine_depth, ks_digit_primes, ks_coarse_from
        prm = hp_params(log_n, len(q), self._q, self.P, self.t, max_depth, ks_fine_depth, ks_digit_primes,
                        ks_coarse_from)
        h = ctypes.c_void_p()
        _check(self.lib.hp_create(ctypes.byref(prm), None, max_tile_ct, ctypes.byref(h)))
        self.h = h
        self.sk = None
        self.max_tile = max_tile_ct

    def close(self):
        if getattr(self, "h", None):
            self.lib.hp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shapes -------------------------------------------------------------
    def ct_empty(self, n: int, device="cuda"):
        return self.torch.empty((n, 2, self.L, self.N), dtype=self.torch.int64, device=device)

    # -- client helpers -------------------------------------------------------
    def keygen(self, seed: int, stream=None):
        torch = self.torch
        sk = torch.empty(self.N, dtype=torch.int8, device="cuda")
        rk = torch.empty((self.D, 2, self.L + 1, self.N), dtype=torch.int64, device="cuda")
        _check(self.lib.hp_keygen(self.h, seed, _ptr(sk), _ptr(rk), _stream(stream)), self.h)
        self.sk = sk
        return sk, rk

    def set_relin_key(self, rk):
        _check(self.lib.hp_set_relin_key(self.h, _ptr(rk)), self.h)

    def keygen_fine(self, seed: int, sk=None, stream=None):
        """The per-prime relinearisation key ([L, 2, L+1, N]) from the secret, installed."""
        torch = self.torch
        sk = self.sk if sk is None else sk
        rk = torch.empty((self.L, 2, self.L + 1, self.N), dtype=torch.int64, device="cuda")
        _check(self.lib.hp_keygen_fine(self.h, seed, _ptr(sk), _ptr(rk), _stream(stream)), self.h)
        return rk

    def set_relin_key_fine(self, rk):
        _check(self.lib.hp_set_relin_key_fine(self.h, _ptr(rk)), self.h)

    def keygen_coarse(self, seed: int, sk=None, stream=None):
        """The two-digit relinearisation key ([2, 2, L+1, N]) from the secret, installed."""
        torch = self.torch
        sk = self.sk if sk is None else sk
        rk = torch.empty((2, 2, self.L + 1, self.N), dtype=torch.int64, device="cuda")
        _check(self.lib.hp_keygen_coarse(self.h, seed, _ptr(sk), _ptr(rk), _stream(stream)), self.h)
        return rk

    def set_relin_key_coarse(self, rk):
        _check(self.lib.hp_set_relin_key_coarse(self.h, _ptr(rk)), self.h)

    def encrypt(self, slots, seed: int, ct_index0: int = 0, sk=None, stream=None):
        torch = self.torch
        sk = self.sk if sk is None else sk
        sl = torch.as_tensor(np.ascontiguousarray(slots, dtype=np.uint32).view(np.int32)).to("cuda")
        n = sl.numel() // self.N
        ct = self.ct_empty(n)
        _check(self.lib.hp_encrypt(self.h, _ptr(sk), _ptr(sl), n, seed, ct_index0, _ptr(ct), _stream(stream)), self.h)
        return ct

    def decrypt(self, ct, sk=None, stream=None) -> np.ndarray:
        torch = self.torch
        sk = self.sk if sk is None else sk
        n = ct.numel() // (2 * self.L * self.N)
        out = torch.empty(n * self.N, dtype=torch.int32, device="cuda")
        _check(self.lib.hp_decrypt(self.h, _ptr(sk), _ptr(ct), n, _ptr(out), _stream(stream)), self.h)
        return out.cpu().numpy().view(np.uint32).reshape(n, self.N)

    # -- hot path ---------------------------------------------------------------
    def run(self, op: int, x, y=None, const_val: int = 0, out=None, stream=None):
        """hp_run on device tensors (or host numpy arrays: synchronous)."""
        n = x.shape[0] if len(x.shape) == 4 else x.size // (2 * self.L * self.N)
        if out is None:
            out = self.ct_empty(n) if hasattr(x, "data_ptr") else np.empty_like(x)
        _check(self.lib.hp_run(self.h, op, _ptr(x), _ptr(y), const_val, _ptr(out), n, _stream(stream)), self.h)
        return out

    def eq(self, x, y=None, const_val: int = 0, out=None, stream=None):
        op = HP_EQ_CT_CT if y is not None else HP_EQ_CT_CONST
        return self.run(op, x, y, const_val, out, stream)

    def run_batched(self, op: int, instances, x, y=None, out=None, stream=None):
        n = x.shape[0]
        arr = (hp_instance * len(instances))()
        for i, ins in enumerate(instances):
            arr[i] = hp_instance(*ins) if not isinstance(ins, hp_instance) else ins
        if out is None:
            out = self.ct_empty(n)
        _check(self.lib.hp_run_batched(self.h, op, arr, len(instances), _ptr(x), _ptr(y), _ptr(out), n,
                                       _stream(stream)), self.h)
        return out

    def between(self, x, lo: int, hi: int, out=None, stream=None):
        """[lo <= x <= hi] slot-wise for plaintext bounds (device ciphertexts)."""
        n = x.shape[0]
        if out is None:
            out = self.ct_empty(n)
        _check(self.lib.hp_between(self.h, _ptr(x), n, lo, hi, _ptr(out), _stream(stream)), self.h)
        return out

    def select_mask(self, col, mask, mask_depth: int, mask_bits: float, out=None, stream=None):
        """SELECT (Eq. 5) with any mask: col * mask, relinearised; the mask lies at
        depth mask_depth with estimated budget mask_bits (see budget_estimate)."""
        n = col.shape[0]
        if out is None:
            out = self.ct_empty(n)
        _check(self.lib.hp_select_mask(self.h, _ptr(col), _ptr(mask), n, mask_depth, float(mask_bits), _ptr(out),
                                       _stream(stream)), self.h)
        return out

    def params(self, max_depth: int = 17) -> hp_params:
        return hp_params(self.log_n, self.L, self._q, self.P, self.t, max_depth, self.ks_fine_depth,
                         self.ks_digit_primes, self.ks_coarse_from)

    def eq_fanout(self, x, consts, masks=True, in_set=True, stream=None):
        """GROUP BY masks EQ(x, c_k) ([n_const, n_ct, 2, L, N]) and/or IN(x, consts)
        ([n_ct, 2, L, N]).  `masks` / `in_set`: True (allocate), False/None (skip)
        or a preallocated device tensor to write."""
        n = x.shape[0]
        k = len(consts)
        c = (ctypes.c_uint64 * max(1, k))(*[int(v) for v in consts])
        if masks is True:
            masks = self.torch.empty((k, n, 2, self.L, self.N), dtype=self.torch.int64, device="cuda")
        if in_set is True:
            in_set = self.ct_empty(n)
        m = masks if masks is not False else None
        io = in_set if in_set is not False else None
        _check(self.lib.hp_eq_fanout(self.h, _ptr(x), n, c, k, _ptr(m), _ptr(io), _stream(stream)), self.h)
        return m, io

    def galois_keygen(self, seed: int, sk=None, keep: bool = False, stream=None):
        """Galois keys of the rotate-and-add reduction (installed); returned as
        [logN, D, 2, L+1, N] (D key-switching digits) when `keep`."""
        sk = self.sk if sk is None else sk
        gk = self.torch.empty((self.log_n, self.D, 2, self.L + 1, self.N), dtype=self.torch.int64,
                              device="cuda") if keep else None
        _check(self.lib.hp_galois_keygen(self.h, seed, _ptr(sk), _ptr(gk), _stream(stream)), self.h)
        return gk

    def set_galois_keys(self, gk):
        _check(self.lib.hp_set_galois_keys(self.h, _ptr(gk)), self.h)

    def rotate_sum(self, x, group: int = 1, out=None, stream=None):
        """COUNT / SUM reduction: ceil(n / group) ciphertexts whose every slot holds
        the sum of all slots of a group of `group` consecutive ciphertexts."""
        n = x.shape[0]
        if out is None:
            out = self.ct_empty((n + max(group, 1) - 1) // max(group, 1))
        _check(self.lib.hp_rotate_sum(self.h, _ptr(x), n, group, _ptr(out), _stream(stream)), self.h)
        return out

    def ct_sum(self, x, group: int, out=None, stream=None):
        """Sums of groups of `group` consecutive ciphertexts (mod Q)."""
        n = x.shape[0]
        if out is None:
            out = self.ct_empty((n + max(group, 1) - 1) // max(group, 1))
        _check(self.lib.hp_ct_sum(self.h, _ptr(x), n, group, _ptr(out), _stream(stream)), self.h)
        return out

    def extract_broadcast(self, column, row0: int, n_rows: int = 1, out=None, stream=None):
        """Ciphertexts whose every slot holds row row0 + k of the column (k < n_rows)."""
        if out is None:
            out = self.ct_empty(n_rows)
        _check(self.lib.hp_extract_broadcast(self.h, _ptr(column), column.shape[0], row0, n_rows, _ptr(out),
                                             _stream(stream)), self.h)
        return out

    def join(self, a_key, b_key, b_attrs, n_rows: int, out=None, stream=None):
        """Equi-join A.key = B.key over the first n_rows rows of B: [max(1, n_attr), n_a] ciphertexts."""
        n_a = a_key.shape[0]
        attrs = self.torch.stack(list(b_attrs)).contiguous() if len(b_attrs) else None
        k = 0 if attrs is None else attrs.shape[0]
        if out is None:
            out = self.torch.empty((max(1, k), n_a, 2, self.L, self.N), dtype=self.torch.int64, device="cuda")
        _check(self.lib.hp_join(self.h, _ptr(a_key), n_a, _ptr(b_key), _ptr(attrs), k, n_rows, _ptr(out),
                                _stream(stream)), self.h)
        return out

    def backward(self, op: int, grad_out, grad_x, n: int):
        return self.lib.hp_backward(self.h, op, _ptr(grad_out), _ptr(grad_x), n, None)

    def autotune(self) -> int:
        t = ctypes.c_size_t()
        _check(self.lib.hp_autotune(self.h, ctypes.byref(t)), self.h)
        return int(t.value)

    def tile(self) -> int:
        return int(self.lib.hp_tile_size(self.h))

    def launch_count(self) -> int:
        return int(self.lib.hp_launch_count(self.h))

    def check_status(self):
        _check(self.lib.hp_check_status(self.h), self.h)

    def profile(self, class_mask: int):
        _check(self.lib.hp_profile(self.h, class_mask), self.h)

    def profile_read(self, cls: int):
        ms, n, w = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_double()
        _check(self.lib.hp_profile_read(self.h, cls, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)), self.h)
        return ms.value, int(n.value), w.value


def _bf16_bits(x: np.ndarray) -> np.ndarray:
    """bf16 bit patterns of values exactly representable in bf16 (top half of f32)."""
    return (np.ascontiguousarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def probe_tc_gemm(A: np.ndarray, B: np.ndarray, bf16: bool = False) -> np.ndarray:
    """Tensor-core probe: A [128, 112] and B [n, 112] (f16, or bf16 when `bf16`;
    given as numbers) -> A @ B.T as f32 [128, n]."""
    lib = load()
    if bf16:
        A, B = _bf16_bits(A), _bf16_bits(B)
    else:
        A = np.ascontiguousarray(A, dtype=np.float16).view(np.uint16)
        B = np.ascontiguousarray(B, dtype=np.float16).view(np.uint16)
    D = np.zeros((128, B.shape[0]), dtype=np.float32)
    _check(lib.hp_probe_tc_gemm(A.ctypes.data, B.ctypes.data, D.ctypes.data, B.shape[0], int(bf16)))
    return D


def galois_elements(log_n: int):
    """Galois elements of the rotate-and-add reduction, in application order."""
    lib = load()
    g = (ctypes.c_uint64 * log_n)()
    _check(lib.hp_galois_elements(log_n, g))
    return [int(v) for v in g]


def lt_coefficients() -> np.ndarray:
    """Odd coefficients of the LT polynomial (Eq. 4), computed by the library."""
    out = np.zeros(32768, dtype=np.uint32)
    _check(load().hp_lt_coefficients(out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return out


def budget_estimate(params: hp_params, op: int, in_depth: int = 0, in_bits: float = 0.0) -> float:
    """The library's static noise-budget estimate (bits) for `op` (HP_BUDGET_*);
    host computation, no GPU."""
    v = ctypes.c_double()
    _check(load().hp_budget_estimate(ctypes.byref(params), op, in_depth, float(in_bits), ctypes.byref(v)))
    return v.value


def probe_peak(kind: int) -> float:
    """Register-only peak rate on the current device: 0 = butterflies/s, 1 = MACs/s, 2 = 32-bit-word
    butterflies/s (a 30-bit prime)."""
    v = ctypes.c_double()
    _check(load().hp_probe_peak(kind, ctypes.byref(v)))
    return v.value


def to_u64(t) -> np.ndarray:
    """torch int64 tensor -> numpy uint64 view (host copy)."""
    return t.cpu().numpy().view(np.uint64)


def from_u64(a, device="cuda"):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)
