"""Plain CPU oracle for exact decimal multiplication (arXiv 2011.11524).

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library ``libdmul.so`` and its Python
binding) never imports, links or calls anything here; only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s cpu_baseline / reference leg do.  The oracle shares no code, header, table or
constant with the GPU path.

Everything computes by definition (Sec. 3.1-3.2 of the paper: convolution of the zero-padded limb
vectors, then the carry recurrence) or by an independent slow textbook route (two 63-bit primes,
plain ``%``, radix-2 with explicit bit reversal, the two-prime CRT of Sec. 8.2.2).  See
``oracle.c`` for the passage each function follows.

Limb vectors are little-endian base-10^9 ``uint32`` numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

B = 10**9


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (plain C, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           "-Wall", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        sz = ctypes.c_size_t
        lib.or_conv_schoolbook.argtypes = [u32p, sz, u32p, sz, u64p, ctypes.c_int]
        lib.or_conv_schoolbook.restype = None
        lib.or_conv_at.argtypes = [u32p, sz, u32p, sz, sz, u64p]
        lib.or_conv_at.restype = None
        lib.or_carry.argtypes = [u64p, sz, u32p]
        lib.or_carry.restype = ctypes.c_uint64
        lib.or_mul_schoolbook.argtypes = [u32p, sz, u32p, sz, u32p, ctypes.c_int]
        lib.or_mul_schoolbook.restype = ctypes.c_int
        lib.or_ntt_mul.argtypes = [u32p, sz, u32p, sz, u32p]
        lib.or_ntt_mul.restype = ctypes.c_int
        lib.or_powmod.argtypes = [ctypes.c_uint64] * 3
        lib.or_powmod.restype = ctypes.c_uint64
        lib.or_is_prime_mr.argtypes = [ctypes.c_uint64]
        lib.or_is_prime_mr.restype = ctypes.c_int
        lib.or_find_primes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p]
        lib.or_find_primes.restype = ctypes.c_int
        lib.or_primitive_root.argtypes = [ctypes.c_uint64]
        lib.or_primitive_root.restype = ctypes.c_uint64
        lib.or_dft_naive.argtypes = [u64p, sz, ctypes.c_uint64, ctypes.c_uint64, u64p]
        lib.or_dft_naive.restype = None
        lib.or_tau_dif.argtypes = [u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        lib.or_tau_dif.restype = None
        lib.or_tau_dit.argtypes = [u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
        lib.or_tau_dit.restype = None
        lib.or_cyclic_conv_mod.argtypes = [u64p, u64p, ctypes.c_int, ctypes.c_uint64]
        lib.or_cyclic_conv_mod.restype = None
        lib.or_fingerprint.argtypes = [u32p, sz, ctypes.c_uint64]
        lib.or_fingerprint.restype = ctypes.c_uint64
        lib.or_fingerprint_many.argtypes = [u64p, u64p, sz, u64p, sz, u64p, ctypes.c_int]
        lib.or_fingerprint_many.restype = None
        lib.or_transpose.argtypes = [u32p, sz, sz, u32p]
        lib.or_transpose.restype = None
        lib.or_permute_rows_rho.argtypes = [u32p, sz, sz, u32p]
        lib.or_permute_rows_rho.restype = None
        _lib = lib
        return lib


def _u32(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return a


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def default_threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


# ----------------------------------------------------------------------------------------------
# The product by definition
# ----------------------------------------------------------------------------------------------
def conv_schoolbook(x, y, nthreads: int | None = None) -> list[int]:
    """c_k = sum_{i+j=k} x_i y_j for k in [0, n+m) as Python ints (Sec. 3.1-3.2, exact)."""
    c = conv_schoolbook_words(x, y, nthreads)
    return [int(lo) | (int(hi) << 64) for lo, hi in c]


def conv_schoolbook_words(x, y, nthreads: int | None = None) -> np.ndarray:
    """Same as conv_schoolbook, as an (n+m, 2) uint64 array of (lo, hi) words."""
    lib = _load()
    x, y = _u32(x), _u32(y)
    L = len(x) + len(y)
    c = np.zeros((L, 2), dtype=np.uint64)
    lib.or_conv_schoolbook(_p32(x), len(x), _p32(y), len(y), _p64(c),
                           nthreads or default_threads())
    return c


def conv_at(x, y, k: int) -> int:
    """One exact coefficient c_k = sum_{i+j=k} x_i y_j (Sec. 3.2), for sampled checks."""
    lib = _load()
    x, y = _u32(x), _u32(y)
    out = np.zeros(2, dtype=np.uint64)
    lib.or_conv_at(_p32(x), len(x), _p32(y), len(y), k, _p64(out))
    return int(out[0]) | (int(out[1]) << 64)


def carry(c_words: np.ndarray) -> tuple[np.ndarray, int]:
    """Carry recurrence of Sec. 3.2 on (L, 2) uint64 coefficient words -> (z limbs, final carry)."""
    lib = _load()
    c = np.ascontiguousarray(c_words, dtype=np.uint64)
    L = c.shape[0]
    z = np.zeros(L, dtype=np.uint32)
    top = lib.or_carry(_p64(c), L, _p32(z))
    return z, int(top)


def mul_schoolbook(x, y, nthreads: int | None = None) -> np.ndarray:
    """Exact product x*y as n+m base-10^9 limbs (by definition: schoolbook + carry)."""
    lib = _load()
    x, y = _u32(x), _u32(y)
    z = np.zeros(len(x) + len(y), dtype=np.uint32)
    rc = lib.or_mul_schoolbook(_p32(x), len(x), _p32(y), len(y), _p32(z),
                               nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"or_mul_schoolbook failed: {rc}")
    return z


def mul_ntt(x, y) -> np.ndarray:
    """Exact product by the independent slow NTT route (two 63-bit primes, plain %)."""
    lib = _load()
    x, y = _u32(x), _u32(y)
    z = np.zeros(len(x) + len(y), dtype=np.uint32)
    if x is y or (len(x) == len(y) and x.ctypes.data == y.ctypes.data):
        rc = lib.or_ntt_mul(_p32(x), len(x), _p32(x), len(x), _p32(z))
    else:
        rc = lib.or_ntt_mul(_p32(x), len(x), _p32(y), len(y), _p32(z))
    if rc != 0:
        raise RuntimeError(f"or_ntt_mul failed: {rc}")
    return z


def mul(x, y, nthreads: int | None = None) -> np.ndarray:
    """Exact product: schoolbook when n*m is small enough, else the slow NTT route."""
    x, y = _u32(x), _u32(y)
    if len(x) * len(y) <= 4_000_000_000:
        return mul_schoolbook(x, y, nthreads)
    return mul_ntt(x, y)


def normalize(z: np.ndarray) -> np.ndarray:
    """Strip leading zero limbs, keeping at least one limb."""
    z = np.asarray(z, dtype=np.uint32)
    nz = np.flatnonzero(z)
    n = int(nz[-1]) + 1 if nz.size else 1
    return z[:n]


# ----------------------------------------------------------------------------------------------
# Fingerprints, primes, field transforms
# ----------------------------------------------------------------------------------------------
def fingerprint(limbs, q: int) -> int:
    """sum_i limbs[i] 10^(9 i) mod q by Horner's rule (q < 2^64)."""
    lib = _load()
    a = _u32(limbs)
    return int(lib.or_fingerprint(_p32(a), len(a), q))


def fingerprint_many(vectors, qs, nthreads: int | None = None) -> np.ndarray:
    """fingerprint(v, q) for every vector v and modulus q: a (len(vectors), len(qs)) array, the
    vectors spread over threads (each Horner chain stays on one thread)."""
    lib = _load()
    vecs = [_u32(v) for v in vectors]
    ptrs = np.array([v.ctypes.data for v in vecs], dtype=np.uint64)
    lens = np.array([len(v) for v in vecs], dtype=np.uint64)
    qa = np.array([int(q) for q in qs], dtype=np.uint64)
    out = np.zeros((len(vecs), len(qa)), dtype=np.uint64)
    if len(vecs) and len(qa):
        lib.or_fingerprint_many(_p64(ptrs), _p64(lens), len(vecs), _p64(qa), len(qa), _p64(out),
                                nthreads or default_threads())
    return out


def powmod(a: int, e: int, p: int) -> int:
    return int(_load().or_powmod(a, e, p))


def is_prime_mr(n: int) -> bool:
    return bool(_load().or_is_prime_mr(n))


def find_primes(w: int, n_min: int, l: int) -> list[int]:
    """FindPrimes(w, n_min, l) of Sec. 4.5, largest first."""
    out = np.zeros(l, dtype=np.uint64)
    rc = _load().or_find_primes(w, n_min, l, _p64(out))
    if rc != 0:
        raise ValueError("cannot find the requested primes")
    return [int(v) for v in out]


def primitive_root(p: int) -> int:
    return int(_load().or_primitive_root(p))


def dft_naive(a, w: int, p: int) -> np.ndarray:
    """Sec. 3.3 eq. dft by definition: out[k] = sum_i a[i] w^(ik) mod p."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    out = np.zeros_like(a)
    _load().or_dft_naive(_p64(a), len(a), w, p, _p64(out))
    return out


def tau_dif(a, w: int, p: int) -> np.ndarray:
    a = np.array(a, dtype=np.uint64)
    lg = int(len(a)).bit_length() - 1
    _load().or_tau_dif(_p64(a), lg, w, p)
    return a


def tau_dit(a, w: int, p: int) -> np.ndarray:
    a = np.array(a, dtype=np.uint64)
    lg = int(len(a)).bit_length() - 1
    _load().or_tau_dit(_p64(a), lg, w, p)
    return a


def cyclic_conv_mod(a, b, p: int) -> np.ndarray:
    """Cyclic convolution mod p via the convolution theorem (length a power of two)."""
    a = np.array(a, dtype=np.uint64)
    b = np.array(b, dtype=np.uint64)
    lg = int(len(a)).bit_length() - 1
    _load().or_cyclic_conv_mod(_p64(a), _p64(b), lg, p)
    return a


def transpose(a, rows: int, cols: int) -> np.ndarray:
    """Out-of-place transpose of a row-major rows x cols matrix (flat in, flat out)."""
    a = _u32(a)
    out = np.zeros(rows * cols, dtype=np.uint32)
    _load().or_transpose(_p32(a), rows, cols, _p32(out))
    return out


def permute_rows_rho(a, n: int, cols: int) -> np.ndarray:
    """Sec. 7.6 rho on the rows of a (2n) x cols matrix: row i -> n*(i mod 2) + i div 2."""
    a = _u32(a)
    out = np.zeros(2 * n * cols, dtype=np.uint32)
    _load().or_permute_rows_rho(_p32(a), n, cols, _p32(out))
    return out


def residues(c_words: np.ndarray, p: int) -> np.ndarray:
    """c_k mod p from (L, 2) uint64 coefficient words."""
    lo = c_words[:, 0].astype(object)
    hi = c_words[:, 1].astype(object)
    return np.array([(int(h) * (1 << 64) + int(l)) % p for l, h in zip(lo, hi)], dtype=np.uint64)
