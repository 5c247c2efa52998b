"""CPU oracle -- TEST INFRASTRUCTURE, not the product.

A plain, slow, obviously correct implementation of what the CUDA path
computes (the C file ``he_oracle.c`` holds the arithmetic, with ``%`` on
128-bit products; ``ckks.py`` holds the host-side CKKS encode, decode,
key generation, encryption and decryption in FP64 and Python integers).
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import it. It shares no code with the CUDA library; the only
module both use is the seeded input generator
``paper_2109_14704_gb300.synth``, which holds none of the method's
arithmetic.

Every function is pinned by ``tests/test_oracle_*.py``; see the header of
``he_oracle.c`` for the passage of the paper each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "he_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler at -O3 (plain C, no SIMD
    intrinsics). Rebuilds when the source or these build flags (this file)
    are newer than the library."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(__file__)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u64, i32 = ctypes.c_uint64, ctypes.c_int
        lib.or_is_prime.argtypes = [u64]
        lib.or_is_prime.restype = i32
        lib.or_find_primes.argtypes = [i32, u64, i32, _u64p, i32, _u64p]
        lib.or_find_primes.restype = i32
        lib.or_find_psi.argtypes = [u64, u64]
        lib.or_find_psi.restype = u64
        lib.or_ntt_fwd.argtypes = [_u64p, u64, u64, u64]
        lib.or_ntt_inv.argtypes = [_u64p, u64, u64, u64]
        lib.or_dyadic.argtypes = [_u64p, _u64p, _u64p, u64, u64]
        lib.or_tensor.argtypes = [_u64p, _u64p, _u64p, u64, i32, _u64p]
        lib.or_relin.argtypes = [_u64p, _u64p, _u64p, u64, i32, _u64p, u64, i32]
        lib.or_rescale.argtypes = [_u64p, _u64p, u64, _u64p, i32]
        lib.or_negacyclic_mul.argtypes = [_u64p, _u64p, _u64p, u64, u64, u64]
        lib.or_pow_mod.argtypes = [u64, u64, u64]
        lib.or_pow_mod.restype = u64
        lib.or_mul_mod.argtypes = [u64, u64, u64]
        lib.or_mul_mod.restype = u64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


# ---- parameters -------------------------------------------------------------

def is_prime(n: int) -> bool:
    return bool(_load().or_is_prime(int(n)))


def find_primes(bits: int, two_n: int, count: int, exclude=()) -> list[int]:
    """The `count` largest `bits`-bit primes q = 1 mod two_n, descending."""
    ex = _u64(list(exclude) or [0])
    out = np.zeros(max(count, 1), dtype=np.uint64)
    got = _load().or_find_primes(bits, two_n, count, _ptr(ex), len(exclude), _ptr(out))
    return [int(x) for x in out[:got]]


_psi_cache: dict = {}


def find_psi(q: int, N: int) -> int:
    """The smallest primitive 2N-th root of unity mod q."""
    key = (int(q), int(N))
    if key not in _psi_cache:
        _psi_cache[key] = int(_load().or_find_psi(int(q), int(N)))
    return _psi_cache[key]


def chain_primes(N: int, data_bits: list[int], special_bits: int, two_n: int | None = None):
    """A modulus chain: data primes of the given bit sizes and one special
    prime, all distinct and = 1 mod 2N (or mod `two_n`). Each size takes the
    largest unused primes of that size, data primes first in chain order."""
    two_n = two_n or 2 * N
    used: list[int] = []
    data = []
    for b in data_bits:
        q = find_primes(b, two_n, 1, exclude=used)[0]
        used.append(q)
        data.append(q)
    P = find_primes(special_bits, two_n, 1, exclude=used)[0]
    return data, P


# ---- transforms and products on [limbs][N] arrays -----------------------------

def ntt_fwd(a: np.ndarray, moduli) -> np.ndarray:
    """Forward negacyclic NTT of each row of a [limbs][N] array (copy)."""
    a = _u64(a).copy()
    lib = _load()
    N = a.shape[-1]
    for l, q in enumerate(moduli):
        row = a[l]
        lib.or_ntt_fwd(_ptr(row), N, int(q), find_psi(q, N))
    return a


def ntt_inv(a: np.ndarray, moduli) -> np.ndarray:
    """Inverse negacyclic NTT (with the factor N^-1) of each row (copy)."""
    a = _u64(a).copy()
    lib = _load()
    N = a.shape[-1]
    for l, q in enumerate(moduli):
        row = a[l]
        lib.or_ntt_inv(_ptr(row), N, int(q), find_psi(q, N))
    return a


def dyadic(a: np.ndarray, b: np.ndarray, moduli) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    out = np.empty_like(a)
    lib = _load()
    N = a.shape[-1]
    for l, q in enumerate(moduli):
        lib.or_dyadic(_ptr(out[l]), _ptr(a[l]), _ptr(b[l]), N, int(q))
    return out


def negacyclic_mul(a: np.ndarray, b: np.ndarray, moduli) -> np.ndarray:
    """a * b in Z_q[X]/(X^N+1) for each limb, coefficient domain."""
    a, b = _u64(a), _u64(b)
    out = np.empty_like(a)
    lib = _load()
    N = a.shape[-1]
    for l, q in enumerate(moduli):
        lib.or_negacyclic_mul(_ptr(out[l]), _ptr(a[l]), _ptr(b[l]), N, int(q), find_psi(q, N))
    return out


def tensor(ct_a: np.ndarray, ct_b: np.ndarray, moduli) -> np.ndarray:
    """Mul: [2][n][N] x [2][n][N] -> [3][n][N] (NTT domain)."""
    ct_a, ct_b = _u64(ct_a), _u64(ct_b)
    n, N = ct_a.shape[1], ct_a.shape[2]
    out = np.empty((3, n, N), dtype=np.uint64)
    _load().or_tensor(_ptr(out), _ptr(ct_a), _ptr(ct_b), N, n, _ptr(_u64(moduli)))
    return out


def relin(ct3: np.ndarray, evk: np.ndarray, moduli, P: int, level: int) -> np.ndarray:
    """Relin: [3][l+1][N] -> [2][l+1][N]. evk is [n_max][2][n_max+1][N]."""
    ct3, evk = _u64(ct3), _u64(evk)
    n_max = evk.shape[0]
    N = ct3.shape[2]
    assert ct3.shape[1] == level + 1 and evk.shape == (n_max, 2, n_max + 1, N)
    out = np.empty((2, level + 1, N), dtype=np.uint64)
    for q in list(moduli)[:level + 1] + [P]:
        find_psi(q, N)
    _load().or_relin(_ptr(out), _ptr(ct3), _ptr(evk), N, n_max, _ptr(_u64(moduli)), int(P), level)
    return out


def rescale(ct: np.ndarray, moduli, level: int) -> np.ndarray:
    """RS: [2][l+1][N] -> [2][l][N]."""
    ct = _u64(ct)
    N = ct.shape[2]
    assert ct.shape[1] == level + 1 and level >= 1
    out = np.empty((2, level, N), dtype=np.uint64)
    _load().or_rescale(_ptr(out), _ptr(ct), N, _ptr(_u64(moduli)), level)
    return out


def mul_relin_rescale(ct_a, ct_b, evk, moduli, P, level) -> np.ndarray:
    """MulLinRS: tensor, relinearize, rescale (Sec. IV-C routines)."""
    ct3 = tensor(ct_a, ct_b, list(moduli)[:level + 1])
    ct2 = relin(ct3, evk, moduli, P, level)
    return rescale(ct2, moduli, level)


def add(ct_a: np.ndarray, ct_b: np.ndarray, moduli) -> np.ndarray:
    """Add (Sec. II-A): componentwise (a + b) mod q_l on [c][n][N] residues
    (any number of components c; moduli q_0..q_{n-1})."""
    a, b = _u64(ct_a), _u64(ct_b)
    qs = np.array([int(q) for q in list(moduli)[:a.shape[-2]]], dtype=np.uint64)[:, None]
    return (a + b) % qs


def automorphism(a: np.ndarray, g: int, moduli) -> np.ndarray:
    """The ring automorphism a(X) -> a(X^g) of Z_q[X]/(X^N + 1) (g odd) on
    coefficient-domain residues [limbs][N]: coefficient j moves to g j mod 2N,
    negated when that exponent is N or more (X^N = -1). Behind Rotate
    (Sec. IV-C): X -> X^(5^k) rotates the slots by k."""
    a = _u64(a)
    N = a.shape[-1]
    assert g % 2 == 1
    e = (np.arange(N, dtype=np.int64) * (g % (2 * N))) % (2 * N)
    dest, neg = e % N, e >= N
    qs = np.array([int(q) for q in list(moduli)[:a.shape[0]]], dtype=np.uint64)[:, None]
    out = np.zeros_like(a)
    out[:, dest] = np.where(neg[None, :], (qs - a) % qs, a)
    return out


def ntt_automorphism(a_ntt: np.ndarray, g: int, moduli) -> np.ndarray:
    """The automorphism on NTT-domain residues, through the coefficient
    domain (inverse transform, automorphism, forward transform)."""
    return ntt_fwd(automorphism(ntt_inv(a_ntt, moduli), g, moduli), moduli)


def rotate(ct: np.ndarray, g: int, gk: np.ndarray, moduli, P: int, level: int) -> np.ndarray:
    """Rotate (Sec. IV-C): (sigma(c0), sigma(c1)) with sigma: X -> X^g, then
    c1's key switched back to s with the Galois key gk (the relinearization
    of (sigma(c0), 0, sigma(c1)))."""
    ct = _u64(ct)
    qs = list(moduli)[:level + 1]
    c3 = np.stack([ntt_automorphism(ct[0], g, qs), np.zeros_like(ct[0]), ntt_automorphism(ct[1], g, qs)])
    return relin(c3, gk, moduli, P, level)


def matmul_tensor(A, B, moduli) -> np.ndarray:
    """Tensor part of the encrypted matrix product C += A B (Sec. IV-E
    matMul_mxnxk): A is [m][k] and B [k][n] two-component ciphertexts
    ([2][n_limbs][N] each); returns [m][n][3][n_limbs][N] with
    T[i][j] = sum over l of the Mul tensor (Sec. II-A) of A[i][l] and B[l][j],
    summed limb by limb mod q."""
    A, B = _u64(A), _u64(B)
    m, k, n = A.shape[0], A.shape[1], B.shape[1]
    assert B.shape[0] == k
    qs = list(moduli)[:A.shape[-2]]
    out = np.empty((m, n, 3) + A.shape[-2:], dtype=np.uint64)
    for i in range(m):
        for j in range(n):
            acc = tensor(A[i, 0], B[0, j], qs)
            for l in range(1, k):
                acc = add(acc, tensor(A[i, l], B[l, j], qs), qs)
            out[i, j] = acc
    return out


# ---- multi-threaded runners for the timed CPU baseline -------------------------

def ntt_fwd_many(polys: np.ndarray, moduli, threads: int) -> np.ndarray:
    """Forward NTT of polys[poly][limb][N] over (poly, limb) units on
    `threads` host threads (ctypes releases the GIL during each call)."""
    polys = _u64(polys).copy()
    lib = _load()
    N = polys.shape[-1]
    psis = [find_psi(q, N) for q in moduli]

    def unit(idx):
        p, l = divmod(idx, polys.shape[1])
        lib.or_ntt_fwd(_ptr(polys[p, l]), N, int(moduli[l]), psis[l])

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(unit, range(polys.shape[0] * polys.shape[1])))
    return polys


def ntt_inv_many(polys: np.ndarray, moduli, threads: int) -> np.ndarray:
    polys = _u64(polys).copy()
    lib = _load()
    N = polys.shape[-1]
    psis = [find_psi(q, N) for q in moduli]

    def unit(idx):
        p, l = divmod(idx, polys.shape[1])
        lib.or_ntt_inv(_ptr(polys[p, l]), N, int(moduli[l]), psis[l])

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(unit, range(polys.shape[0] * polys.shape[1])))
    return polys


def mul_relin_rescale_many(cts_a, cts_b, evk, moduli, P, level, threads: int):
    """MulLinRS over a batch of ciphertext pairs, one pair per host thread."""
    def unit(i):
        return mul_relin_rescale(cts_a[i], cts_b[i], evk, moduli, P, level)

    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(unit, range(len(cts_a))))
