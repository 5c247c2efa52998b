"""Python binding of libhe.so: the same entry points as include/he.h, with
argument marshalling only (tensor data pointers, the current CUDA stream,
host arrays). Every step of the computation runs in the library's CUDA
kernels; there is no CPU fallback. If the library cannot be built or loaded,
every call raises.

Device buffers are torch tensors of dtype int64 or uint64 holding the 64-bit
words (the bits are used as is), contiguous and 32-byte aligned.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p

HE_OK, HE_EINVAL, HE_ENOMEM, HE_ECUDA, HE_EUNSUPPORTED, HE_ETIMEOUT = 0, -1, -2, -3, -4, -5
_NAMES = {-1: "HE_EINVAL", -2: "HE_ENOMEM", -3: "HE_ECUDA", -4: "HE_EUNSUPPORTED", -5: "HE_ETIMEOUT"}


class HeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_NAMES.get(status, status)}: {message}")
        self.status = status


class PolyDesc(ctypes.Structure):
    _fields_ = [("data", _vp), ("tables", _vp), ("N", ctypes.c_uint32), ("limbs", ctypes.c_uint32),
                ("first_prime", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class MrrJob(ctypes.Structure):
    _fields_ = [("ct_out", ctypes.c_void_p), ("ct_a", ctypes.c_void_p), ("ct_b", ctypes.c_void_p),
                ("count", ctypes.c_uint32), ("level", ctypes.c_uint32)]


class MrrMultiJob(ctypes.Structure):
    _fields_ = [("ct_out", ctypes.c_void_p), ("ct_a", ctypes.c_void_p), ("ct_b", ctypes.c_void_p),
                ("count", ctypes.c_uint32), ("level", ctypes.c_uint32), ("ctx", ctypes.c_void_p),
                ("key", ctypes.c_void_p)]


class NttShape(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("log_block", ctypes.c_uint32), ("log_thread_words", ctypes.c_uint32),
                ("persistent", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32)]


_SIGS = {
    "he_last_error": (ctypes.c_int32, [ctypes.c_char_p, ctypes.c_size_t]),
    "he_version": (ctypes.c_uint32, []),
    "he_primes_generate": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, _u64p,
                                            ctypes.c_uint32, _u64p]),
    "he_ntt_tables_create": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_uint32, _u64p, ctypes.POINTER(_vp)]),
    "he_ntt_tables_destroy": (ctypes.c_int32, [_vp]),
    "he_ntt_tables_psi": (ctypes.c_int32, [_vp, ctypes.c_uint32, _u64p]),
    "he_ntt_fwd": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u64p, _vp, _vp]),
    "he_ntt_inv": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u64p, _vp, _vp]),
    "he_ntt_fwd_naive": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u64p, _vp,
                                          _vp]),
    "he_ntt_inv_naive": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u64p, _vp,
                                          _vp]),
    "he_dyadic_mul": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u64p,
                                       _vp, _vp]),
    "he_context_create": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_uint32, _u64p, ctypes.c_uint64,
                                           ctypes.POINTER(_vp)]),
    "he_context_destroy": (ctypes.c_int32, [_vp]),
    "he_context_set_eval_shape": (ctypes.c_int32, [_vp, ctypes.c_uint32]),
    "he_relin_key_upload": (ctypes.c_int32, [_vp, _u64p, ctypes.POINTER(_vp)]),
    "he_relin_key_destroy": (ctypes.c_int32, [_vp]),
    "he_ct_mul": (ctypes.c_int32, [_vp, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
    "he_relin_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32]),
    "he_relin": (ctypes.c_int32, [_vp, _vp, _vp, _vp, ctypes.c_uint32, _vp, ctypes.c_size_t, _vp]),
    "he_rescale_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32]),
    "he_rescale": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, _vp, ctypes.c_size_t, _vp]),
    "he_mul_relin_rescale_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32, ctypes.c_uint32]),
    "he_mul_relin_rescale_scratch_bytes_ex": (ctypes.c_size_t, [_vp, ctypes.c_uint32, ctypes.c_uint32,
                                                                ctypes.c_uint32]),
    "he_mul_relin_rescale": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, _vp, _vp, ctypes.c_uint32, _vp,
                                              ctypes.c_size_t, _vp]),
    "he_ntt_plan_create": (ctypes.c_int32, [ctypes.POINTER(PolyDesc), ctypes.c_uint32, ctypes.POINTER(NttShape),
                                            ctypes.c_uint32, ctypes.POINTER(_vp)]),
    "he_ntt_plan_fwd": (ctypes.c_int32, [_vp, _vp]),
    "he_ntt_plan_inv": (ctypes.c_int32, [_vp, _vp]),
    "he_plan_destroy": (ctypes.c_int32, [_vp]),
    "he_plan_launches": (ctypes.c_uint32, [_vp]),
    "he_ntt_host": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u64p, _vp,
                                     ctypes.c_uint32, _vp, ctypes.c_size_t, _vp]),
    "he_ntt_shapes": (ctypes.c_int32, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_uint32)]),
    "he_ntt_set_shape": (ctypes.c_int32, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_uint32]),
    "he_butterfly_probe": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp]),
    "he_butterfly_apply": (ctypes.c_int32, [_vp, _vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, _vp]),
    "he_sqr_relin_rescale": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, _vp, _vp, ctypes.c_uint32, _vp,
                                              ctypes.c_size_t, _vp]),
    "he_mul_relin_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32, ctypes.c_uint32]),
    "he_mul_relin": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, _vp, _vp, ctypes.c_uint32, _vp,
                                      ctypes.c_size_t, _vp]),
    "he_relin_rescale": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, _vp, _vp, ctypes.c_uint32, _vp,
                                          ctypes.c_size_t, _vp]),
    "he_ct_add": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, _vp, ctypes.c_uint32, _vp]),
    "he_ct_matmul_tensor": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             _vp, ctypes.c_uint32, _vp]),
    "he_ct_automorph": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp,
                                         ctypes.c_uint32, _vp]),
    "he_rotate_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32, ctypes.c_uint32]),
    "he_rotate": (ctypes.c_int32, [_vp, _vp, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp, ctypes.c_uint32, _vp,
                                   ctypes.c_size_t, _vp]),
    "he_mul_relin_rescale_noalloc": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, _vp, _vp, ctypes.c_uint32,
                                                      _vp]),
    "he_encoder_create": (ctypes.c_int32, [_vp, ctypes.POINTER(_vp)]),
    "he_encoder_destroy": (ctypes.c_int32, [_vp]),
    "he_encode_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32]),
    "he_decode_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32, ctypes.c_uint32]),
    "he_encode": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32, _vp,
                                   ctypes.c_size_t, _vp]),
    "he_decode": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32, _vp,
                                   ctypes.c_size_t, _vp]),
    "he_crt_compose": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, _vp]),
    "he_fp64_probe": (ctypes.c_int32, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp]),
    "he_negacyclic_mul": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u64p,
                                           _vp, _vp]),
    "he_encrypt_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32, ctypes.c_uint32]),
    "he_sample_encryption_draws": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                                    _vp]),
    "he_encrypt_seeded": (ctypes.c_int32, [_vp, _vp, _vp, ctypes.c_uint64, ctypes.c_uint32, _vp, ctypes.c_uint32, _vp,
                                           ctypes.c_size_t, _vp]),
    "he_encrypt": (ctypes.c_int32, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_uint32, _vp, ctypes.c_uint32, _vp,
                                    ctypes.c_size_t, _vp]),
    "he_mul_relin_rescale_batch_scratch_bytes": (ctypes.c_size_t, [_vp, ctypes.POINTER(MrrJob), ctypes.c_uint32]),
    "he_mul_relin_rescale_multi_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(MrrMultiJob), ctypes.c_uint32]),
    "he_mul_relin_rescale_multi": (ctypes.c_int32, [ctypes.POINTER(MrrMultiJob), ctypes.c_uint32, _vp,
                                                    ctypes.c_size_t, _vp]),
    "he_mul_relin_rescale_batch": (ctypes.c_int32, [ctypes.POINTER(MrrJob), ctypes.c_uint32, _vp, _vp, _vp,
                                                    ctypes.c_size_t, _vp]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libhe.so (building it first if its sources are newer)."""
    global _lib
    if _lib is None:
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library missing: {_build.LIB} (run __graft_entry__.build())")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def declared_symbols() -> list[str]:
    return sorted(_SIGS)


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    load().he_last_error(buf, 512)
    return buf.value.decode()


def _check(status: int):
    if status != HE_OK:
        raise HeError(status, last_error())


def _ptr(x, words: int | None = None):
    """Device pointer of a torch tensor (or an int address, or None). With
    `words`, the tensor must hold at least that many 64-bit words: the C ABI
    takes bare pointers, so the binding is where a short buffer is caught
    (an int address is passed through unchecked)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if x.element_size() != 8:
        raise ValueError("expected 64-bit words (int64 or uint64)")
    if words is not None and x.numel() < words:
        raise ValueError(f"device tensor holds {x.numel()} words, the call needs {words}")
    return x.data_ptr()


def _fptr(x, doubles: int):
    """Device pointer of a float64 or complex128 torch tensor holding at least
    `doubles` FP64 values."""
    import torch
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    per = {torch.float64: 1, torch.complex128: 2}.get(x.dtype)
    if per is None:
        raise ValueError("expected float64 or complex128")
    if x.numel() * per < doubles:
        raise ValueError(f"device tensor holds {x.numel() * per} doubles, the call needs {doubles}")
    return x.data_ptr()


def _i8ptr(x, values: int):
    """Device pointer of an int8 torch tensor holding at least `values` entries."""
    import torch
    if not x.is_cuda or not x.is_contiguous() or x.dtype != torch.int8:
        raise ValueError("expected a contiguous int8 CUDA tensor")
    if x.numel() < values:
        raise ValueError(f"device tensor holds {x.numel()} values, the call needs {values}")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _host_u64(values) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(values, dtype=np.uint64))


def _hp(a: np.ndarray):
    return a.ctypes.data_as(_u64p)


def version() -> int:
    return int(load().he_version())


def primes_generate(bits: int, two_n: int, count: int, exclude=()) -> list[int]:
    ex = _host_u64(list(exclude) or [0])
    out = np.zeros(max(count, 1), dtype=np.uint64)
    _check(load().he_primes_generate(bits, two_n, count, _hp(ex), len(exclude), _hp(out)))
    return [int(v) for v in out[:count]]


def chain_primes(N: int, data_bits, special_bits: int, two_n: int | None = None):
    """Data primes of the given bit sizes then one special prime, each the
    largest unused prime of its size that is 1 mod 2N (or mod two_n)."""
    two_n = two_n or 2 * N
    used: list[int] = []
    for b in data_bits:
        used += primes_generate(b, two_n, 1, exclude=used)
    P = primes_generate(special_bits, two_n, 1, exclude=used)[0]
    return used, P


class NttTables:
    """he_ntt_tables: device-resident twiddles of `moduli` at degree N."""

    def __init__(self, N: int, moduli):
        self.N = int(N)
        self.moduli = [int(q) for q in moduli]
        self._m = _host_u64(self.moduli)
        h = _vp()
        _check(load().he_ntt_tables_create(self.N, len(self.moduli), _hp(self._m), ctypes.byref(h)))
        self.handle = h

    def psi(self, index: int) -> int:
        out = np.zeros(1, dtype=np.uint64)
        _check(load().he_ntt_tables_psi(self.handle, index, _hp(out)))
        return int(out[0])

    def close(self):
        if getattr(self, "handle", None):
            load().he_ntt_tables_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ntt_shapes(N: int) -> list[tuple[int, int, int]]:
    """Transform shapes (log_block, log_thread_words, ctas_per_sm) built for
    degree N, default first (ctas_per_sm 0: the shape's default register
    budget)."""
    n = ctypes.c_uint32()
    buf = (ctypes.c_uint32 * 48)()
    _check(load().he_ntt_shapes(N, buf, 16, ctypes.byref(n)))
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(min(n.value, 16))]


FORWARD, INVERSE, BOTH = 1, 2, 0


def ntt_set_shape(N: int, log_block: int = 0, log_thread_words: int = 0, persistent: int = 0,
                  direction: int = BOTH, ctas_per_sm: int = 0):
    """Shape used by ntt_fwd (direction 1) / ntt_inv (2) / both (0) at
    degree N (all zero = default)."""
    _check(load().he_ntt_set_shape(N, direction, log_block, log_thread_words, int(persistent), ctas_per_sm))


def _moduli_arg(tables: NttTables, limbs: int, moduli):
    m = _host_u64(tables.moduli[:limbs] if moduli is None else list(moduli)[:limbs])
    return m


def ntt_fwd(poly, N, limbs, count, tables: NttTables, moduli=None, stream=None):
    m = _moduli_arg(tables, limbs, moduli)
    _check(load().he_ntt_fwd(_ptr(poly, N * limbs * count), N, limbs, count, _hp(m), tables.handle, _stream(stream)))


def ntt_inv(poly, N, limbs, count, tables: NttTables, moduli=None, stream=None):
    m = _moduli_arg(tables, limbs, moduli)
    _check(load().he_ntt_inv(_ptr(poly, N * limbs * count), N, limbs, count, _hp(m), tables.handle, _stream(stream)))


NTT_OP_FORWARD, NTT_OP_INVERSE = 1, 2


def _host_ptr(x, words: int):
    """Host address of a numpy array or CPU torch tensor of >= `words`
    64-bit words (or an int address)."""
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"] or x.itemsize != 8:
            raise ValueError("expected a contiguous array of 64-bit words")
        if x.size < words:
            raise ValueError(f"host array holds {x.size} words, need {words}")
        return x.ctypes.data
    if x.is_cuda:
        raise ValueError("expected a host (CPU) tensor")
    if not x.is_contiguous() or x.element_size() != 8:
        raise ValueError("expected a contiguous tensor of 64-bit words")
    if x.numel() < words:
        raise ValueError(f"host tensor holds {x.numel()} words, need {words}")
    return x.data_ptr()


def ntt_host(inp, out, N, limbs, count, tables: NttTables, ops, work, moduli=None, stream=None):
    """he_ntt_host: transform host-resident polynomials through the device
    (copy in, ops = NTT_OP_FORWARD / NTT_OP_INVERSE / both, copy out),
    pipelined over chunks; `work` is device scratch."""
    m = _moduli_arg(tables, limbs, moduli)
    words = N * limbs * count
    nbytes = work.numel() * work.element_size()
    _check(load().he_ntt_host(_host_ptr(inp, words), _host_ptr(out, words), N, limbs, count, _hp(m),
                              tables.handle, ops, _ptr(work), nbytes, _stream(stream)))


def ntt_fwd_naive(poly, N, limbs, count, tables: NttTables, moduli=None, stream=None):
    m = _moduli_arg(tables, limbs, moduli)
    _check(load().he_ntt_fwd_naive(_ptr(poly, N * limbs * count), N, limbs, count, _hp(m), tables.handle, _stream(stream)))


def ntt_inv_naive(poly, N, limbs, count, tables: NttTables, moduli=None, stream=None):
    m = _moduli_arg(tables, limbs, moduli)
    _check(load().he_ntt_inv_naive(_ptr(poly, N * limbs * count), N, limbs, count, _hp(m), tables.handle, _stream(stream)))


def dyadic_mul(out, a, b, N, limbs, count, tables: NttTables, moduli=None, stream=None):
    m = _moduli_arg(tables, limbs, moduli)
    w = N * limbs * count
    _check(load().he_dyadic_mul(_ptr(out, w), _ptr(a, w), _ptr(b, w), N, limbs, count, _hp(m), tables.handle,
                                _stream(stream)))


def negacyclic_mul(c, a, b, N, limbs, count, tables: NttTables, moduli=None, stream=None):
    """Fused negacyclic product c = a b mod (X^N + 1, q) in one launch
    (coefficient domain in and out)."""
    m = _moduli_arg(tables, limbs, moduli)
    w = N * limbs * count
    _check(load().he_negacyclic_mul(_ptr(c, w), _ptr(a, w), _ptr(b, w), N, limbs, count, _hp(m), tables.handle,
                                    _stream(stream)))


class Context:
    """he_context: modulus chain q_0..q_L and special prime P at degree N."""

    def __init__(self, N: int, data_moduli, special_modulus: int):
        self.N = int(N)
        self.data_moduli = [int(q) for q in data_moduli]
        self.P = int(special_modulus)
        m = _host_u64(self.data_moduli)
        h = _vp()
        _check(load().he_context_create(self.N, len(self.data_moduli), _hp(m), self.P, ctypes.byref(h)))
        self.handle = h

    @property
    def n_data(self) -> int:
        return len(self.data_moduli)

    def set_eval_shape(self, log_thread_words: int):
        """Words per thread (2^3 or 2^4; 0 = default) of the context's
        key-switching and rescale kernels."""
        _check(load().he_context_set_eval_shape(self.handle, log_thread_words))

    def relin_scratch_bytes(self, level: int) -> int:
        return int(load().he_relin_scratch_bytes(self.handle, level))

    def rescale_scratch_bytes(self, level: int) -> int:
        return int(load().he_rescale_scratch_bytes(self.handle, level))

    def rotate_scratch_bytes(self, level: int, count: int) -> int:
        return int(load().he_rotate_scratch_bytes(self.handle, level, count))

    def mul_relin_scratch_bytes(self, level: int, count: int) -> int:
        return int(load().he_mul_relin_scratch_bytes(self.handle, level, count))

    def mrr_scratch_bytes(self, level: int, count: int, expand_group: int | None = None) -> int:
        """Scratch bytes of mul_relin_rescale; expand_group bounds the
        expanded mod-up's group (0: the fused minimum, None: the default)."""
        if expand_group is None:
            return int(load().he_mul_relin_rescale_scratch_bytes(self.handle, level, count))
        return int(load().he_mul_relin_rescale_scratch_bytes_ex(self.handle, level, count, expand_group))

    def encrypt_scratch_bytes(self, level: int, count: int) -> int:
        return int(load().he_encrypt_scratch_bytes(self.handle, level, count))

    def mrr_batch_scratch_bytes(self, jobs) -> int:
        """Scratch bytes of mul_relin_rescale_batch for jobs given as
        (count, level) pairs (or full job tuples)."""
        arr = (MrrJob * max(1, len(jobs)))()
        for i, j in enumerate(jobs):
            count, level = (j[0], j[1]) if len(j) == 2 else (j[3], j[4])
            arr[i] = MrrJob(None, None, None, count, level)
        return int(load().he_mul_relin_rescale_batch_scratch_bytes(self.handle, arr, len(jobs)))

    def close(self):
        if getattr(self, "handle", None):
            load().he_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RelinKey:
    """he_relin_key: evk [n_data][2][n_data+1][N] (host array) uploaded."""

    def __init__(self, ctx: Context, evk_host: np.ndarray):
        evk = _host_u64(evk_host)
        nd = ctx.n_data
        if evk.shape != (nd, 2, nd + 1, ctx.N):
            raise ValueError(f"evk must have shape {(nd, 2, nd + 1, ctx.N)}, got {evk.shape}")
        h = _vp()
        _check(load().he_relin_key_upload(ctx.handle, _hp(evk), ctypes.byref(h)))
        self.handle = h
        self.ctx = ctx

    def close(self):
        if getattr(self, "handle", None):
            load().he_relin_key_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ct_mul(out3, ct_a, ct_b, ctx: Context, level: int, stream=None):
    w = (level + 1) * ctx.N
    _check(load().he_ct_mul(_ptr(out3, 3 * w), _ptr(ct_a, 2 * w), _ptr(ct_b, 2 * w), ctx.handle, level,
                            _stream(stream)))


def relin(ct_out2, ct_in3, key: RelinKey, ctx: Context, level: int, scratch, stream=None):
    w = (level + 1) * ctx.N
    _check(load().he_relin(_ptr(ct_out2, 2 * w), _ptr(ct_in3, 3 * w), key.handle, ctx.handle, level, _ptr(scratch),
                           scratch.numel() * 8, _stream(stream)))


def rescale(ct_out, ct_in, ctx: Context, level: int, scratch, stream=None):
    _check(load().he_rescale(_ptr(ct_out, 2 * level * ctx.N), _ptr(ct_in, 2 * (level + 1) * ctx.N), ctx.handle,
                             level, _ptr(scratch), scratch.numel() * 8,
                             _stream(stream)))


def mul_relin_rescale(ct_out, ct_a, ct_b, count: int, key: RelinKey, ctx: Context, level: int, scratch,
                      stream=None):
    w_in, w_out = count * 2 * (level + 1) * ctx.N, count * 2 * level * ctx.N
    _check(load().he_mul_relin_rescale(_ptr(ct_out, w_out), _ptr(ct_a, w_in), _ptr(ct_b, w_in), count, key.handle,
                                       ctx.handle, level, _ptr(scratch), scratch.numel() * 8, _stream(stream)))


def encrypt(ct_out, pt, pk, v, e0, e1, count: int, ctx: Context, level: int, scratch, stream=None):
    """Public-key encryption (Sec. II-A) of NTT-domain plaintexts with the
    given randomness: v, e0, e1 are int8 tensors [count][N]; pk is the
    public key [2][n_data][N] (NTT domain)."""
    N, n = ctx.N, level + 1
    _check(load().he_encrypt(_ptr(ct_out, count * 2 * n * N), _ptr(pt, count * n * N), _ptr(pk, 2 * ctx.n_data * N),
                             _i8ptr(v, count * N), _i8ptr(e0, count * N), _i8ptr(e1, count * N), count, ctx.handle,
                             level, _ptr(scratch), scratch.numel() * 8, _stream(stream)))


def sample_encryption_draws(v, e0, e1, count: int, N: int, seed: int, stream=None):
    """The encryption randomness drawn on the device from `seed` (int8
    tensors [count][N]: ternary mask, two centred-binomial errors)."""
    _check(load().he_sample_encryption_draws(_i8ptr(v, count * N), _i8ptr(e0, count * N), _i8ptr(e1, count * N),
                                             count, N, seed & ((1 << 64) - 1), _stream(stream)))


def encrypt_seeded(ct_out, pt, pk, seed: int, count: int, ctx: Context, level: int, scratch, stream=None):
    """Public-key encryption with the randomness drawn on the device from
    `seed` (the draws of sample_encryption_draws)."""
    N, n = ctx.N, level + 1
    _check(load().he_encrypt_seeded(_ptr(ct_out, count * 2 * n * N), _ptr(pt, count * n * N),
                                    _ptr(pk, 2 * ctx.n_data * N), seed & ((1 << 64) - 1), count, ctx.handle, level,
                                    _ptr(scratch), scratch.numel() * 8, _stream(stream)))


# Jobs of a mixed-level batch that one pass of he_mul_relin_rescale_batch takes.
MAX_BATCH_JOBS = 16


def mul_relin_rescale_batch(jobs, key: RelinKey, ctx: Context, scratch, stream=None):
    """MulLinRS of a mixed-level batch, one launch per pipeline stage: jobs
    are (ct_out, ct_a, ct_b, count, level) tuples of device tensors."""
    arr = (MrrJob * max(1, len(jobs)))()
    for i, (out, a, b, count, level) in enumerate(jobs):
        w_in, w_out = count * 2 * (level + 1) * ctx.N, count * 2 * level * ctx.N
        arr[i] = MrrJob(_ptr(out, w_out), _ptr(a, w_in), _ptr(b, w_in), count, level)
    _check(load().he_mul_relin_rescale_batch(arr, len(jobs), key.handle, ctx.handle, _ptr(scratch),
                                             scratch.numel() * 8, _stream(stream)))


def _multi_jobs(jobs, with_pointers: bool):
    arr = (MrrMultiJob * max(1, len(jobs)))()
    for i, (out, a, b, count, level, key, ctx) in enumerate(jobs):
        if with_pointers:
            w_in, w_out = count * 2 * (level + 1) * ctx.N, count * 2 * level * ctx.N
            arr[i] = MrrMultiJob(_ptr(out, w_out), _ptr(a, w_in), _ptr(b, w_in), count, level, ctx.handle.value,
                                 key.handle.value)
        else:
            arr[i] = MrrMultiJob(None, None, None, count, level, ctx.handle.value, key.handle.value)
    return arr


def mul_relin_rescale_multi_scratch_bytes(jobs) -> int:
    """Scratch of mul_relin_rescale_multi for (count, level, key, ctx) jobs."""
    return int(load().he_mul_relin_rescale_multi_scratch_bytes(
        _multi_jobs([(None, None, None, c, l, k, x) for c, l, k, x in jobs], False), len(jobs)))


def mul_relin_rescale_multi(jobs, scratch, stream=None):
    """MulLinRS of jobs of different degrees, one launch per pipeline stage:
    jobs are (ct_out, ct_a, ct_b, count, level, key, ctx) tuples."""
    _check(load().he_mul_relin_rescale_multi(_multi_jobs(jobs, True), len(jobs), _ptr(scratch),
                                             scratch.numel() * 8, _stream(stream)))


def sqr_relin_rescale(ct_out, ct_a, count: int, key: RelinKey, ctx: Context, level: int, scratch, stream=None):
    """SqrLinRS: he_mul_relin_rescale(a, a) (Sec. IV-C routine set)."""
    w_in, w_out = count * 2 * (level + 1) * ctx.N, count * 2 * level * ctx.N
    _check(load().he_sqr_relin_rescale(_ptr(ct_out, w_out), _ptr(ct_a, w_in), count, key.handle, ctx.handle, level,
                                       _ptr(scratch), scratch.numel() * 8, _stream(stream)))


def mul_relin(ct_out, ct_a, ct_b, count: int, key: RelinKey, ctx: Context, level: int, scratch, stream=None):
    """MulLin: Mul then Relin of `count` pairs, no rescale."""
    w = count * 2 * (level + 1) * ctx.N
    _check(load().he_mul_relin(_ptr(ct_out, w), _ptr(ct_a, w), _ptr(ct_b, w), count, key.handle, ctx.handle, level,
                               _ptr(scratch), scratch.numel() * 8, _stream(stream)))


def relin_rescale(ct_out, ct3, count: int, key: RelinKey, ctx: Context, level: int, scratch, stream=None):
    """Relin then RS of `count` three-component ciphertexts."""
    _check(load().he_relin_rescale(_ptr(ct_out, count * 2 * level * ctx.N), _ptr(ct3, count * 3 * (level + 1) * ctx.N),
                                   count, key.handle, ctx.handle, level, _ptr(scratch), scratch.numel() * 8,
                                   _stream(stream)))


def ct_add(ct_out, ct_a, ct_b, count: int, components: int, ctx: Context, level: int, stream=None):
    """Add: ct_out = ct_a + ct_b mod q_i (2- or 3-component ciphertexts)."""
    w = count * components * (level + 1) * ctx.N
    _check(load().he_ct_add(_ptr(ct_out, w), _ptr(ct_a, w), _ptr(ct_b, w), count, components, ctx.handle, level,
                            _stream(stream)))


def ct_matmul_tensor(t_out, a, b, m: int, k: int, n: int, ctx: Context, level: int, stream=None):
    """Tensor part of C += A B over matrices of ciphertexts (row-major)."""
    w = 2 * (level + 1) * ctx.N
    _check(load().he_ct_matmul_tensor(_ptr(t_out, m * n * 3 * (level + 1) * ctx.N), _ptr(a, m * k * w),
                                      _ptr(b, k * n * w), m, k, n, ctx.handle, level, _stream(stream)))


def ct_automorph(ct_out, ct_in, count: int, components: int, galois_elt: int, ctx: Context, level: int,
                 stream=None):
    """The automorphism X -> X^galois_elt on NTT-domain ciphertexts."""
    w = count * components * (level + 1) * ctx.N
    _check(load().he_ct_automorph(_ptr(ct_out, w), _ptr(ct_in, w), count, components, galois_elt, ctx.handle, level,
                                  _stream(stream)))


def rotate(ct_out, ct_in, count: int, galois_elt: int, galois_key: RelinKey, ctx: Context, level: int, scratch,
           stream=None):
    """Rotate: automorphism then key switch with the Galois key."""
    w = count * 2 * (level + 1) * ctx.N
    _check(load().he_rotate(_ptr(ct_out, w), _ptr(ct_in, w), count, galois_elt, galois_key.handle, ctx.handle, level,
                            _ptr(scratch), scratch.numel() * 8, _stream(stream)))


class Encoder:
    """he_encoder: slot FFT and CRT tables of a context (Sec. II-A Encode /
    Decode on the device). Slots are complex128 tensors [count][N/2] (or
    float64 [count][N/2][2])."""

    def __init__(self, ctx: Context):
        h = _vp()
        _check(load().he_encoder_create(ctx.handle, ctypes.byref(h)))
        self.handle = h
        self.ctx = ctx

    def encode_scratch_bytes(self, count: int) -> int:
        return int(load().he_encode_scratch_bytes(self.handle, count))

    def decode_scratch_bytes(self, level: int, count: int) -> int:
        return int(load().he_decode_scratch_bytes(self.handle, level, count))

    def encode(self, pt_out, slots, count: int, scale: float, level: int, scratch, stream=None):
        """pt_out [count][level+1][N] (NTT domain) = residues of the rounded
        scale-times-slots polynomial."""
        N = self.ctx.N
        _check(load().he_encode(self.handle, _ptr(pt_out, count * (level + 1) * N), _fptr(slots, count * N), count,
                                float(scale), level, _ptr(scratch), scratch.numel() * 8, _stream(stream)))

    def decode(self, slots_out, pt, count: int, scale: float, level: int, scratch, stream=None):
        """slots_out [count][N/2] = slot values of the NTT-domain plaintexts / scale."""
        N = self.ctx.N
        _check(load().he_decode(self.handle, _fptr(slots_out, count * N), _ptr(pt, count * (level + 1) * N), count,
                                float(scale), level, _ptr(scratch), scratch.numel() * 8, _stream(stream)))

    def crt_compose(self, out, coeffs, count: int, level: int, stream=None):
        """out [count][N] (float64) = nearest doubles of the centred CRT lifts
        of coefficient-domain residues coeffs [count][level+1][N]."""
        N = self.ctx.N
        _check(load().he_crt_compose(self.handle, _fptr(out, count * N), _ptr(coeffs, count * (level + 1) * N), count,
                                     level, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().he_encoder_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NttPlan:
    """he_plan over a list of (tensor, tables, N, limbs, first_prime).
    `shapes` maps N to log_block, (log_block, log_thread_words),
    (log_block, log_thread_words, persistent) or (log_block,
    log_thread_words, persistent, ctas_per_sm)."""

    def __init__(self, polys, shapes=None):
        arr = (PolyDesc * max(len(polys), 1))()
        self._keep = []
        for i, (data, tables, N, limbs, first) in enumerate(polys):
            arr[i].data = _ptr(data, N * limbs)
            arr[i].tables = tables.handle.value
            arr[i].N = N
            arr[i].limbs = limbs
            arr[i].first_prime = first
            self._keep.append((data, tables))
        shapes = shapes or {}
        sh = (NttShape * max(len(shapes), 1))()
        for i, (N, shape) in enumerate(shapes.items()):
            lb, le, pe, oc = (shape, 4, 0, 0) if isinstance(shape, int) else (tuple(shape) + (0, 0))[:4]
            sh[i].N, sh[i].log_block, sh[i].log_thread_words, sh[i].persistent = N, lb, le, pe
            sh[i].ctas_per_sm = oc
        h = _vp()
        _check(load().he_ntt_plan_create(arr, len(polys), sh, len(shapes), ctypes.byref(h)))
        self.handle = h

    def fwd(self, stream=None):
        _check(load().he_ntt_plan_fwd(self.handle, _stream(stream)))

    def inv(self, stream=None):
        _check(load().he_ntt_plan_inv(self.handle, _stream(stream)))

    @property
    def launches(self) -> int:
        return int(load().he_plan_launches(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            load().he_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def butterfly_probe(sink, blocks: int, threads: int, iters: int, stream=None):
    """Launch the register-resident butterfly probe (16 * iters butterflies
    per thread)."""
    _check(load().he_butterfly_probe(_ptr(sink), blocks, threads, iters, _stream(stream)))


def fp64_probe(sink, blocks: int, threads: int, iters: int, stream=None):
    """Launch the FP64 probe (16 * iters FLOP per thread); sink is a float64
    tensor of blocks * threads entries."""
    _check(load().he_fp64_probe(_fptr(sink, blocks * threads), blocks, threads, iters, _stream(stream)))


# Bytes of the scratch buffer built into the library (HE_NOALLOC_SCRATCH_BYTES).
NOALLOC_SCRATCH_BYTES = 16 << 20


def mul_relin_rescale_noalloc(ct_out, ct_a, ct_b, count: int, key: RelinKey, ctx: Context, level: int,
                              stream=None):
    """MulLinRS without a scratch argument, for callers that cannot allocate
    device memory at call time (stream capture, allocator-free serving paths,
    externally budgeted memory): the library's built-in buffer is used.
    Calls that can overlap on the GPU share that buffer and must be ordered."""
    w_in, w_out = count * 2 * (level + 1) * ctx.N, count * 2 * level * ctx.N
    _check(load().he_mul_relin_rescale_noalloc(_ptr(ct_out, w_out), _ptr(ct_a, w_in), _ptr(ct_b, w_in), count,
                                               key.handle, ctx.handle, level, _stream(stream)))


def butterfly_apply(x, y, w, w_shoup, p: int, inverse: bool = False, stream=None):
    """Apply the transform butterfly elementwise (device arrays, in place)."""
    n = x.numel()
    _check(load().he_butterfly_apply(_ptr(x), _ptr(y, n), _ptr(w, n), _ptr(w_shoup, n), n, p, int(inverse),
                                     _stream(stream)))
