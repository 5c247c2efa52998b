"""The C ABI without a GPU: libhe.so loads, exports every entry point that
include/he.h declares, generates the same RNS primes as the oracle, and
rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest
import sympy

import oracle
from paper_2109_14704_gb300 import he

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "he.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(he_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = he.load()
    declared = _declared()
    assert len(declared) >= 20
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    # the binding covers the whole ABI too
    assert set(declared) == set(he.declared_symbols())


def test_version():
    assert he.version() == 0x000100


@pytest.mark.parametrize("bits,two_n", [(60, 2 ** 13), (60, 2 ** 16), (50, 2 ** 15), (40, 2 ** 14), (31, 2 ** 11)])
def test_primes_match_oracle(bits, two_n):
    assert he.primes_generate(bits, two_n, 5) == oracle.find_primes(bits, two_n, 5)


def test_chain_primes_match_oracle():
    for N, bits in [(16384, [60] + [50] * 6), (8192, [60, 40, 40]), (32768, [60] + [50] * 15)]:
        assert he.chain_primes(N, bits, 60) == oracle.chain_primes(N, bits, 60)



def test_invalid_arguments_rejected_on_host():
    lib = he.load()
    h = ctypes.c_void_p()
    q = np.array(he.primes_generate(60, 2 * 4096, 1), dtype=np.uint64)
    qp = q.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    # N not a power of two, N out of range
    assert lib.he_ntt_tables_create(3000, 1, qp, ctypes.byref(h)) == he.HE_EINVAL
    assert lib.he_ntt_tables_create(1 << 17, 1, qp, ctypes.byref(h)) == he.HE_EUNSUPPORTED
    assert lib.he_ntt_tables_create(512, 1, qp, ctypes.byref(h)) == he.HE_EUNSUPPORTED
    # modulus not 1 mod 2N, not prime, too large
    composite = next(8192 * k + 1 for k in range(3, 100) if not sympy.isprime(8192 * k + 1))
    for bad in (int(q[0]) + 2, (1 << 60) + 1, composite):
        b = np.array([bad], dtype=np.uint64)
        assert lib.he_ntt_tables_create(4096, 1, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                        ctypes.byref(h)) == he.HE_EINVAL
    assert "modulus" in he.last_error()
    # null output handle, no moduli
    assert lib.he_ntt_tables_create(4096, 1, qp, None) == he.HE_EINVAL
    assert lib.he_ntt_tables_create(4096, 0, qp, ctypes.byref(h)) == he.HE_EINVAL
    # null tables on a transform, on a host-buffer transform
    assert lib.he_ntt_fwd(None, 4096, 1, 1, qp, None, None) == he.HE_EINVAL
    host = np.zeros(4096, dtype=np.uint64)
    assert lib.he_ntt_host(host.ctypes.data, host.ctypes.data, 4096, 1, 1, qp, None, 1, None, 1 << 20,
                           None) == he.HE_EINVAL
    # contexts: too many primes, duplicates, small primes
    assert lib.he_context_create(4096, 0, qp, int(q[0]), ctypes.byref(h)) == he.HE_EINVAL
    assert lib.he_context_create(4096, 1, qp, int(q[0]), ctypes.byref(h)) == he.HE_EINVAL
    assert "twice" in he.last_error()
    small = np.array(he.primes_generate(20, 2 * 4096, 1), dtype=np.uint64)
    assert lib.he_context_create(4096, 1, small.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), int(q[0]),
                                 ctypes.byref(h)) == he.HE_EINVAL
    # prime search out of range
    out = np.zeros(4, dtype=np.uint64)
    assert lib.he_primes_generate(61, 8192, 1, None, 0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))) == \
        he.HE_EINVAL
    assert lib.he_primes_generate(10, 1 << 12, 4, None, 0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))) == \
        he.HE_EINVAL
    # plans with missing tables
    d = (he.PolyDesc * 1)()
    d[0].N, d[0].limbs = 4096, 1
    assert lib.he_ntt_plan_create(d, 1, None, 0, ctypes.byref(h)) == he.HE_EINVAL


def test_error_message_buffer():
    lib = he.load()
    buf = ctypes.create_string_buffer(8)
    assert lib.he_ntt_tables_create(3000, 1, None, None) == he.HE_EINVAL
    assert lib.he_last_error(buf, 8) == 0 and len(buf.value) == 7
    assert lib.he_last_error(None, 0) == he.HE_EINVAL


def test_error_type():
    with pytest.raises(he.HeError) as e:
        he.primes_generate(61, 8192, 1)
    assert e.value.status == he.HE_EINVAL


def test_binding_rejects_short_device_buffers():
    """The C ABI takes bare pointers; the binding checks every tensor against
    the words the call will touch before anything is launched."""
    import types
    fake = types.SimpleNamespace(is_cuda=True, is_contiguous=lambda: True, element_size=lambda: 8,
                                 numel=lambda: 99, data_ptr=lambda: 4096)
    assert he._ptr(fake) == 4096
    assert he._ptr(fake, 99) == 4096
    with pytest.raises(ValueError, match="needs 100"):
        he._ptr(fake, 100)
    assert he._ptr(12345, 1 << 40) == 12345      # raw addresses pass unchecked


# Entry points that accept all-NULL / zero arguments as a no-op.
_NOOP_OK = {"he_ntt_tables_destroy", "he_context_destroy", "he_relin_key_destroy", "he_plan_destroy",
            "he_encoder_destroy", "he_mul_relin_rescale_multi"}   # the last: zero jobs, nothing to do


def test_every_entry_point_rejects_null_arguments_on_the_host():
    """Each status-returning call, given NULL for every pointer and 0 for
    every number, returns HE_EINVAL with a message (or HE_OK where that is a
    no-op: a destroy of NULL, an empty job list), before any device work; the
    size queries return 0. Runs without a GPU."""
    lib = he.load()
    checked = 0
    for name in he.declared_symbols():
        f = getattr(lib, name)
        args = [0.0 if t is ctypes.c_double else
                0 if t in (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t) else None
                for t in f.argtypes]
        r = f(*args)
        if name in ("he_version",):
            continue
        if f.restype is ctypes.c_size_t or name == "he_plan_launches":
            assert r == 0, name
        elif name in _NOOP_OK:
            assert r == he.HE_OK, name
        else:
            assert r == he.HE_EINVAL, name
            if name != "he_last_error":
                assert he.last_error(), name
        checked += 1
    assert checked >= 60


def test_last_error_is_per_thread():
    """he_last_error reports the calling thread's own last failure: two
    threads failing in different ways at the same time each read their own
    message (ctypes releases the interpreter lock around every call)."""
    import threading
    lib = he.load()
    out = np.zeros(1, dtype=np.uint64)
    op = out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    start = threading.Barrier(2)
    wrong = []

    def worker(kind):
        buf = ctypes.create_string_buffer(256)
        h = ctypes.c_void_p()
        start.wait()
        for _ in range(2000):
            if kind == 0:
                assert lib.he_ntt_tables_create(3000, 1, op, ctypes.byref(h)) == he.HE_EINVAL
                want = b"power of two"
            else:
                assert lib.he_primes_generate(61, 8192, 1, None, 0, op) == he.HE_EINVAL
                want = b"bits must be"
            lib.he_last_error(buf, 256)
            if want not in buf.value:
                wrong.append((kind, buf.value))

    ts = [threading.Thread(target=worker, args=(k,)) for k in (0, 1)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not wrong, wrong[:3]
