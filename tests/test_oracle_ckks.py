"""Pins for the oracle's host-side CKKS routines (Sec. II-A): encoding against
direct evaluation of the polynomial at the slot roots, and round trips
(encode/decode, encrypt/decrypt, encrypt/MulLinRS/decrypt) against exact
complex arithmetic.

Tolerance: max_j |z'_j - z_j| <= tol * max(1, max_j |z_j|). At scale 2^40 the
stated bar is 1e-5. The 16384-point chain of one 60-bit and six 50-bit primes
leaves the product at scale 2^80 / q_6 ~ 2^30, 2^10 coarser, so its bound is
5e-5 (measured 1.2e-5)."""
import numpy as np
import pytest

import oracle
from oracle import ckks
from paper_2109_14704_gb300.synth import Rng


def _err(z, ref):
    return float(np.abs(z - ref).max() / max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("N", [16, 1024])
def test_encode_matches_direct_evaluation(N):
    scale = 2.0 ** 40
    z = Rng(N).complex_slots(N // 2)
    m = ckks.encode_real(z, N, scale)
    k = np.arange(N)
    for j in (0, 1, 2, N // 4, N // 2 - 1):
        e = pow(5, j, 2 * N)
        val = np.sum(m.astype(np.float64) * np.exp(1j * np.pi * e * k / N)) / scale
        assert abs(val - z[j]) < 1e-8, j
        # the conjugate root gives the conjugate slot (m is real)
        val_c = np.sum(m.astype(np.float64) * np.exp(-1j * np.pi * e * k / N)) / scale
        assert abs(val_c - np.conj(z[j])) < 1e-8


def test_crt_centred_lift():
    qs = [97, 101, 103]
    Q = 97 * 101 * 103
    vals = [0, 1, -1, Q // 2, -(Q // 2), 12345, -54321]
    res = np.array([[v % q for v in vals] for q in qs], dtype=np.uint64)
    assert ckks.crt_centered(res, qs) == vals


def test_encode_decode_round_trip():
    N, scale = 4096, 2.0 ** 40
    data, _ = oracle.chain_primes(N, [60, 40, 40], 60)
    z = Rng(1).complex_slots(N // 2)
    m = ckks.encode_real(z, N, scale)
    assert _err(ckks.decode(ckks.to_residues(m, data), data, scale), z) < 1e-9


def test_encrypt_decrypt():
    N, scale = 4096, 2.0 ** 40
    data, P = oracle.chain_primes(N, [60, 40, 40], 60)
    r = Rng(2)
    keys = ckks.keygen(N, data, P, r)
    z = r.complex_slots(N // 2)
    ct = ckks.encrypt(ckks.encode_real(z, N, scale), keys, r)
    assert _err(ckks.decrypt_decode(ct, keys, scale), z) < 1e-6


def test_relin_preserves_decryption():
    """decrypt(relin(d)) - decrypt(d) is small noise (the key-switching error)."""
    N = 1024
    data, P = oracle.chain_primes(N, [60, 40, 40], 60)
    r = Rng(3)
    keys = ckks.keygen(N, data, P, r)
    scale = 2.0 ** 40
    za, zb = r.complex_slots(N // 2), r.complex_slots(N // 2)
    ca = ckks.encrypt(ckks.encode_real(za, N, scale), keys, r)
    cb = ckks.encrypt(ckks.encode_real(zb, N, scale), keys, r)
    d = oracle.tensor(ca, cb, data)
    c2 = oracle.relin(d, keys.evk, data, P, 2)
    m3 = ckks.crt_centered(ckks.decrypt_residues(d, keys), data)
    m2 = ckks.crt_centered(ckks.decrypt_residues(c2, keys), data)
    noise = max(abs(a - b) for a, b in zip(m3, m2))
    assert noise < 2 ** 20, noise  # tiny against the scale^2 = 2^80 message


@pytest.mark.parametrize("N,data_bits,tol", [
    (8192, [60, 40, 40], 1e-5),                       # element-wise matrix workload
    (16384, [60, 50, 50, 50, 50, 50, 50], 5e-5),      # CKKS evaluation workload
])
def test_mul_relin_rescale_round_trip(N, data_bits, tol):
    scale = 2.0 ** 40
    data, P = oracle.chain_primes(N, data_bits, 60)
    r = Rng(4)
    keys = ckks.keygen(N, data, P, r)
    za, zb = r.complex_slots(N // 2), r.complex_slots(N // 2)
    ca = ckks.encrypt(ckks.encode_real(za, N, scale), keys, r)
    cb = ckks.encrypt(ckks.encode_real(zb, N, scale), keys, r)
    L = len(data) - 1
    out = oracle.mul_relin_rescale(ca, cb, keys.evk, data, P, L)
    assert out.shape == (2, L, N)
    scale_out = scale * scale / data[L]
    assert _err(ckks.decrypt_decode(out, keys, scale_out), za * zb) < tol


def test_add_brute_force_and_decryption():
    """Add: residue by residue against Python integers, and decrypt(a + b) =
    decrypt(a) + decrypt(b) on decoded slots."""
    qs = [97, 113]
    a = np.array([[[96, 5, 0], [112, 1, 50]]], dtype=np.uint64)
    b = np.array([[[1, 96, 0], [112, 112, 63]]], dtype=np.uint64)
    got = oracle.add(a, b, qs)
    for l, q in enumerate(qs):
        for x in range(3):
            assert int(got[0, l, x]) == (int(a[0, l, x]) + int(b[0, l, x])) % q
    N, scale = 1024, 2.0 ** 40
    data, P = oracle.chain_primes(N, [60, 40, 40], 60)
    r = Rng(11)
    keys = ckks.keygen(N, data, P, r)
    za, zb = r.complex_slots(N // 2), r.complex_slots(N // 2)
    ca = ckks.encrypt(ckks.encode_real(za, N, scale), keys, r)
    cb = ckks.encrypt(ckks.encode_real(zb, N, scale), keys, r)
    assert _err(ckks.decrypt_decode(oracle.add(ca, cb, data), keys, scale), za + zb) < 1e-6


def test_matmul_tensor_decrypts_to_slot_matrix_product():
    """T = sum_l A_il (x) B_lj decrypts (with 1, s, s^2) to the slot-wise
    matrix product sum_l z(A_il) z(B_lj): exact numpy arithmetic on the
    plaintext slots, independent of the oracle's ring code."""
    N, scale = 1024, 2.0 ** 40          # product scale 2^80 under the 180-bit chain
    data, P = oracle.chain_primes(N, [60, 60, 60], 60)
    r = Rng(12)
    keys = ckks.keygen(N, data, P, r)
    m, k, n = 2, 3, 2
    zA = np.array([[r.complex_slots(N // 2) for _ in range(k)] for _ in range(m)])
    zB = np.array([[r.complex_slots(N // 2) for _ in range(n)] for _ in range(k)])
    A = np.stack([np.stack([ckks.encrypt(ckks.encode_real(zA[i, l], N, scale), keys, r) for l in range(k)])
                  for i in range(m)])
    B = np.stack([np.stack([ckks.encrypt(ckks.encode_real(zB[l, j], N, scale), keys, r) for j in range(n)])
                  for l in range(k)])
    T = oracle.matmul_tensor(A, B, data)
    assert T.shape == (m, n, 3, len(data), N)
    for i in range(m):
        for j in range(n):
            z = ckks.decrypt_decode(T[i, j], keys, scale * scale)
            exact = sum(zA[i, l] * zB[l, j] for l in range(k))
            assert _err(z, exact) < 1e-5


@pytest.mark.parametrize("N", [16, 2048])
def test_encode_unrounded_recovers_integer_polynomial(N):
    """Slots of an integer polynomial (evaluated directly at the slot roots)
    encode back to that polynomial's coefficients before any rounding."""
    r = Rng(N + 1)
    m = (r.unit_doubles(N) * 2e6 - 1e6).round()
    k = np.arange(N)
    z = np.array([np.sum(m * np.exp(1j * np.pi * pow(5, j, 2 * N) * k / N)) for j in range(N // 2)])
    got = ckks.encode_unrounded(z, N, 1.0)
    assert np.abs(got - m).max() < 1e-6
    assert np.array_equal(ckks.encode_real(z, N, 1.0), m.astype(np.int64))
