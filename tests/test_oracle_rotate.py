"""Pins for the oracle's automorphism and Rotate (Sec. IV-C routine set):
brute force against polynomial arithmetic on Python integers, the ring
homomorphism property, composition, and decrypted slots rotated exactly as
numpy.roll rotates the plaintext slot vector."""
import numpy as np
import pytest

import oracle
from oracle import ckks
from paper_2109_14704_gb300.synth import Rng


def _poly_automorphism_bruteforce(a, g, q):
    """a(X^g) mod (X^N + 1, q) by reducing each monomial X^(g j) by hand."""
    N = len(a)
    out = [0] * N
    for j, c in enumerate(a):
        e = g * j
        sign = 1
        while e >= N:          # X^N = -1
            e -= N
            sign = -sign
        out[e] = (out[e] + sign * int(c)) % q
    return out


@pytest.mark.parametrize("g", [5, 25, 15, 3])
def test_automorphism_brute_force(g):
    q, N = 97, 8
    a = np.array([[3, 0, 96, 5, 1, 40, 7, 2]], dtype=np.uint64)
    assert list(oracle.automorphism(a, g, [q])[0]) == _poly_automorphism_bruteforce(list(a[0]), g, q)


def test_automorphism_is_a_ring_homomorphism_and_composes():
    N = 256
    qs = oracle.find_primes(50, 2 * N, 2)
    r = Rng(21)
    a, b = r.uniform_limbs(qs, N), r.uniform_limbs(qs, N)
    for g in (5, 125, 2 * N - 1):
        lhs = oracle.automorphism(oracle.negacyclic_mul(a, b, qs), g, qs)
        rhs = oracle.negacyclic_mul(oracle.automorphism(a, g, qs), oracle.automorphism(b, g, qs), qs)
        assert np.array_equal(lhs, rhs)
    assert np.array_equal(oracle.automorphism(oracle.automorphism(a, 5, qs), 25, qs),
                          oracle.automorphism(a, 125, qs))
    assert np.array_equal(oracle.automorphism(a, 1, qs), a)


@pytest.mark.parametrize("k", [1, 3])
def test_rotate_decrypts_to_rolled_slots(k):
    N, scale = 1024, 2.0 ** 40
    data, P = oracle.chain_primes(N, [60, 40, 40], 60)
    r = Rng(22)
    keys = ckks.keygen(N, data, P, r)
    g = pow(5, k, 2 * N)
    gk = ckks.galois_key(keys, g, r)
    z = r.complex_slots(N // 2)
    ct = ckks.encrypt(ckks.encode_real(z, N, scale), keys, r)
    out = oracle.rotate(ct, g, gk, data, P, len(data) - 1)
    got = ckks.decrypt_decode(out, keys, scale)
    assert float(np.abs(got - np.roll(z, -k)).max()) < 1e-5


def test_conjugation_decrypts_to_conjugate_slots():
    N, scale = 1024, 2.0 ** 40
    data, P = oracle.chain_primes(N, [60, 40, 40], 60)
    r = Rng(23)
    keys = ckks.keygen(N, data, P, r)
    g = 2 * N - 1
    gk = ckks.galois_key(keys, g, r)
    z = r.complex_slots(N // 2)
    ct = ckks.encrypt(ckks.encode_real(z, N, scale), keys, r)
    got = ckks.decrypt_decode(oracle.rotate(ct, g, gk, data, P, len(data) - 1), keys, scale)
    assert float(np.abs(got - np.conj(z)).max()) < 1e-5
