"""Pins for the oracle's parameter generation: primality, the prime search of
the RNS chain (Sec. II-B; primes below 2^60, Sec. III-A-1) and psi, the
primitive 2N-th root of unity (Sec. II-B)."""
import random

import pytest
import sympy
from sympy.ntheory.residue_ntheory import nthroot_mod

import oracle


def test_is_prime_small_exhaustive():
    for n in range(0, 20000):
        assert oracle.is_prime(n) == sympy.isprime(n), n


def test_is_prime_large_random_and_special():
    rnd = random.Random(7)
    cases = [rnd.getrandbits(64) | 1 for _ in range(2000)]
    # Carmichael numbers and strong pseudoprimes to small bases
    cases += [561, 41041, 825265, 3215031751, 3825123056546413051, 318665857834031151167461 % (1 << 64)]
    cases += [(1 << 61) - 1, (1 << 64) - 59, (1 << 62) - 57]
    for n in cases:
        assert oracle.is_prime(n) == sympy.isprime(n), n


@pytest.mark.parametrize("bits,two_n", [(60, 2 ** 13), (60, 2 ** 16), (50, 2 ** 15), (40, 2 ** 14)])
def test_find_primes_descending_first(bits, two_n):
    ps = oracle.find_primes(bits, two_n, 4)
    assert len(ps) == 4
    top = ((1 << bits) - 2) // two_n * two_n + 1
    cand = top
    for p in ps:
        assert p.bit_length() == bits and p % two_n == 1 and sympy.isprime(p)
        # every skipped candidate of the same residue class is composite
        while cand > p:
            assert not sympy.isprime(cand), cand
            cand -= two_n
        assert cand == p
        cand -= two_n


def test_find_primes_exclusion():
    first = oracle.find_primes(60, 2 ** 16, 3)
    again = oracle.find_primes(60, 2 ** 16, 2, exclude=[first[0]])
    assert again == first[1:3]


def test_psi_toy_by_hand():
    # 3^8 = 6561 = 16 = -1 (mod 17); 2^8 = 256 = 1 (mod 17), so 2 is no 16th root.
    assert oracle.find_psi(17, 8) == 3


def _psi_brute(q, N):
    return min(x for x in range(2, q) if pow(x, N, q) == q - 1)


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
def test_psi_brute_force_small_primes(N):
    found = 0
    q = 2 * N + 1
    while found < 6 and q < 40000:
        if sympy.isprime(q):
            assert oracle.find_psi(q, N) == _psi_brute(q, N), (q, N)
            found += 1
        q += 2 * N


@pytest.mark.parametrize("N", [1024, 4096, 8192])
def test_psi_large_against_sympy_roots(N):
    for bits in (60, 50):
        q = oracle.find_primes(bits, 2 * N, 1)[0]
        roots = nthroot_mod(q - 1, N, q, all_roots=True)
        psi = oracle.find_psi(q, N)
        assert len(roots) == N and psi == min(roots)
        assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1
