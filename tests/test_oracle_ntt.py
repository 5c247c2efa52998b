"""Pins for the oracle's negacyclic NTT (Sec. II-B): the defining sum
evaluated directly, monomials and the constant polynomial in closed form,
linearity, exact inversion, and the convolution theorem against schoolbook
negacyclic convolution."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300.synth import Rng
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_toy_q17():
    g = json.load(open(os.path.join(GOLDEN, "toy_ntt_q17_n8.json")))
    a = np.array([g["input"]], dtype=np.uint64)
    assert oracle.find_psi(g["q"], g["N"]) == g["psi"]
    assert list(oracle.ntt_fwd(a, [g["q"]])[0]) == g["ntt_fwd"]
    # the stored values are the defining sum
    assert bf.ntt_definition(g["input"], g["q"], g["psi"]) == g["ntt_fwd"]


def test_golden_n4096_samples():
    g = json.load(open(os.path.join(GOLDEN, "ntt_n4096_seed1.json")))
    qs, N = g["moduli"], g["N"]
    assert oracle.find_primes(60, 2 * N, 2) == qs
    x = Rng(g["seed"]).uniform_limbs(qs, N)
    assert [int(v) for v in x[0, :4]] == g["input_head"]
    X = oracle.ntt_fwd(x, qs)
    for l, key in enumerate(("ntt_fwd_limb0", "ntt_fwd_limb1")):
        assert [int(X[l, i]) for i in g["sample_index"]] == g[key]
        assert bf.ntt_definition(x[l], qs[l], g["psi"][l], g["sample_index"]) == g[key]


@pytest.mark.parametrize("N", [2, 4, 16, 64, 256])
@pytest.mark.parametrize("bits", [60, 50, 30])
def test_forward_equals_definition_small(N, bits):
    q = oracle.find_primes(bits, 2 * N, 1)[0]
    x = Rng(100 + N).uniform_limbs([q], N)
    psi = oracle.find_psi(q, N)
    assert [int(v) for v in oracle.ntt_fwd(x, [q])[0]] == bf.ntt_definition(x[0], q, psi)


@pytest.mark.parametrize("N", [1024, 4096, 8192, 16384, 32768, 65536])
def test_forward_sampled_outputs_full_size(N):
    qs = oracle.find_primes(60, 2 * N, 1) + oracle.find_primes(50, 2 * N, 1)
    x = Rng(N).uniform_limbs(qs, N)
    X = oracle.ntt_fwd(x, qs)
    idx = [0, 1, N // 2 - 1, N // 2, N - 2, N - 1, 12345 % N, 777 % N]
    for l, q in enumerate(qs):
        assert [int(X[l, i]) for i in idx] == bf.ntt_definition(x[l], q, oracle.find_psi(q, N), idx)


@pytest.mark.parametrize("N", [16, 256, 4096])
def test_monomials_and_constant(N):
    q = oracle.find_primes(60, 2 * N, 1)[0]
    psi = oracle.find_psi(q, N)
    logn = N.bit_length() - 1
    one = np.zeros((1, N), dtype=np.uint64)
    one[0, 0] = 1
    assert (oracle.ntt_fwd(one, [q]) == 1).all()
    for k in (1, 2, N // 2, N - 1):
        mono = np.zeros((1, N), dtype=np.uint64)
        mono[0, k] = 1
        out = oracle.ntt_fwd(mono, [q])[0]
        for i in (0, 1, N // 3, N - 1):
            assert int(out[i]) == pow(psi, (2 * bf.brv(i, logn) + 1) * k, q)


def test_linearity():
    N = 2048
    q = oracle.find_primes(60, 2 * N, 1)[0]
    r = Rng(5)
    a, b = r.uniform_limbs([q], N), r.uniform_limbs([q], N)
    c = 987654321987
    comb = np.array([[(int(x) + c * int(y)) % q for x, y in zip(a[0], b[0])]], dtype=np.uint64)
    lhs = oracle.ntt_fwd(comb, [q])
    A, B = oracle.ntt_fwd(a, [q]), oracle.ntt_fwd(b, [q])
    rhs = [(int(A[0, i]) + c * int(B[0, i])) % q for i in range(N)]
    assert [int(v) for v in lhs[0]] == rhs


@pytest.mark.parametrize("logn", list(range(1, 17)))
def test_inverse_round_trip(logn):
    N = 1 << logn
    qs = oracle.find_primes(60, max(2 * N, 2 ** 13), 1) + oracle.find_primes(50, max(2 * N, 2 ** 13), 1)
    x = Rng(logn).uniform_limbs(qs, N)
    assert (oracle.ntt_inv(oracle.ntt_fwd(x, qs), qs) == x).all()
    assert (oracle.ntt_fwd(oracle.ntt_inv(x, qs), qs) == x).all()


def test_inverse_of_all_ones_is_unit_constant():
    N = 1024
    q = oracle.find_primes(60, 2 * N, 1)[0]
    y = np.ones((1, N), dtype=np.uint64)
    out = oracle.ntt_inv(y, [q])[0]
    assert int(out[0]) == 1 and not out[1:].any()


@pytest.mark.parametrize("N", [4, 32, 256])
def test_convolution_theorem_small(N):
    q = oracle.find_primes(60, 2 * N, 1)[0]
    r = Rng(9 + N)
    a, b = r.uniform_limbs([q], N), r.uniform_limbs([q], N)
    exact = bf.negacyclic_bigint(a[0], b[0])
    assert [int(v) for v in oracle.negacyclic_mul(a, b, [q])[0]] == [v % q for v in exact]


def test_convolution_theorem_plain_workload():
    """Plain workload: N = 4096, two 60-bit primes, seed 1, checked against
    schoolbook O(N^2) negacyclic convolution."""
    N = 4096
    qs = oracle.find_primes(60, 2 * N, 2)
    r = Rng(1)
    a, b = r.uniform_limbs(qs, N), r.uniform_limbs(qs, N)
    prod = oracle.negacyclic_mul(a, b, qs)
    for l, q in enumerate(qs):
        assert [int(v) for v in prod[l]] == bf.negacyclic_schoolbook(a[l], b[l], q)
