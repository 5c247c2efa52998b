"""Pins for the oracle's evaluation routines (Sec. II-A): Mul against the
decryption identity with schoolbook ring products, Relin and RS against
big-integer CRT arithmetic in Z_{PQ}[X]/(X^N+1) (Python integers)."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300.synth import Rng
from tests import bruteforce as bf


def _ring_mod(poly, q):
    return [v % q for v in poly]


@pytest.mark.parametrize("n", [1, 3])
def test_tensor_decryption_identity(n):
    """(a0 + a1 s)(b0 + b1 s) = d0 + d1 s + d2 s^2 in R_q for every limb."""
    N = 32
    qs = [oracle.find_primes(60, 2 * N, 1)[0]] + oracle.find_primes(50, 2 * N, n)[: n - 1]
    r = Rng(11)
    coef = [r.uniform_limbs(qs, N) for _ in range(4)]  # a0, a1, b0, b1 (coefficients)
    s = r.ternary(N)
    ct_a = np.stack([oracle.ntt_fwd(coef[0], qs), oracle.ntt_fwd(coef[1], qs)])
    ct_b = np.stack([oracle.ntt_fwd(coef[2], qs), oracle.ntt_fwd(coef[3], qs)])
    d = oracle.tensor(ct_a, ct_b, qs)
    dc = [oracle.ntt_inv(d[c], qs) for c in range(3)]
    s_list = [int(v) for v in s]
    s2 = bf.negacyclic_bigint(s_list, s_list)
    for l, q in enumerate(qs):
        a0, a1, b0, b1 = ([int(v) for v in c[l]] for c in coef)
        lhs_a = [x + y for x, y in zip(a0, bf.negacyclic_bigint(a1, s_list))]
        lhs_b = [x + y for x, y in zip(b0, bf.negacyclic_bigint(b1, s_list))]
        lhs = _ring_mod(bf.negacyclic_bigint(lhs_a, lhs_b), q)
        d0, d1, d2 = ([int(v) for v in dc[c][l]] for c in range(3))
        rhs = [x + y + z for x, y, z in zip(d0, bf.negacyclic_bigint(d1, s_list), bf.negacyclic_bigint(d2, s2))]
        assert lhs == _ring_mod(rhs, q)


def _chain(N, n_max):
    data = [oracle.find_primes(60, 2 * N, 1)[0]] + oracle.find_primes(50, 2 * N, n_max - 1)
    P = oracle.find_primes(60, 2 * N, 2)[1]
    return data, P


@pytest.mark.parametrize("N,n_max,level", [(16, 3, 2), (16, 3, 0), (32, 4, 1), (32, 4, 3), (64, 2, 1)])
def test_relin_bigint_bruteforce(N, n_max, level):
    """c'_k = d_k + round(x_k / P) mod q_i with x_k = sum_j c2_j evk[j][k]
    computed exactly in Z[X]/(X^N+1) and reduced mod P * Q_l."""
    data, P = _chain(N, n_max)
    n = level + 1
    qs = data[:n]
    r = Rng(1000 + N + level)
    # coefficient-domain inputs
    d_coef = [r.uniform_limbs(qs, N) for _ in range(3)]
    evk_coef = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(n_max)])
    # NTT-domain oracle inputs
    ct3 = np.stack([oracle.ntt_fwd(d_coef[c], qs) for c in range(3)])
    evk = np.empty_like(evk_coef)
    for j in range(n_max):
        for k in range(2):
            evk[j, k] = oracle.ntt_fwd(evk_coef[j, k], data + [P])
    out = oracle.relin(ct3, evk, data, P, level)
    out_coef = [oracle.ntt_inv(out[k], qs) for k in range(2)]

    PQ = P
    for q in qs:
        PQ *= q
    limb_sel = list(range(n)) + [n_max]  # q_0..q_l, then P
    mods = qs + [P]
    for k in range(2):
        x = [0] * N
        for j in range(n):
            digit = [int(v) for v in d_coef[2][j]]  # c2_j in [0, q_j)
            key = bf.crt([evk_coef[j, k, t] for t in limb_sel], mods)  # in [0, P Q_l)
            prod = bf.negacyclic_bigint(digit, key)
            x = [a + b for a, b in zip(x, prod)]
        x = [v % PQ for v in x]
        rounded = [(v + (P - 1) // 2) // P for v in x]  # round half up, P odd
        for i, q in enumerate(qs):
            expect = [(int(d) + v) % q for d, v in zip(d_coef[k][i], rounded)]
            assert [int(v) for v in out_coef[k][i]] == expect, (k, i)


@pytest.mark.parametrize("N,n,level", [(16, 3, 2), (32, 5, 4), (32, 5, 1), (64, 2, 1)])
def test_rescale_bigint_bruteforce(N, n, level):
    """c' = round(c / q_l) mod q_i for i < l, via the canonical CRT lift of
    c over Q_l = q_0 ... q_l."""
    data, _ = _chain(N, n)
    qs = data[: level + 1]
    r = Rng(2000 + N + level)
    coef = np.stack([r.uniform_limbs(qs, N) for _ in range(2)])
    ct = np.stack([oracle.ntt_fwd(coef[k], qs) for k in range(2)])
    out = oracle.rescale(ct, data, level)
    ql = qs[level]
    for k in range(2):
        X = bf.crt(coef[k], qs)
        rounded = [(v + (ql - 1) // 2) // ql for v in X]
        got = oracle.ntt_inv(out[k], qs[:level])
        for i in range(level):
            assert [int(v) for v in got[i]] == [v % qs[i] for v in rounded], (k, i)


def test_rescale_exact_division_property():
    """When every coefficient is a multiple of q_l, rescale is exact division."""
    N, level = 64, 2
    data, _ = _chain(N, 3)
    qs = data[: level + 1]
    r = Rng(3)
    small = [int(v) for v in r.uniform_mod(1 << 40, N)]
    ql = qs[level]
    coef = np.array([[(v * ql) % q for v in small] for q in qs], dtype=np.uint64)
    ct = np.stack([oracle.ntt_fwd(coef, qs), oracle.ntt_fwd(coef, qs)])
    out = oracle.rescale(ct, data, level)
    got = oracle.ntt_inv(out[0], qs[:level])
    for i in range(level):
        assert [int(v) for v in got[i]] == [v % qs[i] for v in small]
