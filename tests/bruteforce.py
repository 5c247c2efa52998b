"""Brute-force references that pin the oracle: direct evaluation of the
transform's defining sum, schoolbook negacyclic convolution and big-integer
CRT arithmetic. Written independently of ``oracle/`` (Python integers and
numpy integer convolution only) so that a mistake in the oracle shows up as a
disagreement here."""
from __future__ import annotations

import numpy as np


def brv(x: int, logn: int) -> int:
    r = 0
    for _ in range(logn):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


def ntt_definition(a, q: int, psi: int, indices=None) -> list[int]:
    """out[i] = sum_j a_j psi^((2 brv(i) + 1) j) mod q, by Horner's rule, for
    the requested output indices (all by default)."""
    N = len(a)
    logn = N.bit_length() - 1
    coeffs = [int(x) for x in a]
    if indices is None:
        indices = range(N)
    out = []
    for i in indices:
        x = pow(psi, 2 * brv(i, logn) + 1, q)
        acc = 0
        for c in reversed(coeffs):
            acc = (acc * x + c) % q
        out.append(acc)
    return out


def negacyclic_schoolbook(a, b, q: int) -> list[int]:
    """c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j mod q, for
    coefficients below 2^60, with exact int64 numpy convolutions of 20-bit
    pieces (every partial sum stays below 2^53)."""
    a = np.asarray([int(x) for x in a], dtype=object)
    b = np.asarray([int(x) for x in b], dtype=object)
    N = len(a)
    mask = (1 << 20) - 1
    pa = [np.array([(int(x) >> (20 * s)) & mask for x in a], dtype=np.int64) for s in range(3)]
    pb = [np.array([(int(x) >> (20 * s)) & mask for x in b], dtype=np.int64) for s in range(3)]
    lin = [0] * (2 * N - 1)
    for s in range(3):
        for t in range(3):
            conv = np.convolve(pa[s], pb[t])
            shift = 20 * (s + t)
            for k in range(2 * N - 1):
                v = int(conv[k])
                if v:
                    lin[k] += v << shift
    return [(lin[k] - (lin[k + N] if k + N < 2 * N - 1 else 0)) % q for k in range(N)]


def negacyclic_bigint(a, b) -> list[int]:
    """Exact product in Z[X]/(X^N+1) of integer coefficient lists (small N)."""
    N = len(a)
    c = [0] * N
    for i in range(N):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(N):
            k = i + j
            if k < N:
                c[k] += ai * int(b[j])
            else:
                c[k - N] -= ai * int(b[j])
    return c


def crt(residues, moduli) -> list[int]:
    """Canonical representatives in [0, prod(moduli)) of [limbs][N] residues."""
    Q = 1
    for q in moduli:
        Q *= int(q)
    out = []
    N = len(residues[0])
    for i in range(N):
        x = 0
        for l, q in enumerate(moduli):
            Qi = Q // int(q)
            x += int(residues[l][i]) * Qi * pow(Qi, -1, int(q))
        out.append(x % Q)
    return out
