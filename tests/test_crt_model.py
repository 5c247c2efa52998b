"""CPU check of the CRT-lift arithmetic that decoding uses on the device
(Sec. II-A decoding, Sec. II-B RNS): with y_i = [c_i (Q/q_i)^-1]_{q_i} and
acc = sum_i y_i (Q/q_i) held in NW = ceil((log2 Q + 6) / 64) words, the
multiple of Q to subtract is estimated from acc's top two words as a double
against Q / 2^(64 (NW - 2)), rounded to the nearest integer, and one exact
correction brings the result into [-(Q-1)/2, (Q-1)/2]. This model follows
those steps with Python integers and IEEE doubles and checks the result
against the centred residue on random values and on values next to the
centring boundaries and zero (where the estimate is most often off by one),
for chains of 1 to 32 primes."""
import math
import random

import pytest

import oracle


def _words(x, nw):
    return [(x >> (64 * w)) & ((1 << 64) - 1) for w in range(nw)]


def _lift(residues, qs):
    Q = math.prod(qs)
    nw = max(2, (Q.bit_length() + 6 + 63) // 64)
    acc = 0
    for c, q in zip(residues, qs):
        Qi = Q // q
        acc += (c * pow(Qi % q, -1, q) % q) * Qi
    assert acc < 1 << (64 * nw - 1)                       # no carry out, sign bit clear
    aw, qw = _words(acc, nw), _words(Q, nw)
    top = math.ldexp(float(aw[nw - 1]), 64) + float(aw[nw - 2])     # fma(hi, 2^64, lo)
    qtop = math.ldexp(float(qw[nw - 1]), 64) + float(qw[nw - 2])
    assert qtop >= 2.0 ** 58 or nw == 2
    k = round(top * (1.0 / qtop))                          # nearest, ties to even (rint)
    r = acc - k * Q
    h = (Q - 1) // 2
    if r < -h:
        r += Q
    elif r > h:
        r -= Q
    return r


def _chain(n, bits):
    return oracle.find_primes(bits, 1 << 17, n)


@pytest.mark.parametrize("n,bits", [(1, 50), (1, 60), (2, 60), (3, 40), (8, 50), (17, 50), (20, 60), (32, 60)])
def test_lift_matches_centred_residue(n, bits):
    qs = _chain(n, bits)
    Q = math.prod(qs)
    h = (Q - 1) // 2
    rnd = random.Random(n * 100 + bits)
    values = [rnd.randrange(-h, h + 1) for _ in range(300)]
    for d in range(0, 40):
        values += [h - d, -h + d, d, -d, (Q // 3) - d, -(Q // 3) + d]
    values += [rnd.randrange(-(1 << 60), 1 << 60) for _ in range(50)]
    for x in values:
        if not -h <= x <= h:
            continue
        assert _lift([x % q for q in qs], qs) == x, x
