"""CPU pins of the modular-arithmetic bounds the kernels rely on (Algorithm 1
and its widened lazy ranges, Barrett reduction for Sec. III-A-1's mad_mod),
checked on an exact Python-integer model of each step as the device code
performs it (64-bit wrap-around made explicit), over random and extreme
inputs and primes from 2^30 to just below 2^60:

* the Shoup quotient from three 32 x 32 partial products is short of the
  exact quotient by at most 2, so W Y + Q' (2^64 - p) mod 2^64 is the
  integer W Y - Q' p in [0, 4p);
* the forward butterfly keeps x, y in [0, 8p + 2^32) with a high-word test;
* four conditional subtractions bring [0, 8p + 2^32) to [0, p);
* the forward transform's last butterfly, which reduces its input and the
  lazy product before the sum and the difference, gives canonical outputs;
* the inverse butterfly keeps [0, 4p);
* Barrett with one correction reduces any z < 2 p^2;
* the sign of the 64-bit difference decides x >= m for x, m < 2^63."""
import random

import pytest

import oracle

M64 = (1 << 64) - 1


def shoup_pre(w, p):
    return (w << 64) // p


def quotient_approx(w_sh, y):
    wl, wh = w_sh & 0xFFFFFFFF, w_sh >> 32
    yl, yh = y & 0xFFFFFFFF, y >> 32
    return wh * yh + ((wh * yl) >> 32) + ((wl * yh) >> 32)


def lazy4(y, w, w_sh, p):
    return (w * y + quotient_approx(w_sh, y) * ((1 << 64) - p)) & M64


def ct_butterfly(x, y, w, w_sh, p):
    h4 = (4 * p + 0xFFFFFFFF) >> 32
    X = x - 4 * p if (x >> 32) >= h4 else x
    T = lazy4(y, w, w_sh, p)
    return (X + T) & M64, (X + 4 * p - T) & M64


def reduce_once(x, m):
    d = (x - m) & M64
    return x if d >= 1 << 63 else d


def sub_mod(a, b, p):
    d = (a - b) & M64
    return (d + p) & M64 if d >= 1 << 63 else d


def ct_butterfly_canon(x, y, w, w_sh, p):
    T = lazy4(y, w, w_sh, p)
    X = reduce_from_fwd_range(x, p)
    T = reduce_once(reduce_once(T, 2 * p), p)
    return reduce_once(X + T, p), sub_mod(X, T, p)


def reduce_from_fwd_range(x, p):
    for m in (8 * p, 4 * p, 2 * p, p):
        x = reduce_once(x, m)
    return x


def gs_butterfly(x, y, w, w_sh, p):
    X = reduce_once(x + y, 4 * p)
    T = (x - y + 4 * p) & M64
    return X, lazy4(T, w, w_sh, p)


def barrett(z, p):
    b = p.bit_length()
    mu = (1 << (2 * b + 2)) // p
    q3 = ((z >> (b - 2)) * mu) >> (b + 4)
    return reduce_once((z - q3 * p) & M64, p)


PRIMES = [oracle.find_primes(30, 1 << 17, 1)[0], oracle.find_primes(31, 1 << 17, 1)[0],
          oracle.find_primes(45, 1 << 17, 1)[0], oracle.find_primes(50, 1 << 17, 1)[0],
          oracle.find_primes(60, 1 << 17, 1)[0], (1 << 30) + 1, (1 << 60) - 93]


def _cases(p, rnd, top):
    xs = [0, 1, p - 1, p, top - 1, top - 2, top // 2, (1 << 32) - 1, 1 << 32]
    return [x for x in xs if 0 <= x < top] + [rnd.randrange(top) for _ in range(400)]


@pytest.mark.parametrize("p", PRIMES)
def test_shoup_quotient_and_lazy_product(p):
    rnd = random.Random(p)
    for w in (1, 2, p - 1, p // 2, rnd.randrange(p)):
        w_sh = shoup_pre(w, p)
        for y in _cases(p, rnd, 1 << 64):
            q = (w_sh * y) >> 64
            qa = quotient_approx(w_sh, y)
            assert q - 2 <= qa <= q
            t = lazy4(y, w, w_sh, p)
            assert t < 4 * p and (t - w * y) % p == 0


@pytest.mark.parametrize("p", PRIMES)
def test_forward_butterfly_range(p):
    rnd = random.Random(p + 1)
    top = 8 * p + (1 << 32)
    assert top < 1 << 64
    for w in (1, p - 1, rnd.randrange(p)):
        w_sh = shoup_pre(w, p)
        xs, ys = _cases(p, rnd, top), _cases(p, rnd, top)
        for x, y in zip(xs, ys):
            x2, y2 = ct_butterfly(x, y, w, w_sh, p)
            assert x2 < top and y2 < top
            assert (x2 - (x + w * y)) % p == 0 and (y2 - (x - w * y)) % p == 0
            assert reduce_from_fwd_range(x2, p) == (x + w * y) % p


@pytest.mark.parametrize("p", PRIMES)
def test_forward_last_butterfly_canonical(p):
    rnd = random.Random(p + 5)
    top = 8 * p + (1 << 32)
    for w in (1, p - 1, rnd.randrange(p)):
        w_sh = shoup_pre(w, p)
        xs, ys = _cases(p, rnd, top), _cases(p, rnd, top)
        for x, y in zip(xs + xs[::-1], ys + ys):
            x2, y2 = ct_butterfly_canon(x, y, w, w_sh, p)
            assert x2 == (x + w * y) % p and y2 == (x - w * y) % p


@pytest.mark.parametrize("p", PRIMES)
def test_inverse_butterfly_range(p):
    rnd = random.Random(p + 2)
    for w in (1, p - 1, rnd.randrange(p)):
        w_sh = shoup_pre(w, p)
        for x, y in zip(_cases(p, rnd, 4 * p), _cases(p, rnd, 4 * p)):
            x2, y2 = gs_butterfly(x, y, w, w_sh, p)
            assert x2 < 4 * p and y2 < 4 * p
            assert (x2 - (x + y)) % p == 0 and (y2 - (x - y) * w) % p == 0


@pytest.mark.parametrize("p", PRIMES)
def test_barrett_one_correction(p):
    rnd = random.Random(p + 3)
    zs = [0, 1, p - 1, p, 2 * p * p - 1, p * p, 2 * p * p - p] + [rnd.randrange(2 * p * p) for _ in range(2000)]
    for z in zs:
        assert barrett(z, p) == z % p


def test_sign_tested_comparison():
    rnd = random.Random(9)
    vals = [0, 1, (1 << 63) - 1, (1 << 62), (1 << 60)] + [rnd.randrange(1 << 63) for _ in range(2000)]
    for x in vals:
        for m in (0, 1, x, (1 << 63) - 1, rnd.randrange(1 << 63)):
            assert reduce_once(x, m) == (x - m if x >= m else x)
