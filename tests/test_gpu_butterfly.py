"""Algorithm 1's contract on the device primitive: the GPU butterflies give
x + W y and x - W y (forward) or x + y and (x - y) W (inverse) modulo p, with
outputs inside the documented lazy ranges, for random and extreme inputs --
checked against Python integers."""
import numpy as np
import pytest

from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, host  # noqa: E402

PRIMES = [he.primes_generate(60, 1 << 16, 1)[0], he.primes_generate(50, 1 << 16, 1)[0],
          he.primes_generate(40, 1 << 14, 1)[0], he.primes_generate(31, 1 << 11, 1)[0]]


def _cases(p, hi_bound, n, seed):
    r = Rng(seed)
    x = r.uniform_mod(hi_bound, n)
    y = r.uniform_mod(hi_bound, n)
    w = r.uniform_mod(p, n)
    edges_xy = [e for e in (0, hi_bound - 1, 4 * p - 1, 4 * p, 4 * p + (1 << 32) - 1, p, p - 1) if e < hi_bound]
    edges_w = [0, 1, p - 1]
    k = 0
    for ex in edges_xy:
        for ey in edges_xy:
            for ew in edges_w:
                x[k], y[k], w[k] = ex, ey, ew
                k += 1
    wsh = np.array([(int(v) << 64) // p for v in w], dtype=np.uint64)
    return x, y, w, wsh


@pytest.mark.parametrize("p", PRIMES)
def test_forward_butterfly_contract(p):
    bound = 8 * p + (1 << 32)
    x, y, w, wsh = _cases(p, bound, 4096, p % 1000)
    dx, dy = dev(x), dev(y)
    he.butterfly_apply(dx, dy, dev(w), dev(wsh), p)
    X, Y = host(dx), host(dy)
    for i in range(len(x)):
        a, b, c = int(x[i]), int(y[i]), int(w[i])
        assert int(X[i]) < bound and int(Y[i]) < bound, i
        assert int(X[i]) % p == (a + c * b) % p and int(Y[i]) % p == (a - c * b) % p, i


@pytest.mark.parametrize("p", PRIMES)
def test_inverse_butterfly_contract(p):
    x, y, w, wsh = _cases(p, 4 * p, 4096, p % 997)
    dx, dy = dev(x), dev(y)
    he.butterfly_apply(dx, dy, dev(w), dev(wsh), p, inverse=True)
    X, Y = host(dx), host(dy)
    for i in range(len(x)):
        a, b, c = int(x[i]), int(y[i]), int(w[i])
        assert int(X[i]) < 4 * p and int(Y[i]) < 4 * p, i
        assert int(X[i]) % p == (a + b) % p and int(Y[i]) % p == ((a - b) * c) % p, i
