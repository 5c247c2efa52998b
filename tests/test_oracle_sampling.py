"""Pins for the oracle's restatement of the device's encryption randomness
(Sec. II-A Encrypt: ternary mask, Gaussian-like errors): the SplitMix64
generator against its published seed-0 reference outputs (Steele, Lea and
Flood 2014; the reference implementation's first outputs), the vectorised
draws against a scalar restatement of the definition on Python integers,
and the mappings against their exact laws (uniform ternary; the centred
binomial of parameter 20, i.e. e + 20 ~ Binomial(40, 1/2))."""
import math

import numpy as np

from oracle import ckks

M64 = (1 << 64) - 1


def _mix_scalar(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_published_outputs():
    got = [int(x) for x in ckks.splitmix64_outputs(0, np.arange(4, dtype=np.uint64))]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_draws_equal_scalar_restatement():
    seed, count, N = 0xDEADBEEFCAFEF00D, 3, 64
    v, e0, e1 = ckks.encryption_draws(seed, count, N)
    for w, arr in enumerate((v, e0, e1)):
        assert arr.shape == (count, N)
        for c in range(count):
            for i in range(N):
                r = _mix_scalar((seed + ((3 * c + w) * N + i + 1) * 0x9E3779B97F4A7C15) & M64)
                if w == 0:
                    want = r % 3 - 1
                else:
                    want = bin(r & 0xFFFFF).count("1") - bin((r >> 20) & 0xFFFFF).count("1")
                assert int(arr[c, i]) == want, (w, c, i)


def test_draw_laws():
    v, e0, e1 = ckks.encryption_draws(12345, 16, 1 << 15)
    n = v.size
    # ternary: each value with probability 1/3 (5-sigma binomial bounds)
    counts = np.bincount((v + 1).ravel(), minlength=3)
    sd = math.sqrt(n * (1 / 3) * (2 / 3))
    assert set(np.unique(v)) <= {-1, 0, 1}
    assert all(abs(cnt - n / 3) < 5 * sd for cnt in counts)
    # centred binomial: e + 20 ~ Binomial(40, 1/2): chi-square over the bins
    # with expectation >= 5 well below its 99.99th percentile
    for e in (e0, e1):
        assert e.min() >= -20 and e.max() <= 20
        hist = np.bincount((e + 20).ravel(), minlength=41)
        pmf = np.array([math.comb(40, k) for k in range(41)], dtype=np.float64) / 2.0 ** 40
        exp = pmf * n
        keep = exp >= 5
        chi2 = float((((hist - exp) ** 2) / exp)[keep].sum())
        assert chi2 < 80.0, chi2       # ~30 degrees of freedom
        assert abs(e.mean()) < 5 * math.sqrt(10 / n) and abs(e.var() - 10.0) < 0.1
    # the three draws of a message are different streams
    assert not np.array_equal(e0, e1)
