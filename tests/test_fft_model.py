"""CPU check of the slot-FFT formulation that the device encoder uses
(Sec. II-A encoding): a numpy model of its steps -- slot j placed at FFT
index t_j = (5^j mod 2N - 1) / 4, an n = N/2-point DFT computed as a
four-step FFT (columns of n1 points, twiddles omega^(k2 t1), rows of n2
points) whose short transforms are the kernel's decimation-in-frequency
stages (one radix-2 stage when the length is an odd power of two, then
radix-4 stages, output in bit-reversed order), the twist by zeta^-k and the
split of w_k into m_k and m_{k+n} -- must give the oracle's unrounded
encoding, and the reverse direction the oracle's slot evaluation. A wrong
index, twiddle, twist or stage formula in this formulation fails here
without a GPU."""
import numpy as np
import pytest

from oracle import ckks
from paper_2109_14704_gb300.synth import Rng


def _brev(t, bits):
    return int(format(t, f"0{bits}b")[::-1], 2) if bits else 0


def _dif(x, sign, n_full):
    """Decimation in frequency of len(x) points with omega = exp(sign 2 pi i /
    n_full)^(n_full / len): radix-2 first for odd log2, then radix-4 stages."""
    x = np.array(x, dtype=np.complex128)
    L = len(x)
    logL = L.bit_length() - 1
    w = lambda e: np.exp(sign * 2j * np.pi * e / n_full)
    log_g = logL
    if logL & 1:
        h = L // 2
        for r in range(h):
            a, b = x[r], x[r + h]
            x[r], x[r + h] = a + b, (a - b) * w(r * (n_full // (2 * h)))
        log_g -= 1
    while log_g >= 2:
        g, h = 1 << log_g, 1 << (log_g - 2)
        sh = n_full // g
        for base in range(0, L, g):
            for r in range(h):
                x0, x1, x2, x3 = x[base + r], x[base + r + h], x[base + r + 2 * h], x[base + r + 3 * h]
                s02, d02, s13, t = x0 + x2, x0 - x2, x1 + x3, x1 - x3
                d13 = t * (-1j if sign < 0 else 1j)
                x[base + r] = s02 + s13
                x[base + r + h] = (s02 - s13) * w(2 * r * sh)
                x[base + r + 2 * h] = (d02 + d13) * w(r * sh)
                x[base + r + 3 * h] = (d02 - d13) * w(3 * r * sh)
        log_g -= 2
    return np.array([x[_brev(t, logL)] for t in range(L)])


def _four_step(x, sign):
    n = len(x)
    log_n = n.bit_length() - 1
    n1 = 1 << (log_n // 2)
    n2 = n // n1
    Y = np.empty((n1, n2), dtype=np.complex128)
    for k2 in range(n2):
        col = _dif(x[k2::n2], sign, n)
        for t1 in range(n1):
            Y[t1, k2] = col[t1] * np.exp(sign * 2j * np.pi * k2 * t1 / n)
    X = np.empty(n, dtype=np.complex128)
    for t1 in range(n1):
        row = _dif(Y[t1], sign, n)
        for t2 in range(n2):
            X[t1 + n1 * t2] = row[t2]
    return X


def _slot_index(N):
    n = N // 2
    t = np.empty(n, dtype=np.int64)
    e = 1
    for j in range(n):
        t[j] = (e - 1) // 4
        e = e * 5 % (2 * N)
    return t


@pytest.mark.parametrize("N", [32, 64, 512, 2048])
def test_encode_formulation_matches_oracle(N):
    n, scale = N // 2, 2.0 ** 20
    z = Rng(N).complex_slots(n)
    t = _slot_index(N)
    assert sorted(t) == list(range(n))          # 5^j mod 2N covers every 1 mod 4 once
    X = np.zeros(n, dtype=np.complex128)
    X[t] = scale * z
    u = _four_step(X, -1) / n
    w = u * np.exp(-1j * np.pi * np.arange(n) / N)
    m = np.concatenate([w.real, w.imag])
    ref = ckks.encode_unrounded(z, N, scale)
    assert np.abs(m - ref).max() < 1e-6 * scale


@pytest.mark.parametrize("N", [32, 256, 1024])
def test_decode_formulation_matches_oracle(N):
    n = N // 2
    m = np.array(Rng(N + 7).uniform_limbs([1 << 20], N)[0], dtype=np.float64) - (1 << 19)
    w = (m[:n] + 1j * m[n:]) * np.exp(1j * np.pi * np.arange(n) / N)
    X = _four_step(w, +1)
    z = X[_slot_index(N)]
    ref = ckks.eval_slots(m, N)
    assert np.abs(z - ref).max() < 1e-9 * np.abs(ref).max()
