"""GPU parity at the rounding boundaries of key switching and rescaling
(Sec. II-A Relin and RS), bit-exact against the oracle.

Random residues almost never reach the values where the device takes its
rare branches, so these inputs plant them. In the coefficient domain:
  * the special-prime limb of the key-switching accumulator (the value that
    the mod-down by P rounds away) takes 0, 1, floor(P/2) - 1, floor(P/2),
    floor(P/2) + 1, P - 2 and P - 1 at chosen positions, or one of them at
    every position. This uses a key whose P limbs are the constants +1
    (component 0) and -1 (component 1) for digit 0 and 0 for the other
    digits, so that the accumulator's P limb is +-(digit 0 mod P);
  * the dropped limb q_l of a rescale takes the same values for q_l;
  * the digits are all zero or all q_j - 1.
A constant coefficient polynomial also makes every forward-transform output
of the rounding correction equal, which drives the lazy a + 12p - x
subtraction of the epilogues to the ends of its range.
Inputs reach the NTT domain through the oracle's forward transform. The
chains are the CKKS evaluation chain (N = 2^14: 60 + six 50-bit primes,
60-bit special prime) and the matrix chain with 40-bit primes (N = 2^13:
60/40/40, 60-bit special prime)."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests import edge_inputs as ei  # noqa: E402
from tests.gpu_util import dev, empty, host  # noqa: E402

CHAINS = {
    "ckks16k": (16384, [60] + [50] * 6, 60),
    "matrix8k": (8192, [60, 40, 40], 60),
}
LEVELS = {"ckks16k": 6, "matrix8k": 2}


def _ntt_rows(rows, qs):
    return oracle.ntt_fwd(np.stack(rows), qs)


def _setup(name):
    N, bits, pbits = CHAINS[name]
    data, P = he.chain_primes(N, bits, pbits)
    assert data == oracle.chain_primes(N, bits, pbits)[0]
    ctx = he.Context(N, data, P)
    return N, data, P, ctx


def _modup_scratch(ctx, N, level, modup):
    if modup == "expanded":
        return empty(ctx.relin_scratch_bytes(level) // 8)
    return empty((3 * (level + 1) + 2) * N)


# (key mode, digit mode): special-prime boundaries, constants at the
# boundary, and extreme digits with a random key
RELIN_CASES = [("pmod", "pedges"), ("pmod", "pconst:0"), ("pmod", "pconst:1"), ("pmod", "pconst:-1"),
               ("random", "zero"), ("random", "max"), ("random", "edges")]


@pytest.mark.parametrize("modup", ["expanded", "fused"])
@pytest.mark.parametrize("keymode,digmode", RELIN_CASES)
@pytest.mark.parametrize("name", ["ckks16k", "matrix8k"])
def test_relin_rounding_edges(name, keymode, digmode, modup):
    N, data, P, ctx = _setup(name)
    level = LEVELS[name]
    qs = data[:level + 1]
    r = Rng(700 + level)
    evk = ei.key(data, P, N, r, keymode)
    key = he.RelinKey(ctx, evk)
    d2 = _ntt_rows(ei.digits(qs, P, N, r, digmode), qs)
    c3 = np.stack([r.uniform_limbs(qs, N), r.uniform_limbs(qs, N), d2])
    out = empty(2, level + 1, N)
    he.relin(out, dev(c3), key, ctx, level, _modup_scratch(ctx, N, level, modup))
    assert np.array_equal(host(out), oracle.relin(c3, evk, data, P, level))


@pytest.mark.parametrize("mode", ["edges", "zero", "max", "h", "h+1", "h-1"])
@pytest.mark.parametrize("name", ["ckks16k", "matrix8k"])
def test_rescale_rounding_edges(name, mode):
    """The dropped limb q_l at its boundaries; the other limbs random."""
    N, data, P, ctx = _setup(name)
    r = Rng(710)
    for level in (LEVELS[name], 1):
        qs = data[:level + 1]
        ql = qs[level]
        m = {"h": f"const:{ql // 2}", "h+1": f"const:{ql // 2 + 1}", "h-1": f"const:{ql // 2 - 1}"}.get(mode, mode)
        comps = []
        for k in range(2):
            rows = [r.uniform_mod(q, N) for q in qs[:level]] + [ei.planted(ql, N, r, m)]
            comps.append(_ntt_rows(rows, qs))
        c = np.stack(comps)
        out = empty(2, level, N)
        he.rescale(out, dev(c), ctx, level, empty(ctx.rescale_scratch_bytes(level) // 8))
        assert np.array_equal(host(out), oracle.rescale(c, data, level)), level


def _ones(qs, N):
    return np.ones((len(qs), N), dtype=np.uint64)


@pytest.mark.parametrize("modup", ["expanded", "fused"])
@pytest.mark.parametrize("case", ["rescale_edges", "rescale_h", "moddown_edges", "moddown_const", "digits_max"])
@pytest.mark.parametrize("name", ["ckks16k", "matrix8k"])
def test_mul_relin_rescale_rounding_edges(name, case, modup):
    """The fused MulLinRS on planted inputs. With a = (1, 0) in the NTT
    domain the tensor is (b0, b1, 0): all-zero digits, and with the zero key
    the rescale input is b itself, so b's dropped limb carries the q_l
    boundaries. With a = (1, 1) the last tensor component is b1, which
    carries the digit patterns of the Relin cases."""
    N, data, P, ctx = _setup(name)
    level = LEVELS[name]
    qs = data[:level + 1]
    ql = qs[level]
    r = Rng(720)
    count = 3
    cas, cbs = [], []
    if case.startswith("rescale"):
        evk = ei.key(data, P, N, r, "zero")
        for c in range(count):
            a = np.stack([_ones(qs, N), np.zeros((len(qs), N), dtype=np.uint64)])
            mode = "edges" if case == "rescale_edges" else f"const:{ql // 2 + c - 1}"
            b = np.stack([_ntt_rows([r.uniform_mod(q, N) for q in qs[:level]] + [ei.planted(ql, N, r, mode)], qs)
                          for _ in range(2)])
            cas.append(a)
            cbs.append(b)
    else:
        evk = ei.key(data, P, N, r, "random" if case == "digits_max" else "pmod")
        for c in range(count):
            a = np.stack([r.uniform_limbs(qs, N), _ones(qs, N)])
            dmode = {"moddown_edges": "pedges", "moddown_const": f"pconst:{c - 1}", "digits_max": "max"}[case]
            b = np.stack([r.uniform_limbs(qs, N), _ntt_rows(ei.digits(qs, P, N, r, dmode), qs)])
            cas.append(a)
            cbs.append(b)
    ca, cb = np.stack(cas), np.stack(cbs)
    key = he.RelinKey(ctx, evk)
    out = empty(count, 2, level, N)
    if modup == "expanded":
        scratch = empty(ctx.mrr_scratch_bytes(level, count) // 8)
    else:
        scratch = empty((3 * (level + 1) + 4) * N * count)
    he.mul_relin_rescale(out, dev(ca), dev(cb), count, key, ctx, level, scratch)
    got = host(out)
    for c in range(count):
        assert np.array_equal(got[c], oracle.mul_relin_rescale(ca[c], cb[c], evk, data, P, level)), c


@pytest.mark.parametrize("digmode", ["pedges", "pconst:0", "zero", "max"])
@pytest.mark.parametrize("name", ["ckks16k", "matrix8k"])
def test_rotate_rounding_edges(name, digmode):
    """Rotate key-switches sigma(c1): planted c1 limbs (their automorphic
    images keep the boundary values, some negated) with the +-1 key on P or
    a random key."""
    N, data, P, ctx = _setup(name)
    level = LEVELS[name]
    qs = data[:level + 1]
    r = Rng(730)
    gk = ei.key(data, P, N, r, "pmod" if digmode.startswith("p") else "random")
    key = he.RelinKey(ctx, gk)
    g = pow(5, 3, 2 * N)
    c1 = _ntt_rows(ei.digits(qs, P, N, r, digmode), qs)
    ct = np.stack([r.uniform_limbs(qs, N), c1])
    out = empty(1, 2, level + 1, N)
    he.rotate(out, dev(ct[None]), 1, g, key, ctx, level, empty(ctx.rotate_scratch_bytes(level, 1) // 8))
    assert np.array_equal(host(out)[0], oracle.rotate(ct, g, gk, data, P, level))
