"""CPU checks of the planted inputs that the rounding-boundary GPU tests use
(Sec. II-A Relin and RS), on the oracle alone: the boundary values land where
claimed, and with the +-1 key on the special prime the key-switching
accumulator's P limb equals +-(digit 0 mod P) in the coefficient domain, so
the mod-down's rounding input v = (x + floor(P/2)) mod P reaches both ends of
[0, P)."""
import numpy as np

import oracle
from paper_2109_14704_gb300.synth import Rng
from tests import edge_inputs as ei


def _chain():
    N = 1024
    data, P = oracle.chain_primes(N, [60, 40, 40], 60)
    return N, data, P


def test_boundary_values_planted():
    N, data, P = _chain()
    r = Rng(741)
    for q in data + [P]:
        vals = ei.boundary_values(q)
        assert vals == [0, 1, q // 2 - 1, q // 2, q // 2 + 1, q - 2, q - 1]
        x = ei.planted(q, N, r, "edges")
        for base in (0, N // 2, N - len(vals)):
            assert [int(v) for v in x[base:base + len(vals)]] == vals
        assert (x < q).all()
        assert (ei.planted(q, N, r, "max") == q - 1).all() and (ei.planted(q, N, r, "zero") == 0).all()
        assert (ei.planted(q, N, r, f"const:{q // 2 + 1}") == q // 2 + 1).all()


def test_pmod_key_exposes_digit_zero_on_the_special_prime():
    N, data, P = _chain()
    assert P < data[0]                  # the P boundary values are valid digits mod q_0
    r = Rng(742)
    evk = ei.key(data, P, N, r, "pmod")
    nd = len(data)
    # the NTT-domain key limbs are the transforms of the constants +1 and -1
    one = np.zeros((1, N), dtype=np.uint64)
    one[0, 0] = 1
    assert np.array_equal(evk[0, 0, nd][None], oracle.ntt_fwd(one, [P]))
    assert np.array_equal(evk[0, 1, nd][None], oracle.ntt_fwd(np.array([[P - 1] + [0] * (N - 1)], dtype=np.uint64), [P]))
    assert not evk[1:, :, nd].any()
    rows = ei.digits(data, P, N, r, "pedges")
    c2_0 = rows[0]
    # accumulator's P limb: sum_j NTT_P(c2_j mod P) * evk[j][k][P] = NTT_P(+-c2_0)
    for k, sign in ((0, 1), (1, -1)):
        acc = oracle.dyadic(oracle.ntt_fwd((c2_0 % np.uint64(P))[None], [P]), evk[0, k, nd][None], [P])
        x = oracle.ntt_inv(acc, [P])[0]
        expect = np.array([(sign * int(c)) % P for c in c2_0], dtype=np.uint64)
        assert np.array_equal(x, expect)
        v = [(int(t) + P // 2) % P for t in x[:7]]
        assert 0 in v and P - 1 in v
    # the constant digit modes put v at one point everywhere
    for k_off, v_want in ((0, P - 1), (1, 0), (-1, P - 2)):
        c = ei.digits(data, P, N, r, f"pconst:{k_off}")[0]
        assert ((c.astype(object) + P // 2) % P == v_want).all()
