"""GPU parity of device encoding and decoding (Sec. II-A Encode / Decode).

* CRT lift: bit-exact against the oracle's centred lift (Python integers)
  converted to the nearest double, on random residues, on the values that
  decide the centring (0, +-1, +-(Q-1)/2) and on rounding ties.
* Decode: slots against the oracle's decode of the same plaintext.
* Encode: the FFT differs from the oracle's in rounding order, so a
  coefficient whose exact value sits next to a half-integer may round either
  way. Every coefficient must be within 1/2 + delta of the oracle's
  unrounded value (delta bounds the FP64 error of both FFTs), must equal the
  oracle's rounding wherever the value is farther than delta from a tie, and
  every limb must hold the residue of the same integer.
* Round trips decode(encode(z)) = z within FP64 accuracy.
The decoded-slot bar is 1e-5 relative (normwise); the tests assert 1e-9."""
import math

import numpy as np
import pytest

import oracle
from oracle import ckks
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import dev, empty, host  # noqa: E402

CHAINS = {
    "n1k": (1024, [60, 50], 60),
    "n4k": (4096, [60, 50, 50, 50], 60),
    "n8k": (8192, [60, 40, 40], 60),
    "n16k": (16384, [60] + [50] * 6, 60),
    "n64k": (65536, [60, 50], 60),
    "long": (2048, [60] + [50] * 18, 60),   # Q up to 960 bits: 16-word lifts
}
_ctx_cache = {}


def _setup(name):
    if name not in _ctx_cache:
        N, bits, pbits = CHAINS[name]
        data, P = he.chain_primes(N, bits, pbits)
        ctx = he.Context(N, data, P)
        _ctx_cache[name] = (N, data, ctx, he.Encoder(ctx))
    return _ctx_cache[name]


def _err(z, ref):
    return float(np.abs(z - ref).max() / max(1.0, np.abs(ref).max()))


def _residues(vals, qs):
    """[limbs][len(vals)] residues of Python integers."""
    return np.array([[v % q for v in vals] for q in qs], dtype=np.uint64)


def _crt_expected(res, qs):
    return np.array([float(v) for v in ckks.crt_centered(res, qs)])


def _slots_dev(z):
    return torch.from_numpy(np.ascontiguousarray(z, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("name,level,count", [("n1k", 1, 3), ("n4k", 0, 2), ("n4k", 3, 2), ("n16k", 6, 1),
                                              ("long", 18, 2), ("long", 9, 1)])
def test_crt_compose_bit_exact(name, level, count):
    N, data, ctx, enc = _setup(name)
    qs = data[:level + 1]
    r = Rng(300 + level)
    res = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    out = torch.empty((count, N), dtype=torch.float64, device="cuda")
    enc.crt_compose(out, dev(res), count, level)
    got = out.cpu().numpy()
    for c in range(count):
        assert np.array_equal(got[c], _crt_expected(res[c], qs)), c


@pytest.mark.parametrize("name,level", [("n4k", 0), ("n4k", 3), ("long", 18)])
def test_crt_compose_edges(name, level):
    """Centring boundaries, small values and round-to-nearest-even ties
    (with and without bits below the tie)."""
    N, data, ctx, enc = _setup(name)
    qs = data[:level + 1]
    Q = math.prod(qs)
    h = (Q - 1) // 2
    vals = [0, 1, -1, 2, -2, h, -h, h - 1, -(h - 1), 2 ** 53, 2 ** 53 + 1, -(2 ** 53 + 1), 2 ** 53 + 3,
            2 ** 60 + 2 ** 7, 2 ** 60 + 2 ** 7 + 1, 2 ** 60 + 3 * 2 ** 7, -(2 ** 60 + 3 * 2 ** 7)]
    for top in (100, 200, 400, 800):
        if top < Q.bit_length() - 2:
            ulp = 2 ** (top - 52)
            vals += [2 ** top + ulp // 2, 2 ** top + ulp // 2 + 1, 2 ** top + 3 * ulp // 2, -(2 ** top + ulp // 2 + 1),
                     2 ** top + ulp // 2 + 2 ** (top - 150 if top > 150 else 0)]
    vals = [v for v in vals if -h <= v <= h]
    r = Rng(400 + level)
    res = r.uniform_limbs(qs, N)
    res[:, :len(vals)] = _residues(vals, qs)
    out = torch.empty((1, N), dtype=torch.float64, device="cuda")
    enc.crt_compose(out, dev(res), 1, level)
    got = out.cpu().numpy()[0]
    exp = _crt_expected(res, qs)
    assert np.array_equal(got, exp)
    assert [float(v) for v in vals] == list(got[:len(vals)])


@pytest.mark.parametrize("name,level,count", [("n1k", 1, 2), ("n4k", 3, 3), ("n8k", 2, 2), ("n64k", 1, 1)])
def test_decode_matches_oracle(name, level, count):
    """Encoded messages (scale 2^40) and random residues (values up to Q/2)."""
    N, data, ctx, enc = _setup(name)
    qs = data[:level + 1]
    r = Rng(500 + level)
    scale = 2.0 ** 40
    pts, refs = [], []
    for c in range(count):
        if c % 2 == 0:
            coef = ckks.to_residues(ckks.encode_real(r.complex_slots(N // 2), N, scale), qs)
        else:
            coef = r.uniform_limbs(qs, N)
        pts.append(oracle.ntt_fwd(coef, qs))
        refs.append(ckks.decode(coef, qs, scale))
    pt = dev(np.stack(pts))
    before = host(pt).copy()
    z = torch.empty((count, N // 2), dtype=torch.complex128, device="cuda")
    enc.decode(z, pt, count, scale, level, empty(enc.decode_scratch_bytes(level, count) // 8))
    got = z.cpu().numpy()
    for c in range(count):
        assert _err(got[c], refs[c]) < 1e-9, c
    assert np.array_equal(host(pt), before)   # the input is not modified


def _check_encoding(pt_ntt, z, N, qs, scale):
    """Validity of one device-encoded plaintext against the oracle."""
    coef = oracle.ntt_inv(pt_ntt, qs)
    q0 = int(qs[0])
    m = coef[0].astype(object)
    m = np.array([int(v) - q0 if int(v) > q0 // 2 else int(v) for v in m], dtype=object)
    for l, q in enumerate(qs):   # every limb holds the same integer
        assert np.array_equal(coef[l], np.array([v % int(q) for v in m], dtype=np.uint64)), l
    exact = ckks.encode_unrounded(z, N, scale)
    md = m.astype(np.float64)
    delta = 2.0 ** -48 * scale * max(1.0, float(np.abs(z).max())) * math.log2(N)
    dev_from_exact = np.abs(md - exact)
    assert dev_from_exact.max() <= 0.5 + delta, dev_from_exact.max()
    frac = np.abs(exact - np.floor(exact) - 0.5)
    differs = md != np.rint(exact)
    assert np.all(frac[differs] <= delta), frac[differs].max()
    assert differs.sum() <= max(2, N // 100)
    return int(differs.sum())


@pytest.mark.parametrize("name,level,count,scale", [("n1k", 1, 2, 2.0 ** 40), ("n4k", 3, 3, 2.0 ** 40),
                                                    ("n8k", 2, 2, 2.0 ** 30), ("n16k", 6, 1, 2.0 ** 40),
                                                    ("n64k", 1, 1, 2.0 ** 45), ("n4k", 0, 1, 1.0)])
def test_encode_valid_rounding(name, level, count, scale):
    N, data, ctx, enc = _setup(name)
    qs = data[:level + 1]
    r = Rng(600 + level)
    z = np.stack([r.complex_slots(N // 2) for _ in range(count)])
    if scale == 1.0:
        z = z * 1000.0
    pt = empty(count, level + 1, N)
    enc.encode(pt, _slots_dev(z), count, scale, level, empty(enc.encode_scratch_bytes(count) // 8))
    got = host(pt)
    for c in range(count):
        _check_encoding(got[c], z[c], N, qs, scale)


def test_encode_matches_oracle_limbs_exactly_on_integer_slots():
    """Slots that make every coefficient an exact small integer (m = sum of
    a few monomials, encoded by the oracle first): no rounding freedom, so the
    NTT-domain limbs equal the oracle's bit for bit."""
    N, data, ctx, enc = _setup("n4k")
    level, qs = 3, data[:4]
    m = np.zeros(N, dtype=np.int64)
    m[[0, 1, 7, N // 2, N - 1]] = [5, -3, 1 << 20, -(1 << 30), 12345]
    z = ckks.eval_slots(m.astype(np.float64), N)   # slots of m at scale 1
    pt = empty(1, level + 1, N)
    enc.encode(pt, _slots_dev(z[None]), 1, 1.0, level, empty(enc.encode_scratch_bytes(1) // 8))
    assert np.array_equal(host(pt)[0], oracle.ntt_fwd(ckks.to_residues(m, qs), qs))


@pytest.mark.parametrize("name,level,count", [("n1k", 1, 4), ("n8k", 2, 3), ("n16k", 6, 2), ("n64k", 1, 2)])
def test_round_trip(name, level, count):
    N, data, ctx, enc = _setup(name)
    r = Rng(700 + level)
    z = np.stack([r.complex_slots(N // 2) for _ in range(count)])
    scale = 2.0 ** 40
    pt = empty(count, level + 1, N)
    enc.encode(pt, _slots_dev(z), count, scale, level, empty(enc.encode_scratch_bytes(count) // 8))
    out = torch.empty((count, N // 2), dtype=torch.complex128, device="cuda")
    enc.decode(out, pt, count, scale, level, empty(enc.decode_scratch_bytes(level, count) // 8))
    got = out.cpu().numpy()
    for c in range(count):
        assert _err(got[c], z[c]) < 1e-9, c


def test_full_size_sampled():
    """The routine-set size (N = 2^15, 60 + 7 x 50-bit primes, level 7),
    16 messages: round trip for all, oracle checks on two of them."""
    N = 32768
    data, P = he.chain_primes(N, [60] + [50] * 7, 60)
    ctx = he.Context(N, data, P)
    enc = he.Encoder(ctx)
    level, count, scale = 7, 16, 2.0 ** 40
    r = Rng(800)
    z = np.stack([r.complex_slots(N // 2) for _ in range(count)])
    pt = empty(count, level + 1, N)
    enc.encode(pt, _slots_dev(z), count, scale, level, empty(enc.encode_scratch_bytes(count) // 8))
    out = torch.empty((count, N // 2), dtype=torch.complex128, device="cuda")
    enc.decode(out, pt, count, scale, level, empty(enc.decode_scratch_bytes(level, count) // 8))
    got_pt, got_z = host(pt), out.cpu().numpy()
    for c in range(count):
        assert _err(got_z[c], z[c]) < 1e-9, c
    for c in (0, count - 1):
        _check_encoding(got_pt[c], z[c], N, data, scale)
        ref = ckks.decode(oracle.ntt_inv(got_pt[c], data), data, scale)
        assert _err(got_z[c], ref) < 1e-9


def test_edge_cases():
    N, data, ctx, enc = _setup("n4k")
    sc = empty(enc.decode_scratch_bytes(3, 2) // 8)
    pt = empty(2, 4, N)
    z0 = torch.zeros((2, N // 2), dtype=torch.complex128, device="cuda")
    enc.encode(pt, z0, 0, 2.0 ** 40, 3, sc)          # count 0: nothing to do
    enc.encode(pt, z0, 2, 2.0 ** 40, 3, sc)          # zero slots -> zero plaintext
    assert not host(pt).any()
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(he.HeError):
            enc.encode(pt, z0, 2, bad, 3, sc)
    with pytest.raises(he.HeError):
        enc.encode(empty(2, 5, N), z0, 2, 2.0 ** 40, 4, sc)   # level beyond the chain
    with pytest.raises(he.HeError):
        enc.decode(z0, pt, 2, 2.0 ** 40, 3, empty(16))   # short scratch
    with pytest.raises(ValueError):
        enc.decode(z0[:1], pt, 2, 2.0 ** 40, 3, sc)      # short output (binding check)


def _i8(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int8)).cuda()


@pytest.mark.parametrize("level", [3, 1])
def test_encrypt_matches_oracle(level):
    """Public-key encryption (Sec. II-A) with the same draws as the oracle's
    (v ternary, e0 and e1 rounded Gaussian, in that order from one seeded
    generator): bit-exact ciphertexts."""
    N, data, ctx, enc = _setup("n4k")
    P = ctx.P
    keys = ckks.keygen(N, data, P, Rng(900))
    qs = data[:level + 1]
    count = 2
    m = [ckks.encode_real(Rng(901 + c).complex_slots(N // 2), N, 2.0 ** 40) for c in range(count)]
    ref = [ckks.encrypt(m[c], keys, Rng(910 + c), level) for c in range(count)]
    draws = [Rng(910 + c) for c in range(count)]
    v, e0, e1 = [], [], []
    for r in draws:
        v.append(r.ternary(N))
        e0.append(r.gaussian(N))
        e1.append(r.gaussian(N))
    pt = dev(np.stack([oracle.ntt_fwd(ckks.to_residues(m[c], qs), qs) for c in range(count)]))
    ct = empty(count, 2, level + 1, N)
    he.encrypt(ct, pt, dev(keys.pk), _i8(np.stack(v)), _i8(np.stack(e0)), _i8(np.stack(e1)), count, ctx, level,
               empty(ctx.encrypt_scratch_bytes(level, count) // 8))
    got = host(ct)
    for c in range(count):
        assert np.array_equal(got[c], ref[c]), c


def test_device_ckks_pipeline():
    """Encode, encrypt, MulLinRS and decode on the device (decryption with the
    secret key on the host): the decoded product matches the exact complex
    product within the 1e-5 bar."""
    N, data, ctx, enc = _setup("n8k")
    P, L, scale = ctx.P, len(data) - 1, 2.0 ** 40
    keys = ckks.keygen(N, data, P, Rng(920))
    key = he.RelinKey(ctx, keys.evk)
    r = Rng(921)
    za, zb = r.complex_slots(N // 2), r.complex_slots(N // 2)
    pt = empty(2, L + 1, N)
    enc.encode(pt, _slots_dev(np.stack([za, zb])), 2, scale, L, empty(enc.encode_scratch_bytes(2) // 8))
    draws = [[r.ternary(N), r.gaussian(N), r.gaussian(N)] for _ in range(2)]
    ct = empty(2, 2, L + 1, N)
    he.encrypt(ct, pt, dev(keys.pk), *[_i8(np.stack([d[w] for d in draws])) for w in range(3)], 2, ctx, L,
               empty(ctx.encrypt_scratch_bytes(L, 2) // 8))
    out = empty(1, 2, L, N)
    he.mul_relin_rescale(out, ct[0:1], ct[1:2], 1, key, ctx, L, empty(ctx.mrr_scratch_bytes(L, 1) // 8))
    dec = ckks.decrypt_residues(host(out)[0], keys)                  # coefficient domain
    z = torch.empty((1, N // 2), dtype=torch.complex128, device="cuda")
    enc.decode(z, dev(oracle.ntt_fwd(dec, data[:L])[None]), 1, scale * scale / data[L], L - 1,
               empty(enc.decode_scratch_bytes(L - 1, 1) // 8))
    exact = za * zb
    assert _err(z.cpu().numpy()[0], exact) < 1e-5


@pytest.mark.parametrize("N,count,seed", [(4096, 3, 1), (32768, 2, 0xFFFFFFFFFFFFFFFF), (1024, 5, 77)])
def test_device_sampled_draws_match_oracle(N, count, seed):
    """The encryption randomness drawn on the device (SplitMix64 counter
    form, ternary mask, centred-binomial errors) equals the oracle's
    restatement of the same definition bit for bit."""
    v, e0, e1 = (torch.empty((count, N), dtype=torch.int8, device="cuda") for _ in range(3))
    he.sample_encryption_draws(v, e0, e1, count, N, seed)
    ref = ckks.encryption_draws(seed, count, N)
    for got, want in zip((v, e0, e1), ref):
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy().astype(np.int64), want)


@pytest.mark.parametrize("level", [3, 1])
def test_encrypt_seeded_matches_oracle(level):
    """Encryption with the randomness drawn on the device equals the oracle's
    encryption with the oracle's draws for the same seed, bit for bit, and
    decrypts to the message (the errors are small)."""
    N, data, ctx, enc = _setup("n4k")
    keys = ckks.keygen(N, data, ctx.P, Rng(930))
    qs = data[:level + 1]
    count, seed = 3, 0x1234_5678_9ABC_DEF0
    m = [ckks.encode_real(Rng(931 + c).complex_slots(N // 2), N, 2.0 ** 40) for c in range(count)]
    v, e0, e1 = ckks.encryption_draws(seed, count, N)
    ref = [ckks.encrypt_with_draws(m[c], keys, v[c], e0[c], e1[c], level) for c in range(count)]
    pt = dev(np.stack([oracle.ntt_fwd(ckks.to_residues(m[c], qs), qs) for c in range(count)]))
    ct = empty(count, 2, level + 1, N)
    he.encrypt_seeded(ct, pt, dev(keys.pk), seed, count, ctx, level,
                      empty(ctx.encrypt_scratch_bytes(level, count) // 8))
    got = host(ct)
    for c in range(count):
        assert np.array_equal(got[c], ref[c]), c
        # m' - m = v e + e0 + e1 s: far below the scale
        diff = ckks.crt_centered(ckks.decrypt_residues(got[c], keys), qs) - np.asarray(m[c], dtype=object)
        assert max(abs(int(x)) for x in diff) < 2 ** 20
    # the same seed through he_sample_encryption_draws + he_encrypt
    dv, d0, d1 = (torch.empty((count, N), dtype=torch.int8, device="cuda") for _ in range(3))
    he.sample_encryption_draws(dv, d0, d1, count, N, seed)
    ct2 = empty(count, 2, level + 1, N)
    he.encrypt(ct2, pt, dev(keys.pk), dv, d0, d1, count, ctx, level,
               empty(ctx.encrypt_scratch_bytes(level, count) // 8))
    assert np.array_equal(host(ct2), got)
