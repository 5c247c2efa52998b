"""Host-side CKKS routines of the oracle -- TEST INFRASTRUCTURE.

KeyGen, Encode, Decode, Encrypt and Decrypt as the paper describes them in
Sec. II-A; the paper keeps all five on the CPU (Sec. III), and so does this
oracle. Encoding is FP64 (numpy FFT as a library step), the CRT lift of
decoding uses Python integers, and every ring product goes through the oracle
NTT (``oracle.negacyclic_mul``). Random draws (secret, errors, masks) come
from the shared seeded generator and are inputs here, never drawn inside the
arithmetic.

Conventions (readings of the paper, which states none of them):
* slot j sits at the root zeta^(5^j mod 2N), zeta = exp(i pi / N);
* ciphertexts and keys are [component][limb][N] in the NTT domain;
* the relinearization key has one RNS digit per data prime and one special
  prime P: evk[j] = (-a_j s + e_j + [j = i] (P mod q_i) s^2, a_j) over the
  limbs {q_0..q_L, P}; on the P limb the s^2 term is 0.
"""
from __future__ import annotations

import numpy as np

import oracle as _o


def slot_positions(N: int) -> tuple[np.ndarray, np.ndarray]:
    """Index i (root zeta^(2i+1)) of slot j and of its conjugate."""
    e = np.empty(N // 2, dtype=np.int64)
    x = 1
    for j in range(N // 2):
        e[j] = x
        x = (x * 5) % (2 * N)
    return (e - 1) // 2, (2 * N - e - 1) // 2


def encode_unrounded(z: np.ndarray, N: int, scale: float) -> np.ndarray:
    """Encode (Sec. II-A) before rounding: the real coefficients of the
    polynomial m with m(zeta^(5^j)) = scale * z_j and m(zeta^(-5^j)) =
    scale * conj(z_j), as float64."""
    pos, cpos = slot_positions(N)
    E = np.zeros(N, dtype=np.complex128)
    E[pos] = scale * z
    E[cpos] = scale * np.conj(z)
    k = np.arange(N)
    zeta_k = np.exp(1j * np.pi * k / N)
    m = np.fft.fft(E) / N / zeta_k
    return m.real


def encode_real(z: np.ndarray, N: int, scale: float) -> np.ndarray:
    """Encode (Sec. II-A): encode_unrounded rounded to integers (int64)."""
    return np.rint(encode_unrounded(z, N, scale)).astype(np.int64)


def eval_slots(m: np.ndarray, N: int) -> np.ndarray:
    """m(zeta^(5^j)) for every slot j, m given as real coefficients."""
    pos, _ = slot_positions(N)
    k = np.arange(N)
    zeta_k = np.exp(1j * np.pi * k / N)
    E = np.fft.ifft(np.asarray(m, dtype=np.float64) * zeta_k) * N
    return E[pos]


def to_residues(m_int: np.ndarray, moduli) -> np.ndarray:
    """Signed integer coefficients -> [limbs][N] residues."""
    m_int = np.asarray(m_int, dtype=np.int64)
    out = np.empty((len(moduli), len(m_int)), dtype=np.uint64)
    for l, q in enumerate(moduli):
        out[l] = _signed_mod(m_int, int(q))
    return out


def _signed_mod(v: np.ndarray, q: int) -> np.ndarray:
    neg = v < 0
    mag = np.abs(v).astype(np.uint64)
    r = mag % np.uint64(q)
    return np.where(neg & (r != 0), np.uint64(q) - r, r).astype(np.uint64)


def crt_centered(res: np.ndarray, moduli) -> list[int]:
    """CRT lift of [limbs][N] residues to centred integers in (-Q/2, Q/2]."""
    moduli = [int(q) for q in moduli]
    Q = 1
    for q in moduli:
        Q *= q
    basis = []
    for q in moduli:
        Qi = Q // q
        basis.append(Qi * pow(Qi, -1, q) % Q)
    N = res.shape[1]
    rows = [[int(x) for x in res[l]] for l in range(len(moduli))]
    out = []
    half = Q // 2
    for i in range(N):
        x = 0
        for l in range(len(moduli)):
            x += rows[l][i] * basis[l]
        x %= Q
        out.append(x - Q if x > half else x)
    return out


def decode(res: np.ndarray, moduli, scale: float) -> np.ndarray:
    """Decode (Sec. II-A): CRT-lift, centre, evaluate at the slots, / scale."""
    m = np.array([float(v) for v in crt_centered(res, moduli)])
    return eval_slots(m, res.shape[1]) / scale


class Keys:
    """Secret, public and relinearization keys for one modulus chain."""

    def __init__(self, N, data_moduli, P, s, pk, evk):
        self.N, self.data_moduli, self.P = N, list(data_moduli), P
        self.s = s          # int64 ternary coefficients
        self.pk = pk        # [2][L+1][N], NTT domain
        self.evk = evk      # [L+1][2][L+2][N], NTT domain


def keygen(N: int, data_moduli, P: int, rng) -> Keys:
    """KeyGen (Sec. II-A). rng is a paper_2109_14704_gb300.synth.Rng."""
    data_moduli = [int(q) for q in data_moduli]
    L1 = len(data_moduli)
    all_mod = data_moduli + [int(P)]
    s = rng.ternary(N)
    s_res = to_residues(s, all_mod)
    s2_res = _o.negacyclic_mul(s_res, s_res, all_mod)

    a = rng.uniform_limbs(data_moduli, N)
    e = to_residues(rng.gaussian(N), data_moduli)
    as_ = _o.negacyclic_mul(a, s_res[:L1], data_moduli)
    pk0 = np.stack([(np.uint64(q) - as_[l] + e[l]) % np.uint64(q) for l, q in enumerate(data_moduli)])
    pk = np.stack([_o.ntt_fwd(pk0, data_moduli), _o.ntt_fwd(a, data_moduli)])

    evk = _switching_key(s_res, s2_res, data_moduli, int(P), rng)
    return Keys(N, data_moduli, int(P), s, pk, evk)


def _switching_key(s_res: np.ndarray, from_res: np.ndarray, data_moduli, P: int, rng) -> np.ndarray:
    """Key switching from the secret `from` (residues on q_0..q_L, P) to s:
    one RNS digit per data prime, evk[j] = (-a_j s + e_j + [t = j] (P mod q_t)
    from, a_j) on the limbs t of {q_0..q_L, P}, in the NTT domain
    ([L+1][2][L+2][N]). With from = s^2 it is the relinearization key."""
    all_mod = list(data_moduli) + [P]
    L1, N = len(data_moduli), s_res.shape[1]
    evk = np.empty((L1, 2, L1 + 1, N), dtype=np.uint64)
    for j in range(L1):
        aj = rng.uniform_limbs(all_mod, N)
        ej = to_residues(rng.gaussian(N), all_mod)
        ajs = _o.negacyclic_mul(aj, s_res, all_mod)
        k0 = np.empty_like(aj)
        for t, q in enumerate(all_mod):
            qq = np.uint64(q)
            v = (qq - ajs[t] + ej[t]) % qq
            if t == j:
                v = (v + _mulmod_vec(from_res[t], P % q, q)) % qq
            k0[t] = v
        evk[j, 0] = _o.ntt_fwd(k0, all_mod)
        evk[j, 1] = _o.ntt_fwd(aj, all_mod)
    return evk


def galois_key(keys: "Keys", g: int, rng) -> np.ndarray:
    """Rotation (Galois) key for the automorphism X -> X^g: the switching key
    from s(X^g) to s, in the relinearization key's layout."""
    all_mod = keys.data_moduli + [keys.P]
    s_res = to_residues(keys.s, all_mod)
    return _switching_key(s_res, _o.automorphism(s_res, g, all_mod), keys.data_moduli, keys.P, rng)


def _mulmod_vec(x: np.ndarray, c: int, q: int) -> np.ndarray:
    """x * c mod q elementwise through the oracle's dyadic product."""
    cvec = np.full((1, len(x)), c % q, dtype=np.uint64)
    return _o.dyadic(x.reshape(1, -1), cvec, [q])[0]


def encrypt(m_int: np.ndarray, keys: Keys, rng, level: int | None = None) -> np.ndarray:
    """Encrypt (Sec. II-A): c = (v pk0 + m + e0, v pk1 + e1) mod q_L, as
    [2][L+1][N] in the NTT domain (optionally truncated to `level`), with v
    ternary and e0, e1 rounded Gaussians drawn from `rng`."""
    N = keys.N
    return encrypt_with_draws(m_int, keys, rng.ternary(N), rng.gaussian(N), rng.gaussian(N), level)


# ---- the device's encryption randomness, restated -----------------------------
# A counter-based generator and two integer mappings, written here from their
# definitions (SplitMix64: Steele, Lea and Flood, "Fast splittable
# pseudorandom number generators", 2014; the centred binomial distribution),
# so that draws made on the device can be reproduced without sharing code.

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64_outputs(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output k of the SplitMix64 stream with key `seed`, for every k in
    `counters` (uint64): z = seed + (k + 1) gamma, then the two xor-shift-
    multiply steps and a final xor-shift, all mod 2^64."""
    k = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (k + np.uint64(1)) * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _popcount(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint64)
    c = np.zeros(x.shape, dtype=np.int64)
    for b in range(64):
        c += ((x >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return c


def encryption_draws(seed: int, count: int, N: int):
    """(v, e0, e1), each int64 [count][N]: draw w (0 v, 1 e0, 2 e1) of message
    c at coefficient i takes output (3c + w) N + i of the stream: v = r mod 3
    - 1 (ternary); e = popcount of the low 20 bits minus popcount of the next
    20 bits (centred binomial, parameter 20, variance 10)."""
    out = []
    i = np.arange(N, dtype=np.uint64)
    for w in range(3):
        rows = []
        for c in range(count):
            r = splitmix64_outputs(seed, np.uint64((3 * c + w) * N) + i)
            if w == 0:
                rows.append((r % np.uint64(3)).astype(np.int64) - 1)
            else:
                mask = np.uint64((1 << 20) - 1)
                rows.append(_popcount(r & mask) - _popcount((r >> np.uint64(20)) & mask))
        out.append(np.stack(rows) if rows else np.zeros((0, N), dtype=np.int64))
    return tuple(out)


def encrypt_with_draws(m_int: np.ndarray, keys: Keys, v_int, e0_int, e1_int, level: int | None = None) -> np.ndarray:
    """Encrypt (Sec. II-A) with the given mask and errors (integer
    coefficient vectors): c = (v pk0 + m + e0, v pk1 + e1)."""
    mods = keys.data_moduli
    v = to_residues(np.asarray(v_int, dtype=np.int64), mods)
    e0 = to_residues(np.asarray(e0_int, dtype=np.int64), mods)
    e1 = to_residues(np.asarray(e1_int, dtype=np.int64), mods)
    m = to_residues(m_int, mods)
    v_ntt = _o.ntt_fwd(v, mods)
    c0 = _o.dyadic(v_ntt, keys.pk[0], mods)
    c1 = _o.dyadic(v_ntt, keys.pk[1], mods)
    me = np.stack([(m[l] + e0[l]) % np.uint64(q) for l, q in enumerate(mods)])
    c0 = np.stack([(c0[l] + x) % np.uint64(q) for l, (q, x) in enumerate(zip(mods, _o.ntt_fwd(me, mods)))])
    c1 = np.stack([(c1[l] + x) % np.uint64(q) for l, (q, x) in enumerate(zip(mods, _o.ntt_fwd(e1, mods)))])
    ct = np.stack([c0, c1])
    if level is not None:
        ct = np.ascontiguousarray(ct[:, :level + 1])
    return ct


def decrypt_residues(ct: np.ndarray, keys: Keys) -> np.ndarray:
    """Decrypt (Sec. II-A): m' = c0 + c1 s (+ c2 s^2 for a 3-component
    ciphertext) mod q_l, returned as coefficient-domain residues."""
    n = ct.shape[1]
    mods = keys.data_moduli[:n]
    s_ntt = _o.ntt_fwd(to_residues(keys.s, mods), mods)
    acc = ct[0].copy()
    power = s_ntt
    for c in range(1, ct.shape[0]):
        term = _o.dyadic(ct[c], power, mods)
        acc = np.stack([(acc[l] + term[l]) % np.uint64(q) for l, q in enumerate(mods)])
        power = _o.dyadic(power, s_ntt, mods)
    return _o.ntt_inv(acc, mods)


def decrypt_decode(ct: np.ndarray, keys: Keys, scale: float) -> np.ndarray:
    n = ct.shape[1]
    return decode(decrypt_residues(ct, keys), keys.data_moduli[:n], scale)
