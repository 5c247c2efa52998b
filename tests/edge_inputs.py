"""Planted inputs for the rounding-boundary tests of key switching and
rescaling (Sec. II-A Relin and RS): coefficient-domain residues that put the
values the mod-down by P and the rescale by q_l round away at their
boundaries, and keys whose special-prime limbs expose a digit directly.
Shared by the GPU parity tests and the CPU checks of the construction; no
method arithmetic here beyond filling arrays."""
import numpy as np

from paper_2109_14704_gb300.synth import Rng


def boundary_values(m: int) -> list[int]:
    h = m // 2
    return [0, 1, h - 1, h, h + 1, m - 2, m - 1]


def planted(m: int, N: int, r: Rng, mode: str, values=None) -> np.ndarray:
    """One coefficient-domain limb mod m: "edges" plants the boundary values
    (or `values`) at the first positions and after N/2 over random residues;
    "const:<v>" is the constant v; "zero", "max" are 0 and m - 1 everywhere."""
    if mode == "zero":
        return np.zeros(N, dtype=np.uint64)
    if mode == "max":
        return np.full(N, m - 1, dtype=np.uint64)
    if mode.startswith("const:"):
        return np.full(N, int(mode[6:]) % m, dtype=np.uint64)
    assert mode == "edges"
    x = r.uniform_mod(m, N)
    vals = [int(v) % m for v in (values if values is not None else boundary_values(m))]
    for base in (0, N // 2, N - len(vals)):
        x[base:base + len(vals)] = np.array(vals, dtype=np.uint64)
    return x


def key(data, P, N, r, mode):
    """evk [digit][2][limb][N] (NTT domain). "random"; "pmod": random data
    limbs, P limbs +1 / -1 (components 0 / 1) for digit 0 and 0 for the
    other digits; "zero": the zero key."""
    nd = len(data)
    if mode == "zero":
        return np.zeros((nd, 2, nd + 1, N), dtype=np.uint64)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(nd)])
    if mode == "pmod":
        evk[:, :, nd, :] = 0
        evk[0, 0, nd, :] = 1          # NTT of the constant 1 is all ones
        evk[0, 1, nd, :] = P - 1      # and of the constant -1 all P - 1
    return evk


def digits(data, P, N, r, mode):
    """d2 in the coefficient domain, one row per data limb: "pedges" plants
    the special-prime boundaries in digit 0 (random elsewhere), "pconst:<k>"
    makes digit 0 the constant floor(P/2) + k, "zero" / "max" all digits,
    "edges" the q_j boundaries in every digit."""
    rows = []
    for j, q in enumerate(data):
        if mode == "pedges":
            rows.append(planted(q, N, r, "edges", boundary_values(P)) if j == 0 else r.uniform_mod(q, N))
        elif mode.startswith("pconst:"):
            v = P // 2 + int(mode[7:])
            rows.append(planted(q, N, r, f"const:{v}") if j == 0 else r.uniform_mod(q, N))
        else:
            rows.append(planted(q, N, r, mode))
    return rows
