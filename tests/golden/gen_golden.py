"""Writes the stored expected values under tests/golden/ by calling only the
CPU oracle (oracle/) and the seeded input generator. Run from the repository
root: python tests/golden/gen_golden.py"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2109_14704_gb300.synth import Rng  # noqa: E402


def main():
    # Toy transform: q = 17, N = 8 (psi = 3, the smallest primitive 16th root).
    q, N = 17, 8
    a = np.arange(1, N + 1, dtype=np.uint64).reshape(1, N)
    toy = {
        "q": q, "N": N, "psi": oracle.find_psi(q, N),
        "input": [int(x) for x in a[0]],
        "ntt_fwd": [int(x) for x in oracle.ntt_fwd(a, [q])[0]],
    }
    with open(os.path.join(HERE, "toy_ntt_q17_n8.json"), "w") as f:
        json.dump(toy, f, indent=1)

    # Plain NTT workload of N = 4096, two 60-bit primes (seed 1): the primes,
    # psi and sampled outputs of the forward transform of the first limb.
    N = 4096
    qs = oracle.find_primes(60, 2 * N, 2)
    x = Rng(1).uniform_limbs(qs, N)
    X = oracle.ntt_fwd(x, qs)
    idx = [0, 1, 2, 3, 1000, 2047, 2048, 4095]
    c1 = {
        "N": N, "moduli": qs, "psi": [oracle.find_psi(q, N) for q in qs], "seed": 1,
        "sample_index": idx,
        "input_head": [int(v) for v in x[0, :4]],
        "ntt_fwd_limb0": [int(X[0, i]) for i in idx],
        "ntt_fwd_limb1": [int(X[1, i]) for i in idx],
    }
    with open(os.path.join(HERE, "ntt_n4096_seed1.json"), "w") as f:
        json.dump(c1, f, indent=1)


if __name__ == "__main__":
    main()
