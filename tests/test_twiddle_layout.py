"""CPU pins of the inverse twiddle table's layout (inv_tw_pos, used by the
host table builder and every inverse-transform kernel): the function itself
is compiled for the host with nvcc and checked, for every supported degree,
against the properties the kernels rely on:

* each stage S keeps its 2^S pairs inside [2^S, 2^(S+1)), one per group
  (a permutation), so no twiddle is lost or doubled;
* stages below log N - 4 keep the natural order 2^S + G (the cross-CTA
  stages and every shape's earlier rounds read them directly);
* in the last four stages, for Q = S - (log N - 4) >= 1, the pair of an
  even group G sits at an even position with G + 1 right after it (one
  aligned 32-byte load of two pairs), and run t + 1's pair lies two pairs
  after run t's (lane-consecutive loads in the inverse's first round).

The expected properties are stated here; the positions come from the
library's own function, not from a restatement of its formula."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_14704_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "ntt_core.cuh"
int main()
{
    for (int log_n = 10; log_n <= 16; log_n++)
        for (int S = 1; S < log_n; S++)
            for (int G = 0; G < (1 << S); G++)
                std::printf("%d %d %d %d\n", log_n, S, G, he::inv_tw_pos(log_n, S, G));
    return 0;
}
"""


@pytest.fixture(scope="module")
def positions(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("twl")
    src, exe = d / "layout.cu", d / "layout"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout
    table = {}
    for line in out.splitlines():
        log_n, S, G, pos = map(int, line.split())
        table.setdefault((log_n, S), {})[G] = pos
    return table


@pytest.mark.parametrize("log_n", range(10, 17))
def test_each_stage_is_a_permutation_of_its_slice(positions, log_n):
    for S in range(1, log_n):
        pos = positions[(log_n, S)]
        assert sorted(pos.values()) == list(range(1 << S, 1 << (S + 1))), S


@pytest.mark.parametrize("log_n", range(10, 17))
def test_natural_order_below_the_last_four_stages(positions, log_n):
    for S in range(1, log_n - 3):
        pos = positions[(log_n, S)]
        assert all(pos[G] == (1 << S) + G for G in pos), S


@pytest.mark.parametrize("log_n", range(10, 17))
def test_last_stages_keep_pairs_aligned_and_runs_lane_consecutive(positions, log_n):
    for S in range(log_n - 3, log_n):
        Q = S - (log_n - 4)
        pos = positions[(log_n, S)]
        for G in range(0, 1 << S, 2):
            assert pos[G] % 2 == 0 and pos[G + 1] == pos[G] + 1, (S, G)
        # group r of run t and of run t + 1 (runs of 2^Q groups)
        runs = (1 << S) >> Q
        for t in range(runs - 1):
            for r in range(1 << Q):
                assert pos[((t + 1) << Q) + r] == pos[(t << Q) + r] + 2, (S, t, r)
