"""The paper's operation counts (Table I) and operational densities (Sec. V-B
roofline analysis), stored in tests/golden/paper_table1.json, against the
work accounting the benchmark's rooflines use: a transform of N points is
(N/2) log2 N radix-2 butterflies, a radix-2^k round holds 2^(k-1) k of them
per group of 2^k words. The fixture's figures are the paper's, quoted with
their passage in the file."""
import json
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

T = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_table1.json")))
BFLY_OPS = T["ops_per_round"]["radix-2"]["butterfly"]      # operations of one radix-2 butterfly


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_butterfly_operations_per_round(k):
    row = T["ops_per_round"][f"radix-{1 << k}"]
    assert row["butterfly"] == (1 << (k - 1)) * k * BFLY_OPS
    assert row["total"] == row["butterfly"] + row["other"]


def test_rounds_cover_the_transform_once():
    """Radix-8 rounds at N = 2^15 (five rounds of N/8 groups) perform exactly
    the (N/2) log2 N butterflies the roofline counts per limb."""
    N = T["N"]
    log_n = int(math.log2(N))
    assert log_n % 3 == 0
    rounds, groups = log_n // 3, N // 8
    assert rounds * groups * 4 * 3 == (N // 2) * log_n
    assert bench.NTT_LOG_N == log_n


def test_operational_densities():
    N = T["N"]
    log_n = int(math.log2(N))
    # naive radix-2: every stage reads and writes all N words
    stage_ops = (N // 2) * T["ops_per_round"]["radix-2"]["total"]
    assert stage_ops / (2 * N * 8) == T["operational_density"]["naive_radix2"]
    # radix-8 in shared memory: log_8 N rounds, two global rounds of load and store
    ops = (log_n // 3) * (N // 8) * T["ops_per_round"]["radix-8"]["total"]
    assert round(ops / (4 * N * 8), 1) == T["operational_density"]["radix8_slm"]

