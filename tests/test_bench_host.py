"""Host logic of the benchmark line, on the CPU: the clock sampler's reading
of nvidia-smi's CSV (median SM clock under load, the throttle reasons that
make a run invalid, malformed rows skipped), and the roofline entries that
the sub-results carry."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def __init__(self):
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def wait(self, timeout=None):
        return 0


def _stop(tmp_path, rows):
    """ClockSampler.stop over `rows` as nvidia-smi wrote them (the sampler's
    own field order, csv, noheader, nounits)."""
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s.fh = open(s.path, "a")
    s.proc = _Proc()
    out = s.stop()
    assert s.proc.terminated and not os.path.exists(s.path)
    return out


NA = "Not Active"


def _row(sm, util, hw=NA, hw_th=NA, sw_th=NA, pcap=NA, mx=2070):
    return f"0, {sm}, {mx}, 812.40, {util}, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {pcap}"


def test_field_order_matches_the_parser():
    fields = bench.ClockSampler.FIELDS.split(",")
    assert fields[1] == "clocks.sm" and fields[2] == "clocks.max.sm" and fields[4] == "utilization.gpu"
    assert fields[6:10] == ["clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                            "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


def test_median_under_load_and_no_reasons(tmp_path):
    out = _stop(tmp_path, [_row(345, 0), _row(2070, 100), _row(2055, 98), _row(2070, 100), _row(210, 0)])
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_each_throttle_reason_is_reported(tmp_path):
    for kw, name in (({"hw": "Active"}, "hw_slowdown"), ({"hw_th": "Active"}, "hw_thermal_slowdown"),
                     ({"sw_th": "Active"}, "sw_thermal_slowdown"), ({"pcap": "Active"}, "sw_power_cap")):
        out = _stop(tmp_path, [_row(2070, 100), _row(1980, 100, **kw), _row(2070, 100)])
        assert out["reasons"] == [name], name


def test_reasons_while_idle_do_not_count(tmp_path):
    out = _stop(tmp_path, [_row(300, 0, hw_th="Active"), _row(2070, 100), _row(2070, 99)])
    assert out["reasons"] == [] and out["samples"] == 2


def test_malformed_rows_are_skipped_and_all_idle_falls_back_to_every_row(tmp_path):
    rows = ["", "0, [N/A], 2070, 80.0, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage", _row(1500, 0), _row(1600, 0)]
    out = _stop(tmp_path, rows)
    assert out["samples"] == 2 and out["sm_mhz"] == 1550.0


def test_no_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}


def test_roof_entry_and_nested_attachment():
    work = {"bfly": 2e9, "products": 1e9, "bytes": 4e9}
    e = bench.roof_entry(work, 0.5, alu_peak=1e12, hbm_peak=8000.0)
    assert e["tbfly_per_s"] == pytest.approx(4e-3) and e["alu_frac_transforms"] == pytest.approx(4e-3)
    assert e["alu_frac_with_products"] == pytest.approx(6e-3)
    assert e["gbs"] == pytest.approx(8.0) and e["hbm_frac"] == pytest.approx(1e-3)
    obj = {"a": {"_work": dict(work, seconds=0.5), "x": 1}, "b": [{"_work": dict(work, products=0, seconds=1.0)}]}
    bench.attach_rooflines(obj, 1e12, 8000.0)
    assert "_work" not in obj["a"] and obj["a"]["roofline"] == e and obj["a"]["x"] == 1
    assert "alu_frac_with_products" not in obj["b"][0]["roofline"]
    assert obj["b"][0]["roofline"]["gbs"] == pytest.approx(4.0)


def test_mul_relin_rescale_transform_count():
    """n^2 + 5n + 2 transforms per MulLinRS at n data limbs (with one
    special prime): the tensor's d2 to coefficients (n), its digits lifted
    to the n - 1 other data primes and P (n^2), the two P limbs back (2) and
    into the n data primes (2n), the two q_l limbs back (2) and into the
    n - 1 remaining primes (2(n - 1))."""
    for n in (2, 3, 7, 17):
        stages = n + n * ((n - 1) + 1) + 2 + 2 * n + 2 + 2 * (n - 1)
        for N in (4096, 16384):
            w = bench.mrr_work(n, N)
            assert w["bfly"] == stages * (N // 2) * (N.bit_length() - 1)
            assert w["bytes"] == (2 * 2 * n + 2 * (n - 1)) * N * 8
