"""The arithmetic behind the bench line's measurement keys, on the CPU: the whole-job value over
ranks, the roofline entry (butterflies of the NTT against the measured butterfly rate; bytes of
the other regions against the measured copy bandwidth), the key-switch aggregate, and the clock
record's parsing of nvidia-smi samples (throttle reasons, median SM clock)."""
import json
import os

import pytest

import bench


class FakeFr:
    def __init__(self, peak):
        self.peak = peak

    def butterfly_peak(self, device):
        return self.peak


def regions(ntt_ms, ntt_bytes, ntt_n, ip_ms=0.5, ip_bytes=2e9):
    r = {k: {"ms": 0.0, "bytes": 0.0, "launches": 0} for k in ("ntt", "modup", "ip", "moddown", "mac")}
    r["ntt"] = {"ms": ntt_ms, "bytes": ntt_bytes, "launches": ntt_n}
    r["ip"] = {"ms": ip_ms, "bytes": ip_bytes, "launches": 3}
    r["modup"] = {"ms": 0.25, "bytes": 0.5e9, "launches": 2}
    r["moddown"] = {"ms": 0.25, "bytes": 0.5e9, "launches": 2}
    return r


def test_whole_job_value_is_all_units_over_slowest_rank():
    assert bench.whole_job_value(1, 32768, 5.0) == pytest.approx(32768 / 0.005)
    assert bench.whole_job_value(4, 1000, 250.0) == pytest.approx(4 * 1000 / 0.25)


def test_peaks_come_from_the_measured_file():
    hbm, kind = bench.load_peaks()
    p = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            assert hbm == pytest.approx(float(json.load(f)["hbm_gbs"]))
        assert kind == "measured"
    else:
        assert (hbm, kind) == (6800.0, "fallback")


@pytest.mark.parametrize("valid", [False, True])
def test_ntt_roofline_counts_butterflies(monkeypatch, valid):
    monkeypatch.setattr(bench, "launch_list_valid", lambda: valid)
    log_n = 16
    n_transforms = 70
    polys = 5616 // 2                       # limb-polynomial transforms of one step
    nbytes = 16.0 * polys * (1 << log_n)    # one read and one write per coefficient and pass pair
    ms = 3.0
    peak = 965e9
    roof = bench.roofline(regions(ms, nbytes, n_transforms), log_n, 0, FakeFr(peak))
    butterflies = polys * (1 << log_n) / 2 * log_n
    assert roof["kernel"] == "ntt" and roof["bound"] == "alu"
    assert roof["butterflies_per_launch"] == pytest.approx(butterflies / n_transforms)
    assert roof["achieved"] == pytest.approx(butterflies / (ms / 1000) / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / (peak / 1e9))
    assert roof["avg_launch_us"] == pytest.approx(1000.0 * ms / n_transforms)
    hbm, _ = bench.load_peaks()
    assert roof["hbm_view"]["achieved"] == pytest.approx(nbytes / (ms / 1000) / 1e9)
    assert roof["hbm_view"]["frac"] == pytest.approx(roof["hbm_view"]["achieved"] / hbm)
    if valid:
        ratio = bench.LAUNCH_LIST["ntt_dram_per_alg_byte"]
        assert roof["traffic"] == pytest.approx(ratio * nbytes / n_transforms)
    else:
        assert roof["traffic"] is None


def test_memory_region_roofline_uses_copy_bandwidth(monkeypatch):
    monkeypatch.setattr(bench, "launch_list_valid", lambda: False)
    r = regions(0.1, 1e8, 2, ip_ms=2.0, ip_bytes=9e9)
    roof = bench.roofline(r, 16, 0, FakeFr(1e12))
    hbm, kind = bench.load_peaks()
    assert roof["kernel"] == "ip" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(9e9 / 2e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / hbm)
    assert roof["peak_kind"] == kind


@pytest.mark.parametrize("valid", [False, True])
def test_keyswitch_aggregate(monkeypatch, valid):
    monkeypatch.setattr(bench, "launch_list_valid", lambda: valid)
    r = regions(3.0, 1e9, 70, ip_ms=0.75, ip_bytes=4e9)
    e = bench.keyswitch_entry(r, 6800.0, "measured")
    assert e["ms_per_step"] == pytest.approx(0.25 + 0.75 + 0.25)
    assert e["algorithmic_bytes"] == pytest.approx(5e9)
    assert e["achieved"] == pytest.approx(5e9 / 1.25e-3 / 1e9)
    assert e["frac"] == pytest.approx(e["achieved"] / 6800.0)
    if valid:
        g = bench.LAUNCH_LIST["keyswitch_dram_gbs"]
        assert e["dram_view"]["achieved"] == g and e["dram_view"]["frac"] == pytest.approx(g / 6800.0)
    else:
        assert e["dram_view"] is None


def test_launch_list_shares_cover_every_region_once():
    share = bench.LAUNCH_LIST["share"]
    assert set(share) == set(bench.REGIONS)
    assert sum(share.values()) == pytest.approx(1.0, abs=2e-3)
    assert all(v >= 0 for v in share.values())


def test_launch_list_applies_to_the_headline_configuration_only(monkeypatch):
    monkeypatch.setattr(bench, "_RUN_CONFIG", dict(bench.LAUNCH_LIST_CONFIG, ell=128))
    assert not bench.launch_list_valid()
    monkeypatch.setattr(bench, "_RUN_CONFIG", dict(bench.LAUNCH_LIST_CONFIG))
    monkeypatch.setattr(bench, "csrc_sha256", lambda: "0" * 64)
    assert not bench.launch_list_valid()


class FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def sampled(lines):
    s = bench.ClockSampler(0)
    s.proc = FakeProc()
    s.lines = lines
    return s.stop()


def test_clock_record_median_and_reasons():
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active"
    r = sampled([ok, ok, cap])
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    r = sampled([ok, hot, "garbage", "0, [N/A], 2070, 1, 0, a, b, c, d"])
    assert r["samples"] == 2 and r["sm_mhz"] == pytest.approx((2070 + 1500) / 2)
    assert r["reasons"] == ["hw_thermal_slowdown"]
    assert sampled([])["sm_mhz"] is None
