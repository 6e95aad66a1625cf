"""Host-side arithmetic of the benchmark line (no GPU): the roofline of the
dominant kernel and the DRAM traffic taken from the committed ncu summary."""
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_roofline_picks_the_dominant_kernel_and_the_nearer_ceiling(bench):
    hbm_peak, _ = bench.measured_peaks()
    bf_peak, mac_peak = 800e9, 1000e9
    # (launches, ms, algorithmic bytes, butterflies, conversion products) per step
    prof = {
        "conv": (10, 20.0, 1e9, 4e9, 6e9),     # integer-bound pass
        "copy": (5, 10.0, 40e9, 0.0, 0.0),      # HBM-bound kernel, less time
    }
    r = bench.roofline_of(prof, bf_peak, 3e12, 16, mac_peak)
    assert r["kernel"] == "conv" and r["bound"] == "alu"
    sec = 0.020
    equiv = 4e9 + 6e9 * bf_peak / mac_peak      # products in butterfly equivalents
    assert r["frac"] == pytest.approx(equiv / sec / bf_peak)
    assert r["butterflies_only_frac"] == pytest.approx(4e9 / sec / bf_peak)
    assert r["other"]["bound"] == "hbm"
    assert r["other"]["frac"] == pytest.approx(1e9 / sec / 1e9 / hbm_peak)
    assert r["launches_per_step"] == 10 and r["avg_launch_us"] == pytest.approx(2000.0)
    assert r["share_of_step"] == pytest.approx(20.0 / 30.0)
    assert r["traffic"] is None                  # no capture of a kernel named "conv"
    assert list(r["kernels"]) == ["conv", "copy"]

    # the same kernel with ten times the bytes: HBM becomes the nearer ceiling
    prof["conv"] = (10, 20.0, 10e12, 4e9, 6e9)
    r = bench.roofline_of(prof, bf_peak, 3e12, 16, mac_peak)
    assert r["bound"] == "hbm" and r["other"]["bound"] == "alu"
    assert r["frac"] == pytest.approx(10e12 / sec / 1e9 / hbm_peak)


def test_traffic_scales_with_the_batch_and_follows_the_source_hash(bench, tmp_path, monkeypatch):
    j = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    name, k = next(iter(j["kernels"].items()))
    per16 = k["dram_bytes_per_launch_full_size"]
    if j["csrc_hash"] == bench.csrc_hash():
        assert bench.ncu_traffic(name, j["batch"]) == pytest.approx(per16)
        assert bench.ncu_traffic(name, 4 * j["batch"]) == pytest.approx(4 * per16)
    assert bench.ncu_traffic("no_such_kernel", 16) is None
    # a capture taken on other sources is not used
    fake = dict(j, csrc_hash="0" * 16)
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(fake))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_hash", lambda: "f" * 16)
    assert bench.ncu_traffic(name, 16) is None


def test_issue_block_against_the_hardware_limit(bench, tmp_path, monkeypatch):
    """roofline.issue: warp instructions per SM cycle from the committed record
    against 4 per SM per clock x 148 SMs x the sampled clock; unused when the
    record was taken on other kernel sources."""
    j = json.load(open(os.path.join(ROOT, "profiles", "ncu_issue_rates.json")))
    name, k = next(iter(j["kernels"].items()))
    if j["csrc_hash"] == bench.csrc_hash():
        r = bench.ncu_issue(name, 2000.0)
        ipc = k["inst_per_active_sm_cycle"]
        assert r["frac"] == pytest.approx(ipc / 4)
        assert r["peak_warp_inst_per_s"] == pytest.approx(4 * 148 * 2000e6)
        assert r["achieved_warp_inst_per_s"] == pytest.approx(ipc * 148 * 2000e6)
    assert bench.ncu_issue("no_such_kernel", 2000.0) is None
    fake = dict(j, csrc_hash="0" * 16)
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "ncu_issue_rates.json").write_text(json.dumps(fake))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_hash", lambda: "f" * 16)
    assert bench.ncu_issue(name, 2000.0) is None


def test_line_carries_the_committed_accuracy_and_learned_records(bench):
    """The bench line's accuracy and learned-vs-plain blocks come from the
    committed GPU records, with the fields the line promises."""
    acc = bench.accuracy_line()
    assert acc["windows"] == 64 and acc["below_floor"] == 0 and acc["above_ceiling"] == 0
    assert acc["within_1e-3_bpm_both_bands"] == acc["windows"] and acc["max_bpm"] < 1e-3
    assert acc["copies_per_window"] == pytest.approx(acc["copies"] / acc["windows"])
    lv = bench.learned_line()
    assert lv["learned"]["depth"] < lv["plain"]["depth"]
    assert lv["learned"]["windows_per_s"] > lv["plain"]["windows_per_s"]
    assert lv["speedup_learned_over_plain"] == pytest.approx(lv["learned"]["windows_per_s"] /
                                                              lv["plain"]["windows_per_s"])
