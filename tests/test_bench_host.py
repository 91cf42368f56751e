"""Host-side helpers of the benchmark on the CPU: the ncu CSV reader behind
profiles/traffic.json, the source-hash gate of the traffic counters, and the
summary of the clock samples taken during the timed region."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

HDR = ['"ID"', '"Process ID"', '"Process Name"', '"Host Name"', '"Kernel Name"', '"Context"', '"Stream"',
       '"Block Size"', '"Grid Size"', '"Device"', '"CC"', '"Section Name"', '"Metric Name"', '"Metric Unit"',
       '"Metric Value"']


def _row(i, kernel, metric, unit, value):
    vals = [str(i), "1", "python", "h", kernel, "1", "7", "(256, 1, 1)", "(608, 1, 1)", "0", "10.3", "Command line",
            metric, unit, value]
    return ",".join(f'"{v}"' for v in vals)


def test_ncu_csv_sums_dram_bytes_per_kernel_kind(tmp_path):
    lines = ["==PROF== Connected to process 1", ",".join(HDR),
             _row(0, "void lcg::k_parse<unsigned char>(lcg::RoundArgs)", "dram__bytes_read.sum", "Mbyte", "369.5"),
             _row(0, "void lcg::k_parse<unsigned char>(lcg::RoundArgs)", "dram__bytes_write.sum", "Mbyte", "321"),
             _row(0, "void lcg::k_parse<unsigned char>(lcg::RoundArgs)", "gpu__time_duration.sum", "msecond", "1.1"),
             _row(1, "void lcg::k_parse<unsigned int>(lcg::RoundArgs)", "dram__bytes_read.sum", "Gbyte", "0.826"),
             _row(1, "void lcg::k_parse<unsigned int>(lcg::RoundArgs)", "dram__bytes_write.sum", "Kbyte", "1,500"),
             _row(2, "lcg::k_rewrite(const unsigned int *, unsigned long long)", "dram__bytes_read.sum", "byte",
                  "4096")]
    path = tmp_path / "ncu.csv"
    path.write_text("\n".join(lines) + "\n")
    got = bench._ncu_dram_bytes(str(path))
    assert set(got) == {"k_parse", "k_rewrite"}
    assert got["k_parse"]["launches"] == 2
    assert got["k_parse"]["dram_bytes"] == pytest.approx(369.5e6 + 321e6 + 0.826e9 + 1.5e6)
    assert got["k_rewrite"] == {"dram_bytes": 4096.0, "launches": 1}


def test_traffic_is_used_only_for_the_sources_it_was_taken_from(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"source_hash": "abc", "kernels": {"k_parse": {"dram_bytes_per_alg_byte": 1.25}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.profiled_traffic("k_parse") == 1.25
    assert bench.profiled_traffic("k_rules") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.profiled_traffic("k_parse") is None


def test_measured_peak_falls_back_without_the_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6761.9}))
    assert bench.measured_peak() == (6761.9, "measured")


def test_kernel_source_hash_covers_the_kernel_sources():
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = _Proc()
    s.rows = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["0", "2055", "2070", "1200", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
              ["0", "2070", "2070", "1100", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    got = s.stop()
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_algorithmic_bytes_follow_the_stated_formulas():
    """The roofline's byte counts, recomputed by hand for a two-round build:
    round 1 reads its bytes (1 B each), round 2 its ranks (4 B each); a table
    larger than L2 adds one 32-byte sector per phrase; the whole path counts
    the input once, each round's next sequence written and read (8 B per
    phrase) and its new rules (4 B per symbol, 12 B per rule)."""
    import bench
    small = 1024                                   # slots: 32 KB, inside L2
    big = int(bench.L2_BYTES // 32) + 1            # one slot past L2
    r1 = {"n": 1000, "phrases": 300, "g": 20, "G": 70, "table_cap": small}
    r2 = {"n": 300, "phrases": 100, "g": 60, "G": 200, "table_cap": big}
    assert bench.parse_alg_bytes(r1, 1) == 1000.0
    assert bench.parse_alg_bytes(r2, 2) == 4 * 300 + 32 * 100
    assert bench.parse_alg_bytes(r2, 2, tables=False) == 4 * 300
    streams = 1000 + (8 * 300 + 4 * 70 + 12 * 20) + (8 * 100 + 4 * 200 + 12 * 60)
    assert bench.path_alg_bytes([r1, r2], tables=False) == streams
    assert bench.path_alg_bytes([r1, r2]) == streams + 32 * 100
    assert bench.path_alg_bytes([]) == 0.0
