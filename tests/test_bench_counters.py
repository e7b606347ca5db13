"""bench.py's counters file: written from an ncu CSV of one sweep launch,
divided by the MC steps the launch covered, and used only while its source
hash matches the sweep kernels' sources (CPU only; a temporary file stands
in for the committed one)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HDR = ['"ID"', '"Process ID"', '"Process Name"', '"Host Name"', '"Kernel Name"', '"Context"',
       '"Stream"', '"Block Size"', '"Grid Size"', '"Device"', '"CC"', '"Section Name"',
       '"Metric Name"', '"Metric Unit"', '"Metric Value"']


def _csv(tmp_path, kernel, values):
    lines = ["==PROF== a line ncu prints before the table", ",".join(HDR)]
    for name, val in values.items():
        row = ['"0"', '"1"', '"python3"', '"127.0.0.1"', '"%s"' % kernel, '"1"', '"13"',
               '"(256, 1, 1)"', '"(608, 1, 1)"', '"0"', '"10.3"', '"Command line profiler metrics"',
               '"%s"' % name, '""', '"%s"' % val]
        lines.append(",".join(row))
    p = tmp_path / "counters.csv"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_counters_per_step_and_hash(tmp_path, monkeypatch):
    out = tmp_path / "k_sweep_wave_L4096_counters.json"
    monkeypatch.setattr(bench, "COUNTERS_FILE", str(out))
    cells = 4096 * 4096
    steps = 20
    inst = 88_000_000 * steps
    csv_path = _csv(tmp_path, "void k_sweep_wave<1, 0, 64, 64, 1>(LatticeArgs)",
                    {"dram__bytes_read.sum": "1,000,000", "dram__bytes_write.sum": "3000000",
                     "smsp__inst_executed.sum": str(inst)})
    assert bench.record_counters(csv_path, steps) == 0
    d = json.loads(out.read_text())
    assert d["steps_in_launch"] == steps
    assert d["dram_bytes"] == 4_000_000 / steps
    assert d["inst_executed_warp"] == inst / steps
    assert d["instructions_per_update"] == inst * 32 / (4 * cells * steps)
    assert d["source_hash"] == bench.sweep_source_hash()
    assert bench.sweep_counters() == d
    # a capture of other sources is not used
    d["source_hash"] = "0" * 16
    out.write_text(json.dumps(d))
    assert bench.sweep_counters() is None


def test_counters_of_the_tiled_sweep(tmp_path, monkeypatch):
    out = tmp_path / "c.json"
    monkeypatch.setattr(bench, "COUNTERS_FILE", str(out))
    csv_path = _csv(tmp_path, "void k_sweep_tiled<1, 0, 0, 1>(LatticeArgs)",
                    {"dram__bytes_read.sum": "34000000", "dram__bytes_write.sum": "400000",
                     "smsp__inst_executed.sum": "90000000"})
    assert bench.record_counters(csv_path, 1) == 0
    d = json.loads(out.read_text())
    assert d["dram_bytes"] == 34_400_000 and d["steps_in_launch"] == 1
    assert "k_sweep_tiled" in d["kernel"]

