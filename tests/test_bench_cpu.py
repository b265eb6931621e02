"""bench.py's reference arm (the FP64 oracle on the host cores) runs without a
GPU; its JSON line carries the contract's keys."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--grid", "128", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better",
                "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_kernel_source_hash_tracks_sources():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_sources_sha256()
    assert len(h) == 64 and h == bench.kernel_sources_sha256()


def test_traffic_record_from_an_ncu_log(tmp_path):
    """The traffic record is computed from the capture's CSV log and keyed to
    the kernel sources as they are when it is written (the log here is a
    hand-made stand-in of ncu's CSV format: two launches, one other kernel)."""
    sys.path.insert(0, ROOT)
    import bench
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
           '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
           '"Metric Value"\n')
    rows = []
    for i, (rd, wr) in enumerate(((800.0, 480.0), (820.0, 470.0))):
        k = "void rdc::k_step1<float, 0>(const float *, ...)"
        for name, val in (("dram__bytes_read.sum", rd), ("dram__bytes_write.sum", wr),
                          ("gpu__time_duration.sum", 190.0)):
            unit = "Mbyte" if name.startswith("dram") else "usecond"
            rows.append(f'"{i}","1","python","h","{k}","1","7","(128, 1, 1)","(16, 1024, 1)",'
                        f'"0","10.3","Command line profiler metrics","{name}","{unit}","{val}"\n')
    rows.append('"2","1","python","h","void rdc::k_seed<float>()","1","7","(128, 1, 1)",'
                '"(1, 1, 1)","0","10.3","Command line profiler metrics",'
                '"dram__bytes_read.sum","Mbyte","5"\n')
    log = tmp_path / "launches.csv"
    log.write_text("==PROF== Connected to process\n" + hdr + "".join(rows))
    rec = bench.record_traffic(str(log))["k_step1<float>"]
    assert rec["launches"] == 2
    assert rec["dram_bytes_read_per_launch"] == 810e6
    assert rec["dram_bytes_write_per_launch"] == 475e6
    assert abs(rec["bytes_per_cell"] - 1285e6 / (8192 * 8192)) < 1e-12
    assert rec["sources_sha256"] == bench.kernel_sources_sha256()
