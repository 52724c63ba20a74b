"""The benchmark's reference arm (the CPU oracle timed on the host) prints one
JSON line with the keys the benchmark contract asks for; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "cell-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "gaussian_pulse_2048x2048"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_traffic_record_is_keyed_to_the_sources(tmp_path):
    """bench.py --record-traffic sums DRAM reads and writes per launch from an
    ncu CSV (the x2 sweep's second kernel counted with its first) and keys them
    to the digest of the kernel sources, so a stale capture is never used."""
    sys.path.insert(0, ROOT)
    import bench
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
           '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
           '"Metric Value"')
    def row(i, name, metric, v):
        return (f'"{i}","1","python","h","{name}","1","7","(32, 1, 1)","(9, 1, 1)","0","10.3",'
                f'"Command line profiler metrics","{metric}","byte","{v}"')
    # the names as ncu prints them: no namespaces, bools as 0 / 1
    x = "void k_sweep_x32<32, 0, 1>(StepArgs)"
    y1 = "void k_sweep_y32<0, 1, 0>(StepArgs)"
    y2 = "void k_sweep_y32<0, 1, 1>(StepArgs)"
    lines = ["==PROF== Connected", hdr]
    for s in range(2):
        b = 10 * s
        lines += [row(b, x, "dram__bytes_read.sum", "50,000,000"),
                  row(b, x, "dram__bytes_write.sum", 6000000 + s * 2),
                  row(b + 1, y1, "dram__bytes_read.sum", 30000000),
                  row(b + 1, y1, "dram__bytes_write.sum", 20000000),
                  row(b + 2, y2, "dram__bytes_read.sum", 1000)]
    csv_path = tmp_path / "t.csv"
    csv_path.write_text("\n".join(lines) + "\n")
    out = bench.record_traffic(str(csv_path), str(tmp_path / "t.json"))
    assert out["k_sweep_x_fp32_2048x2048"]["dram_bytes_per_launch"] == 56000001
    assert out["k_sweep_y_fp32_2048x2048"]["dram_bytes_per_launch"] == 50001000
    assert out["k_sweep_y_fp32_2048x2048"]["launches"] == 2
    assert out["k_sweep_x_fp32_2048x2048"]["source_digest"] == bench.source_digest()
    assert json.loads((tmp_path / "t.json").read_text()) == out
