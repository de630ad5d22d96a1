"""bench.py's reference arm (the FP64 oracle on the host cores) on a small
case: one JSON line with the keys the benchmark contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--rays", "20000", "--depth", "6", "--cpu-sample", "4096"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_kernel_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The committed DRAM capture is matched to the render kernel's code by
    this hash: a comment or layout edit keeps it, a code edit does not."""
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "paper_2207_05009_gb300" / "csrc"
    csrc.mkdir(parents=True)
    files = {"render.cu": "// a kernel\nint f(int x) { return x + 1; }  /* tail */\n",
             "tree.cu": "int g;\n", "plo_internal.h": "#pragma once\n"}
    for name, text in files.items():
        (csrc / name).write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (csrc / "render.cu").write_text("/* the same kernel,\n   reworded */ int f(int x)  {\n  return x + 1; } // ok\n")
    assert bench.kernel_source_hash() == h0
    (csrc / "render.cu").write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_source_hash() != h0
