"""Host-side checks of the benchmark's contract and of the binding's failure
mode, with no GPU: the reference arm (the oracle on the host cores) prints
one JSON line with the keys the contract names, and the binding raises when
the library is missing instead of computing anything on the CPU."""
import json
import os
import subprocess
import sys

import pytest

import paper_2310_19925_b300 as orand

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(orand, "LIB_PATH", str(tmp_path / "liborand.so"))
    monkeypatch.setattr(orand, "_LIB", None)
    with pytest.raises(RuntimeError, match="not built"):
        orand._lib()
    with pytest.raises(RuntimeError, match="not built"):
        orand.orand_fill(0, 0, 1, 0, 1, 4, 16, 0)
