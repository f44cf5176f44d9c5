"""Host-side pieces of bench.py that need no GPU: the traffic lookup keyed by
the kernel sources, the oracle sample behind the CPU baseline, and the
reference arm's JSON line."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_is_reported_only_for_the_captured_kernel_sources(tmp_path, monkeypatch):
    src = bench._kernel_source_hash()
    assert len(src) == 16 and int(src, 16) >= 0
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.txt").write_text(f"# comment\nusolve {src} 123\nlsolve 0000000000000000 456\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: src)
    assert bench._traffic("usolve") == 123.0
    assert bench._traffic("lsolve") is None          # captured on other kernel sources
    assert bench._traffic("residual") is None        # never captured


def test_committed_traffic_file_parses():
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert rows and all(len(r) == 3 and int(r[1], 16) >= 0 and float(r[2]) > 0 for r in rows)


def test_oracle_sample_counts_dofs_times_cycles(monkeypatch):
    monkeypatch.setattr(bench, "LOG2H", 4)
    value, secs, steps = bench._oracle_sample(0.05, degrees=(2, 3))
    assert steps >= 1 and secs > 0 and value > 0
    # the sample's units are sum_p N_p * cycles_p per step: a lower bound is one cycle per degree
    from oracle import oracle as O
    n = sum(O.Hierarchy(O.ANNULUS, p, 4).N[0] for p in (2, 3))
    assert value * 1e6 * secs >= steps * n


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "LOG2H", 4)
    monkeypatch.setattr(bench, "DEGREES", (2, 3))
    args = bench.argparse.Namespace(gpus=1, steps=1, warmup=1)
    monkeypatch.delenv("RANK", raising=False)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(bench.argparse.Namespace(gpus=2, steps=1, warmup=1))
    assert capsys.readouterr().out == ""
