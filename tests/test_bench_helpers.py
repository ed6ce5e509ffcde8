"""The bench line's arithmetic on the host: algorithmic bytes per stage, the
HBM fractions built from them, the ncu traffic record that is reported only
for the sources it was taken of, and the peak used when no measured one is
present."""
import hashlib
import json
import os

import pytest

import bench


def test_stage_bytes_per_stage():
    n, D, mesh = 1000, 3, 16
    real = 4 * D * mesh ** 3
    spec = 8 * D * mesh * mesh * (mesh // 2 + 1)
    b = bench.stage_bytes(n, D, mesh, passes=6)
    assert b["keys"] == 37 * n                      # 24 B position + 1 B species in, 12 B out
    assert b["radix"] == 6 * 32 * n                 # per pass: 8 B histogram + 12 B in + 12 B out
    assert b["gather"] == (2 * 45 + 4) * n
    assert b["type_order"] == 36 * n
    assert b["interp"] == 41 * n + real
    assert b["deposit"] == 33 * n + real
    assert b["fft_fwd"] == real + spec and b["fft_inv"] == spec + real
    assert b["kspace"] == 2 * spec
    nopm = bench.stage_bytes(n, D, 0)
    assert not {"deposit", "fft_fwd", "kspace", "fft_inv"} & set(nopm)


def test_hbm_block_fractions(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: (1000.0, "measured"))
    n, D, mesh = 1 << 20, 2, 32
    times = {"keys": 0.5, "radix": 2.0, "walk": 7.0, "monopoles": 1.0, "interp": 0.0}
    h = bench.hbm_block(times, n, D, mesh, passes=4)
    assert h["radix_passes"] == 4 and h["peak_gbs"] == 1000.0
    gbs = 37 * n / 0.5e-3 / 1e9
    assert h["keys"]["gbs"] == round(gbs, 1) and h["keys"]["frac"] == round(gbs / 1000.0, 4)
    assert h["radix"]["bytes"] == 4 * 32 * n
    assert "interp" not in h                         # not timed: no fraction
    assert h["walk"]["bound"] == "FP32" and h["monopoles"]["bound"] == "latency / FP64"


def _fake_repo(tmp_path, walk_src, tree_src, record_sha, leaf=32, cell=256):
    csrc = tmp_path / "paper_1502_07442_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "ng_walk.cu").write_bytes(walk_src)
    (csrc / "ng_tree.cu").write_bytes(tree_src)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_walk_clustered16m_d4_yukawa_dram.md").write_text(
        f"notes\ntraffic: leaf={leaf} cell={cell} read=1000 write=24 source_sha256={record_sha}\n")
    return str(tmp_path)


def test_walk_traffic_only_for_recorded_sources(tmp_path, monkeypatch):
    walk, tree = b"walk source", b"tree source"
    sha = hashlib.sha256(walk + tree).hexdigest()
    monkeypatch.setattr(bench, "ROOT", _fake_repo(tmp_path, walk, tree, sha))
    assert bench.walk_traffic(bench.DEFAULT_WORKLOAD, None, 32, 256) == 1024
    assert bench.walk_traffic(bench.DEFAULT_WORKLOAD, None, 16, 256) is None     # other leaf
    assert bench.walk_traffic(bench.DEFAULT_WORKLOAD, 4194304, 32, 256) is None  # other size
    assert bench.walk_traffic("batch64", None, 32, 256) is None                  # other workload


def test_walk_traffic_stale_after_a_source_change(tmp_path, monkeypatch):
    sha = hashlib.sha256(b"old walk" + b"tree").hexdigest()
    monkeypatch.setattr(bench, "ROOT", _fake_repo(tmp_path, b"new walk", b"tree", sha))
    assert bench.walk_traffic(bench.DEFAULT_WORKLOAD, None, 32, 256) is None


def test_measured_peaks_file_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench.measured_peaks()
    assert src == "fallback" and peak > 0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6543.2}))
    assert bench.measured_peaks() == (6543.2, "measured")


def test_job_totals_single_process():
    assert bench.job_totals(123.0, 4.5, 1) == (123.0, 4.5)
