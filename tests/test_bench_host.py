"""Host-side pieces of bench.py on CPU: argument defaults, the confidence
interval, the clock-record parser, the committed-profile lookup and the
breadth-first ablation order.  No GPU and no oracle call.
"""
from __future__ import annotations

import os
import statistics

import pytest

import bench


def test_defaults_meet_the_timing_rules():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.impl == "gpu"
    assert a.warmup >= 3 and a.steps >= 1
    assert a.scale == 20                      # the full R-MAT workload by default
    assert bench.L2_FLUSH_BYTES > 129 * 10**6  # larger than the 129 MB L2


def test_mean_ci_student_t():
    scipy = pytest.importorskip("scipy")
    assert scipy
    xs = [10.0, 12.0, 11.0, 13.0, 9.0]
    m, h = bench.mean_ci(xs)
    assert m == 11.0
    # t(0.975, 4) = 2.776445; s = sqrt(2.5)
    assert h == pytest.approx(2.776445 * statistics.stdev(xs) / 5 ** 0.5, rel=1e-6)
    assert bench.mean_ci([4.0]) == (4.0, 0.0)


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _FakeThread:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc, s._t, s.lines = _FakeProc(), _FakeThread(), lines
    return s


def test_clock_record_median_max_and_reasons():
    ok = "0, {sm}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {pc}"
    lines = [ok.format(sm=sm, pc=pc) for sm, pc in
             [(2070, "Not Active"), (2055, "Active"), (1980, "Not Active")]]
    lines += ["", "garbage", "0, [N/A], 2070, 1, 0x0, a, b, c, d"]
    rec = _sampler(lines).stop()
    assert rec["sm_mhz"] == 2055 and rec["sm_max_mhz"] == 2070
    assert rec["reasons"] == ["sw_power_cap"] and rec["samples"] == 3


def test_clock_record_flags_thermal_slowdown():
    line = "0, 1500, 2070, 1300, 0x48, Not Active, Not Active, Active, Active"
    rec = _sampler([line]).stop()
    assert rec["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["unavailable"]


def _fake_tree(tmp_path, kernels_text, profile_hash, per_launch="6.2e9"):
    csrc = tmp_path / "paper_2507_04130_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "hm_kernels.cuh").write_text(kernels_text)
    (csrc / "hm_internal.cuh").write_text("// helpers\n")
    (csrc / "hm_match.cu").write_text("// orchestration\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_extend_rmat20.md").write_text(
        f"# summary\n\nkernel_source_sha256: {profile_hash}\ndram_bytes_per_launch: {per_launch}\n")


def test_committed_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _fake_tree(tmp_path, "// kernels v1\n", "0" * 16)
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h != "0" * 16
    assert bench.committed_traffic("k_extend", "rmat20") is None          # stale profile
    (tmp_path / "profiles" / "k_extend_rmat20.md").write_text(
        f"kernel_source_sha256: {h}\ndram_bytes_per_launch: 6.2e9\n")
    assert bench.committed_traffic("k_extend", "rmat20") == 6.2e9        # same source
    (tmp_path / "paper_2507_04130_gb300" / "csrc" / "hm_kernels.cuh").write_text("// kernels v2\n")
    assert bench.kernel_source_hash() != h
    assert bench.committed_traffic("k_extend", "rmat20") is None          # kernel changed since
    assert bench.committed_traffic("k_extend", "er1k") is None            # no such profile


def test_committed_profile_names_a_source_hash():
    text = open(os.path.join(bench.ROOT, "profiles", "k_extend_rmat20.md")).read()
    assert "kernel_source_sha256:" in text and "dram_bytes_per_launch:" in text


@pytest.mark.parametrize("k,src,dst", [
    (4, [0, 1, 0, 2], [1, 2, 2, 3]),            # feed-forward loop plus out-edge
    (4, [0, 0, 1, 1], [2, 3, 2, 3]),            # bi-fan: 1 is reached through 2
    (5, [3, 4, 2, 1], [0, 3, 4, 2]),            # a path given backwards
])
def test_bfs_order_anchors_every_position(k, src, dst):
    order = bench.bfs_order(k, src, dst)
    assert sorted(order) == list(range(k)) and order[0] == 0
    und = {(a, b) for a, b in zip(src, dst)} | {(b, a) for a, b in zip(src, dst)}
    for i in range(1, k):
        assert any((order[i], order[j]) in und for j in range(i))


class _FakeOracleGraph:
    def __init__(self):
        self.calls = []

    def match(self, p, mode, rows=True, threads=1, root_mask=None):
        self.calls.append((p.name, mode, rows, int(root_mask.sum())))
        return 7, None


def test_reference_arm_line(monkeypatch, capsys):
    """The reference arm's JSON line: the contract's keys, values from the oracle's own timing."""
    import json

    import synth

    small = synth.config2_graph(scale=8)
    monkeypatch.setattr(synth, "cached", lambda name, fn, **kw: small)
    og = _FakeOracleGraph()
    monkeypatch.setattr(bench, "oracle_sample", lambda g, pats, mode, target_s: (21, 0.5, 64, 4, og))
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.main(["--impl", "reference", "--steps", "2", "--warmup", "3"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["unit"] == "matches/s" and line["higher_is_better"] is True
    assert line["data"] == "synthetic" and "workload" in line["config"]
    # 5 steps x 3 induced queries, every one with rows, each on its own 64-root sample
    assert len(og.calls) == 15 and all(c[1] == 1 and c[2] and c[3] == 64 for c in og.calls)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 4 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "matches/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["value"] > 0 and line["ms_per_step"] > 0


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: pytest.fail("rank 1 ran the oracle"))
    assert bench.main(["--impl", "reference"]) == 0
    assert capsys.readouterr().out == ""
