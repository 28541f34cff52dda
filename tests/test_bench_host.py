"""Host logic of the benchmark (no GPU): the per-launch DRAM traffic recorded with
an ncu capture is reported only while the kernel's source is the one captured."""
import hashlib
import json
import os

import bench


def _tree(tmp_path, source_text, recorded_hash):
    src_dir = tmp_path / "paper_2404_14691_b300" / "csrc"
    src_dir.mkdir(parents=True)
    (src_dir / "k.cu").write_text(source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(
        {"wl": {"kern": {"source": "k.cu", "source_sha256_16": recorded_hash, "dram_bytes_per_launch": 1234,
                         "capture": "test"}}}))


def test_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    text = "__global__ void k() {}\n"
    _tree(tmp_path, text, hashlib.sha256(text.encode()).hexdigest()[:16])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("kern", "wl") == 1234
    assert bench.traffic_for("kern", "other-workload") is None
    assert bench.traffic_for("other-kernel", "wl") is None
    # the kernel changed since the capture: no traffic figure
    (tmp_path / "paper_2404_14691_b300" / "csrc" / "k.cu").write_text(text + "// edited\n")
    assert bench.traffic_for("kern", "wl") is None


def test_committed_traffic_entries_name_existing_sources():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for wl, kernels in d.items():
        for kind, rec in kernels.items():
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2404_14691_b300", "csrc", rec["source"])), (wl, kind)
            assert rec["dram_bytes_per_launch"] > 0 and len(rec["source_sha256_16"]) == 16


def test_roofline_of_each_kernel_kind():
    """Gather: achieved = DRAM bytes per launch (from an ncu capture) / mean launch time,
    against the HBM copy rate, beside the effective (algorithmic) rate; GEMMs:
    algorithmic flops / mean launch time against the burst tensor peak."""
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1500.0, "sm_max_mhz": 2000.0}
    # 4 launches in 2 ms in all, 8e9 algorithmic bytes in all: 2e9 B per 0.5 ms = 4000 GB/s effective;
    # 1e9 DRAM bytes per launch: 2000 GB/s of DRAM = 1/3 of the copy rate
    g = bench.roofline_of("gather", 4, 2.0, 8e9, peaks, "test", traffic=1e9)
    assert g["bound"] == "hbm" and g["unit"] == "GB/s"
    assert abs(g["effective_GBs"] - 4000.0) < 1e-6 and abs(g["effective_over_hbm"] - 4000.0 / 6000.0) < 1e-4
    assert abs(g["achieved"] - 2000.0) < 1e-6 and abs(g["frac"] - 2000.0 / 6000.0) < 1e-4
    assert g["traffic"] == 1e9
    # without a capture of the current source there is no DRAM figure, only the effective one
    g0 = bench.roofline_of("gather", 4, 2.0, 8e9, peaks, "test")
    assert g0["achieved"] is None and g0["frac"] is None and abs(g0["effective_GBs"] - 4000.0) < 1e-6
    # bf16 GEMMs against the burst bf16 peak: 3e12 flop in 2 ms over 2 launches = 1500 TF/s
    t = bench.roofline_of("gemm_tc", 2, 2.0, 3e12, peaks, "test")
    assert t["bound"] == "tensor" and abs(t["achieved"] - 1500.0) < 1e-6 and abs(t["frac"] - 1500.0 / 1800.0) < 1e-4
    # fp32 as three tf32 products (and the fused bottom kernel): tf32 = bf16 burst x 1.1 / 2.25, / 3
    ceiling = 1800.0 * 1.1 / 2.25 / 3.0
    for kind in ("gemm_tf32x3", "bottom01"):
        f = bench.roofline_of(kind, 1, 1.0, 1e11, peaks, "test")   # 100 TF/s
        assert f["bound"] == "tensor" and abs(f["peak"] - round(ceiling, 1)) < 1e-6
        assert abs(f["frac"] - 100.0 / ceiling) < 1e-3
    # anything else: the FP32 pipes at the maximum SM clock
    a = bench.roofline_of("bottom0", 1, 1.0, 1e10, peaks, "test")
    assert a["bound"] == "alu" and abs(a["peak"] - 148 * 128 * 2 * 2000e6 / 1e12) < 0.01


def test_stratified_order_is_a_permutation_spread_over_sizes():
    """Every invocation once; the first four cover the quartiles of the size mix."""
    sizes = [5, 1, 9, 3, 7, 2, 8, 4, 6, 10, 11, 12]
    o = bench.stratified_order(sizes)
    assert sorted(o) == list(range(len(sizes)))
    first = sorted(sizes[i] for i in o[:4])
    ranks = sorted(sorted(sizes).index(v) for v in first)
    assert ranks[0] < 3 and ranks[-1] >= 9 and len(set(r // 3 for r in ranks)) == 4


def test_oracle_rate_recovers_the_whole_mix_from_any_prefix():
    """With a per-invocation cost c + B * t, the fit over any timed prefix (two or more
    sizes) predicts the whole workload's time exactly, so both oracle legs agree however
    many invocations their budgets allowed."""
    c, t = 0.030, 0.0019
    batches = [1, 3, 17, 40, 90, 250, 400, 700, 1500, 4096]
    want = len(batches) / sum(c + b * t for b in batches)
    order = bench.stratified_order(batches)
    for m in (2, 3, 5, len(batches)):
        recs = [(batches[i], c + batches[i] * t) for i in order[:m]]
        rate, c_fit, t_fit = bench.oracle_rate(recs, batches)
        assert abs(rate / want - 1) < 1e-9 and abs(c_fit - c) < 1e-9 and abs(t_fit - t) < 1e-12
    # one size only: no intercept can be fitted; the per-sample rate is used (c = 0)
    rate, c_fit, _ = bench.oracle_rate([(100, 0.2), (100, 0.2)], [100, 100, 100])
    assert c_fit == 0.0 and abs(rate - 5.0) < 1e-9


def test_oracle_timing_records_each_invocation(monkeypatch):
    """oracle_timing walks the stratified order from `start` and times every invocation."""
    import time as _t
    import oracle
    calls = []

    def fake_forward(spec, w, v, **kw):
        calls.append(v["batch"])
        _t.sleep(0.002 + 0.0005 * v["batch"])

    monkeypatch.setattr(oracle, "forward", fake_forward)
    monkeypatch.setattr(bench.workload, "weights_arrays", lambda spec: None)
    invs = [{"batch": b} for b in (10, 30, 50, 70)]
    order = bench.stratified_order([v["batch"] for v in invs])
    recs, el = bench.oracle_timing(None, invs, 0.15, 1, start=1)
    assert [r[0] for r in recs] == calls
    assert calls[:3] == [invs[order[(1 + k) % 4]]["batch"] for k in range(3)]
    assert all(r[1] >= 0.002 + 0.0005 * r[0] for r in recs) and el >= sum(r[1] for r in recs)
    rate, c, t = bench.oracle_rate(recs, [v["batch"] for v in invs])
    want = 4 / sum(0.002 + 0.0005 * v["batch"] for v in invs)
    assert 0.6 * want < rate <= 1.05 * want


def test_cold_run_summary():
    """A function's setup ends at its first launch; a cold request's time after setup is
    its completion minus max(arrival, that launch)."""
    # fn 0 ready at 1.0 s: requests at 0.1 (done 1.010), 0.5 (done 1.020), 1.2 warm (done 1.201)
    # fn 1 ready at 0.3 s: request at 0.2 (done 0.305)
    reqs = [(0, 0.1), (0, 0.5), (1, 0.2), (0, 1.2)]
    res = [{"queue_ms": 900.0, "latency_ms": 910.0, "cold": 1},
           {"queue_ms": 500.0, "latency_ms": 520.0, "cold": 1},
           {"queue_ms": 100.0, "latency_ms": 105.0, "cold": 1},
           {"queue_ms": 0.0, "latency_ms": 1.0, "cold": 0}]
    s = bench.cold_run_summary(reqs, res, 3)
    assert s["first_launch_s_by_function"] == [1.0, 0.3, -1.0]
    # after setup: 10, 20 and 5 ms (the warm request is not counted): median 10, p99 20
    assert abs(s["cold_after_setup_p50_ms"] - 10.0) < 1e-6
    assert abs(s["cold_after_setup_p99_ms"] - 20.0) < 1e-6


def test_cpu_baseline_is_the_reference_arm_in_a_child_process(monkeypatch):
    """cpu_baseline runs `bench.py --impl reference` for the same workload in a fresh
    process (two steps of half the budget each) and reports that line's cpu_baseline."""
    import argparse
    import json
    import subprocess
    seen = {}

    class Done:
        returncode = 0
        stderr = ""
        stdout = "noise\n" + json.dumps({"impl": "reference", "cpu_baseline": {
            "value": 2.5, "unit": "invocations/s", "cores": 16, "kind": "oracle", "sample": "fitted"}}) + "\n"

    def fake_run(cmd, **kw):
        seen["cmd"], seen["env"] = cmd, kw.get("env", {})
        return Done()

    monkeypatch.setattr(subprocess, "run", fake_run)
    monkeypatch.setenv("RANK", "3")
    cb = bench.cpu_baseline(argparse.Namespace(workload="c3", cpu_budget_s=12.0))
    cmd = seen["cmd"]
    assert cmd[cmd.index("--impl") + 1] == "reference" and cmd[cmd.index("--workload") + 1] == "c3"
    assert float(cmd[cmd.index("--ref-step-s") + 1]) == 6.0 and cmd[cmd.index("--steps") + 1] == "2"
    assert "RANK" not in seen["env"]                      # the child is a single process
    assert cb["value"] == 2.5 and cb["kind"] == "oracle" and cb["sample"].endswith("fitted")
    assert "fresh process" in cb["sample"]
