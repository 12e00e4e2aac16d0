"""Host-side arithmetic of bench.py's roofline objects (no GPU).

The algorithmic bytes per dof and instance that bench.py divides by each
kernel's CUDA-event time are checked against the DRAM traffic ncu measured
for the same kernels at full size (the committed summary of the one-pass
capture under profiles/): a count that included bytes a kernel does not
move, or left out a vector it does, shows up as a ratio away from 1.
The traffic lookup is checked to follow the kernel-source hash."""
import os
import re

import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
TRAFFIC = os.path.join(ROOT, "profiles", "traffic_mixed_diff3d_128.md")


def _measured_bytes_per_unit():
    """kernel -> DRAM read + write per dof and instance, from the summary."""
    out = {}
    for line in open(TRAFFIC):
        m = re.match(r"\| `(k_\w+)<[^`]*>` \| ([0-9.]+) \| ([0-9.]+) \|", line)
        if m and m.group(1) not in out:  # the first table: read | write | ...
            out[m.group(1)] = float(m.group(2)) + float(m.group(3))
    return out


def test_mixed_algorithmic_bytes_match_the_measured_full_size_traffic():
    meas = _measured_bytes_per_unit()
    # the headline configuration: 3D, k = 60 BF16 modes shared by 128 instances
    k, phi_bytes, B = 60, 2, 128
    names = {"update": "k_update_v3p", "spmv": "k_spmv3p", "expand": "k_expand_tc",
             "project": "k_proj_tc"}
    assert set(names.values()) <= set(meas), meas
    for name, kern in names.items():
        _, byts = bench.kernel_work(name, 3, k, phi_bytes, 4, True, B)
        ratio = meas[kern] / byts
        # traffic may exceed the count a little (halo sectors at tile edges),
        # never fall short of it at this size (every vector is 1.07 GB)
        assert 0.99 <= ratio <= 1.05, (name, byts, meas[kern], ratio)


def test_loop_floor_is_below_the_sum_of_the_kernels():
    # the per-iteration floor of one fused pass (bench.loop_roofline) against
    # what the four launches move: the split re-reads p, r, the mask and v
    prof = {"mean_ms": {"expand": 1.0, "spmv": 1.0, "update": 1.0, "project": 1.0,
                        "resid": 10.0}}
    w = type("Wk", (), {"dim": 3})()
    loop = bench.loop_roofline(prof, w, 60, True, 2, 128, 1)
    kernels = sum(bench.kernel_work(n, 3, 60, 2, 4, True, 128)[1]
                  for n in ("update", "spmv", "expand", "project"))
    assert loop["bytes_per_unit"] < kernels
    assert loop["ms_per_iter"] == pytest.approx(4.0 + 10.0 / 100)


def test_profile_traffic_follows_the_kernel_source_hash(monkeypatch):
    path = os.path.join(ROOT, "profiles", "k_update_mixed_diff3d_128.md")
    txt = open(path).read()
    h = re.search(r"source_hash:\s*([0-9a-f]+)", txt).group(1)
    t = float(re.search(r"traffic_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt).group(1))
    monkeypatch.setattr(bench, "source_hash", lambda: h)
    assert bench.profile_traffic("update_mixed", "diff3d_128") == t
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.profile_traffic("update_mixed", "diff3d_128") is None
    assert bench.profile_traffic("update_mixed", "no_such_workload") is None


def test_fp64_batch_projection_bytes_match_its_capture():
    # k_proj_gemm64 on the convection-diffusion law at 384^2, batch 64, k = 48
    # (its small-case capture under profiles/): v of every instance and the
    # modes once per launch
    txt = open(os.path.join(ROOT, "profiles", "k_project_fp64_convdiff2d_512.md")).read()
    read_mb = float(re.search(r"\| DRAM read \+ write \| ([0-9.]+) \+", txt).group(1))
    _, byts = bench.kernel_work_fp64("project", 2, 48, True, 64)
    units = 384 * 384 * 64
    assert read_mb * 1e6 / (byts * units) == pytest.approx(1.0, abs=0.03)


def _reference_line(monkeypatch, capsys, argv):
    # the oracle sample is replaced by fixed timings: only the line's shape
    # is under test here
    monkeypatch.setattr(bench, "cpu_sample", lambda w, inst, m=20: (2.0, 0.5, 4))
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"] + argv)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    bench.main()
    import json
    return json.loads(capsys.readouterr().out.strip().splitlines()[-1])


def test_reference_arm_prints_the_headline_workload_config(monkeypatch, capsys):
    line = _reference_line(monkeypatch, capsys, ["--steps", "2", "--warmup", "1"])
    cfg = line["config"]
    # the headline: 128^3, k = 60 BF16 modes, 1024 held-out instances in 8
    # batches of 128; vectors of a batch are 1.07 GB, the modes 0.25 GB
    assert cfg == {"workload": "diff3d_128", "grid": [128, 128, 128], "k": 60, "alpha": 1e-4,
                   "instances_per_step": 128, "batch_per_gpu": 128, "held_out": 1024,
                   "held_out_batches": 8,
                   "l2": "inputs larger than L2: Phi is 0.25 GB and each vector 1.07 GB",
                   "parallelism": "1 GPU"}
    assert line["impl"] == "reference" and line["path"].startswith("CPU oracle")
    assert line["steps"] == 2 and line["warmup"] == 1
    # one outer set-up plus the golden CG count at 0.5 s per iteration
    assert line["value"] == pytest.approx(1.0 / (2.0 * 1.0 + 0.5 * 5542), rel=1e-2)


def test_both_arms_share_the_config_of_an_overridden_mode(monkeypatch, capsys):
    # the same overrides give the same config object on both arms: the GPU
    # arm's line and the reference arm's come from workload_config
    line = _reference_line(monkeypatch, capsys, ["--steps", "1", "--warmup", "0",
                                                 "--path", "plain", "--batch", "16"])
    import argparse
    args = argparse.Namespace(workload="diff3d_128", path="plain", phi="", modes="", batch=16,
                              no_learned=False, held_out=0)
    mode = bench.resolve_mode(args)
    assert not mode["learned"]
    from paper_2606_17971_b300 import workloads as W
    assert line["config"] == bench.workload_config(W.WORKLOADS["diff3d_128"], mode, 1, args)
    assert line["config"]["l2"] == "inputs larger than L2 (2.15 GB of vectors per batch)"
    assert "held_out" not in line["config"]


def test_clock_summary_parses_the_sampled_lines():
    # nvidia-smi --format=csv,noheader,nounits lines as the sampler reads
    # them: index, SM clock, max SM clock, power, active mask, then the four
    # throttle reasons of the query
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2032, 2032, 850.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2010, 2032, 1098.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 345, 2032, 120.0, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2032, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    s = c.summary()
    # the idle sample (345 MHz, below half the maximum) is not under load;
    # the unreadable and short lines are skipped
    assert s["samples"] == 3 and s["sm_max_mhz"] == 2032.0
    assert s["sm_mhz"] == pytest.approx(2021.0)
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1500, 2032, 900, 0x8, Not Active, Active, Not Active, Not Active"]
    assert bench.ClockSampler.summary(c)["reasons"] == ["hw_thermal_slowdown"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    # under torchrun the oracle runs once: rank 0 prints the line for the
    # whole job's config, the other ranks exit without work
    calls = []
    monkeypatch.setattr(bench, "cpu_sample", lambda w, inst, m=20: calls.append(m) or (2.0, 0.5, 4))
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2",
                                     "--steps", "1", "--warmup", "0"])
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.main()
    assert capsys.readouterr().out.strip() == "" and not calls
    monkeypatch.setenv("RANK", "0")
    bench.main()
    import json
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["n_gpus"] == 2 and line["config"]["instances_per_step"] == 256
    assert line["config"]["parallelism"] == "replicas x2" and calls == [10]


def test_roofline_peak_comes_from_the_measured_file_else_the_labelled_fallback(monkeypatch):
    prof = {"mean_ms": {"expand": 1.3, "spmv": 1.2, "update": 2.2, "project": 0.7,
                        "resid": 19.0},
            "samples": {"expand": 10, "spmv": 10, "update": 10, "project": 10, "resid": 1}}
    w = type("Wk", (), {"dim": 3, "name": "diff3d_128"})()
    units = 128**3 * 128
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6480.8})
    dom = bench.dominant_roofline(prof, w, 60, True, 2, 128, units, False)
    assert dom["kernel"] == "k_update" and dom["peak"] == 6480.8
    assert dom["peak_source"].startswith("measured")
    # 29 B per unit moved in 2.2 ms
    assert dom["achieved"] == pytest.approx(29 * units / 2.2e-3 / 1e9)
    assert dom["frac"] == pytest.approx(dom["achieved"] / 6480.8)
    loop = bench.loop_roofline(prof, w, 60, True, 2, 128, units)
    assert loop["peak"] == 6480.8 and loop["ms_per_iter"] == pytest.approx(5.4 + 0.19)
    monkeypatch.setattr(bench, "peaks", lambda: {})
    dom = bench.dominant_roofline(prof, w, 60, True, 2, 128, units, False)
    loop = bench.loop_roofline(prof, w, 60, True, 2, 128, units)
    for r in (dom, loop):
        assert r["peak"] == bench.HBM_FALLBACK_GBS and r["peak_source"].startswith("fallback")
        assert r["frac"] == pytest.approx(r["achieved"] / bench.HBM_FALLBACK_GBS)
