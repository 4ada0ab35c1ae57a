"""Host logic of bench.py on CPU: the kernel-source digest that ties the committed ncu traffic to the code it was
measured on, the clock sampler (an NVML reader tested against a fake NVML, with nvidia-smi as the fallback), and
the contract line (short enough for a reader that keeps only the end of the output, and printed last)."""
import ctypes
import json
import os
import shutil
import time

import bench

CSRC = bench.DIGEST_SOURCES


def copy_tree(tmp_path):
    """The digest's sources and the committed profile in a scratch root."""
    root = tmp_path / "root"
    os.makedirs(root / "paper_2112_10517_gb300" / "csrc")
    os.makedirs(root / "profiles")
    for f in CSRC:
        shutil.copy(os.path.join(bench.ROOT, "paper_2112_10517_gb300", "csrc", f),
                    root / "paper_2112_10517_gb300" / "csrc" / f)
    shutil.copy(os.path.join(bench.ROOT, bench.PROFILE_JSON), root / "profiles")
    return str(root)


def test_digest_ignores_comments_and_blank_lines_but_not_code(tmp_path):
    root = copy_tree(tmp_path)
    d0 = bench.source_digest(root)
    assert d0 == bench.source_digest()
    path = os.path.join(root, "paper_2112_10517_gb300", "csrc", "volume_pipe.cuh")
    text = open(path).read()
    open(path, "w").write("// a new comment line\n\n" + text.replace("\n", "  // trailing comment\n", 1))
    assert bench.source_digest(root) == d0
    open(path, "w").write(text + "\nstatic const int a_new_constant = 1;\n")
    assert bench.source_digest(root) != d0
    open(path, "w").write(text)
    # the tile schedule decides which tiles the kernel runs: a change to it is a change of the kernel
    plan = os.path.join(root, "paper_2112_10517_gb300", "csrc", "tile_plan.h")
    open(plan, "a").write("\nstatic const int changed_plan = 3;\n")
    assert bench.source_digest(root) != d0


def test_committed_traffic_only_for_the_source_it_was_measured_on(tmp_path):
    root = copy_tree(tmp_path)
    cap = json.load(open(os.path.join(root, bench.PROFILE_JSON)))
    cap["source_digest"] = bench.source_digest(root)  # as if captured on the current source
    json.dump(cap, open(os.path.join(root, bench.PROFILE_JSON), "w"))
    nd = 32 ** 3 * 64
    for precision in ("fp64", "fp32"):
        t = bench.committed_traffic(precision, nd, root)
        assert t == cap[precision]["traffic_bytes_per_dof"] * nd
        # a capture moves every DOF's state, metric terms and fluxes at least once: 160 B/DOF and more in FP64
        assert t / nd > (160 if precision == "fp64" else 100)
        assert bench.committed_utilization(precision, root)["dram_throughput"] == cap[precision]["dram_throughput"]
    path = os.path.join(root, "paper_2112_10517_gb300", "csrc", "kernels.cuh")
    open(path, "a").write("\nstatic const int changed_code = 2;\n")
    assert bench.committed_traffic("fp64", nd, root) is None
    assert bench.committed_traffic("fp32", nd, root) is None
    assert bench.committed_utilization("fp64", root) is None


class FakeNvml:
    """The four NVML calls the sampler makes; SM clock and reason bits replayed from a list."""

    def __init__(self, samples, max_mhz=2070):
        self.samples = list(samples)
        self.i = 0
        lib = self

        def clock(handle, kind, out):
            assert kind == bench.NvmlClockSampler.NVML_CLOCK_SM
            out._obj.value = lib.samples[min(lib.i, len(lib.samples) - 1)][0]
            return 0

        def max_clock(handle, kind, out):
            out._obj.value = max_mhz
            return 0

        def reasons(handle, out):
            out._obj.value = lib.samples[min(lib.i, len(lib.samples) - 1)][1]
            lib.i += 1
            return 0

        self.nvmlDeviceGetClockInfo = clock
        self.nvmlDeviceGetMaxClockInfo = max_clock
        self.nvmlDeviceGetCurrentClocksEventReasons = reasons


def test_nvml_sampler_reports_median_clock_and_reasons():
    lib = FakeNvml([(2070, 0x0), (1980, 0x4), (2070, 0x4 | 0x8), (2070, 0x0), (1500, 0x20)])
    s = bench.NvmlClockSampler(lib, ctypes.c_void_p(1))
    s.start()
    deadline = time.time() + 10.0
    while lib.i < len(lib.samples) and time.time() < deadline:
        time.sleep(0.001)
    r = s.stop()
    assert r["sm_max_mhz"] == 2070
    assert r["samples"] >= len(lib.samples)
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert r["sm_mhz"] in (1500, 1980, 2070)


def test_sampler_falls_back_to_nvidia_smi_without_nvml(monkeypatch):
    monkeypatch.setattr(bench.NvmlClockSampler, "open", classmethod(lambda cls, device: None))
    s = bench.clock_sampler(0, None)
    assert isinstance(s, bench.ClockSampler)
    assert s.stop()["sm_mhz"] is None  # never started: reported as unavailable, not as a clock


def stub_run(label, pid, frac, precision):
    """A result record of run_ours with the full-precision floats a real run produces."""
    return {"ms_per_step": pid * 4 * 262144 / 1e6 + 1e-9 / 3, "pid_ns": pid + 1e-7 / 3, "pid_std_ns": 0.0012345678,
            "launches": 80, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070, "reasons": ["sw_power_cap"],
                                       "samples": 4321, "source": "NVML, every 5 ms during the timed region"},
            "volume_ms_avg": 0.17234567, "interface_ms_avg": 0.0491234, "volume_share_of_step": 0.79123,
            "graph_ms_per_step": 0.8812345, "graph_pid_ns": pid * 0.99, "noprof_pid_ns": pid * 0.98,
            "e2e_pid_ns": pid * 1.1 + 1e-7 / 3, "e2e_bytes": 262144 * 5 * 8,
            "roofline": {"bound": "alu" if precision == "fp64" else "hbm", "achieved": 0.7654321 / 3,
                         "peak": 1.2574551016763027, "unit": "TFLOP/s" if precision == "fp64" else "GB/s",
                         "frac": frac + 1e-9 / 3, "traffic": 77700034.56789,
                         "peak_src": "FP64 FMA rate measured live (libdgpeaks) x 2 flop",
                         "algorithmic_flops_per_launch": 1.23456789e8,
                         "ncu_utilization": {"fp64_pipe_active": 0.86, "dram_throughput": 0.062,
                                             "capture": bench.PROFILE_JSON}},
            "ndofs": 262144}


def stub_results():
    return {"fp64_16": stub_run("fp64_16", 0.8349499518089942, 0.6012345, "fp64"),
            "fp32_16": stub_run("fp32_16", 0.0967932134443572, 0.4987654, "fp32"),
            "fp64_32": stub_run("fp64_32", 0.7618354777605418, 0.6512345, "fp64"),
            "fp32_32": stub_run("fp32_32", 0.0622070311351308, 0.5012345, "fp32")}


def stub_cpu():
    return {"value": 1604.2085449218848, "unit": "ns/DOF/RHS", "cores": 1, "kind": "oracle", "reps": 23,
            "sample": "23 oracle RHS evaluations of the full 16^3 p=3 mesh (262144 DOF each), 1 core",
            "all_cores": {"value": 101.23456789, "unit": "ns/DOF/RHS", "cores": 16, "sample": "..."}}


def test_contract_line_is_short_and_carries_every_contract_key():
    args = bench.parse_args(["--steps", "20", "--warmup", "5"])
    line = bench.contract_line(args, 1, stub_results(), bench.compact_cpu_baseline(stub_cpu()))
    text = json.dumps(line, separators=(",", ":"))
    assert len(text) < bench.CONTRACT_LINE_MAX_BYTES, len(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert line["higher_is_better"] is False and line["steps"] == 20 and line["warmup"] == 5
    assert abs(line["value"] - 0.8349499518089942) < 1e-3
    assert set(line["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == e2e["d2h_bytes_per_step"] == 262144 * 5 * 8
    assert e2e["value"] != line["value"]
    assert line["clocks"]["reasons"] == ["sw_power_cap"]
    assert "workload" in line["config"]
    assert 0 < line["fp32"]["value"] < line["value"]


def test_main_prints_the_contract_line_last(monkeypatch, capsys):
    monkeypatch.setattr(bench, "run_ours", lambda args, rank, world, local_rank: (stub_results(),
                                                                                 {"fp64": 1.2e12, "fp32": 7.8e13}))
    monkeypatch.setattr(bench, "oracle_pid", lambda seconds: (1604.2, 23, 262144))
    monkeypatch.setattr(bench, "oracle_pid_all_cores", lambda: (101.2, 16))
    monkeypatch.setattr(bench, "run_batch", lambda args, dev: {"fp64": {"pid_ns": 1.8}, "workload": "stub"})
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.main(["--steps", "20", "--warmup", "5", "--extras", "batch"])
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    last = json.loads(lines[-1])
    assert last["metric"] == bench.METRIC and last["steps"] == 20
    assert len(lines[-1]) < bench.CONTRACT_LINE_MAX_BYTES
    details = [json.loads(ln)["bench_detail"] for ln in lines[:-1]]
    assert "batch" in details and "cpu_baseline" in details and "fp64_16" in details
