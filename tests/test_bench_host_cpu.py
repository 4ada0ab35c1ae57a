"""Host logic of bench.py on CPU: the kernel-source digest that ties the committed ncu traffic to the code it was
measured on, and the clock sampler (an NVML reader tested against a fake NVML, with nvidia-smi as the fallback)."""
import ctypes
import os
import shutil
import time

import bench

CSRC = ("dgmath.cuh", "kernels.cuh", "volume.cu", "volume_impl.cuh", "volume_inst.cu", "volume_pipe.cuh")


def copy_tree(tmp_path):
    """The digest's sources and the committed profile in a scratch root."""
    root = tmp_path / "root"
    os.makedirs(root / "paper_2112_10517_gb300" / "csrc")
    os.makedirs(root / "profiles")
    for f in CSRC:
        shutil.copy(os.path.join(bench.ROOT, "paper_2112_10517_gb300", "csrc", f),
                    root / "paper_2112_10517_gb300" / "csrc" / f)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "volume_kernel_tgv32_p3.md"), root / "profiles")
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


def test_committed_traffic_only_for_the_source_it_was_measured_on(tmp_path):
    root = copy_tree(tmp_path)
    nd = 32 ** 3 * 64
    for precision in ("fp64", "fp32"):
        t = bench.committed_traffic(precision, nd, root)
        assert t is not None and t == bench.committed_traffic(precision, nd)
        # the capture moves every DOF's state, metric terms and fluxes at least once: 160 B/DOF and more in FP64
        assert t / nd > (160 if precision == "fp64" else 100)
    path = os.path.join(root, "paper_2112_10517_gb300", "csrc", "kernels.cuh")
    open(path, "a").write("\nstatic const int changed_code = 2;\n")
    assert bench.committed_traffic("fp64", nd, root) is None
    assert bench.committed_traffic("fp32", nd, root) is None


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
