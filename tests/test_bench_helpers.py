"""bench.py's measurement helpers on the CPU: the clock record it attaches to
every line (median SM clock under load, throttle reasons seen), the SIMT
peaks derived from unit counts, and the per-kernel roofline rows."""
import bench


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_median_and_reasons():
    s = bench.ClockSampler(0)
    s.proc = _Done()
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = s.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_without_nvidia_smi():
    rec = bench.ClockSampler(0).stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["nvidia-smi unavailable"]


def test_simt_peaks_from_unit_counts():
    p = bench.alu_peaks({"sm_max_mhz": 2070.0})
    assert abs(p["fp32"] - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert abs(p["fp64"] - 152 * 4 * 2.07e9 / 1e12) < 1e-9


def test_kernel_roofline_rows():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1500.0, "sm_max_mhz": 2000.0}
    prof = {
        "fold_kernel": {"ranges": 2, "ms": 500.0, "flops": 1e12, "bytes": 0.0},
        "sweep": {"ranges": 1, "ms": 10.0, "bytes": 6e9, "flops": 0.0},
        "direct_sum_short": {"ranges": 2, "ms": 1000.0, "flops": 3e13, "bytes": 0.0},
        "big_T_kernel": {"ranges": 1, "ms": 1.0, "flops": 0.0, "bytes": 0.0},
        "id_kernel": {"ranges": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0},
    }
    rows = {r["kernel"]: r for r in bench.kernel_rooflines(prof, peaks, "fp32")}
    assert "id_kernel" not in rows                                  # no ranges: no row
    fold = rows["fold_kernel"]
    assert fold["bound"] == "alu" and abs(fold["achieved"] - 2.0) < 1e-12
    assert abs(fold["frac"] - 2.0 / bench.alu_peaks(peaks)["fp32"]) < 1e-12
    sw = rows["sweep"]
    assert sw["bound"] == "hbm" and abs(sw["achieved"] - 600.0) < 1e-9 and abs(sw["frac"] - 0.1) < 1e-12
    ds = rows["direct_sum_short"]
    assert ds["bound"] == "tensor" and abs(ds["achieved"] - 30.0) < 1e-9 and abs(ds["frac"] - 0.02) < 1e-12
    assert "frac" not in rows["big_T_kernel"]                       # no bound assigned: time only
