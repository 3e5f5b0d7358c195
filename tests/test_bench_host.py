"""Host logic of bench.py on CPU: the clock-sample parser that decides which
throttle reasons were active during the timed region, and the gate that
reports the committed DRAM traffic only for the kernel source it was
measured on."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


class _Done:
    """Stands in for the finished nvidia-smi process."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_are_parsed(tmp_path):
    b = _bench()
    s = b.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070 MHz, 2070 MHz, 900.1 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2062 MHz, 2070 MHz, 1390.0 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055 MHz, 2070 MHz, 1400.0 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070 MHz, 1.0 W, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s.proc = _Done()
    s.f = open(os.devnull, "w")
    c = s.stop()
    assert c["samples"] == 3 and c["sm_mhz"] == 2062.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    # a throttle that rejects a run is reported by name
    with open(s.path, "w") as f:
        f.write("0, 1500 MHz, 2070 MHz, 700 W, 0x8, Not Active, Active, Not Active, Not Active\n")
    s.proc = _Done()
    s.f = open(os.devnull, "w")
    assert s.stop()["reasons"] == ["hw_thermal_slowdown"]


def test_unsampled_clocks_say_so():
    b = _bench()
    s = b.ClockSampler(0)
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_traffic_only_for_the_kernel_it_was_measured_on(tmp_path):
    b = _bench()
    prof = json.load(open(b.TV_PROFILE))
    assert prof["kernel_hash"] == b.kernel_hash()          # the committed capture is current
    per_voxel = prof["launch_kinds"]["tv_mid"]["dram_bytes_per_voxel"]
    assert b.measured_traffic(1000, "k_tv_step2") == per_voxel * 1000
    assert b.measured_traffic(1000, "k_tv_step") is None   # another kernel
    stale = dict(prof, kernel_hash="0" * 16)
    path = tmp_path / "stale.json"
    path.write_text(json.dumps(stale))
    b.TV_PROFILE = str(path)
    assert b.measured_traffic(1000, "k_tv_step2") is None  # the kernel changed since


def test_kernel_hash_ignores_comments(tmp_path):
    b = _bench()
    src = tmp_path / "a.cu"
    src.write_text("int f();  // one comment\n\n// a whole comment line\nint g();\n")
    lines = list(b._code_lines(str(src)))
    assert lines == ["int f();", "int g();"]
