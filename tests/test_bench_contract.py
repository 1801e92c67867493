"""The benchmark's JSON contract and its roofline arithmetic, checked on the CPU: the reference arm (the
FP64 oracle timed on the host) prints one line with the contract's keys, and the HBM roofline and the
per-cell operation count follow their stated definitions."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "advected_wave_128", "--steps", "2", "--warmup", "3"], capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["config"]["workload"] == "advected_wave_128"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["value"] == pytest.approx(128 * 128 * 2 / (d["ms_per_step"] * 2e-3), rel=1e-9)


def test_hbm_roofline_and_operation_count():
    sys.path.insert(0, ROOT)
    import bench
    cells, ms = 8192 * 8192, 3.7
    hbm, none = bench.roofline(5, 4, cells, ms)
    assert none is None
    alg = 8 * 5 * 4 * cells / 3.0  # 8 F B bytes per cell and RK3 step, over 3 launches
    assert hbm["alg_bytes_per_launch"] == pytest.approx(alg)
    assert hbm["achieved"] == pytest.approx(alg / (ms * 1e-3) / 1e9)
    assert hbm["frac"] == pytest.approx(hbm["achieved"] / hbm["peak"])
    assert hbm["bound"] == "hbm" and hbm["unit"] == "GB/s"
    # the method's FP32 operations per cell and stage (no halo): per hydro line cell flux + split 5, two
    # triplets of 23, one face of 15, one difference of 2 and half an accumulation; per level-set line cell
    # 2 + 25 + 14; primitives 8; the cell phase 61 (40 without the level set)
    assert bench.method_ops_per_cell_stage(5) == pytest.approx(8 * 68.5 + 8 + 2 * 41 + 61)
    assert bench.method_ops_per_cell_stage(4) == pytest.approx(8 * 68.5 + 8 + 40)
    # the kernel's count with its line halos: 8 hydro lines of 1210.5 / 15, 2 level-set lines of 700 / 15,
    # primitives on the halo box 12.3
    assert bench.kernel_ops_per_cell_stage(5) == pytest.approx(8 * 1210.5 / 15 + 12.3 + 2 * 700 / 15 + 61, abs=0.5)
    assert bench.kernel_ops_per_cell_stage(4) == pytest.approx(8 * 1210.5 / 15 + 12.3 + 40, abs=0.5)
    # a 15-cell line's halo costs the kernel 12-15 % over the method
    assert 1.12 < bench.kernel_ops_per_cell_stage(5) / bench.method_ops_per_cell_stage(5) < 1.2


def _smi(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 1012.45, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def test_clock_record_rejection_rules():
    """A hardware or thermal slowdown rejects the timed region's number, a power cap alone keeps it (and is
    reported), and a median SM clock well below the maximum with no reason active rejects it."""
    sys.path.insert(0, ROOT)
    import bench
    ok = bench.Clocks.summarise([_smi(1965, 2070), _smi(1980, 2070), "garbage\n", _smi(1950, 2070)])
    assert ok == {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    assert bench.clocks_rejected(ok) is None
    capped = bench.Clocks.summarise([_smi(1500, 2070, cap="Active"), _smi(1490, 2070, cap="Active")])
    assert capped["reasons"] == ["sw_power_cap"] and bench.clocks_rejected(capped) is None
    for kw, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown")):
        rec = bench.Clocks.summarise([_smi(1900, 2070), _smi(1200, 2070, **{kw: "Active"})])
        assert rec["reasons"] == [name] and bench.clocks_rejected(rec) == name
    locked = bench.Clocks.summarise([_smi(1200, 2070)] * 5)
    assert "no reason" in bench.clocks_rejected(locked)
    assert bench.Clocks.summarise([]) is None and bench.clocks_rejected(None) is None


def test_forward_path_times_again_after_a_rejected_clock_record(monkeypatch, capsys):
    """The forward path on the CPU with the context, the CUDA events and the clock sampler replaced by fakes:
    the first timed region's record shows a thermal slowdown, so the region is timed once more and the line
    carries the second region's time, stage launches and clock record (naming why)."""
    sys.path.insert(0, ROOT)
    import torch
    import bench
    from paper_1507_08549_gb300 import hydro

    region_ms = iter([50.0, 20.0])
    records = iter([{"sm_mhz": 1400.0, "sm_max_mhz": 2070.0, "reasons": ["hw_thermal_slowdown"], "samples": 9},
                    {"sm_mhz": 1960.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 9}])

    class Event:  # each region records a start and an end event; the end carries the region's time
        count = 0

        def __init__(self, enable_timing=False):
            self.at = 0.0

        def record(self):
            Event.count += 1
            self.at = next(region_ms) if Event.count % 2 == 0 else 0.0

        def elapsed_time(self, end):
            return end.at - self.at

    class Clocks:
        def __init__(self, index):
            pass

        def start(self):
            pass

        def stop(self):
            return dict(next(records))

    class Ctx:
        launches = 0

        def __init__(self, prob, dtype):
            self.steps = 0

        def state(self, U0):
            return torch.from_numpy(U0.copy())

        def step(self, U, n):
            self.steps += n
            Ctx.launches += 3 * n
            return 0.01 * self.steps, 0.01

        def launch_count(self):
            return Ctx.launches

        def profile(self, on):
            if on:
                self.first = Ctx.launches

        def stage_timing(self):
            return Ctx.launches - self.first, 0.5 * (Ctx.launches - self.first)

        def tile_variants(self):
            return 1, 0

        def autotune(self, U, steps=3):
            return [0.5]

        def tile_info(self, v):
            return {"variant": v, "tile_x": 60, "tile_y": 15, "threads": 320}

        def close(self):
            pass

    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(bench, "Clocks", Clocks)
    monkeypatch.setattr(hydro, "Hydro", Ctx)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "advected_wave_128", "--steps", "4", "--warmup", "3",
                                      "--quick"])
    assert bench.main() == 0
    d = json.loads([l for l in capsys.readouterr().out.splitlines() if l.startswith("{")][-1])
    assert d["ms_per_step"] == pytest.approx(20.0 / 4)
    assert d["value"] == pytest.approx(128 * 128 * 4 / 20e-3)
    assert d["clocks"]["remeasured_after"] == "hw_thermal_slowdown" and d["clocks"]["sm_mhz"] == 1960.0
    assert d["gpu_launches"] == 12 and d["roofline"]["avg_launch_ms"] == pytest.approx(0.5)


def test_alu_roofline_arithmetic(monkeypatch):
    """The FP32 stage kernel's roofline: algorithmic operations per launch (operations per cell and stage
    times cells) over the launch time, against 152 SMs x 128 FP32 lanes x the sampled SM clock; the HBM
    roofline comes along as the second object."""
    sys.path.insert(0, ROOT)
    import torch
    import bench

    class Props:
        multi_processor_count = 152

    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: Props())
    cells, ms = 8192 * 8192, 3.72
    alu, hbm = bench.roofline(5, 4, cells, ms, sm_mhz=2070.0, alu=True, traffic=3.4664e9)
    ops = bench.method_ops_per_cell_stage(5) * cells
    assert alu["bound"] == "alu" and alu["alg_ops_per_launch"] == pytest.approx(ops)
    assert alu["achieved"] == pytest.approx(ops / (ms * 1e-3) / 1e12)
    assert alu["peak"] == pytest.approx(152 * 128 * 2070e6 / 1e12)
    assert alu["frac"] == pytest.approx(alu["achieved"] / alu["peak"])
    assert 0.28 < alu["frac"] < 0.34  # a 3.72 ms launch of the 8192^2 blobs + blast stage
    assert alu["kernel_ops_frac"] == pytest.approx(alu["frac"] * bench.kernel_ops_per_cell_stage(5)
                                                   / bench.method_ops_per_cell_stage(5))
    assert alu["traffic"] == hbm["traffic"] == 3.4664e9
    assert hbm["bound"] == "hbm" and hbm["frac"] == pytest.approx(8 * 5 * 4 * cells / 3 / (ms * 1e-3) / 1e9 / hbm["peak"])


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm's other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "advected_wave_128", "--steps", "2", "--warmup", "3"], capture_output=True, text=True,
                       cwd=ROOT, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_crop_keeps_rows_and_columns_apart():
    """The oracle legs time a crop of the workload; a grid with fewer rows than columns keeps its rows."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1507_08549_gb300 import workloads as wl
    p = wl.advected_wave(24, ny=10)
    sub = bench.crop(p, 16)
    assert (sub.nx, sub.ny) == (16, 10) and sub.U0.shape == (4, 10, 16)
    assert sub.dx == p.dx and sub.dy == p.dy and sub.cells == 160
    oracle.step(sub, sub.U0, 1)  # a consistent problem the oracle accepts
    line = bench.cpu_baseline(p.with_(nx=24, ny=10), seconds=0.05)
    assert line["kind"] == "oracle" and line["sample"].startswith("24x10 crop")


def test_traffic_figure_is_tied_to_the_kernel_source(monkeypatch):
    """The measured DRAM traffic per stage launch is reported only for the stage-kernel source it was
    captured on: a changed source (another SHA-256) gives null, so a stale capture is never reported."""
    sys.path.insert(0, ROOT)
    import bench
    per_cell = bench.stage_traffic_per_cell("60x15")
    assert per_cell is not None and 53.0 < per_cell < 80.0  # algorithmic 160/3 = 53.3 bytes per cell and launch
    assert bench.stage_traffic_per_cell("61x17") is None  # no capture for that tile shape
    monkeypatch.setattr(bench, "stage_kernel_sha256", lambda: "0" * 64)
    assert bench.stage_traffic_per_cell("60x15") is None
