"""Host logic of bench.py that needs no GPU: the hash tying the committed ncu
figures (profiles/traffic.json) to the kernel sources they were taken on, the
roofline views built from them, and the clock record (median SM clock under
load, throttle reasons) that decides whether a bench line stands."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_strip_comments_keeps_code_and_literals():
    b = _bench()
    src = ('int a = 1;  // note\n/* block\n comment */ asm("mov.u32 %0, %%smid; // not a comment" : "=r"(s));\n'
           "char q = '/'; char e = '\\''; const char* t = \"a /* b */ c\";")
    out = b.strip_comments(src)
    assert "note" not in out and "block" not in out
    assert 'asm("mov.u32 %0, %%smid; // not a comment" : "=r"(s));' in out
    assert "char q = '/';" in out and "char e = '\\'';" in out
    assert 'const char* t = "a /* b */ c";' in out


def test_hash_ignores_comments_and_layout_but_not_code():
    b = _bench()
    base = "double f(double x) {\n    return x * x;  // square\n}\n"
    same = "/* the square */\ndouble f(double x) { return x * x; }\n"
    other = "double f(double x) {\n    return x * x * x;\n}\n"
    assert b.strip_comments(base) == b.strip_comments(same)
    assert b.strip_comments(base) != b.strip_comments(other)



def test_roofline_views_from_recorded_figures(monkeypatch):
    b = _bench()
    cells = 8192 * 8192
    rec = {"source_hash": "h", "dram_bytes_per_sweep": 4.9e9, "fp64_flops_per_cell_sweep": 216.0}
    monkeypatch.setattr(b, "recorded_profile", lambda key: dict(rec) if key == "modes8192_fp64" else {})
    monkeypatch.setattr(b, "load_peaks", lambda: {"hbm_gbs": 6788.3})
    # FP64: the FP64-pipe view (216 flops per cell-sweep) outweighs the HBM view
    r = b.roofline_for("modes8192_fp64", 64, cells, {"sweep_ms": 20.0})
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 216.0 * cells / 20e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / b.FP64_PEAK_TFLOPS) < 1e-12
    assert abs(r["hbm_view"]["achieved"] - 2 * 4 * 8 * cells / 20e-3 / 1e9) < 1e-6
    assert r["traffic"] == 4.9e9 and r["algorithmic_bytes_per_launch"] == 2 * 4 * 8 * cells
    # a fused launch does both sweeps: twice the flops and the step kernel's time
    f = b.roofline_for("modes8192_fp64", 64, cells, {"step_kernels_ms": 40.0}, fused=True)
    assert f["traffic"] is None and f["bound"] == "hbm"  # no recorded figures for the fused key
    # FP32: the HBM view with the measured peak; no recorded traffic -> null
    r = b.roofline_for("modes8192_fp32", 32, cells, {"sweep_ms": 0.8})
    assert r["bound"] == "hbm" and r["peak"] == 6788.3 and r["peak_source"] == "measured"
    assert abs(r["achieved"] - 2 * 4 * 4 * cells / 0.8e-3 / 1e9) < 1e-6
    assert r["traffic"] is None
    # without the measured peaks: the fallback, said so
    monkeypatch.setattr(b, "load_peaks", lambda: {})
    r = b.roofline_for("modes8192_fp32", 32, cells, {"sweep_ms": 0.8})
    assert r["peak"] == 6800.0 and r["peak_source"] == "fallback"


def test_recorded_figures_only_for_the_current_sources(monkeypatch):
    b = _bench()
    import json
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    key = next(k for k in rec if not k.startswith("_"))
    monkeypatch.setattr(b, "kernel_source_hash", lambda: rec[key]["source_hash"])
    assert b.recorded_profile(key)["dram_bytes_per_sweep"] == rec[key]["dram_bytes_per_sweep"]
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "0000000000000000")
    assert b.recorded_profile(key) == {}
    assert b.recorded_profile("no_such_workload") == {}


class _FakeProc:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def test_clock_sampler_median_under_load_and_reasons(monkeypatch):
    b = _bench()
    monkeypatch.setattr(b.time, "sleep", lambda s: None)
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    rows = ["0, 345, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # idle
            "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    s = b.ClockSampler(None)
    s.proc = _FakeProc("\n".join(rows) + "\n")
    c = s.stop()
    assert c["samples"] == 5                       # the malformed line is skipped
    assert c["sm_mhz"] == 2070.0                   # median of the loaded samples (idle one left out)
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    s = b.ClockSampler(None)
    s.proc = _FakeProc("0, 1200, 2070, 900.0, 0x8, Active, Not Active, Active, Not Active\n")
    assert b.ClockSampler.stop(s)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert b.ClockSampler(None).stop() is None     # no nvidia-smi: no clock record


def _run_bench(args, env_extra=None):
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    """The reference arm (the oracle on the host cores) runs without a GPU and
    prints one JSON line with the contract's keys; under torchrun only rank 0
    prints; fewer than 3 warm-up steps are refused."""
    import json
    p = _run_bench(["--impl", "reference", "--workload", "sedov128_fp64", "--steps", "2", "--warmup", "3"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["config"]["workload"] == "sedov128_fp64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    p = _run_bench(["--impl", "reference", "--workload", "sedov128_fp64", "--steps", "1", "--warmup", "3",
                    "--gpus", "2"], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0 and p.stdout.strip() == ""
    p = _run_bench(["--impl", "reference", "--workload", "sedov128_fp64", "--steps", "1", "--warmup", "2"])
    assert p.returncode != 0 and "--warmup must be >= 3" in p.stderr
