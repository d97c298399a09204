"""The bench's reference arm on the CPU: one JSON line with the keys the measurement contract
names (the GPU arm's line is checked on the GPU by running the bench itself)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "plain",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "MP/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_every_timed_kernel_has_algorithmic_bytes():
    """Every kernel name the library's per-launch timer reports has algorithmic bytes per pixel in
    the bench (else that kernel would drop out of the bench line's roofline), and the library
    source file the traffic lookup maps it to exists."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    from paper_1805_04590_gb300 import dts

    lib = dts.load()
    names = [n for n in (lib.dts_kernel_name(k).decode() for k in range(256)) if n != "unknown"]
    assert len(names) > 20
    for n in names:
        for s_d, s_t in ((4, 4), (2, 2)):
            b = bench.bytes_per_pixel(n, s_d, s_t)
            assert b is not None and b > 0, n
        src = bench.kernel_source(n)
        assert os.path.exists(src), n
        stem = n.split("<")[0]
        assert stem in open(src).read(), f"{n} not defined in {os.path.basename(src)}"


def test_clock_records_decide_which_runs_are_rejected():
    """A timed run whose clock samples show a hardware or thermal slowdown, or SM clocks stuck
    well below their maximum with no reason given (a leftover clock lock), is rejected; a power cap
    alone is kept and reported."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench

    def summary(rows):
        s = bench.ClockSampler(0)
        s.rows = [[x.strip() for x in r.split(",")] for r in rows]
        return s.summary()

    ok = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1470, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
    hw = "0, 2070, 2070, 900.0, 0x8, Active, Not Active, Not Active, Not Active"
    thermal = "0, 1800, 2070, 900.0, 0x20, Not Active, Not Active, Active, Not Active"
    locked = "0, 900, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active"

    s = summary([ok] * 5)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}
    assert not bench.rejected(s)
    s = summary([ok, capped, capped])
    assert s["reasons"] == ["sw_power_cap"] and not bench.rejected(s)
    assert bench.rejected(summary([ok, hw, ok]))
    assert summary([ok, hw])["reasons"] == ["hw_slowdown"]
    assert bench.rejected(summary([ok, thermal, ok]))
    assert bench.rejected(summary([locked] * 4))
    assert not bench.rejected(summary([]))  # no samples: nothing to judge
