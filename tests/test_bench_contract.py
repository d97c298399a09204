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
    names = []
    for k in range(256):
        n = lib.dts_kernel_name(k).decode()
        if n == "unknown":
            break
        names.append(n)
    assert len(names) > 20
    for n in names:
        for s_d, s_t in ((4, 4), (2, 2)):
            b = bench.bytes_per_pixel(n, s_d, s_t)
            assert b is not None and b > 0, n
        src = bench.kernel_source(n)
        assert os.path.exists(src), n
        stem = n.split("<")[0]
        assert stem in open(src).read(), f"{n} not defined in {os.path.basename(src)}"
