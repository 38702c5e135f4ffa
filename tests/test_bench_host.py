"""bench.py's host-side pieces, without a GPU: the algorithmic byte counts
behind the roofline fractions, the parser of the clock record taken during the
timed region, and the rule that recorded DRAM counters are reported only while
the kernel sources they were taken on are unchanged."""
import hashlib
import json

import bench


def test_algorithmic_bytes_of_one_iteration():
    """Full form, FP32, 20000x2000 / 2000x20000: R read and written (2mn), B
    twice (2qn), one row of A A^T (m), the vectors and the FP64 row norms
    -- 3.52 GB per iteration, 225.33 GB per 64-iteration launch; 3.68 GB when u
    is formed from A (mp instead of m); the row-space form with r = 2000 keeps
    Z (2mr) and reads K once (r^2): 21.55 GB per launch."""
    m, p, q, n = 20000, 2000, 2000, 20000
    full = bench.iter_bytes(m, p, q, n, 4, gram=True)
    assert full == 2 * m * n * 4 + 2 * q * n * 4 + m * 4 + (m + n + q) * 4 + 3 * m * 8
    assert round(full * 64 / 1e9, 2) == 225.33
    assert round(bench.iter_bytes(m, p, q, n, 4) / 1e9, 2) == 3.68
    assert round(bench.iter_bytes(m, p, q, 2000, 4, gram=True, kpath=True) * 64 / 1e9, 2) == 21.55
    # FP64 doubles the bulk terms, not the FP64 row-norm traffic
    assert bench.iter_bytes(m, p, q, n, 8, gram=True) - 3 * m * 8 == 2 * (full - 3 * m * 8)


def test_algorithmic_bytes_of_the_deferred_update():
    """Deferred update, same system, chunks of T = 64: R read once (mn, no store),
    plus on average (T - 1) / 2 of the chunk's kept U' columns (m) and v rows (n)
    per iteration -- 1.93 GB per iteration, 123.25 GB per launch, the figure the
    bench line divides by the launch time."""
    m, p, q, n = 20000, 2000, 2000, 20000
    full = bench.iter_bytes(m, p, q, n, 4, gram=True)
    dfr = bench.iter_bytes(m, p, q, n, 4, gram=True, deferred=True, T=64)
    assert dfr == full - m * n * 4 + 31.5 * (m + n) * 4
    assert round(dfr / 1e9, 2) == 1.93
    assert round(dfr * 64 / 1e9, 2) == 123.25


def test_clock_record_summary():
    c = bench.ClockSampler(0)
    c.lines = [
        "2070, 2070, 901.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1312.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "1905, 2070, 1398.7, 0x0000000000000008, Active, Not Active, Not Active, Active",
        "[N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "truncated line",
    ]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                                               "samples": 0}


def test_recorded_traffic_follows_the_sources(tmp_path, monkeypatch):
    """DRAM bytes of a capture on a smaller case are scaled to the timed launch by
    the ratio of algorithmic bytes; any change of the kernel's sources voids them."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "k.cu").write_bytes(b"kernel v1")
    sha = hashlib.sha256(b"kernel v1").hexdigest()
    rec = {"iterate_kernel<float>": {"sources": ["k.cu"], "sources_sha256": sha,
                                     "dram_bytes_read": 100, "dram_bytes_write": 23, "algorithmic_bytes": 200}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("iterate_kernel<float>", 200) == 123
    assert bench.recorded_traffic("iterate_kernel<float>", 1000) == 615
    assert bench.recorded_traffic("other_kernel", 200) is None
    (tmp_path / "k.cu").write_bytes(b"kernel v2")
    assert bench.recorded_traffic("iterate_kernel<float>", 200) is None


def test_reference_arm_prints_the_contract_line():
    """--impl reference times the oracle on the CPU and prints one JSON line on
    the native arm's workload label, metric and unit."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--workload", "precision_slice"], capture_output=True, text=True,
                         timeout=300, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.workload_label("precision_slice", 64)
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
