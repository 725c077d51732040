"""Host-side accounting of bench.py (no GPU): the algorithmic bytes per site
behind the roofline figures, and the source hash that guards the recorded
DRAM traffic."""
import types

import pytest

import bench


def test_bytes_per_site_int32_and_compact_index():
    # 19 populations read and written, plus the index when the kernel gathers
    assert bench.bytes_per_site(4, "ab") == 19 * 4 * 2 + 18 * 4 == 224
    assert bench.bytes_per_site(4, "aa_even") == 152
    assert bench.bytes_per_site(2, "aa_odd") == 76 + 72
    # compact index: 18 16-bit offsets plus 20 int32 tile bases per 256 sites
    assert bench.bytes_per_site(4, "aa_odd", True) == pytest.approx(152 + 36 + 80 / 256)
    assert bench.bytes_per_site(2, "ab", True) == pytest.approx(76 + 36.3125)
    # AA: the index only on odd steps
    for e in (2, 4, 8):
        for ct in (False, True):
            avg = (bench.bytes_per_site(e, "aa_odd", ct) + bench.bytes_per_site(e, "aa_even", ct)) / 2
            assert bench.bytes_per_site(e, "aa", ct) == pytest.approx(avg)


def test_form_stats_splits_aa_parities():
    lat = types.SimpleNamespace(n=1_000_000)
    steps = 10
    durs = [0.6 if k % 2 else 0.4 for k in range(steps)]   # ms; t_first = 0: odd steps at k = 1, 3, ...
    d = bench.form_stats(lat, "fp32", "aa", sum(durs), durs, 0, steps, 6783.8, True)
    k_odd, k_even = d["kernels"]["k_aa_odd"], d["kernels"]["k_aa_even"]
    assert k_odd["launches"] == k_even["launches"] == 5
    assert k_odd["mean_us"] == pytest.approx(600.0) and k_even["mean_us"] == pytest.approx(400.0)
    assert k_odd["gbs"] == pytest.approx(188.3125 * 1e6 / 600e-6 / 1e9)
    assert d["mlups"] == pytest.approx(1e6 * steps / (sum(durs) * 1e-3) / 1e6)
    assert d["index"] == "compact"


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    code = "__global__ void k(float* a) { a[0] = 1.f; }\n"
    f = tmp_path / "k.cu"
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "TRAFFIC_FILES", ["k.cu"])
    f.write_text(code)
    h0 = bench.kernel_sha()
    f.write_text("// a comment\n/* another\n one */\n" + code.replace("{ ", "{\n  "))
    assert bench.kernel_sha() == h0
    f.write_text(code.replace("1.f", "2.f"))
    assert bench.kernel_sha() != h0


def test_kernel_names_follow_the_launch_rule():
    # the pull step takes two sites a thread on the compact table with 32-bit
    # offsets when the site count is even
    assert bench.kernel_names(20_000_864) == ("k_step2", "k_aa_odd")
    assert bench.kernel_names(20_000_865)[0] == "k_step"
    assert bench.kernel_names(20_000_864, compact=False)[0] == "k_step"
    assert bench.kernel_names(20_000_864, wide=True)[0] == "k_step"


def test_reference_arm_runs_the_requested_steps(tmp_path):
    """The oracle arm runs exactly --warmup and --steps, here on a smaller tree
    of the same generator because the full-lattice steps exceed the budget;
    the line keeps the full workload's config."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, str(bench.ROOT / "bench.py"), "--impl", "reference", "--sites", "2000000",
                        "--steps", "2", "--warmup", "1", "--ref-budget", "0.01"],
                       capture_output=True, text=True, timeout=600, cwd=tmp_path)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["config"]["n_sites"] > 1_900_000 and line["value"] > 0
    assert "smaller tree" in line["cpu_baseline"]["sample"] and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["value"] == line["value"]
