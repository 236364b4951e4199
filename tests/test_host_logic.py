"""Host-side logic with no GPU: ensemble statistics and the benchmark's
source hash that ties the committed ncu traffic to the profiled kernel."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1010_4834_gb300 import ensemble  # noqa: E402


def test_binned_mean_and_error_of_independent_draws():
    # independent normal draws: the binned error is the standard error of
    # the mean, sigma / sqrt(n), whatever the bin count
    rng = np.random.default_rng(3)
    x = rng.normal(2.0, 0.5, 200_000)
    for nbins in (10, 20, 50):
        m, e = ensemble.binned(x, nbins)
        assert abs(m - 2.0) < 5 * 0.5 / np.sqrt(len(x))
        assert 0.6 < e / (0.5 / np.sqrt(len(x))) < 1.6


def test_binned_error_grows_with_autocorrelation():
    # AR(1) series with rho = 0.9: the true error of the mean is larger than
    # the naive one by sqrt((1 + rho) / (1 - rho)) = sqrt(19); long bins see it
    rng = np.random.default_rng(4)
    n, rho = 400_000, 0.9
    eps = rng.normal(0.0, 1.0, n)
    x = np.empty(n)
    x[0] = eps[0]
    for i in range(1, n):
        x[i] = rho * x[i - 1] + np.sqrt(1 - rho * rho) * eps[i]
    _, e = ensemble.binned(x, 20)
    naive = 1.0 / np.sqrt(n)
    assert 0.6 * np.sqrt(19) < e / naive < 1.5 * np.sqrt(19)


def test_binned_drops_the_ragged_tail():
    x = np.arange(23, dtype=float)          # 20 used in 10 bins of 2, 3 dropped
    m, _ = ensemble.binned(x, 10)
    assert m == np.arange(20).mean()


def test_deviation_in_combined_errors():
    assert ensemble.deviation((1.0, 0.3), (0.5, 0.4)) == (0.5 / 0.5)
    assert ensemble.deviation((0.5, 0.3), (1.0, 0.4)) == -1.0


def test_source_hash_ignores_comments_and_follows_code():
    import bench
    c = "int f(int a) { return a + 1; } // add one\n/* block\n comment */\n"
    assert bench._code_only(c) == bench._code_only(c.replace("add one", "increment").replace("block", "x"))
    assert bench._code_only(c) != bench._code_only(c.replace("a + 1", "a + 2"))
    p = "x = 1  # one\ny = x // 2\n"
    assert bench._code_only(p, python=True) == bench._code_only(p.replace("# one", "# first"), python=True)
    assert bench._code_only(p, python=True) != bench._code_only(p.replace("// 2", "// 3"), python=True)
    sha = bench.source_sha()
    assert len(sha) == 16 and all(ch in "0123456789abcdef" for ch in sha)


def test_reference_arm_prints_one_contract_line():
    # the oracle arm of the benchmark (CPU only), on a small extent so the
    # test is quick: one JSON line with the keys the benchmark contract needs
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--extent", "8"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == os.cpu_count()      # the OpenMP build, one thread per core
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_plateau_binning_independent_series():
    # independent draws: the error is flat from the first bin size on
    rng = np.random.default_rng(7)
    x = rng.normal(0.0, 1.0, 64_000)
    m, e, b, ok = ensemble.plateau_binned(x)
    assert ok and b <= 4
    assert 0.85 < e / (1.0 / np.sqrt(len(x))) < 1.15


def test_plateau_binning_finds_the_autocorrelation():
    # AR(1) with rho = 0.95: tau_int = (1 + rho) / (2 (1 - rho)) = 19.5; the
    # error rises with the bin size until bins are several tau long, then
    # stays at sqrt(2 tau_int) = sqrt(39) times the naive error
    rng = np.random.default_rng(8)
    n, rho = 256_000, 0.95
    eps = rng.normal(0.0, 1.0, n)
    x = np.empty(n)
    x[0] = eps[0]
    for i in range(1, n):
        x[i] = rho * x[i - 1] + np.sqrt(1 - rho * rho) * eps[i]
    m, e, b, ok = ensemble.plateau_binned(x)
    assert ok and 32 <= b <= 1024, b
    assert 0.8 * np.sqrt(39) < e / (1.0 / np.sqrt(n)) < 1.2 * np.sqrt(39)


def test_plateau_binning_reports_a_series_too_short():
    # a random walk has no finite autocorrelation time: the error grows with
    # every bin size and no plateau is reported
    rng = np.random.default_rng(9)
    x = np.cumsum(rng.normal(0.0, 1.0, 20_000))
    _, e, b, ok = ensemble.plateau_binned(x)
    assert not ok
    curve = ensemble.binning_curve(x)
    assert e == max(c[1] for c in curve)


def test_thermalisation_drops_the_first_fifth():
    h = np.arange(100.0)[:, None] * np.ones((1, 4))
    assert ensemble.thermalised(h)[0, 0] == 20.0 and len(ensemble.thermalised(h)) == 80


def test_tuning_cache_keys_and_round_trip(tmp_path):
    from paper_1010_4834_gb300 import tuning
    a = tuning.key("NVIDIA GB300", "f32", [(8, 8, 8, 8), (16, 16, 16, 16), (8, 8, 8, 8)])
    b = tuning.key("NVIDIA GB300", "f32", [(16, 16, 16, 16), (8, 8, 8, 8), (8, 8, 8, 8)])
    assert a == b == "NVIDIA GB300|f32|16x16x16x16*1,8x8x8x8*2"        # order-free
    assert tuning.key("NVIDIA GB300", "f64", [(8, 8, 8, 8)]) != tuning.key("NVIDIA GB300", "f32", [(8, 8, 8, 8)])
    p = str(tmp_path / "sub" / "tune.json")
    assert tuning.lookup(a, p) is None
    tuning.store(a, {"groups": 16}, p)
    tuning.store("other", {"groups": 2}, p)
    assert tuning.lookup(a, p) == {"groups": 16} and tuning.lookup("other", p) == {"groups": 2}
