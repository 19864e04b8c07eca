"""Host logic of bench.py's roofline lines, on made-up traces (no GPU): the
fused evaluation's algorithmic bytes (the operand its rows' operator wrote for
a generation, the FP64 rows for a fresh population), the operators' bytes and
FP64 operations, and the choice of the kernel with the largest measured share
as the line's `roofline`."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _St:
    def __init__(self, R):
        self.R = R


def _trace(eval_ms, trial_ms, move_ms):
    # 10 steps of two groups: 20 fused launches, 40 DE trials, 20 PSO moves
    return {"eval_tc_fused": (20, eval_ms), "de_trial": (40, trial_ms),
            "pso_move": (20, move_ms), "de_select": (40, 1.0)}


def test_eval_bytes_count_operand_rows_and_fresh_rows():
    states = [_St(3) for _ in range(6)]  # 6 states x 3 runs x NP rows
    peaks = {"hbm_gbs": 1000.0}
    K, restarts = 10, 1
    ev, stream, shares = bench.rooflines(_trace(2.0, 3.0, 1.0), states, peaks, K, 5e11, restarts)
    step_rows = 6 * 3 * bench.NP
    want = (step_rows * K * (4 * bench.D + 8) + step_rows * restarts * (8 * bench.D + 8)) // 20
    assert ev["algorithmic_bytes_per_launch"] == want
    assert ev["rows_per_launch"] == step_rows * (K + restarts) // 20
    assert abs(ev["achieved"] - want / (2.0 / 20 * 1e-3) / 1e9) < 0.1
    # operators: 5 FP64 rows of D + the TF32 operand, per row (+16 B of
    # partner records for a DE trial); FP64 ops 3 per coordinate for the DE
    # trials (rand/1 2, current-to-pbest 4) and 8 for the PSO move
    rows = 3 * bench.NP
    assert stream["de_trial"]["algorithmic_bytes_per_launch"] == rows * (44 * bench.D + 16)
    assert stream["pso_move"]["algorithmic_bytes_per_launch"] == rows * 44 * bench.D
    f = stream["pso_move"]["fp64_pipe"]
    assert f["ops_per_coordinate"] == 8 and f["bound"] == "alu"
    assert abs(f["achieved"] - 20 * rows * bench.D * 8 / 1e-3) / f["achieved"] < 1e-3
    assert abs(f["frac"] - f["achieved"] / 5e11) < 1e-3


def test_dominant_kernel_is_the_largest_measured_share():
    states = [_St(3) for _ in range(6)]
    peaks = {"hbm_gbs": 1000.0}
    ev, stream, shares = bench.rooflines(_trace(2.0, 3.0, 1.0), states, peaks, 10, 5e11, 0)
    dom = bench.dominant_roofline(shares, ev, stream)
    assert dom["kernel"] == "de_trial" and dom["bound"] == "alu" and dom["unit"] == "FP64 op/s"
    assert dom["frac"] == stream["de_trial"]["fp64_pipe"]["frac"]
    assert dom["hbm"]["frac"] == stream["de_trial"]["frac"]
    ev, stream, shares = bench.rooflines(_trace(4.0, 3.0, 1.0), states, peaks, 10, 5e11, 0)
    assert bench.dominant_roofline(shares, ev, stream) is ev
    ev, stream, shares = bench.rooflines(_trace(1.0, 2.0, 3.0), states, peaks, 10, 5e11, 0)
    assert bench.dominant_roofline(shares, ev, stream)["kernel"] == "pso_move"


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    d = tmp_path / "paper_2505_17430_gb300" / "csrc"
    d.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (d / "k.cu").write_text("// note\nint f(int a) { return a + 1; }  /* old */\n")
    h0 = bench._source_hash(("k.cu",))
    (d / "k.cu").write_text("// a longer note\n/* block\n   comment */\nint f(int a) {\n  return a + 1;\n}\n")
    assert bench._source_hash(("k.cu",)) == h0
    (d / "k.cu").write_text("int f(int a) { return a + 2; }\n")
    assert bench._source_hash(("k.cu",)) != h0


def test_wilson_interval_matches_scipy():
    """bench.py's success-rate interval is the 95 % Wilson score interval
    (rounded to 4 places), as scipy computes it."""
    st = __import__("pytest").importorskip("scipy.stats")
    for k, n in [(0, 51), (1, 51), (31, 51), (50, 51), (51, 51), (3, 11), (7, 7)]:
        ci = st.binomtest(k, n).proportion_ci(confidence_level=0.95, method="wilson")
        lo, hi = bench.wilson(k, n)
        assert abs(lo - ci.low) <= 5e-5 and abs(hi - ci.high) <= 5e-5, (k, n)
    assert bench.wilson(0, 0) == [0.0, 1.0]
