"""Full runs on the GPU in mixed precision against the FP64 oracle, compared
as distributions over 51 seeds (the runs diverge after a few generations,
since the two sides round differently, so single runs cannot be compared).

Workload: shifted-rotated Griewank (multimodal) at D = 10, budget 1e4 * D,
DE/current-to-pbest/1/bin with archive (NP = 18 D, p = 0.11) and ring PSO
(NP = 40), seeds 1..51; the GPU in TF32 and split BF16 with FP64 refinement
below 1e-4, the oracle in FP64.  Success rates (final error <= 1e-8) must
have overlapping 95 % Wilson intervals and the final errors must pass a
two-sample Kolmogorov-Smirnov test at p > 0.01.
"""
import numpy as np
import pytest

import oracle as O

SEEDS = list(range(1, 52))
D, BUDGET = 10, 100000


@pytest.fixture(scope="module")
def S():
    import paper_2505_17430_gb300 as S
    S.build()
    return S


def wilson(k, n, z=1.959963984540054):
    """95 % Wilson score interval of a binomial proportion k / n."""
    p = k / n
    den = 1.0 + z * z / n
    mid = (p + z * z / (2 * n)) / den
    half = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return mid - half, mid + half


def test_wilson_interval_known_values():
    lo, hi = wilson(0, 51)
    assert lo == 0.0 and abs(hi - 0.0700) < 5e-4
    lo, hi = wilson(31, 51)
    assert abs(lo - 0.4711) < 5e-4 and abs(hi - 0.7301) < 5e-4


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
@pytest.mark.parametrize("alg,NP", [("DE_CTPB", 18 * D), ("PSO_RING", 40)])
def test_mixed_runs_match_oracle_distribution(S, prec, alg, NP):
    stats = pytest.importorskip("scipy.stats")
    seed = 0x5EB00000 + O.GRIEWANK
    p, q = S.Problem(seed, S.GRIEWANK, D), O.Problem(seed, O.GRIEWANK, D)
    a = getattr(S, alg)
    res = S.sevo_run_grid([p], [S.alg_params(a, NP, BUDGET, prec=getattr(S, prec))],
                          [(0, 0, s) for s in SEEDS])
    ref = O.run_many([q] * len(SEEDS), [O.make_alg(a, NP, BUDGET)] * len(SEEDS), SEEDS)
    g_best, o_best = np.asarray(res["best"]), np.array([r["best"] for r in ref])
    g_ok, o_ok = int(np.sum(res["success"])), sum(r["success"] for r in ref)
    assert (np.asarray(res["fes"]) == BUDGET).all()
    assert g_ok == int((g_best <= 1e-8).sum()) and o_ok == int((o_best <= 1e-8).sum())
    gl, gh = wilson(g_ok, len(SEEDS))
    ol, oh = wilson(o_ok, len(SEEDS))
    assert gl <= oh and ol <= gh, (g_ok, o_ok)
    ks = stats.ks_2samp(g_best, o_best)
    assert ks.pvalue > 0.01, (ks.statistic, ks.pvalue, np.median(g_best), np.median(o_best))
