"""GPU parity of sevo_evaluate against the FP64 oracle (through the C ABI).

Tolerances are rounding bounds from the oracle's per-row terms
(tests/gpu_util.py): the FP64 path within max(1e-12 |f|, u (E + 2 D G) +
dM Gd), the mixed paths within eps_z G + 2^-23 E on top of that.  Near the
optimum these are far below the 1e-8 success threshold, so the checks there
decide what the method decides.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs
from tests.gpu_util import bound, to_dev, tol64, tol_mixed

pytestmark = pytest.mark.gpu

FAMS = list(range(9))  # the six bodies, hybrid, composition, composition of hybrids
REFINE = 1e-4          # rows whose mixed value is below this are recomputed in FP64


@pytest.fixture(scope="module")
def S():
    import paper_2505_17430_gb300 as S
    S.build()
    return S


def _inputs(q, N, D, seed):
    X = inputs.uniform_pop(N, D, seed=seed)
    o = q.shift(0)
    near = inputs.near(o, 6, 1e-3, seed=seed + 1)
    tiny = inputs.near(o, 3, 1e-7, seed=seed + 2)
    return np.vstack([X, near, tiny, o[None, :]])


def _check_fp64(got, want, bnd, D):
    err = np.abs(got - want)
    tol = tol64(want, bnd)
    assert (err <= tol).all(), (np.max(err / tol), int(np.argmax(err / tol)))
    # where the value is small the tolerance is absolute and tight
    small = want < 1e-6
    if D <= 100:
        assert (tol[small] < 1e-10).all()


def _check_mixed(prec, got, want, bnd, info=None):
    """Every row within the mixed bound; every row whose oracle value is
    below the refinement threshold either came back from the FP64 path
    (FP64 tolerance) or was legitimately left unrefined (its mixed value is
    at or above the threshold, within the mixed bound)."""
    err = np.abs(got - want)
    tm = tol_mixed(prec, want, bnd)
    assert (err <= tm).all(), (np.max(err / tm), int(np.argmax(err / tm)))
    below = want < REFINE
    refined = below & (err <= tol64(want, bnd))
    assert (refined | (got >= REFINE))[below].all()
    # rows below the threshold by more than the mixed bound must be refined
    sure = want + tm < REFINE
    assert refined[sure].all()
    if info is not None:
        assert info["refined"] >= sure.sum()


@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("D", [2, 10, 30, 100, 257])
def test_fp64_path_matches_oracle(S, fam, D):
    """FP64 GPU path within the FP64 rounding bound on random, near-optimum
    (1e-3, 1e-7) and optimum rows; 37+10 rows span several 8-row tiles and a
    ragged tail; D = 257 spans two 256-wide chunks (Rosenbrock carry)."""
    seed = 1000 + 17 * fam + D
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    X = _inputs(q, 37, D, seed)
    got = p.evaluate(to_dev(X), prec=S.FP64).cpu().numpy()
    want = q.eval(X)
    _check_fp64(got, want, bound(p, q, X), D)
    assert got[-1] == 0.0  # f(o) = f* exactly


@pytest.mark.parametrize("fam", FAMS)
def test_fp64_path_d1000_sampled(S, fam):
    D = 1000
    seed = 77 + fam
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    X = _inputs(q, 20, D, seed)
    got = p.evaluate(to_dev(X), prec=S.FP64).cpu().numpy()
    want = q.eval(X)
    _check_fp64(got, want, bound(p, q, X), D)


def _at_level(q, target, n, seed):
    """n points o + t * u (u a random unit direction) with the oracle's g
    within a factor 1.5 of target, t found by bisection on the oracle; None
    where FP64 cannot get that close (a composition whose other components
    keep a weight of order sqrt(s_1) jumps from 0 to large values)."""
    rng = np.random.default_rng(seed)
    o = q.shift(0)
    out = []
    for _ in range(n):
        u = rng.standard_normal(q.D)
        u /= np.linalg.norm(u)
        lo, hi = 0.0, 1.0
        if q.eval(o + hi * u) < target:
            return None
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if q.eval(o + mid * u) < target:
                lo = mid
            else:
                hi = mid
        x = o + hi * u
        if not (target / 1.5 <= q.eval(x) <= target * 1.5):
            return None
        out.append(x)
    return np.array(out)


@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("D", [10, 100])
def test_success_decision_matches_oracle(S, fam, D):
    """Rows placed at g ~ 0.5e-8 and ~ 2e-8 (either side of the 1e-8 success
    threshold): the FP64 path and every mixed path with refinement make the
    oracle's decision, and their values are within the FP64 bound."""
    seed = 2024 + 3 * fam + D
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    rows = [r for r in (_at_level(q, 0.5e-8, 4, seed), _at_level(q, 2e-8, 4, seed + 1))
            if r is not None]
    if not rows:
        assert fam == O.COMPOSITION
        pytest.skip("no FP64 point at g ~ 1e-8 on this composition instance")
    X = np.vstack(rows)
    want = q.eval(X)
    bnd = bound(p, q, X)
    for prec in (S.FP64, S.FP32, S.TF32, S.BF16X3):
        got = p.evaluate(to_dev(X), prec=prec).cpu().numpy()
        assert np.array_equal(got <= 1e-8, want <= 1e-8), prec
        assert (np.abs(got - want) <= tol64(want, bnd)).all(), prec


@pytest.mark.parametrize("prec", ["FP32"])
@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("D", [10, 100])
def test_mixed_path_refines_and_tracks_oracle(S, prec, fam, D):
    """FP32 CUDA-core path: every row within the mixed bound, rows below the
    refinement threshold back from the FP64 path."""
    seed = 555 + fam + D
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    X = np.vstack([_inputs(q, 40, D, seed), inputs.mixed_scales(q.shift(0), 40, D, seed)])
    got, info = p.evaluate(to_dev(X), prec=getattr(S, prec), sync=True)
    got = got.cpu().numpy()
    want = q.eval(X)
    _check_mixed(prec, got, want, bound(p, q, X), info)


def test_nonfinite_rows_reported(S):
    p = S.Problem(3, S.RASTRIGIN, 20)
    X = inputs.uniform_pop(16, 20, seed=3)
    X[5, 7] = np.nan
    X[9, 0] = np.inf
    for prec in (S.FP64, S.FP32):
        out, info = p.evaluate(to_dev(X), prec=prec, sync=True)
        out = out.cpu().numpy()
        assert np.isnan(out[5]) and np.isnan(out[9])
        assert np.isfinite(np.delete(out, [5, 9])).all()
        assert info["nonfinite"] == 2 and info["status"] == -5


def test_empty_and_bad_args(S):
    import ctypes as C
    import torch
    p = S.Problem(3, S.ACKLEY, 10)
    X = torch.zeros((0, 10), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = S.lib()
    assert lib.sevo_evaluate(p.h, C.c_void_p(out.data_ptr()), 0, 10, 10,
                             C.c_void_p(out.data_ptr()), 0, None) == 0
    assert lib.sevo_evaluate(p.h, C.c_void_p(out.data_ptr()), 1, 11, 11,
                             C.c_void_p(out.data_ptr()), 0, None) == -1  # wrong D
    assert lib.sevo_evaluate(p.h, C.c_void_p(out.data_ptr()), 1, 10, 9,
                             C.c_void_p(out.data_ptr()), 0, None) == -1  # ld < D


def test_leading_dimension(S):
    p, q = S.Problem(9, S.GRIEWANK, 30), O.Problem(9, S.GRIEWANK, 30)
    X = inputs.uniform_pop(20, 30, seed=9)
    Xp = np.zeros((20, 34))
    Xp[:, :30] = X
    Xp[:, 30:] = np.nan  # padding must never be read
    import torch
    xt = to_dev(Xp)
    got = p.evaluate(xt[:, :30], prec=S.FP64).cpu().numpy()
    assert np.allclose(got, q.eval(X), rtol=1e-12, atol=0)


def test_bench_shape_sampled(S):
    """N = 4096, D = 100 (the batched-evaluation workload), 6 families; 64
    sampled rows compared with the oracle for FP64 and every mixed mode."""
    X = inputs.uniform_pop(4096, 100, seed=12345)
    rows = np.random.default_rng(0).choice(4096, 64, replace=False)
    xt = to_dev(X)
    for fam in range(6):
        p, q = S.Problem(0x5EB00000 + fam, fam, 100), O.Problem(0x5EB00000 + fam, fam, 100)
        want, bnd = q.eval(X[rows]), bound(p, q, X[rows])
        got = p.evaluate(xt, prec=S.FP64).cpu().numpy()[rows]
        _check_fp64(got, want, bnd, 100)
        for prec in ("FP32", "TF32", "BF16X3"):
            got = p.evaluate(xt, prec=getattr(S, prec)).cpu().numpy()[rows]
            _check_mixed(prec, got, want, bnd)


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("D", [10, 30, 64, 100, 128])
def test_tensor_core_path_matches_oracle(S, prec, fam, D):
    """tcgen05 path (TF32 or split BF16) vs the oracle on 3 row tiles (two
    full, one ragged): every row within the mixed bound; rows below the
    refinement threshold come back from the FP64 path at the FP64 bound;
    f(o) is exactly f*."""
    seed = 4242 + 13 * fam + D
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    X = np.vstack([inputs.uniform_pop(250, D, seed=seed),
                   inputs.mixed_scales(q.shift(0), 40, D, seed),
                   _inputs(q, 0, D, seed)])
    got, info = p.evaluate(to_dev(X), prec=getattr(S, prec), sync=True)
    got = got.cpu().numpy()
    _check_mixed(prec, got, q.eval(X), bound(p, q, X), info)
    assert got[-1] == 0.0


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
def test_tensor_core_many_tiles_per_cta(S, prec):
    """More tiles than SMs (persistent loop, both TMEM/A buffers reused many
    times): 40000 rows at D=100, 200 sampled rows checked."""
    D = 100
    p, q = S.Problem(31, S.RASTRIGIN, D), O.Problem(31, S.RASTRIGIN, D)
    X = inputs.uniform_pop(40000, D, seed=31)
    got = p.evaluate(to_dev(X), prec=getattr(S, prec)).cpu().numpy()
    rows = np.random.default_rng(3).choice(40000, 200, replace=False)
    rows = np.concatenate([rows, [0, 39999]])
    _check_mixed(prec, got[rows], q.eval(X[rows]), bound(p, q, X[rows]))
    assert np.isfinite(got).all()


def test_tensor_core_deterministic(S):
    """Two identical calls give bit-identical results (race canary)."""
    p = S.Problem(5, S.COMPOSITION, 50)
    X = to_dev(inputs.uniform_pop(3000, 50, seed=5))
    for prec in (S.TF32, S.BF16X3):
        a = p.evaluate(X, prec=prec).cpu().numpy()
        b = p.evaluate(X, prec=prec).cpu().numpy()
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("D", [129, 257, 1000])
def test_tensor_core_large_d_matches_oracle(S, prec, fam, D):
    """Large-D tensor-core path (converted operand, 128-column chunk jobs,
    chunk records merged per row): 300 rows over three tiles (one ragged),
    D spanning one, two or eight 128-column chunks with a ragged last chunk
    (Rosenbrock pairs and hybrid groups across chunk borders)."""
    seed = 777 + 7 * fam + D
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    X = np.vstack([inputs.uniform_pop(270, D, seed=seed),
                   inputs.mixed_scales(q.shift(0), 20, D, seed),
                   _inputs(q, 0, D, seed)])
    got, info = p.evaluate(to_dev(X), prec=getattr(S, prec), sync=True)
    got = got.cpu().numpy()
    _check_mixed(prec, got, q.eval(X), bound(p, q, X), info)
    assert got[-1] == 0.0


def test_tensor_core_d5000_sampled(S):
    """D = 5000 (40 chunks of 128 columns, K = 5056): 130 rows, TF32."""
    D = 5000
    p, q = S.Problem(50, S.RASTRIGIN, D), O.Problem(50, O.RASTRIGIN, D)
    X = np.vstack([inputs.uniform_pop(129, D, seed=50), q.shift(0)[None, :]])
    got = p.evaluate(to_dev(X), prec=S.TF32).cpu().numpy()
    _check_mixed("TF32", got, q.eval(X), bound(p, q, X))
    assert got[-1] == 0.0


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("D,N", [(300, 19456), (1000, 4990), (500, 9700)])
def test_tensor_core_large_d_wide_tiles_sampled(S, prec, fam, D, N):
    """Enough rows that the large-D GEMM takes 256-column N tiles (two TMEM
    accumulators, 64-column epilogue slices) by its wave-count rule: TF32 at
    all three sizes (at D = 300 the second tile is half past the padded
    rotation), BF16X3 at D = 500 x 9,700 rows (128-column tiles at the other
    two); sampled rows, the near-optimum probes and the ragged last row tile
    checked against the oracle."""
    seed = 901 + 11 * fam + D
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    X = inputs.uniform_pop(N, D, seed=seed)
    probes = np.vstack([inputs.mixed_scales(q.shift(0), 20, D, seed), _inputs(q, 0, D, seed)])
    X[N - len(probes):] = probes
    got = p.evaluate(to_dev(X), prec=getattr(S, prec)).cpu().numpy()
    rows = np.random.default_rng(seed).choice(N - 128, 160, replace=False)
    rows = np.concatenate([rows, np.arange(N - 128, N)])
    _check_mixed(prec, got[rows], q.eval(X[rows]), bound(p, q, X[rows]))
    assert got[-1] == 0.0
    assert np.isfinite(got).all()


def test_refine_policy_returns_mixed_values(S):
    """SEVO_POLICY_REFINE = 0: sevo_evaluate returns the TF32 values of rows
    below the refinement threshold instead of recomputing them in FP64 (they
    are still counted), within the mixed bound; back on, the same rows come
    back at the FP64 bound.  States keep refining either way."""
    D = 30
    p, q = S.Problem(61, S.RASTRIGIN, D), O.Problem(61, O.RASTRIGIN, D)
    X = np.vstack([inputs.near(q.shift(0), 64, 1e-5, seed=61), inputs.uniform_pop(64, D, seed=61)])
    want, bnd = q.eval(X), bound(p, q, X)
    lib = S.lib()
    assert lib.sevo_get_policy(S.POLICY_REFINE) == 1
    assert lib.sevo_set_policy(S.POLICY_REFINE, 0) == 0
    try:
        raw, info0 = p.evaluate(to_dev(X), prec=S.TF32, sync=True)
    finally:
        assert lib.sevo_set_policy(S.POLICY_REFINE, 1) == 0
    ref, info1 = p.evaluate(to_dev(X), prec=S.TF32, sync=True)
    raw, ref = raw.cpu().numpy(), ref.cpu().numpy()
    assert info0["refined"] == info1["refined"] >= 64
    err_raw, err_ref = np.abs(raw - want), np.abs(ref - want)
    assert (err_raw <= tol_mixed("TF32", want, bnd)).all()
    below = want < 1e-5
    assert below.sum() == 64
    assert (err_ref[below] <= tol64(want, bnd)[below]).all()
    assert (err_raw[below] > tol64(want, bnd)[below]).any()  # really the TF32 values
    assert np.array_equal(raw[~below], ref[~below])
    assert lib.sevo_set_policy(S.POLICY_REFINE, 2) == -1


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
def test_bounded_wait_times_out_and_library_stays_usable(S, prec):
    """SEVO_POLICY_TEST_WAIT makes every CTA of the fused kernel wait on a
    barrier nothing completes, for 20,000 clock cycles, before it issues any
    TMEM, TMA or MMA work: the wait gives up, sevo_evaluate_sync reports
    SEVO_ERR_TIMEOUT, and the next call on the same problem (policy off)
    succeeds and matches the oracle."""
    D = 30
    p, q = S.Problem(71, S.ACKLEY, D), O.Problem(71, O.ACKLEY, D)
    X = inputs.uniform_pop(300, D, seed=71)
    lib = S.lib()
    assert lib.sevo_set_policy(S.POLICY_TEST_WAIT, -1) == S.ERR_ARG
    assert lib.sevo_set_policy(S.POLICY_TEST_WAIT, 20000) == 0
    try:
        import ctypes as C
        import torch
        xt = to_dev(X)
        out = torch.zeros(300, dtype=torch.float64, device="cuda")
        ref, nf = C.c_int64(), C.c_int64()
        rc = lib.sevo_evaluate_sync(p.h, C.c_void_p(xt.data_ptr()), 300, D, D,
                                    C.c_void_p(out.data_ptr()), getattr(S, prec),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                    C.byref(ref), C.byref(nf))
        assert rc == S.ERR_TIMEOUT
    finally:
        assert lib.sevo_set_policy(S.POLICY_TEST_WAIT, 0) == 0
    assert lib.sevo_get_policy(S.POLICY_TEST_WAIT) == 0
    got, info = p.evaluate(to_dev(X), prec=getattr(S, prec), sync=True)
    assert info["status"] == 0
    _check_mixed(prec, got.cpu().numpy(), q.eval(X), bound(p, q, X), info)


def _tune_file(tmp_path, lines=()):
    path = tmp_path / "tune.txt"
    path.write_text("".join(l + "\n" for l in lines))
    return str(path)


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
@pytest.mark.parametrize("fam,D,N", [(6, 1000, 1024), (1, 300, 2000), (8, 257, 700)])
def test_large_d_tile_widths_give_the_same_bits(S, tmp_path, monkeypatch, prec, fam, D, N):
    """The large-D GEMM's N tile (64, 128 or 256 columns, chosen through the
    tuning cache) changes only the speed: records are kept per 32-column
    slice for every width, so all three give bit-identical results, which
    match the oracle (hybrid Rosenbrock pairs and groups across slices,
    compositions of hybrids)."""
    import os
    lib = S.lib()
    p, q = S.Problem(2100 + fam, fam, D), O.Problem(2100 + fam, fam, D)
    X = np.vstack([inputs.uniform_pop(N - 4, D, seed=fam), inputs.near(q.shift(0), 4, 1e-3, seed=fam)])
    xt = to_dev(X)
    pid = getattr(S, prec)
    bucket = 1 << (N - 1).bit_length()
    outs = []
    try:
        for bn in (64, 128, 256):
            monkeypatch.setenv("SEVO_TUNE_FILE", _tune_file(tmp_path, [f"0 {D} {bucket} {pid} {bn}"]))
            assert lib.sevo_set_policy(S.POLICY_AUTOTUNE, 2) == 0
            outs.append(p.evaluate(xt, prec=pid).cpu().numpy())
    finally:
        monkeypatch.delenv("SEVO_TUNE_FILE")
        lib.sevo_set_policy(S.POLICY_AUTOTUNE, 2)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    _check_mixed(prec, outs[0], q.eval(X), bound(p, q, X))


def test_autotuner_ignores_a_width_that_is_not_a_candidate(S, tmp_path, monkeypatch):
    """A cache line whose width is not one of 64, 128, 256 (an edited or
    foreign file) is not used: the call measures the candidates again, appends
    a valid line, and gives the fixed rule's bits."""
    lib = S.lib()
    D, N = 600, 1500
    p = S.Problem(2300, S.RASTRIGIN, D)
    xt = to_dev(inputs.uniform_pop(N, D, seed=23))
    path = _tune_file(tmp_path, [f"0 {D} 2048 {S.TF32} 100"])
    monkeypatch.setenv("SEVO_TUNE_FILE", path)
    try:
        assert lib.sevo_set_policy(S.POLICY_AUTOTUNE, 2) == 0
        S.trace_enable(True)
        got = p.evaluate(xt, prec=S.TF32).cpu().numpy()
        t = S.trace_read()
        S.trace_enable(False)
        assert t["gemm_big"][0] > 1
        lines = [l for l in open(path).read().split("\n") if l.strip()]
        assert len(lines) == 2 and int(lines[1].split()[4]) in (64, 128, 256)
        assert lib.sevo_set_policy(S.POLICY_AUTOTUNE, 0) == 0
        assert np.array_equal(got, p.evaluate(xt, prec=S.TF32).cpu().numpy())
    finally:
        monkeypatch.delenv("SEVO_TUNE_FILE")
        lib.sevo_set_policy(S.POLICY_AUTOTUNE, 2)


def test_autotuner_measures_once_and_caches(S, tmp_path, monkeypatch):
    """SEVO_POLICY_AUTOTUNE: the first large-D call of a (D, row bucket,
    precision) times every width (extra GEMM launches) and writes the choice
    to the cache file; the next call, and a call after the cache is dropped
    and read back from the file, launch the GEMM once; all give the same
    bits, and the same bits as the fixed rule (autotuning off)."""
    import os
    lib = S.lib()
    D, N = 600, 1500
    p = S.Problem(2300, S.RASTRIGIN, D)
    xt = to_dev(inputs.uniform_pop(N, D, seed=23))
    path = _tune_file(tmp_path)
    monkeypatch.setenv("SEVO_TUNE_FILE", path)
    try:
        assert lib.sevo_set_policy(S.POLICY_AUTOTUNE, 2) == 0
        assert lib.sevo_get_policy(S.POLICY_AUTOTUNE) == 1
        outs, gemms = [], []
        for reload in (False, False, True):
            if reload:
                assert lib.sevo_set_policy(S.POLICY_AUTOTUNE, 2) == 0
            S.trace_enable(True)
            outs.append(p.evaluate(xt, prec=S.TF32).cpu().numpy())
            t = S.trace_read()
            S.trace_enable(False)
            gemms.append(t["gemm_big"][0])
        lines = open(path).read().split("\n")
        assert len([l for l in lines if l.strip()]) == 1
        kind, d, bucket, prec, choice = lines[0].split()[:5]
        assert (kind, d, bucket, prec) == ("0", str(D), "2048", str(S.TF32))
        assert int(choice) in (64, 128, 256)
        assert gemms[0] > 1 and gemms[1] == 1 and gemms[2] == 1
        assert lib.sevo_set_policy(S.POLICY_AUTOTUNE, 0) == 0
        outs.append(p.evaluate(xt, prec=S.TF32).cpu().numpy())
        for o in outs[1:]:
            assert np.array_equal(outs[0], o)
        assert lib.sevo_set_policy(S.POLICY_AUTOTUNE, 3) == S.ERR_ARG
    finally:
        monkeypatch.delenv("SEVO_TUNE_FILE")
        lib.sevo_set_policy(S.POLICY_AUTOTUNE, 2)
