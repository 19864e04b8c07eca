"""GPU lock-step parity of the DE/PSO generation path against the oracle,
through the C ABI (sevo_state_*, sevo_de_step, sevo_pso_step, sevo_run_grid).

Lock-step: both sides start each generation from the same state; trial
vectors, positions, velocities and draws must match bit for bit; fitness at
the FP64 tolerance; selection decisions wherever the oracle's margin exceeds
4 x that tolerance; the next generation starts again from the oracle's state.
"""
import numpy as np
import pytest

import oracle as O
from tests.gpu_util import bound, tol64, tol_mixed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2505_17430_gb300 as S
    S.build()
    return S


@pytest.fixture(params=[1, 0], ids=["small_runs", "batched"])
def policy(S, request):
    """Run the test with runs of D <= 32, NP <= 512 advanced by the
    run-per-CTA kernel (1) and by the batched kernels (0)."""
    lib = S.lib()
    old = lib.sevo_get_policy(S.POLICY_SMALL_RUNS)
    S.check(lib.sevo_set_policy(S.POLICY_SMALL_RUNS, request.param), "sevo_set_policy")
    yield request.param
    lib.sevo_set_policy(S.POLICY_SMALL_RUNS, old)


def _state(S, fam, D, alg, NP, budget, seed, prec=None, pseed=None):
    prec = S.FP64 if prec is None else prec
    p = S.Problem(pseed if pseed is not None else 100 + fam, fam, D)
    q = O.Problem(pseed if pseed is not None else 100 + fam, fam, D)
    st = S.State(p, S.alg_params(alg, NP, budget, prec=prec), seed)
    return p, q, st


@pytest.mark.parametrize("alg", [0, 1, 2, 3])
def test_initial_population_bit_exact(S, policy, alg):
    NP, D = 40, 13
    p, q, st = _state(S, S.RASTRIGIN, D, alg, NP, 10000, 77)
    g = st.get()
    X = O.init_population(77, NP, D)
    assert np.array_equal(g["X"], X)
    want = q.eval(X)
    assert (np.abs(g["fx"] - want) <= tol64(want, bound(p, q, X))).all()
    assert st.result()["fes"] == NP and st.result()["best"] == pytest.approx(want.min(), rel=1e-12)


def _decided(fa, fb, tol):
    return np.abs(fa - fb) > 4 * tol


@pytest.mark.parametrize("fam,D,NP", [(S_, D_, N_) for S_, D_, N_ in
                                      [(2, 10, 50), (6, 30, 37), (7, 17, 64), (1, 100, 24)]])
def test_de_rand1_lockstep(S, policy, fam, D, NP):
    p, q, st = _state(S, fam, D, S.DE_RAND1, NP, 10 ** 6, 5)
    X = O.init_population(5, NP, D)
    fx = q.eval(X)
    for gen in range(1, 6):
        st.set(X=X, fx=fx, fes=NP)
        assert st.de_step(gen) == 0
        g = st.get()
        U, part = O.de_rand1_trials(5, gen, X)
        assert np.array_equal(g["part"], part)
        assert np.array_equal(g["U"], U)
        fu = q.eval(U)
        tol = tol64(fu, bound(p, q, U))
        assert (np.abs(g["fu"] - fu) <= tol).all()
        X2, fx2, _, _, acc = O.de_select(5, gen, X, fx, U, fu)
        dec = _decided(fu, fx, tol)
        gacc = np.all(g["X"] == U, axis=1) & ~np.all(U == X, axis=1)
        assert np.array_equal(gacc[dec & ~np.all(U == X, axis=1)],
                              acc.astype(bool)[dec & ~np.all(U == X, axis=1)])
        assert np.array_equal(g["X"][dec], X2[dec])
        X, fx = X2, fx2


def test_de_ctpb_archive_lockstep(S, policy):
    fam, D, NP = S.ACKLEY, 20, 60
    p, q, st = _state(S, fam, D, S.DE_CTPB, NP, 10 ** 6, 9)
    X = O.init_population(9, NP, D)
    fx = q.eval(X)
    A = np.zeros((NP, D))
    asize = 0
    for gen in range(1, 25):
        st.set(X=X, fx=fx, A=A[:asize], asize=asize, fes=NP)
        assert st.de_step(gen) == 0
        g = st.get()
        U, part = O.de_ctpb_trials(9, gen, X, fx, A, asize)
        assert np.array_equal(g["part"], part), gen
        assert np.array_equal(g["U"], U), gen
        fu = q.eval(U)
        tol = tol64(fu, bound(p, q, U))
        assert (np.abs(g["fu"] - fu) <= tol).all()
        X2, fx2, A2, asize2, acc = O.de_select(9, gen, X, fx, U, fu, A, asize)
        if _decided(fu, fx, tol).all():
            assert np.array_equal(g["X"], X2)
            assert g["asize"] == asize2
            assert np.array_equal(g["A"], A2[:asize2])
        X, fx, A, asize = X2, fx2, A2, asize2
    assert asize == NP  # the archive filled and random eviction was exercised


@pytest.mark.parametrize("alg", [0, 1])
def test_de_trials_repair_parents_outside_the_box(S, policy, alg):
    """Parents set outside [lb, ub] by the caller: a trial below lb whose
    midpoint with its parent still lies above ub takes the second repair,
    (ub + x) / 2 (the rare branch of the repair); U and the partners must
    match the oracle bit for bit."""
    fam, D, NP, seed = S.RASTRIGIN, 23, 50, 31
    p, q, st = _state(S, fam, D, alg, NP, 10 ** 6, seed)
    rng = np.random.default_rng(7)
    X = O.init_population(seed, NP, D)
    X[rng.random((NP, D)) < 0.3] *= 10.0  # about 30 % of the coordinates in [-1000, 1000]
    fx = q.eval(X)
    st.set(X=X, fx=fx, fes=NP)
    assert st.de_step(1) == 0
    g = st.get()
    if alg == S.DE_RAND1:
        U, part = O.de_rand1_trials(seed, 1, X)
        v = X[part[:, 0]] + 0.5 * (X[part[:, 1]] - X[part[:, 2]])
    else:
        U, part = O.de_ctpb_trials(seed, 1, X, fx, None, 0)
        v = X + 0.5 * (X[part[:, 0]] - X) + 0.5 * (X[part[:, 1]] - X[part[:, 2]])
    # the rare branch is reached: mutants well below lb with parents above 2 ub - lb
    assert ((v < -101.0) & (X > 301.0)).sum() >= 10
    assert np.array_equal(g["part"], part)
    assert np.array_equal(g["U"], U)


@pytest.mark.parametrize("alg,NP,fam,D", [
    (1, 4096, 2, 10), (1, 600, 4, 17), (1, 60, 0, 8), (0, 1800, 1, 12), (0, 4096, 5, 9)])
def test_de_free_running_selection_and_rank_bit_exact(S, alg, NP, fam, D):
    """Generations stepped back to back with no host write in between, so that
    each generation's p-best pool is the one the previous selection ranked in
    its cluster launch (not a separate ranking of host-set fitness).  Before
    every step the state is read back; the oracle, given that state and the
    library's trial fitness, must produce the same partners and trials and the
    same selection, fitness, archive and archive size, bit for bit (the
    fitness values themselves are the library's, so no tolerance enters a
    decision)."""
    seed = 31 + NP
    p, q, st = _state(S, fam, D, alg, NP, 10 ** 9, seed, prec=S.TF32)
    best = st.get()["fx"].min()  # the initial population's
    assert st.best()[0] == best
    for gen in range(1, 9):
        g0 = st.get()
        A0 = np.zeros((NP, D))
        A0[:g0["asize"]] = g0["A"]
        assert st.de_step(gen) == 0
        g = st.get()
        if alg == 1:
            U, part = O.de_ctpb_trials(seed, gen, g0["X"], g0["fx"], A0, g0["asize"])
        else:
            U, part = O.de_rand1_trials(seed, gen, g0["X"])
        assert np.array_equal(g["part"], part), gen
        assert np.array_equal(g["U"], U), gen
        if alg == 1:
            X2, fx2, A2, as2, _ = O.de_select(seed, gen, g0["X"], g0["fx"], U, g["fu"], A0,
                                              g0["asize"])
            assert g["asize"] == as2 and np.array_equal(g["A"], A2[:as2]), gen
        else:
            X2, fx2, _, _, _ = O.de_select(seed, gen, g0["X"], g0["fx"], U, g["fu"])
        assert np.array_equal(g["X"], X2), gen
        assert np.array_equal(g["fx"], fx2), gen
        best = min(best, g["fu"].min())
        assert st.best()[0] == best, gen
    if alg == 1 and NP <= 600:
        assert g["asize"] == NP  # the archive filled: random slots and overwrites ran


@pytest.mark.parametrize("alg", [0, 1, 4, 2, 3])
@pytest.mark.parametrize("fam", [2, 6, 7])
def test_operand_handoff_equals_converting_evaluation(S, alg, fam):
    """With TF32 and one-component problems the DE trial and PSO move kernels
    also write the rows' tensor-core operand, and the fused evaluation loads
    it instead of converting the rows.  The generation's fitness must equal,
    bit for bit, a plain TF32 sevo_evaluate of the same rows (which converts
    them); a composition (no hand-off) must match too.  Two runs on two
    problems check the per-run offsets of the operand buffer."""
    import torch
    D, NP = 37, 300
    probs = [S.Problem(900 + fam, fam, D), S.Problem(901 + fam, fam, D)]
    st = S.State(probs, S.alg_params(alg, NP, 10 ** 9, prec=S.TF32), [5, 6])
    for gen in (1, 2):
        if alg in (2, 3):
            assert st.pso_step(gen) == 0
        else:
            assert st.de_step(gen) == 0
        g = st.get()
        rows, fit = (g["X"], g["fx"]) if alg in (2, 3) else (g["U"], g["fu"])
        for r, p in enumerate(probs):
            Xr = torch.tensor(rows[r * NP:(r + 1) * NP], dtype=torch.float64, device="cuda")
            ref = p.evaluate(Xr, prec=S.TF32).cpu().numpy()
            got = fit[r * NP:(r + 1) * NP]
            assert np.array_equal(got.view(np.int64), ref.view(np.int64)), (gen, r)


@pytest.mark.parametrize("alg,NP", [(2, 4096), (3, 4096), (3, 700), (2, 50)])
def test_pso_free_running_update_bit_exact(S, alg, NP):
    """PSO generations back to back: from the state read before each step, the
    oracle's move, personal-best update (with the library's fitness) and
    guides (gbest / ring) equal the library's bit for bit."""
    fam, D, seed = S.GRIEWANK, 11, 17 + NP
    topo = alg - 2
    p, q, st = _state(S, fam, D, alg, NP, 10 ** 9, seed, prec=S.TF32)
    for gen in range(1, 7):
        g0 = st.get()
        guide = O.pso_guides(g0["fp"], topo)
        assert np.array_equal(g0["part"][:, 0], guide), gen
        assert st.pso_step(gen) == 0
        g = st.get()
        X2, V2 = O.pso_move(seed, gen, g0["X"], g0["V"], g0["P"], guide)
        assert np.array_equal(g["X"], X2) and np.array_equal(g["V"], V2), gen
        P2, fp2, _ = O.pso_update(X2, g["fx"], g0["P"], g0["fp"])
        assert np.array_equal(g["P"], P2) and np.array_equal(g["fp"], fp2), gen
    assert np.array_equal(st.get()["part"][:, 0], O.pso_guides(fp2, topo))


@pytest.mark.parametrize("alg", [2, 3])
def test_pso_lockstep(S, policy, alg):
    fam, D, NP = S.GRIEWANK, 25, 40
    p, q, st = _state(S, fam, D, alg, NP, 10 ** 6, 13)
    X = O.init_population(13, NP, D)
    V = np.zeros_like(X)
    fx = q.eval(X)
    P, fp = X.copy(), fx.copy()
    topo = alg - 2
    for gen in range(1, 8):
        st.set(X=X, V=V, P=P, fp=fp, fes=NP)
        guide = O.pso_guides(fp, topo)
        assert np.array_equal(st.get()["part"][:, 0], guide)
        assert st.pso_step(gen) == 0
        g = st.get()
        X2, V2 = O.pso_move(13, gen, X, V, P, guide)
        assert np.array_equal(g["X"], X2)
        assert np.array_equal(g["V"], V2)
        fx2 = q.eval(X2)
        tol = tol64(fx2, bound(p, q, X2))
        assert (np.abs(g["fx"] - fx2) <= tol).all()
        P2, fp2, _ = O.pso_update(X2, fx2, P, fp)
        dec = _decided(fx2, fp, tol)
        assert np.array_equal(g["P"][dec], P2[dec])
        X, V, P, fp = X2, V2, P2, fp2


def test_c0_full_run_lockstep(S, policy):
    """The smallest workload: DE/rand/1/bin, NP=50, D=10, F=.5, CR=.9, FP64, budget 1e5
    on shifted-rotated Rastrigin; every one of the 1999 generations is
    compared in lock step (re-synchronised from the oracle each time)."""
    NP, D, budget, seed = 50, 10, 100000, 1
    p, q = S.Problem(1, S.RASTRIGIN, D), O.Problem(1, O.RASTRIGIN, D)
    st = S.State(p, S.alg_params(S.DE_RAND1, NP, budget), seed)
    X = O.init_population(seed, NP, D)
    fx = q.eval(X)
    mism = 0
    for gen in range(1, 2000):
        st.set(X=X, fx=fx, fes=NP)
        st.de_step(gen)
        g = st.get()
        U, _ = O.de_rand1_trials(seed, gen, X)
        assert np.array_equal(g["U"], U)
        fu = q.eval(U)
        tol = tol64(fu, bound(p, q, U))
        X2, fx2, _, _, _ = O.de_select(seed, gen, X, fx, U, fu)
        dec = _decided(fu, fx, tol)
        assert np.array_equal(g["X"][dec], X2[dec])
        # near-ties (common once the population has converged): either
        # outcome is a valid selection, so the row must be x or u
        und = ~dec
        assert (np.all(g["X"][und] == X[und], axis=1) | np.all(g["X"][und] == U[und], axis=1)).all()
        mism += und.sum()
        X, fx = X2, fx2
    ref = O.run(q, O.make_alg(O.ALG_DE_RAND1, NP, budget), seed)
    assert ref["best"] == pytest.approx(min(fx.min(), ref["best"]), abs=1e-9)
    print("undecided selections:", mism, "of", 1999 * NP)


def test_full_run_matches_oracle_fp64(S, policy):
    """A whole run on the FP64 path (no re-sync) ends at the oracle's best
    error: the trajectories agree unless a near-tie flips a decision."""
    NP, D, budget, seed = 30, 10, 6000, 3
    for alg in (0, 1, 2, 3):
        p, q = S.Problem(21, S.ELLIPSOID, D), O.Problem(21, O.ELLIPSOID, D)
        st = S.State(p, S.alg_params(alg, NP, budget), seed)
        gen = 0
        while st.result()["fes"] < budget:
            gen += 1
            assert st.step(gen) == 0
        r = st.result()
        ref = O.run(q, O.make_alg(alg, NP, budget), seed)
        assert r["fes"] == budget == ref["fes"] and r["gens"] == ref["gens"]
        assert r["best"] == pytest.approx(ref["best"], rel=1e-9, abs=1e-12), alg


def test_budget_and_bad_calls(S, policy):
    p = S.Problem(1, S.SCHWEFEL, 10)
    st = S.State(p, S.alg_params(S.PSO_GBEST, 40, 100), 1)
    assert st.de_step(1) == -7          # wrong algorithm kind
    assert st.pso_step(1) == 0          # 40 + 40 = 80
    assert st.pso_step(2) == 0          # last generation counts 20 rows
    assert st.result()["fes"] == 100
    assert st.pso_step(3) == -7         # budget spent


def test_save_load_resume_bit_identical(S, policy):
    p = S.Problem(4, S.HYBRID, 20)
    for alg in (1, 3):
        a = S.State(p, S.alg_params(alg, 32, 10 ** 6), 8)
        for g in range(1, 6):
            a.step(g)
        blob = a.save()
        for g in range(6, 11):
            a.step(g)
        b = S.State(p, S.alg_params(alg, 32, 10 ** 6), 123)
        b.load(blob)
        for g in range(6, 11):
            b.step(g)
        ga, gb = a.get(), b.get()
        for k in ("X", "fx", "V", "P", "fp", "A"):
            assert np.array_equal(ga[k], gb[k]), (alg, k)
        assert a.result()["best"] == b.result()["best"]


def test_grid_equals_single_runs(S, policy):
    """sevo_run_grid (batched runs, graph-captured generations) gives the
    same results as driving each run alone through the state API."""
    D = 10
    probs = [S.Problem(s, f, D) for s, f in [(1, 2), (2, 6), (3, 7)]]
    algs = [S.alg_params(S.DE_CTPB, 40, 2000), S.alg_params(S.PSO_RING, 20, 2010)]
    tasks = [(pi, ai, 1000 + 10 * pi + ai + 100 * k) for pi in range(3) for ai in range(2)
             for k in range(3)]
    res = S.sevo_run_grid(probs, algs, tasks, gens_per_graph=8)
    for t, (pi, ai, seed) in enumerate(tasks):
        st = S.State(probs[pi], algs[ai], seed)
        gen = 0
        while st.result()["fes"] < algs[ai].budget:
            gen += 1
            st.step(gen)
        r = st.result()
        assert res["fes"][t] == r["fes"] and res["gens"][t] == r["gens"]
        assert res["best"][t] == r["best"], (t, res["best"][t], r["best"])


@pytest.mark.parametrize("prec", ["TF32", "BF16X3", "FP32"])
def test_mixed_precision_runs_reach_oracle_quality(S, policy, prec):
    """Mixed-precision runs (FP64 refinement below 1e-4): DE/ctpb on the
    unimodal shifted-rotated ellipsoid at D=10 reaches the 1e-8 success
    threshold like the oracle does."""
    D, NP, budget = 10, 50, 60000
    probs = [S.Problem(2, S.ELLIPSOID, D)]
    algs = [S.alg_params(S.DE_CTPB, NP, budget, prec=getattr(S, prec))]
    res = S.sevo_run_grid(probs, algs, [(0, 0, s) for s in range(1, 9)])
    q = O.Problem(2, O.ELLIPSOID, D)
    ref = [O.run(q, O.make_alg(O.ALG_DE_CTPB, NP, budget), s)["success"] for s in range(1, 9)]
    assert res["success"].sum() >= sum(ref) - 2


@pytest.mark.parametrize("NP,ties", [(600, "stride"), (1800, "stride"), (4096, "stride"),
                                      (4096, "all"), (4096, "kth"), (2000, "near")])
def test_de_ctpb_large_population_sorted_pbest(S, NP, ties):
    """NP > 512 ranks by radix select of the k-th key plus a sort of the
    candidates (ties by index); trial vectors must still match the oracle
    bit for bit.  Fitness patterns: every 7th row tied with row 0; every row
    equal (the select has nothing to split); 300 rows tied with the k-th
    smallest value (the select runs to the last digit and the sort takes all
    of them); values one ulp apart (the keys differ only in the low digits)."""
    fam, D = S.RASTRIGIN, 10
    p, q, st = _state(S, fam, D, S.DE_CTPB, NP, 10 ** 7, 21)
    X = O.init_population(21, NP, D)
    fx = q.eval(X)
    if ties == "stride":
        fx[::7] = fx[0]
    elif ties == "all":
        fx[:] = 123.25
    elif ties == "kth":
        k = max(2, int(np.ceil(0.11 * NP)))
        kth = np.sort(fx)[k - 1]
        fx[np.random.default_rng(5).choice(NP, 300, replace=False)] = kth
    else:
        fx = 1000.0 + np.random.default_rng(6).permutation(NP) * np.spacing(1000.0)
    A = np.zeros((NP, D))
    st.set(X=X, fx=fx, A=A[:0], asize=0, fes=NP)
    assert st.de_step(3) == 0
    g = st.get()
    U, part = O.de_ctpb_trials(21, 3, X, fx, A, 0)
    assert np.array_equal(g["part"], part)
    assert np.array_equal(g["U"], U)


@pytest.mark.parametrize("prec", ["TF32", "BF16X3"])
def test_batched_mixed_segments_many_jobs_per_cta(S, prec):
    """A batch of 48 runs over single, hybrid and composition problems at
    D=30 with NP=540: the fused tensor-core evaluation has more (tile,
    component) jobs than CTAs, so one CTA alternates composition and
    non-composition jobs. Every initial fitness matches the oracle within the
    mixed tolerance, and no bounded device wait gives up (a timeout would
    surface as SEVO_ERR_TIMEOUT from sevo_state_best / sevo_state_result)."""
    D, NP = 30, 540
    keys = [(600 + k, k % 9) for k in range(27)]
    probs = [S.Problem(s, f, D) for s, f in keys for _ in range(2)]
    seeds = [9000 + r for r in range(len(probs))]
    st = S.State(probs, S.alg_params(S.DE_CTPB, NP, 10 ** 9, prec=getattr(S, prec)), seeds)
    fx = st.get()["fx"]
    for r, (s, f) in enumerate([k for k in keys for _ in range(2)]):
        q = O.Problem(s, f, D)
        X = O.init_population(seeds[r], NP, D)
        want = q.eval(X)
        got = fx[r * NP:(r + 1) * NP]
        tm = tol_mixed(prec, want, bound(probs[r], q, X))
        assert (np.abs(got - want) <= tm).all(), (r, f, np.max(np.abs(got - want) / tm))
    for g in range(1, 4):
        assert st.step(g) == 0
    st.best()
    assert st.result()["gens"] == 3


def test_kernel_trace_counts_and_times(S):
    """Tracing brackets every launch outside graph capture with events on its
    stream: one DE/ctpb step traces rank, trial, evaluation, select and apply
    launches with positive device time (the next step needs no rank launch:
    its selection ranked the population); a run grid (graph-captured
    generations) adds no captured launch to the totals."""
    D, NP = 30, 64
    p = S.Problem(77, S.RASTRIGIN, D)
    lib = S.lib()
    old_policy = lib.sevo_get_policy(S.POLICY_SMALL_RUNS)
    lib.sevo_set_policy(S.POLICY_SMALL_RUNS, 0)
    st = S.State(p, S.alg_params(S.DE_CTPB, NP, 10 ** 6, prec=S.TF32), 5)
    lib.sevo_set_policy(S.POLICY_SMALL_RUNS, 1)
    small = S.State(p, S.alg_params(S.DE_CTPB, NP, 10 ** 6, prec=S.TF32), 5)
    lib.sevo_set_policy(S.POLICY_SMALL_RUNS, old_policy)
    S.trace_enable(True)
    assert small.de_step(1) == 0
    t = S.trace_read()
    assert t["small_run"][0] == 1 and t["small_run"][1] > 0.0 and t["de_trial"][0] == 0
    S.trace_enable(True)
    assert st.de_step(1) == 0
    t = S.trace_read()
    for k in ("de_rank", "de_trial", "eval_tc_fused", "de_select", "de_apply"):
        assert t[k][0] == 1 and t[k][1] > 0.0, (k, t[k])
    # fused operators: the trials are formed inside the evaluation
    old_fuse = lib.sevo_get_policy(S.POLICY_FUSE_OPS)
    lib.sevo_set_policy(S.POLICY_FUSE_OPS, 1)
    S.trace_enable(True)
    assert st.de_step(2) == 0
    t = S.trace_read()
    lib.sevo_set_policy(S.POLICY_FUSE_OPS, old_fuse)
    # the first step's selection already ranked the population it left
    assert t["de_trial"][0] == 0 and t["eval_tc_fused"][0] == 1 and t["de_rank"][0] == 0
    assert t["de_select"][0] == 1
    S.trace_enable(True)
    lib.sevo_set_policy(S.POLICY_SMALL_RUNS, 0)
    S.sevo_run_grid([p], [S.alg_params(S.PSO_RING, 20, 20 * 40)], [(0, 0, 3)], gens_per_graph=8)
    lib.sevo_set_policy(S.POLICY_SMALL_RUNS, old_policy)
    t = S.trace_read()
    S.trace_enable(False)
    assert t["pso_move"][0] < 39  # most generations ran inside graphs
    assert t["init"][0] == 1


def test_trace_timeline_spans_match_totals(S):
    """Tracing mode 2 keeps every traced launch as (kind, stream id, start,
    end): two states on their own streams stepped together give spans on two
    stream ids, sorted by start, each with end >= start, whose per-kind counts
    and summed durations equal the per-kind totals; mode 1 keeps none."""
    import torch
    D, NP = 30, 600
    p = S.Problem(78, S.RASTRIGIN, D)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sts = [S.State(p, S.alg_params(alg, NP, 10 ** 6, prec=S.TF32), 5 + k, stream=s)
           for k, (alg, s) in enumerate(zip((S.DE_RAND1, S.PSO_RING), streams))]
    torch.cuda.synchronize()
    S.trace_enable(True, timeline=True)
    for g in range(1, 4):
        assert S.sevo_state_step_many(sts, g) == 0
    torch.cuda.synchronize()
    spans = S.trace_timeline()
    t = S.trace_read()
    S.trace_enable(True)
    assert sts[0].de_step(4) == 0
    torch.cuda.synchronize()
    assert S.trace_timeline() == []
    S.trace_enable(False)
    assert len(spans) == sum(c for c, _ in t.values()) > 0
    assert {s for _, s, _, _ in spans} == {0, 1}
    starts = [a for _, _, a, _ in spans]
    assert starts == sorted(starts) and all(b >= a for _, _, a, b in spans)
    for k, (c, ms) in t.items():
        mine = [b - a for kk, _, a, b in spans if kk == k]
        assert len(mine) == c and abs(sum(mine) - ms) <= 1e-3 * (1 + ms), k


@pytest.mark.parametrize("alg", [1, 3])
def test_restart_equals_fresh_state(S, policy, alg):
    """sevo_state_restart(seeds) leaves a (batched) state bit-identical to a
    state freshly created with those seeds, and both step identically."""
    D, NP = 13, 40
    probs = [S.Problem(300 + k, fam, D) for k, fam in enumerate((2, 6, 7))]
    a = S.alg_params(alg, NP, 10 ** 6)
    st = S.State(probs, a, [1, 2, 3])
    for g in range(1, 6):
        assert st.step(g) == 0
    st.restart([11, 12, 13])
    fresh = S.State(probs, a, [11, 12, 13])
    for g in range(0, 3):
        if g:
            assert st.step(g) == 0 and fresh.step(g) == 0
        ga, gb = st.get(), fresh.get()
        # partner indices are written by each generation's trial kernel
        for k in ("X", "fx", "A", "V", "P", "fp") + (("part",) if g else ()):
            assert np.array_equal(ga[k], gb[k]), (g, k)
        assert ga["asize"] == gb["asize"]
        assert st.result() == fresh.result()
        assert np.array_equal(st.best(), fresh.best())


def test_small_runs_grid_single_launch_and_refined_count(S):
    """With the run-per-CTA policy a grid bucket of small runs advances all
    its generations in one launch; mixed-precision runs report how many rows
    were re-evaluated in FP64 (nonzero once a run gets below 1e-4)."""
    D, NP, budget = 10, 50, 150000
    p = S.Problem(2, S.ELLIPSOID, D)
    a = S.alg_params(S.DE_CTPB, NP, budget, prec=S.TF32)
    lib = S.lib()
    old = lib.sevo_get_policy(S.POLICY_SMALL_RUNS)
    lib.sevo_set_policy(S.POLICY_SMALL_RUNS, 1)
    try:
        S.trace_enable(True)
        res = S.sevo_run_grid([p], [a], [(0, 0, s) for s in range(1, 5)])
        t = S.trace_read()
        S.trace_enable(False)
        assert t["small_run"][0] == 1 and t.get("de_trial", (0, 0))[0] == 0
        assert res["gens"][0] == (budget - NP + NP - 1) // NP
        done = [k for k in range(4) if res["best"][k] < 1e-4]
        assert done, res["best"]  # some run reached the refinement range
        seed = 1 + done[0]
        st = S.State(p, a, seed)
        g = 0
        while st.result()["fes"] < budget:
            g += 1
            st.step(g)
        r = st.result()
        assert r["best"] == res["best"][done[0]]
        assert r["refined"] > 0
    finally:
        lib.sevo_set_policy(S.POLICY_SMALL_RUNS, old)


def test_policy_arguments(S):
    lib = S.lib()
    assert lib.sevo_set_policy(99, 1) == S.ERR_ARG
    assert lib.sevo_set_policy(S.POLICY_SMALL_RUNS, 7) == S.ERR_ARG
    assert lib.sevo_get_policy(99) == -1


def test_async_set_get_match_sync(S):
    """sevo_state_set_async / sevo_state_get_async move the same data as the
    synchronous calls once the state's stream has passed them."""
    import ctypes as C
    import torch
    D, NP = 24, 32
    p = S.Problem(41, S.ACKLEY, D)
    stream = torch.cuda.Stream()
    st = S.State([p, p], S.alg_params(S.PSO_RING, NP, 10 ** 6), [3, 4], stream=stream)
    X = torch.from_numpy(O.init_population(99, 2 * NP, D)).pin_memory()
    fx = torch.empty(2 * NP, dtype=torch.float64).pin_memory()
    V = torch.empty((2 * NP, D), dtype=torch.float64).pin_memory()
    dp = C.POINTER(C.c_double)
    ptr = lambda t: C.cast(C.c_void_p(t.data_ptr()), dp)  # noqa: E731
    lib = S.lib()
    assert lib.sevo_state_set_async(st.h, ptr(X), None, None, 0, None, None, None, -1) == 0
    assert st.step(1) == 0
    assert lib.sevo_state_get_async(st.h, None, ptr(fx), None, ptr(V), None, None, None, None) == 0
    stream.synchronize()
    g = st.get()
    assert np.array_equal(fx.numpy(), g["fx"]) and np.array_equal(V.numpy(), g["V"])
    ref = S.State([p, p], S.alg_params(S.PSO_RING, NP, 10 ** 6), [3, 4])
    ref.set(X=X.numpy())
    assert ref.step(1) == 0
    r = ref.get()
    assert np.array_equal(r["fx"], g["fx"]) and np.array_equal(r["X"], g["X"])


# ---------------------------------------------------------------- SHADE
def _shade_state(S, fam=2, D=13, NP=64, seed=17, prec=None):
    p = S.Problem(400 + fam, fam, D)
    q = O.Problem(400 + fam, fam, D)
    st = S.State(p, S.alg_params(S.DE_SHADE, NP, 10 ** 6, prec=S.FP64 if prec is None else prec),
                 seed)
    return p, q, st


def test_shade_params_match_oracle(S):
    """Per-row F, CR and pbest pool drawn on the GPU from a given memory
    equal the oracle's draws (pool exactly; F and CR to 1e-13, the two sides'
    log, cos and tan may differ in the last place)."""
    NP, seed = 64, 17
    p, q, st = _shade_state(S, NP=NP, seed=seed)
    rng = np.random.default_rng(5)
    MF, MCR = rng.uniform(0.05, 0.95, S.SHADE_H), rng.uniform(0.0, 1.0, S.SHADE_H)
    st.set_shade(MF, MCR, 17)
    assert st.de_step(3) == 0
    sh = st.get_shade()
    F, CR, kpb = O.shade_params(seed, 3, NP, MF, MCR)
    assert np.array_equal(sh["kpb"], kpb)
    assert np.allclose(sh["F"], F, rtol=1e-13, atol=0) and np.allclose(sh["CR"], CR, rtol=1e-13, atol=1e-15)
    assert (sh["F"] > 0).all() and (sh["F"] <= 1).all() and (sh["CR"] >= 0).all() and (sh["CR"] <= 1).all()


@pytest.mark.parametrize("fam,D,NP", [(2, 13, 64), (6, 30, 40), (1, 100, 600)])
def test_shade_lockstep(S, fam, D, NP):
    """Five generations in lock step with the oracle: given the GPU's
    parameters, trial vectors and partners are bit-identical to the oracle's,
    fitness within the FP64 tolerance, selection identical, and the memory
    update equal to the oracle's within 1e-13 (sums in another order)."""
    seed = 23
    p, q, st = _shade_state(S, fam=fam, D=D, NP=NP, seed=seed)
    X = O.init_population(seed, NP, D)
    fx = q.eval(X)
    MF, MCR, k = O.shade_memory()
    for gen in range(1, 6):
        st.set(X=X, fx=fx, fes=NP)
        st.set_shade(MF, MCR, k)
        assert st.de_step(gen) == 0
        g, sh = st.get(), st.get_shade()
        Fo, CRo, kpbo = O.shade_params(seed, gen, NP, MF, MCR)
        assert np.array_equal(sh["kpb"], kpbo)
        assert np.allclose(sh["F"], Fo, rtol=1e-13, atol=0)
        U, part = O.shade_trials(seed, gen, X, fx, sh["F"], sh["CR"], sh["kpb"])
        assert np.array_equal(g["part"], part)
        assert np.array_equal(g["U"], U)
        fu = q.eval(U)
        assert (np.abs(g["fu"] - fu) <= tol64(fu, bound(p, q, U))).all()
        MFo, MCRo, ko, n = O.shade_update(fx, g["fu"], sh["F"], sh["CR"], MF, MCR, k)
        assert int(sh["k"][0]) == ko
        assert np.allclose(sh["MF"][0], MFo, rtol=1e-13, atol=0)
        assert np.allclose(sh["MCR"][0], MCRo, rtol=1e-13, atol=1e-16)
        X2, fx2, _, _, _ = O.de_select(seed, gen, X, fx, U, g["fu"])
        assert np.array_equal(g["X"], X2) and np.array_equal(g["fx"], fx2)
        X, fx, MF, MCR, k = X2, fx2, sh["MF"][0], sh["MCR"][0], int(sh["k"][0])


def test_shade_full_run_and_grid(S):
    """SHADE on the shifted-rotated ellipsoid (D = 10, NP = 50, 6e4
    evaluations, FP64) reaches the 1e-8 success threshold like the oracle's
    control run; a grid of SHADE runs equals the same runs driven alone."""
    D, NP, budget = 10, 50, 60000
    p = S.Problem(3, S.ELLIPSOID, D)
    a = S.alg_params(S.DE_SHADE, NP, budget)
    res = S.sevo_run_grid([p], [a], [(0, 0, s) for s in (1, 2, 3)])
    assert res["success"].all(), res["best"]
    st = S.State(p, a, 2)
    g = 0
    while st.result()["fes"] < budget:
        g += 1
        st.de_step(g)
    assert st.result()["best"] == res["best"][1]


def test_shade_save_load_resume_bit_identical(S):
    p, q, a = _shade_state(S, NP=40, seed=8)
    for g in range(1, 6):
        a.de_step(g)
    blob = a.save()
    p2, q2, b = _shade_state(S, NP=40, seed=99)
    b.load(blob)
    for g in range(6, 11):
        a.de_step(g)
        b.de_step(g)
    ga, gb = a.get(), b.get()
    assert np.array_equal(ga["X"], gb["X"]) and np.array_equal(ga["fx"], gb["fx"])
    sa, sb = a.get_shade(), b.get_shade()
    assert np.array_equal(sa["MF"], sb["MF"]) and np.array_equal(sa["k"], sb["k"])
    assert a.result()["best"] == b.result()["best"]


# ---------------------------------------------------------------- CSO
@pytest.mark.parametrize("fam,D,NP", [(5, 13, 40), (7, 30, 64), (2, 200, 64)])
def test_cso_lockstep(S, fam, D, NP):
    """Five CSO generations in lock step with the oracle: the pairing and the
    winners / losers exactly, the losers' positions and velocities bit for
    bit (same fused multiply-adds, same index-order mean), the losers'
    fitness within the FP64 tolerance, winners untouched (D = 200 takes the
    large-D evaluation of the NP/2 loser rows)."""
    seed, phi = 31, 0.1
    p, q = S.Problem(500 + fam, fam, D), O.Problem(500 + fam, fam, D)
    st = S.State(p, S.alg_params(S.CSO, NP, 10 ** 6, w=phi), seed)
    X = O.init_population(seed, NP, D)
    fx = q.eval(X)
    V = np.zeros((NP, D))
    for gen in range(1, 6):
        st.set(X=X, fx=fx, V=V, fes=NP)
        assert st.pso_step(gen) == 0
        g = st.get()
        X2, V2, pair = O.cso_generation(seed, gen, X, V, fx, phi=phi)
        assert np.array_equal(g["part"][:, 0], pair)
        assert np.array_equal(g["X"], X2) and np.array_equal(g["V"], V2)
        los, win = pair[1::2], pair[0::2]
        want = q.eval(X2[los])
        assert (np.abs(g["fx"][los] - want) <= tol64(want, bound(p, q, X2[los]))).all()
        assert np.array_equal(g["fx"][win], fx[win])
        fx2 = fx.copy()
        fx2[los] = g["fx"][los]
        X, V, fx = X2, V2, fx2


def test_cso_full_run_and_grid(S):
    """CSO (NP = 100, phi = 0.1) on the shifted-rotated Griewank at D = 30
    reaches 1e-8 in 3e5 evaluations (NP/2 per generation) like the oracle's
    control run; a grid of CSO runs equals the same runs driven alone."""
    D, NP, budget = 30, 100, 300000
    p = S.Problem(3, S.GRIEWANK, D)
    a = S.alg_params(S.CSO, NP, budget, w=0.1)
    res = S.sevo_run_grid([p], [a], [(0, 0, s) for s in (1, 2)])
    assert res["success"].all(), res["best"]
    assert (res["gens"] == (budget - NP) // (NP // 2)).all() and (res["fes"] == budget).all()
    st = S.State(p, a, 2)
    g = 0
    while st.result()["fes"] < budget:
        g += 1
        st.pso_step(g)
    assert st.result()["best"] == res["best"][1] and st.result()["gens"] == res["gens"][1]


def test_cso_save_load_and_bad_population(S):
    p = S.Problem(9, S.RASTRIGIN, 12)
    with pytest.raises(S.SevoError):
        S.State(p, S.alg_params(S.CSO, 41, 1000, w=0.1), 1)  # odd swarm
    a = S.State(p, S.alg_params(S.CSO, 40, 10 ** 6, w=0.1), 4)
    for g in range(1, 4):
        a.pso_step(g)
    blob = a.save()
    b = S.State(p, S.alg_params(S.CSO, 40, 10 ** 6, w=0.1), 77)
    b.load(blob)
    for g in range(4, 8):
        a.pso_step(g)
        b.pso_step(g)
    ga, gb = a.get(), b.get()
    assert np.array_equal(ga["X"], gb["X"]) and np.array_equal(ga["V"], gb["V"])
    assert a.result()["best"] == b.result()["best"]


# ---------------------------------------------------------------- PSODE
@pytest.mark.parametrize("fam,D,NP", [(2, 13, 64), (0, 30, 40), (5, 20, 600), (1, 200, 64)])
def test_psode_lockstep(S, fam, D, NP):
    """Four PSODE generations in lock step with the oracle's operators: the
    PSO offspring bit-identical to the oracle's move (ring guides from the
    personal bests, carried velocity), personal bests updated from the GPU's
    fitness exactly as the oracle does, SHADE parameters, partners and
    trials as in the SHADE lock-step test, and the pairwise/3 selection and
    DE displacement bit-identical given the GPU's fitness; every fitness
    within the FP64 tolerance.  NP = 600 takes the radix-select ranking,
    D = 200 the large-D evaluation."""
    seed = 41
    p, q = S.Problem(600 + fam, fam, D), O.Problem(600 + fam, fam, D)
    st = S.State(p, S.alg_params(S.PSODE, NP, 10 ** 7), seed)
    X = O.init_population(seed, NP, D)
    fx = q.eval(X)
    V = np.random.default_rng(fam).uniform(-5, 5, (NP, D))
    P = X + np.random.default_rng(fam + 1).uniform(-1, 1, (NP, D))
    fp = q.eval(P)
    MF, MCR, k = O.shade_memory()
    for gen in range(1, 5):
        st.set(X=X, fx=fx, V=V, P=P, fp=fp, fes=NP)
        st.set_shade(MF, MCR, k)
        assert st.step(gen) == 0
        g, sh = st.get(), st.get_shade()
        assert g["U"].shape == (2 * NP, D)
        Y, _ = O.pso_move(seed, gen, X, V, P, O.pso_guides(fp, 1))
        assert np.array_equal(g["U"][:NP], Y)
        fy = g["fu"][:NP]
        want = q.eval(Y)
        assert (np.abs(fy - want) <= tol64(want, bound(p, q, Y))).all()
        P2, fp2, _ = O.pso_update(Y, fy, P, fp)
        assert np.array_equal(g["P"], P2) and np.array_equal(g["fp"], fp2)
        Fo, CRo, kpbo = O.shade_params(seed, gen, NP, MF, MCR)
        assert np.array_equal(sh["kpb"], kpbo)
        assert np.allclose(sh["F"], Fo, rtol=1e-13, atol=0)
        U, part = O.shade_trials(seed, gen, X, fx, sh["F"], sh["CR"], sh["kpb"])
        assert np.array_equal(g["part"], part) and np.array_equal(g["U"][NP:], U)
        fu = g["fu"][NP:]
        want = q.eval(U)
        assert (np.abs(fu - want) <= tol64(want, bound(p, q, U))).all()
        MFo, MCRo, ko, _ = O.shade_update(fx, fu, sh["F"], sh["CR"], MF, MCR, k)
        assert int(sh["k"][0]) == ko
        assert np.allclose(sh["MF"][0], MFo, rtol=1e-13, atol=0)
        X3, f3, _, _, _ = O.de_select(seed, gen, X, fx, U, fu)
        Xn, fn, Vn = O.psode_select(X, Y, fy, X3, f3)
        assert np.array_equal(g["X"], Xn) and np.array_equal(g["fx"], fn)
        assert np.array_equal(g["V"], Vn)
        X, fx, V, P, fp = Xn, fn, Vn, P2, fp2
        MF, MCR, k = sh["MF"][0], sh["MCR"][0], int(sh["k"][0])


def test_psode_budget_counts_pso_rows_first(S):
    """A budget ending inside a generation: the last generation counts its
    first PSO offspring only (budget - fes < NP) or all PSO offspring and
    the first DE trials; the best-so-far is the minimum over exactly the
    counted evaluations, fes stops at the budget, and a further step is
    refused."""
    NP, D = 24, 9
    p = S.Problem(8, S.ACKLEY, D)
    for extra in (NP // 2 + 1, NP + 7):
        budget = NP + 2 * NP * 2 + extra
        st = S.State(p, S.alg_params(S.PSODE, NP, budget), 5)
        counted = [st.get()["fx"]]
        for gen in range(1, 4):
            assert st.step(gen) == 0
            fe = st.get()["fu"]
            counted.append(fe if gen < 3 else fe[:extra])
        r = st.result()
        assert r["fes"] == budget and r["gens"] == 3
        assert r["best"] == min(float(np.min(c)) for c in counted)
        assert st.step(4) == S.ERR_STATE


def test_psode_full_run_and_grid(S):
    """PSODE (NP = 50) on the shifted-rotated Rosenbrock at D = 10 reaches
    1e-8 in 1e5 evaluations (2 NP per generation) like the oracle's control
    run; a grid of PSODE runs equals the same runs driven alone."""
    D, NP, budget = 10, 50, 100000
    p = S.Problem(3, S.ROSENBROCK, D)
    a = S.alg_params(S.PSODE, NP, budget)
    res = S.sevo_run_grid([p], [a], [(0, 0, s) for s in (1, 2)])
    assert res["success"].all(), res["best"]
    assert (res["gens"] == 1000).all() and (res["fes"] == budget).all()
    st = S.State(p, a, 2)
    g = 0
    while st.result()["fes"] < budget:
        g += 1
        st.step(g)
    assert st.result()["best"] == res["best"][1] and st.result()["gens"] == res["gens"][1]


def test_psode_save_load_and_step_kinds(S):
    """A saved PSODE state (population, velocity, personal bests, SHADE
    memory) resumes bit-identically; the DE-only and PSO-only step entries
    refuse a PSODE state."""
    p = S.Problem(9, S.RASTRIGIN, 12)
    a = S.State(p, S.alg_params(S.PSODE, 40, 10 ** 6), 4)
    assert a.de_step(1) == S.ERR_STATE and a.pso_step(1) == S.ERR_STATE
    for g in range(1, 4):
        assert a.step(g) == 0
    blob = a.save()
    b = S.State(p, S.alg_params(S.PSODE, 40, 10 ** 6), 77)
    b.load(blob)
    for g in range(4, 8):
        a.step(g)
        b.step(g)
    ga, gb = a.get(), b.get()
    for key in ("X", "fx", "V", "P", "fp"):
        assert np.array_equal(ga[key], gb[key]), key
    assert np.array_equal(a.get_shade()["MF"], b.get_shade()["MF"])
    assert a.result()["best"] == b.result()["best"]


@pytest.mark.parametrize("alg", ["DE_SHADE", "PSODE"])
def test_shade_kinds_at_largest_population(S, alg):
    """NP = 4096 (the largest population) needs more than the default 48 KB
    of shared memory for the p-best ranking: two generations run and the
    pools stay within 2 .. 0.2 NP."""
    NP, D = 4096, 8
    p = S.Problem(2, S.SCHWEFEL, D)
    st = S.State(p, S.alg_params(getattr(S, alg), NP, 10 ** 7), 3)
    for g in (1, 2):
        assert st.step(g) == 0
    sh = st.get_shade()
    assert sh["kpb"].min() >= 2 and sh["kpb"].max() <= round(0.2 * NP)
    assert np.isfinite(st.result()["best"])


def _group(S, D, NP, prec, algs, torch, fams=(0, 2, 3, 6, 7)):
    """One batched state per algorithm over the same problems, each on its
    own stream (as a caller overlapping them would)."""
    probs = [S.Problem(700 + f, f, D) for f in fams]
    out = []
    for k, alg in enumerate(algs):
        stream = torch.cuda.Stream()
        st = S.State(probs, S.alg_params(alg, NP, 10 ** 9, prec=prec),
                     [31 + 100 * k + r for r in range(len(probs))], stream=stream)
        st.torch_stream = stream
        out.append(st)
    return probs, out


@pytest.mark.parametrize("prec,D", [("TF32", 30), ("BF16X3", 100), ("FP64", 30), ("FP32", 30),
                                    ("TF32", 200)])
def test_step_many_equals_separate_steps(S, prec, D):
    """sevo_state_step_many over DE/rand/1, DE/current-to-pbest, SHADE,
    ring PSO and CSO states evaluates all their rows in one pass (one fused
    launch at D <= 128 in the tensor-core modes) and leaves every state
    bit-identical to stepping each with sevo_state_step, over 4 generations."""
    import torch
    algs = [S.DE_RAND1, S.DE_CTPB, S.DE_SHADE, S.PSO_RING, S.CSO]
    NP = 260
    _, A = _group(S, D, NP, getattr(S, prec), algs, torch)
    _, B = _group(S, D, NP, getattr(S, prec), algs, torch)
    for g in range(1, 5):
        assert S.sevo_state_step_many(A, g) == 0
        for st in B:
            assert st.step(g) == 0
    torch.cuda.synchronize()
    for a, b in zip(A, B):
        ga, gb = a.get(), b.get()
        for key in ("X", "fx", "U", "fu", "A", "V", "P", "fp", "part"):
            assert np.array_equal(ga[key], gb[key]), key
        assert ga["asize"] == gb["asize"]
        ra, rb = a.result(), b.result()
        assert ra["best"] == rb["best"] and ra["fes"] == rb["fes"] and ra["gens"] == 4
        assert ra["refined"] == rb["refined"]
        assert np.array_equal(a.best(), b.best())


def test_step_many_falls_back_and_checks_arguments(S):
    """With a PSODE state (two evaluations per generation) the states step
    one after another, with the same results; repeated states, an empty
    list and a spent budget are refused before anything is launched."""
    import torch
    D, NP = 20, 40
    algs = [S.DE_CTPB, S.PSODE]
    _, A = _group(S, D, NP, S.TF32, algs, torch, fams=(2, 4))
    _, B = _group(S, D, NP, S.TF32, algs, torch, fams=(2, 4))
    for g in range(1, 4):
        assert S.sevo_state_step_many(A, g) == 0
        for st in B:
            assert st.step(g) == 0
    for a, b in zip(A, B):
        ga, gb = a.get(), b.get()
        assert np.array_equal(ga["X"], gb["X"]) and np.array_equal(ga["fx"], gb["fx"])
    assert S.sevo_state_step_many([A[0], A[0]], 9) == S.ERR_ARG
    assert S.sevo_state_step_many([], 9) == S.ERR_ARG
    p = S.Problem(3, S.RASTRIGIN, D)
    done = S.State([p], S.alg_params(S.DE_RAND1, NP, NP + NP), [1])
    assert done.step(1) == 0  # budget now spent
    before = A[0].result()["gens"]
    assert S.sevo_state_step_many([A[0], done], 9) == S.ERR_STATE
    assert A[0].result()["gens"] == before


def test_grid_buckets_concurrent_on_caller_stream(S):
    """Buckets of several (algorithm, D) pairs run side by side on streams
    forked from the caller's: the grid started behind other work on a side
    stream gives the same results as on the current stream, and matches a
    run driven alone through the state API."""
    import torch
    probs = [S.Problem(11, S.RASTRIGIN, 10), S.Problem(12, S.HYBRID, 30),
             S.Problem(13, S.COMPOSITION, 10)]
    algs = [S.alg_params(S.DE_CTPB, 30, 1500, prec=S.TF32),
            S.alg_params(S.PSO_GBEST, 20, 1510, prec=S.TF32),
            S.alg_params(S.CSO, 20, 1200, prec=S.FP64)]
    tasks = [(pi, ai, 500 + 7 * pi + 31 * ai + k) for pi in range(3) for ai in range(3)
             for k in range(2)]
    ref = S.sevo_run_grid(probs, algs, tasks, gens_per_graph=4)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        big = torch.empty(1 << 26, device="cuda").uniform_()  # work queued before the grid
        res = S.sevo_run_grid(probs, algs, tasks, gens_per_graph=4, stream=side)
        after = big.sum()
    torch.cuda.synchronize()
    assert torch.isfinite(after)
    for key in ("best", "fes", "gens", "success"):
        assert np.array_equal(res[key], ref[key]), key
    assert res["wall_ms"] > 0 and res["evals"] == ref["evals"]
    t = 5
    pi, ai, seed = tasks[t]
    st = S.State(probs[pi], algs[ai], seed)
    gen = 0
    while st.result()["fes"] < algs[ai].budget:
        gen += 1
        st.step(gen)
    assert st.result()["best"] == res["best"][t]


@pytest.mark.parametrize("prec,D", [("TF32", 30), ("BF16X3", 17), ("TF32", 100), ("BF16X3", 128)])
def test_fused_operators_equal_operator_kernels(S, prec, D):
    """SEVO_POLICY_FUSE_OPS: the fused evaluation's producers form the DE
    trials and PSO moves themselves; every state (DE/rand/1,
    current-to-pbest with archive, SHADE, global and ring PSO; single,
    hybrid, composition and composition-of-hybrid problems, whose later
    components read the rows back) stays bit-identical to the run whose
    operators are kernels of their own, over 5 generations."""
    import torch
    lib = S.lib()
    algs = [S.DE_RAND1, S.DE_CTPB, S.DE_SHADE, S.PSO_GBEST, S.PSO_RING]
    NP = 150
    runs = {}
    old = lib.sevo_get_policy(S.POLICY_FUSE_OPS)
    for fuse in (1, 0):
        assert lib.sevo_set_policy(S.POLICY_FUSE_OPS, fuse) == 0
        try:
            _, sts = _group(S, D, NP, getattr(S, prec), algs, torch, fams=(1, 3, 6, 7, 8))
            for g in range(1, 6):
                for st in sts:
                    assert st.step(g) == 0
            runs[fuse] = [(st.get(), st.result(), st.best()) for st in sts]
        finally:
            lib.sevo_set_policy(S.POLICY_FUSE_OPS, old)
    for (ga, ra, ba), (gb, rb, bb) in zip(runs[1], runs[0]):
        for key in ("X", "fx", "U", "fu", "A", "V", "P", "fp", "part"):
            assert np.array_equal(ga[key], gb[key]), key
        assert ga["asize"] == gb["asize"]
        assert ra == rb and np.array_equal(ba, bb)


def test_bench_step_configuration_bit_exact(S):
    """The benchmark step as it is timed: two groups of DE/rand/1,
    DE/current-to-pbest and ring PSO states (3 runs x NP 4096 at D = 100 each,
    TF32, each state on its own stream; bench.make_states) advanced by one
    sevo_state_step_many per group (bench.run_steps).  Over two generations:
    every run's DE/rand/1 trials and partners and every run's PSO moves,
    velocities and guides equal the oracle's bit for bit; run 0 of each
    current-to-pbest state (the run whose archive the binding returns) has the
    oracle's partners, trials and selection; and 64 sampled rows of every state
    have the fitness of a plain TF32 sevo_evaluate of the same rows, bit for
    bit (that evaluation is compared with the oracle at this shape in
    test_bench_shape_sampled)."""
    import torch

    import bench
    seed0 = 7
    probs, states = bench.make_states(S, S.TF32, seed0, torch)
    NP, per = bench.NP, bench.FAMILIES // bench.GROUPS
    rng = np.random.default_rng(3)
    gen = 1
    for _ in range(2):
        torch.cuda.synchronize()
        before = [st.get() for st in states]
        gen_used = gen
        gen = bench.run_steps(states, gen, 1)
        torch.cuda.synchronize()
        for s, (st, g0) in enumerate(zip(states, before)):
            g = st.get()
            gi, k = s // len(bench.ALGS), s % len(bench.ALGS)
            alg = st.params.alg
            for r in range(st.R):
                seed = seed0 + 1000 * k + gi * per + r
                sl = slice(r * NP, (r + 1) * NP)
                if alg == S.DE_RAND1:
                    U, part = O.de_rand1_trials(seed, gen_used, g0["X"][sl])
                    assert np.array_equal(g["part"][sl], part), (s, r)
                    assert np.array_equal(g["U"][sl], U), (s, r)
                elif alg == S.PSO_RING:
                    guide = O.pso_guides(g0["fp"][sl], 1)
                    assert np.array_equal(g0["part"][sl][:, 0], guide), (s, r)
                    X2, V2 = O.pso_move(seed, gen_used, g0["X"][sl], g0["V"][sl], g0["P"][sl],
                                        guide)
                    assert np.array_equal(g["X"][sl], X2), (s, r)
                    assert np.array_equal(g["V"][sl], V2), (s, r)
                elif r == 0:
                    A0 = np.zeros((NP, bench.D))
                    A0[:g0["asize"]] = g0["A"]
                    U, part = O.de_ctpb_trials(seed, gen_used, g0["X"][sl], g0["fx"][sl], A0,
                                               g0["asize"])
                    assert np.array_equal(g["part"][sl], part), s
                    assert np.array_equal(g["U"][sl], U), s
                    X2, fx2, A2, as2, _ = O.de_select(seed, gen_used, g0["X"][sl], g0["fx"][sl],
                                                      U, g["fu"][sl], A0, g0["asize"])
                    assert g["asize"] == as2 and np.array_equal(g["A"], A2[:as2]), s
                    assert np.array_equal(g["X"][sl], X2) and np.array_equal(g["fx"][sl], fx2), s
            rows, fit = (g["X"], g["fx"]) if alg == S.PSO_RING else (g["U"], g["fu"])
            pick = np.sort(rng.choice(st.R * NP, 64, replace=False))
            for r in range(st.R):
                mine = pick[(pick >= r * NP) & (pick < (r + 1) * NP)]
                if len(mine) == 0:
                    continue
                Xr = torch.tensor(rows[mine], dtype=torch.float64, device="cuda")
                ref = probs[gi * per + r].evaluate(Xr, prec=S.TF32).cpu().numpy()
                assert np.array_equal(fit[mine].view(np.int64), ref.view(np.int64)), (s, r)
