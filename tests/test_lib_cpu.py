"""Host-side checks of the product library (no GPU): it builds and loads,
exports every entry point include/sevo.h declares, validates arguments, and
its host-side instance generation agrees with the oracle's."""
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2505_17430_gb300 as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    S.build()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "sevo.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sevo_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    names = header_functions()
    assert "sevo_evaluate" in names and "sevo_run_grid" in names and len(names) >= 18
    lib = S.lib()
    for n in names:
        assert hasattr(lib, n), n
        assert n in S.SIGNATURES, f"binding lacks {n}"


def test_strerror_and_version():
    lib = S.lib()
    assert lib.sevo_version() >= 100
    for code in range(0, -8, -1):
        assert len(lib.sevo_strerror(code)) > 0


def test_argument_validation_without_device():
    import ctypes as C
    h = C.c_void_p()
    lib = S.lib()
    assert lib.sevo_problem_create(1, 99, 10, C.byref(h)) == -1
    assert lib.sevo_problem_create(1, 0, 1, C.byref(h)) == -1
    assert lib.sevo_problem_create(1, 0, 5001, C.byref(h)) == -1
    assert lib.sevo_problem_create(1, 0, 10, None) == -1
    assert lib.sevo_evaluate(None, None, 1, 10, 10, None, 0, None) == -1
    assert lib.sevo_problem_destroy(None) == -1


@pytest.mark.parametrize("fam", range(8))
@pytest.mark.parametrize("D", [2, 10, 100])
def test_host_instances_match_oracle(fam, D):
    """Shift, permutation, groups and composition parameters bit-exact (same
    Philox definition, same IEEE expressions); rotation to FP64 round-off
    (different QR algorithms: Householder in the oracle, Gram-Schmidt twice
    in the library)."""
    seed = 0x5EB00000 + 31 * fam + D
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    assert p.K == (q.K if fam >= 6 else 1)
    for c in range(q.ncomp):
        e = p.export(c)
        assert np.array_equal(e["o"], q.shift(c))
        assert np.abs(e["M"] - q.rotation(c)).max() < 1e-12
    if fam == 6:
        perm, gs, gb = q.hybrid()
        e = p.export()
        assert np.array_equal(e["perm"], perm)
        assert np.array_equal(e["gsize"][:q.K], gs) and np.array_equal(e["gbody"][:q.K], gb)
    if fam == 7:
        b, s, lam, bias = q.comp()
        e = p.export()
        for k, v in (("gbody", b), ("sigma", s), ("lambda", lam), ("bias", bias)):
            assert np.array_equal(e[k][:q.K], v), k


def test_fixed_hybrid_matches_oracle():
    p = S.Problem(5, S.HYBRID, 100, hybrid=([0.3, 0.3, 0.4], [2, 0, 3]))
    q = O.Problem(5, O.HYBRID, 100, hybrid=([0.3, 0.3, 0.4], [2, 0, 3]))
    e = p.export()
    assert list(e["gsize"][:3]) == [30, 30, 40]
    assert np.array_equal(e["perm"], q.hybrid()[0])


def test_large_rotation_orthogonal():
    p = S.Problem(1, S.ELLIPSOID, 500)
    M = p.export()["M"]
    assert np.abs(M.T @ M - np.eye(500)).max() < 1e-13


def test_trace_kinds_match_header_and_read_without_gpu():
    """The tracing kinds enumerated in the header match the binding's count,
    every kind has a distinct name, and enabling / reading with nothing
    traced touches no device."""
    txt = open(os.path.join(ROOT, "include", "sevo.h")).read()
    body = txt[txt.index("enum sevo_trace_kind"):txt.index("SEVO_TRACE_KINDS")]
    kinds = re.findall(r"\b(SEVO_TK_[A-Z_]+)", body)
    assert len(kinds) == S.SEVO_TRACE_KINDS
    lib = S.lib()
    names = [lib.sevo_trace_name(k).decode() for k in range(S.SEVO_TRACE_KINDS)]
    assert all(names) and len(set(names)) == len(names)
    assert lib.sevo_trace_name(S.SEVO_TRACE_KINDS) == b""
    assert lib.sevo_trace_name(-1) == b""
    S.trace_enable(True, timeline=True)
    t = S.trace_read()
    assert S.trace_timeline() == []
    S.trace_enable(False)
    assert set(t) == set(names) and all(v == (0, 0.0) for v in t.values())
    assert lib.sevo_trace_enable(3) == S.ERR_ARG
    assert lib.sevo_trace_timeline(-1, None, None, None, None) == S.ERR_ARG
    assert lib.sevo_trace_timeline(4, None, None, None, None) == S.ERR_ARG


def test_last_cuda_error_empty_before_any_failure():
    assert S.lib().sevo_last_cuda_error() == b""


def test_status_constants_match_header():
    txt = open(os.path.join(ROOT, "include", "sevo.h")).read()
    for name in ("ARG", "CUDA", "OOM", "TIMEOUT", "NAN", "UNSUPPORTED", "STATE"):
        m = re.search(r"#define SEVO_ERR_%s\s+(-?\d+)" % name, txt)
        assert m and int(m.group(1)) == getattr(S, "ERR_" + name), name
    with pytest.raises(S.SevoError) as ei:
        S.check(S.ERR_ARG, "probe")
    assert ei.value.status == S.ERR_ARG


@pytest.mark.parametrize("D", [11, 40])
def test_comp_hybrid_generation_matches_oracle(D):
    """The library's host-side generation of a composition of hybrids draws
    the same instance as the oracle: per component the shift, the permuted
    rotation (to round-off: the two sides' QR differ), the permutation, the
    group sizes and bodies, and sigma, lambda, bias."""
    seed = 0xC0FFEE + D
    p, q = S.Problem(seed, S.COMP_HYBRID, D), O.Problem(seed, O.COMP_HYBRID, D)
    assert p.K == q.K
    _, sig, lam, bias = q.comp()
    for c in range(q.K):
        e = p.export(c)
        perm, gs, gb = q.comp_hybrid(c)
        assert np.array_equal(e["o"], q.shift(c))
        assert np.abs(e["M"] - q.rotation(c)).max() < 1e-12
        assert np.array_equal(e["perm"], perm)
        assert np.array_equal(e["gsize"][:len(gs)], gs) and np.array_equal(e["gbody"][:len(gb)], gb)
        assert np.array_equal(e["sigma"], sig) and np.array_equal(e["lambda"], lam)
        assert np.array_equal(e["bias"], bias)


def _grid_status(p, a):
    """sevo_run_grid's status for one task of algorithm a on problem p
    (called directly, default stream, no device needed to be refused)."""
    import ctypes as C
    ph = (C.c_void_p * 1)(p.h.value)
    aa = (S.AlgParams * 1)(a)
    tt = (S.Task * 1)(S.Task(0, 0, 1))
    best, fes, gens = np.zeros(1), np.zeros(1, np.int64), np.zeros(1, np.int64)
    succ = np.zeros(1, np.int32)
    g = S.Grid(1, C.cast(ph, C.POINTER(C.c_void_p)), 1, C.cast(aa, C.POINTER(S.AlgParams)), 1,
               C.cast(tt, C.POINTER(S.Task)), 0)
    i64 = C.POINTER(C.c_int64)
    r = S.GridResult(best.ctypes.data_as(C.POINTER(C.c_double)), fes.ctypes.data_as(i64),
                     gens.ctypes.data_as(i64), succ.ctypes.data_as(C.POINTER(C.c_int32)), 0.0, 0)
    return S.lib().sevo_run_grid(C.byref(g), C.byref(r), None)


def test_algorithm_parameter_validation_without_device():
    """Every algorithm's parameters are checked before any device work: the
    state, the grid and the step entries refuse what the header rules out
    (unknown algorithm, PSODE and the DE kinds below NP = 4, CSO with an odd
    swarm, empty bounds) with SEVO_ERR_ARG, and a null state with
    SEVO_ERR_ARG from every step entry."""
    import ctypes as C
    lib = S.lib()
    p = S.Problem(3, S.RASTRIGIN, 10)
    bad = [S.alg_params(7, 40, 1000), S.alg_params(-1, 40, 1000),
           S.alg_params(S.PSODE, 3, 1000), S.alg_params(S.DE_SHADE, 3, 1000),
           S.alg_params(S.CSO, 41, 1000), S.alg_params(S.PSODE, 40, 0),
           S.alg_params(S.PSODE, 40, 1000, lb=5.0, ub=5.0)]
    for a in bad:
        out = C.c_void_p()
        assert lib.sevo_state_create(p.h, C.byref(a), 1, None, C.byref(out)) == S.ERR_ARG
        assert not out.value
        assert _grid_status(p, a) == S.ERR_ARG
    for step in (lib.sevo_state_step, lib.sevo_de_step, lib.sevo_pso_step):
        assert step(None, 1) == S.ERR_ARG
    assert lib.sevo_state_get_shade(None, None, None, None, None, None, None) == S.ERR_ARG


def test_enum_constants_match_header_and_oracle():
    """The binding's family, precision and algorithm numbers are the header's
    enums, and the oracle (written independently) numbers families and
    algorithms the same way."""
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sevo.h")).read(), flags=re.S)
    enum = {m.group(1): int(m.group(2)) for m in re.finditer(r"\bSEVO_([A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    fam = {"ELLIPSOID": S.ELLIPSOID, "ROSENBROCK": S.ROSENBROCK, "RASTRIGIN": S.RASTRIGIN,
           "SCHWEFEL": S.SCHWEFEL, "ACKLEY": S.ACKLEY, "GRIEWANK": S.GRIEWANK,
           "HYBRID": S.HYBRID, "COMPOSITION": S.COMPOSITION, "COMP_HYBRID": S.COMP_HYBRID}
    alg = {"DE_RAND1": S.DE_RAND1, "DE_CTPB": S.DE_CTPB, "PSO_GBEST": S.PSO_GBEST,
           "PSO_RING": S.PSO_RING, "DE_SHADE": S.DE_SHADE, "CSO": S.CSO, "PSODE": S.PSODE}
    prec = {"FP64": S.FP64, "TF32": S.TF32, "BF16X3": S.BF16X3, "FP32": S.FP32}
    for table in (fam, alg, prec):
        for name, v in table.items():
            assert enum.get(name) == v, name
    assert [O.ELLIPSOID, O.ROSENBROCK, O.RASTRIGIN, O.SCHWEFEL, O.ACKLEY, O.GRIEWANK, O.HYBRID,
            O.COMPOSITION, O.COMP_HYBRID] == [fam[k] for k in fam]
    assert [O.ALG_DE_RAND1, O.ALG_DE_CTPB, O.ALG_PSO_GBEST, O.ALG_PSO_RING, O.ALG_DE_SHADE,
            O.ALG_CSO, O.ALG_PSODE] == [alg[k] for k in alg]
