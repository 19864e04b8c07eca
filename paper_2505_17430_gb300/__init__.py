"""Thin Python binding over the C ABI in include/sevo.h (libsevo.so).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch tensors are passed by device pointer; streams are the
current torch CUDA stream unless given.  The functions keep the C names
(sevo_problem_create, sevo_evaluate, sevo_de_step, sevo_pso_step,
sevo_run_grid, ...); the small classes below only own handles.

There is no CPU fallback: if libsevo.so is missing the import of the
library fails loudly (run ``build()`` first).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsevo.so")

ELLIPSOID, ROSENBROCK, RASTRIGIN, SCHWEFEL, ACKLEY, GRIEWANK, HYBRID, COMPOSITION = range(8)
COMP_HYBRID = 8  # composition whose components are hybrid functions
FAMILY_NAMES = ["ellipsoid", "rosenbrock", "rastrigin", "schwefel", "ackley", "griewank",
                "hybrid", "composition"]
FP64, TF32, BF16X3, FP32 = 0, 1, 2, 3
PREC_NAMES = {FP64: "fp64", TF32: "tf32", BF16X3: "bf16x3", FP32: "fp32"}
DE_RAND1, DE_CTPB, PSO_GBEST, PSO_RING, DE_SHADE, CSO, PSODE = 0, 1, 2, 3, 4, 5, 6
SHADE_H = 100
OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NAN, ERR_UNSUPPORTED, ERR_STATE = range(-1, -8, -1)
REFINE_THRESHOLD = 1e-4
SUCCESS_THRESHOLD = 1e-8


class SevoError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = _lib().sevo_strerror(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})")


class AlgParams(C.Structure):
    _fields_ = [("alg", C.c_int32), ("NP", C.c_int32), ("F", C.c_double), ("CR", C.c_double),
                ("p", C.c_double), ("w", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
                ("lb", C.c_double), ("ub", C.c_double), ("budget", C.c_int64),
                ("prec", C.c_int32)]


class Task(C.Structure):
    _fields_ = [("problem", C.c_int32), ("alg", C.c_int32), ("seed", C.c_uint64)]


class Grid(C.Structure):
    _fields_ = [("nproblems", C.c_int32), ("problems", C.POINTER(C.c_void_p)),
                ("nalgs", C.c_int32), ("algs", C.POINTER(AlgParams)),
                ("ntasks", C.c_int32), ("tasks", C.POINTER(Task)),
                ("gens_per_graph", C.c_int32)]


class GridResult(C.Structure):
    _fields_ = [("best", C.POINTER(C.c_double)), ("fes", C.POINTER(C.c_int64)),
                ("gens", C.POINTER(C.c_int64)), ("success", C.POINTER(C.c_int32)),
                ("wall_ms", C.c_double), ("evals", C.c_int64)]


# every symbol include/sevo.h declares, with its ctypes signature
_vp, _dp, _ip, _i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
SIGNATURES = {
    "sevo_strerror": (C.c_char_p, [C.c_int32]),
    "sevo_version": (C.c_int32, []),
    "sevo_kernel_launches": (C.c_int64, []),
    "sevo_last_cuda_error": (C.c_char_p, []),
    "sevo_state_create_batch": (C.c_int32, [C.POINTER(_vp), C.c_int32, C.POINTER(AlgParams),
                                            C.POINTER(C.c_uint64), _vp, C.POINTER(_vp)]),
    "sevo_state_best": (C.c_int32, [_vp, _dp]),
    "sevo_problem_create": (C.c_int32, [C.c_uint64, C.c_int32, C.c_int32, C.POINTER(_vp)]),
    "sevo_hybrid_create": (C.c_int32, [C.c_uint64, C.c_int32, C.c_int32, _dp, _ip,
                                       C.POINTER(_vp)]),
    "sevo_problem_destroy": (C.c_int32, [_vp]),
    "sevo_problem_info": (C.c_int32, [_vp, _ip, _ip, _ip, _dp]),
    "sevo_problem_export": (C.c_int32, [_vp, C.c_int32, _dp, _dp, _ip, _ip, _ip, _dp, _dp, _dp]),
    "sevo_evaluate": (C.c_int32, [_vp, _vp, C.c_int64, C.c_int32, C.c_int64, _vp, C.c_int32, _vp]),
    "sevo_evaluate_sync": (C.c_int32, [_vp, _vp, C.c_int64, C.c_int32, C.c_int64, _vp, C.c_int32,
                                       _vp, _i64p, _i64p]),
    "sevo_evaluate_noalloc": (C.c_int32, [_vp, _vp, C.c_int64, C.c_int32, C.c_int64, _vp,
                                          C.c_int32, _vp]),
    "sevo_state_create": (C.c_int32, [_vp, C.POINTER(AlgParams), C.c_uint64, _vp,
                                      C.POINTER(_vp)]),
    "sevo_state_destroy": (C.c_int32, [_vp]),
    "sevo_state_restart": (C.c_int32, [_vp, C.POINTER(C.c_uint64)]),
    "sevo_state_get_shade": (C.c_int32, [_vp, _dp, _dp, _ip, _dp, _dp, _ip]),
    "sevo_state_set_shade": (C.c_int32, [_vp, _dp, _dp, _ip]),
    "sevo_de_step": (C.c_int32, [_vp, C.c_uint64]),
    "sevo_pso_step": (C.c_int32, [_vp, C.c_uint64]),
    "sevo_state_step": (C.c_int32, [_vp, C.c_uint64]),
    "sevo_state_step_many": (C.c_int32, [C.POINTER(_vp), C.c_int32, C.c_uint64]),
    "sevo_state_result": (C.c_int32, [_vp, _dp, _i64p, _i64p, _i64p]),
    "sevo_state_get": (C.c_int32, [_vp, _dp, _dp, _dp, _ip, _dp, _dp, _dp, _dp, _dp, _ip]),
    "sevo_state_set": (C.c_int32, [_vp, _dp, _dp, _dp, C.c_int32, _dp, _dp, _dp, C.c_int64]),
    "sevo_state_set_async": (C.c_int32, [_vp, _dp, _dp, _dp, C.c_int32, _dp, _dp, _dp,
                                         C.c_int64]),
    "sevo_state_get_async": (C.c_int32, [_vp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
    "sevo_state_save": (C.c_int32, [_vp, _vp, C.POINTER(C.c_size_t)]),
    "sevo_state_load": (C.c_int32, [_vp, _vp, C.c_size_t]),
    "sevo_run_grid": (C.c_int32, [C.POINTER(Grid), C.POINTER(GridResult), _vp]),
    "sevo_set_policy": (C.c_int32, [C.c_int32, C.c_int64]),
    "sevo_get_policy": (C.c_int64, [C.c_int32]),
    "sevo_trace_enable": (C.c_int32, [C.c_int32]),
    "sevo_trace_read": (C.c_int32, [_i64p, _dp]),
    "sevo_trace_name": (C.c_char_p, [C.c_int32]),
    "sevo_trace_timeline": (C.c_int64, [C.c_int64, _ip, _ip, _dp, _dp]),
}
SEVO_TRACE_KINDS = 17
POLICY_SMALL_RUNS = 0
POLICY_REFINE = 1
POLICY_TEST_WAIT = 2
POLICY_FUSE_OPS = 3
POLICY_AUTOTUNE = 4

_LIB = None


def build(force: bool = False) -> str:
    """Compile libsevo.so for sm_103a (nvcc; see buildlib.py)."""
    import importlib
    _b = importlib.import_module(__name__ + ".buildlib")
    return _b.build(force=force)


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsevo.so not built ({LIB_PATH}); call "
                              "paper_2505_17430_gb300.build() first -- there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def lib():
    return _lib()


def check(status, what=""):
    if status != OK:
        if status == ERR_CUDA:
            cuda = _lib().sevo_last_cuda_error().decode()
            what = f"{what} ({cuda})" if cuda else what
        raise SevoError(status, what)
    return status


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _np_dp(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _np_ip(a):
    return a.ctypes.data_as(_ip) if a is not None else None


# ---------------------------------------------------------------- problems
class Problem:
    """Owns a sevo_problem handle (seeded instance on the current device)."""

    def __init__(self, seed: int, family: int, D: int, hybrid=None):
        import numpy as np
        h = C.c_void_p()
        if hybrid is not None:
            frac, bodies = hybrid
            fr = np.ascontiguousarray(frac, dtype=np.float64)
            bd = np.ascontiguousarray(bodies, dtype=np.int32)
            check(_lib().sevo_hybrid_create(seed, D, len(bd), _np_dp(fr), _np_ip(bd), C.byref(h)),
                  "sevo_hybrid_create")
        else:
            check(_lib().sevo_problem_create(seed, family, D, C.byref(h)), "sevo_problem_create")
        self.h = h
        fam, d, nc, fs = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        check(_lib().sevo_problem_info(h, C.byref(fam), C.byref(d), C.byref(nc), C.byref(fs)),
              "sevo_problem_info")
        self.family, self.D, self.K, self.fstar = fam.value, d.value, nc.value, fs.value

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _LIB is not None:
            _LIB.sevo_problem_destroy(h)
            self.h = None

    @property
    def ncomp(self):
        return self.K if self.family in (COMPOSITION, COMP_HYBRID) else 1

    def export(self, comp=0):
        import numpy as np
        D, K = self.D, max(self.K, 1)
        o, M = np.zeros(D), np.zeros((D, D))
        G = max(K, 8)  # groups of a hybrid component can exceed the component count
        perm, gs, gb = np.zeros(D, np.int32), np.zeros(G, np.int32), np.zeros(G, np.int32)
        sg, lam, bias = np.zeros(K), np.zeros(K), np.zeros(K)
        check(_lib().sevo_problem_export(self.h, comp, _np_dp(o), _np_dp(M), _np_ip(perm),
                                         _np_ip(gs), _np_ip(gb), _np_dp(sg), _np_dp(lam),
                                         _np_dp(bias)), "sevo_problem_export")
        return {"o": o, "M": M, "perm": perm, "gsize": gs, "gbody": gb, "sigma": sg,
                "lambda": lam, "bias": bias}

    def evaluate(self, pop, out=None, prec=FP64, stream=None, sync=False):
        """out[i] = f(pop_i) - f*  (pop: CUDA float64 tensor N x D, row-major)."""
        import torch
        assert pop.is_cuda and pop.dtype == torch.float64 and pop.dim() == 2
        assert pop.stride(1) == 1
        N = pop.shape[0]
        if out is None:
            out = torch.empty(N, dtype=torch.float64, device=pop.device)
        args = (self.h, C.c_void_p(pop.data_ptr()), N, self.D, pop.stride(0),
                C.c_void_p(out.data_ptr()), prec, _stream_ptr(stream))
        if sync:
            r, n = C.c_int64(), C.c_int64()
            st = _lib().sevo_evaluate_sync(*args, C.byref(r), C.byref(n))
            if st not in (OK, -5):
                check(st, "sevo_evaluate_sync")
            return out, {"refined": r.value, "nonfinite": n.value, "status": st}
        check(_lib().sevo_evaluate(*args), "sevo_evaluate")
        return out


def sevo_problem_create(seed, family, D):
    return Problem(seed, family, D)


def sevo_evaluate(problem, pop, out=None, prec=FP64, stream=None):
    return problem.evaluate(pop, out, prec, stream)


# ---------------------------------------------------------------- runs
def alg_params(alg, NP, budget, F=0.5, CR=0.9, p=0.11, w=0.7298, c1=1.49618, c2=1.49618,
               lb=-100.0, ub=100.0, prec=FP64):
    return AlgParams(alg, NP, F, CR, p, w, c1, c2, lb, ub, int(budget), prec)


class State:
    """Owns a sevo_state handle: one run's device state, or R runs of one
    algorithm (problems = list, seeds = list) stepping together."""

    def __init__(self, problem, params: AlgParams, seed, stream=None):
        h = C.c_void_p()
        self.params = params
        if isinstance(problem, (list, tuple)):
            self.problems = list(problem)  # keep alive
            self.problem = self.problems[0]
            self.R = len(self.problems)
            ph = (C.c_void_p * self.R)(*[p.h.value for p in self.problems])
            sd = (C.c_uint64 * self.R)(*[int(x) for x in seed])
            check(_lib().sevo_state_create_batch(ph, self.R, C.byref(params), sd,
                                                 _stream_ptr(stream), C.byref(h)),
                  "sevo_state_create_batch")
        else:
            self.problems = [problem]
            self.problem = problem
            self.R = 1
            check(_lib().sevo_state_create(problem.h, C.byref(params), seed, _stream_ptr(stream),
                                           C.byref(h)), "sevo_state_create")
        self.h = h

    def best(self):
        import numpy as np
        b = np.zeros(self.R)
        check(_lib().sevo_state_best(self.h, _np_dp(b)), "sevo_state_best")
        return b

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _LIB is not None:
            _LIB.sevo_state_destroy(h)
            self.h = None

    def get_shade(self):
        """SHADE memory and the last generation's per-row parameters."""
        import numpy as np
        R, NP = self.R, self.params.NP
        MF, MCR = np.zeros((R, SHADE_H)), np.zeros((R, SHADE_H))
        k = np.zeros(R, np.int32)
        F, CR, kpb = np.zeros(R * NP), np.zeros(R * NP), np.zeros(R * NP, np.int32)
        check(_lib().sevo_state_get_shade(self.h, _np_dp(MF), _np_dp(MCR), _np_ip(k), _np_dp(F),
                                          _np_dp(CR), _np_ip(kpb)), "sevo_state_get_shade")
        return {"MF": MF, "MCR": MCR, "k": k, "F": F, "CR": CR, "kpb": kpb}

    def set_shade(self, MF=None, MCR=None, k=None):
        import numpy as np
        c = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        kk = None if k is None else np.ascontiguousarray(np.atleast_1d(k), dtype=np.int32)
        check(_lib().sevo_state_set_shade(self.h, _np_dp(c(MF)), _np_dp(c(MCR)), _np_ip(kk)),
              "sevo_state_set_shade")

    def restart(self, seeds):
        """Fresh initial populations for every run (seeds: one per run)."""
        seeds = [seeds] if isinstance(seeds, int) else list(seeds)
        if len(seeds) != self.R:
            raise ValueError("one seed per run")
        sd = (C.c_uint64 * self.R)(*[int(x) for x in seeds])
        check(_lib().sevo_state_restart(self.h, sd), "sevo_state_restart")

    def de_step(self, counter):
        return _lib().sevo_de_step(self.h, counter)

    def pso_step(self, counter):
        return _lib().sevo_pso_step(self.h, counter)

    def step(self, counter):
        """One generation of whatever algorithm the state runs."""
        return _lib().sevo_state_step(self.h, counter)

    def result(self):
        b, f, g, r = C.c_double(), C.c_int64(), C.c_int64(), C.c_int64()
        check(_lib().sevo_state_result(self.h, C.byref(b), C.byref(f), C.byref(g), C.byref(r)),
              "sevo_state_result")
        return {"best": b.value, "fes": f.value, "gens": g.value, "refined": r.value}

    def get(self):
        import numpy as np
        NP, D = self.params.NP * self.R, self.problem.D
        X, fx, A = np.zeros((NP, D)), np.zeros(NP), np.zeros((NP, D))
        V, P, fp = np.zeros((NP, D)), np.zeros((NP, D)), np.zeros(NP)
        ne = 2 * NP if self.params.alg == PSODE else NP  # evaluated rows per generation
        U, fu, part = np.zeros((ne, D)), np.zeros(ne), np.zeros((NP, 4), np.int32)
        asz = C.c_int32()
        check(_lib().sevo_state_get(self.h, _np_dp(X), _np_dp(fx), _np_dp(A), C.byref(asz),
                                    _np_dp(V), _np_dp(P), _np_dp(fp), _np_dp(U), _np_dp(fu),
                                    _np_ip(part)), "sevo_state_get")
        return {"X": X, "fx": fx, "A": A[:asz.value], "asize": asz.value, "V": V, "P": P,
                "fp": fp, "U": U, "fu": fu, "part": part}

    def set(self, X=None, fx=None, A=None, asize=0, V=None, P=None, fp=None, fes=-1):
        import numpy as np
        c = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        X, fx, V, P, fp = c(X), c(fx), c(V), c(P), c(fp)
        Af = None
        if A is not None:
            Af = np.zeros((self.params.NP * self.R, self.problem.D))
            Af[:len(A)] = A
        check(_lib().sevo_state_set(self.h, _np_dp(X), _np_dp(fx), _np_dp(Af), asize, _np_dp(V),
                                    _np_dp(P), _np_dp(fp), fes), "sevo_state_set")

    def save(self) -> bytes:
        n = C.c_size_t(0)
        check(_lib().sevo_state_save(self.h, None, C.byref(n)), "sevo_state_save")
        buf = C.create_string_buffer(n.value)
        check(_lib().sevo_state_save(self.h, buf, C.byref(n)), "sevo_state_save")
        return buf.raw[:n.value]

    def load(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        check(_lib().sevo_state_load(self.h, buf, len(data)), "sevo_state_load")


def sevo_state_step_many(states, counter):
    """One generation of every state in `states`, their rows evaluated in
    one pass (sevo_state_step_many); returns the status."""
    hs = (_vp * len(states))(*[st.h.value for st in states])
    return _lib().sevo_state_step_many(hs, len(states), counter)


STEP_MANY_MAX = 16


def sevo_state_create(problem, params, seed, stream=None):
    return State(problem, params, seed, stream)


def sevo_run_grid(problems, algs, tasks, gens_per_graph=0, stream=None):
    """Run a grid of tasks [(problem index, alg index, seed)] to their budgets."""
    import numpy as np
    n = len(tasks)
    ph = (C.c_void_p * len(problems))(*[p.h.value for p in problems])
    aa = (AlgParams * len(algs))(*algs)
    tt = (Task * n)(*[Task(int(a), int(b), int(s)) for a, b, s in tasks])
    best, fes, gens = np.zeros(n), np.zeros(n, np.int64), np.zeros(n, np.int64)
    succ = np.zeros(n, np.int32)
    g = Grid(len(problems), C.cast(ph, C.POINTER(C.c_void_p)), len(algs),
             C.cast(aa, C.POINTER(AlgParams)), n, C.cast(tt, C.POINTER(Task)), gens_per_graph)
    r = GridResult(_np_dp(best), fes.ctypes.data_as(_i64p),
                   gens.ctypes.data_as(_i64p), succ.ctypes.data_as(_ip), 0.0, 0)
    check(_lib().sevo_run_grid(C.byref(g), C.byref(r), _stream_ptr(stream)), "sevo_run_grid")
    return {"best": best, "fes": fes, "gens": gens, "success": succ.astype(bool),
            "wall_ms": r.wall_ms, "evals": r.evals}


def trace_enable(on=True, timeline=False):
    """Start (clearing the totals; timeline: also keep every launch's span)
    or stop per-kernel event tracing."""
    check(_lib().sevo_trace_enable((2 if timeline else 1) if on else 0), "sevo_trace_enable")


def trace_timeline():
    """The launches traced with timeline=True: a list of (kind name, stream
    id, start ms, end ms), sorted by start."""
    import numpy as np
    n = _lib().sevo_trace_timeline(0, None, None, None, None)
    check(n if n < 0 else 0, "sevo_trace_timeline")
    kinds, streams = np.zeros(n, np.int32), np.zeros(n, np.int32)
    t0, t1 = np.zeros(n), np.zeros(n)
    m = _lib().sevo_trace_timeline(n, kinds.ctypes.data_as(_ip), streams.ctypes.data_as(_ip),
                                   _np_dp(t0), _np_dp(t1))
    check(m if m < 0 else 0, "sevo_trace_timeline")
    m = min(n, m)
    names = [_lib().sevo_trace_name(k).decode() for k in range(SEVO_TRACE_KINDS)]
    return [(names[kinds[i]], int(streams[i]), float(t0[i]), float(t1[i])) for i in range(m)]


def trace_read():
    """{kernel kind: (launches, device ms)} of the traced launches so far."""
    counts = (C.c_int64 * SEVO_TRACE_KINDS)()
    ms = (C.c_double * SEVO_TRACE_KINDS)()
    check(_lib().sevo_trace_read(counts, ms), "sevo_trace_read")
    return {_lib().sevo_trace_name(k).decode(): (counts[k], ms[k])
            for k in range(SEVO_TRACE_KINDS)}
