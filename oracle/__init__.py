"""Plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

ctypes wrapper over ``oracle/sevo_oracle.c``.  Only the tests, the smoke check
and the benchmark's CPU-baseline leg may import this package; the product
package never does.  The C source is the statement of what the GPU path
computes (see the header comment of ``sevo_oracle.h`` for what each function
follows in arXiv 2505.17430).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = [os.path.join(HERE, "sevo_oracle.c")]

ELLIPSOID, ROSENBROCK, RASTRIGIN, SCHWEFEL, ACKLEY, GRIEWANK, HYBRID, COMPOSITION = range(8)
COMP_HYBRID = 8  # composition whose components are hybrids
P_INIT, P_PART, P_CROSS, P_ARCH, P_PSO = 1, 2, 3, 4, 5

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, -ffp-contract=off)."""
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SRC + [os.path.join(HERE, "sevo_oracle.h")])
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-D_GNU_SOURCE", *SRC, "-o", tmp, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


class Alg(C.Structure):
    _fields_ = [("alg", C.c_int), ("NP", C.c_int), ("F", C.c_double), ("CR", C.c_double),
                ("p", C.c_double), ("w", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
                ("lb", C.c_double), ("ub", C.c_double), ("budget", C.c_int64)]


class Result(C.Structure):
    _fields_ = [("best", C.c_double), ("fes", C.c_int64), ("gens", C.c_int64),
                ("success", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, ip, u8p = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_uint8)
            vp = C.c_void_p
            sig = {
                "orc_philox": (None, [C.c_uint32] * 6 + [C.POINTER(C.c_uint32)]),
                "orc_u53": (C.c_double, [C.c_uint32, C.c_uint32]),
                "orc_below": (C.c_uint32, [C.c_uint32, C.c_uint32]),
                "orc_problem_create": (vp, [C.c_uint64, C.c_int, C.c_int]),
                "orc_hybrid_create": (vp, [C.c_uint64, C.c_int, C.c_int, dp, ip]),
                "orc_problem_destroy": (None, [vp]),
                "orc_problem_info": (None, [vp, ip, dp]),
                "orc_problem_get": (C.c_int, [vp, C.c_int, dp, dp]),
                "orc_problem_hybrid": (C.c_int, [vp, ip, ip, ip]),
                "orc_problem_comp": (C.c_int, [vp, ip, dp, dp, dp]),
                "orc_problem_comp_hybrid": (C.c_int, [vp, C.c_int, ip, ip, ip]),
                "orc_eval": (C.c_double, [vp, dp]),
                "orc_eval_batch": (None, [vp, dp, C.c_int64, C.c_int64, dp]),
                "orc_eval_bound": (None, [vp, dp, dp]),
                "orc_eval_bound_batch": (None, [vp, dp, C.c_int64, C.c_int64, dp]),
                "orc_body": (C.c_double, [C.c_int, dp, C.c_int]),
                "orc_transform": (None, [vp, C.c_int, dp, dp]),
                "orc_init_population": (None, [C.c_uint64, C.c_int, C.c_int, C.c_double,
                                               C.c_double, dp]),
                "orc_de_rand1_trials": (None, [C.c_uint64, C.c_uint64, dp, C.c_int, C.c_int,
                                               C.c_double, C.c_double, C.c_double, C.c_double,
                                               dp, ip]),
                "orc_pbest_k": (C.c_int, [C.c_double, C.c_int]),
                "orc_rank": (None, [dp, C.c_int, ip]),
                "orc_de_ctpb_trials": (None, [C.c_uint64, C.c_uint64, dp, dp, C.c_int, C.c_int,
                                              C.c_double, C.c_double, C.c_double, dp, C.c_int,
                                              C.c_double, C.c_double, dp, ip]),
                "orc_de_select": (C.c_int, [C.c_uint64, C.c_uint64, dp, dp, dp, dp, C.c_int,
                                            C.c_int, dp, ip, u8p]),
                "orc_shade_params": (None, [C.c_uint64, C.c_uint64, C.c_int, C.c_int, dp, dp,
                                            dp, dp, ip]),
                "orc_shade_kmax": (C.c_int, [C.c_int]),
                "orc_shade_trials": (None, [C.c_uint64, C.c_uint64, dp, dp, C.c_int, C.c_int,
                                            dp, dp, ip, C.c_double, C.c_double, dp, ip]),
                "orc_shade_update": (C.c_int, [C.c_int, C.c_int, dp, dp, dp, dp, dp, dp, ip]),
                "orc_cso_generation": (None, [C.c_uint64, C.c_uint64, dp, dp, dp, C.c_int,
                                              C.c_int, C.c_double, C.c_double, C.c_double, ip]),
                "orc_pso_guides": (None, [dp, C.c_int, C.c_int, ip]),
                "orc_pso_move": (None, [C.c_uint64, C.c_uint64, dp, dp, dp, ip, C.c_int,
                                        C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_double]),
                "orc_pso_update": (C.c_int, [dp, dp, dp, dp, C.c_int, C.c_int]),
                "orc_psode_select": (None, [dp, dp, dp, dp, dp, C.c_int, C.c_int, dp, dp, dp]),
                "orc_psode_generation": (None, [vp, C.c_uint64, C.c_uint64, C.c_int, dp, dp, dp,
                                                dp, dp, ip, dp, dp, ip, C.c_double, C.c_double,
                                                C.c_double, C.c_double, C.c_double, dp, dp, dp,
                                                dp]),
                "orc_run": (None, [vp, C.POINTER(Alg), C.c_uint64, C.POINTER(Result),
                                   C.POINTER(C.c_int64), dp, C.c_int64]),
                "orc_run_many": (None, [C.POINTER(vp), C.POINTER(Alg), C.POINTER(C.c_uint64),
                                        C.c_int, C.c_int, C.POINTER(Result)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


def f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- Philox
def philox(ctr, key):
    out = (C.c_uint32 * 4)()
    lib().orc_philox(*[int(c) & 0xFFFFFFFF for c in ctr], *[int(k) & 0xFFFFFFFF for k in key],
                     out)
    return [int(v) for v in out]


def u53(w0, w1):
    return lib().orc_u53(w0, w1)


def below(w, n):
    return lib().orc_below(w, n)


# ---------------------------------------------------------------- problems
class Problem:
    """An oracle problem instance (family, D) generated from a seed."""

    def __init__(self, seed: int, family: int, D: int, *, hybrid=None):
        L = lib()
        if hybrid is not None:
            frac, bodies = hybrid
            fr = f64(frac)
            bd = np.ascontiguousarray(bodies, dtype=np.int32)
            self.h = L.orc_hybrid_create(seed, D, len(bd), _dp(fr), _ip(bd))
        else:
            self.h = L.orc_problem_create(seed, family, D)
        if not self.h:
            raise ValueError("oracle: bad problem arguments")
        info = np.zeros(3, np.int32)
        fs = np.zeros(1)
        L.orc_problem_info(self.h, _ip(info), _dp(fs))
        self.family, self.D, self.K = (int(v) for v in info)
        self.fstar = float(fs[0])

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.orc_problem_destroy(h)
            self.h = None

    @property
    def ncomp(self):
        return self.K if self.family in (COMPOSITION, COMP_HYBRID) else 1

    def shift(self, comp=0):
        o = np.zeros(self.D)
        assert lib().orc_problem_get(self.h, comp, _dp(o), None) == 0
        return o

    def rotation(self, comp=0):
        M = np.zeros((self.D, self.D))
        assert lib().orc_problem_get(self.h, comp, None, _dp(M)) == 0
        return M

    def hybrid(self):
        perm = np.zeros(self.D, np.int32)
        gs = np.zeros(self.K, np.int32)
        gb = np.zeros(self.K, np.int32)
        assert lib().orc_problem_hybrid(self.h, _ip(perm), _ip(gs), _ip(gb)) == 0
        return perm, gs, gb

    def comp_hybrid(self, c):
        """Component c of a composition of hybrids: (perm, group sizes, bodies)."""
        perm = np.zeros(self.D, np.int32)
        gs, gb = np.zeros(8, np.int32), np.zeros(8, np.int32)
        K = lib().orc_problem_comp_hybrid(self.h, c, _ip(perm), _ip(gs), _ip(gb))
        assert K > 0
        return perm, gs[:K], gb[:K]

    def comp(self):
        n = self.K
        b = np.zeros(n, np.int32)
        s, lam, bias = np.zeros(n), np.zeros(n), np.zeros(n)
        assert lib().orc_problem_comp(self.h, _ip(b), _dp(s), _dp(lam), _dp(bias)) == 0
        return b, s, lam, bias

    def eval(self, x):
        x = f64(x)
        if x.ndim == 1:
            return lib().orc_eval(self.h, _dp(x))
        out = np.zeros(x.shape[0])
        lib().orc_eval_batch(self.h, _dp(x), x.shape[0], x.shape[1], _dp(out))
        return out

    def bound(self, x):
        """Rounding-error bound terms (E, G, Gd) of the plain FP64 evaluation
        at each row of x (see orc_eval_bound); each an array of len(x)."""
        x = np.atleast_2d(f64(x))
        out = np.zeros((x.shape[0], 3))
        lib().orc_eval_bound_batch(self.h, _dp(x), x.shape[0], x.shape[1], _dp(out))
        return out[:, 0], out[:, 1], out[:, 2]

    def transform(self, x, comp=0):
        x = f64(x)
        z = np.zeros(self.D)
        lib().orc_transform(self.h, comp, _dp(x), _dp(z))
        return z


def body(family, z):
    z = f64(z)
    return lib().orc_body(family, _dp(z), len(z))


# ---------------------------------------------------------------- operators
def init_population(seed, NP, D, lb=-100.0, ub=100.0):
    X = np.zeros((NP, D))
    lib().orc_init_population(seed, NP, D, lb, ub, _dp(X))
    return X


def de_rand1_trials(seed, gen, X, F=0.5, CR=0.9, lb=-100.0, ub=100.0):
    X = f64(X)
    NP, D = X.shape
    U = np.zeros_like(X)
    part = np.zeros((NP, 4), np.int32)
    lib().orc_de_rand1_trials(seed, gen, _dp(X), NP, D, F, CR, lb, ub, _dp(U), _ip(part))
    return U, part


def pbest_k(p, NP):
    return lib().orc_pbest_k(p, NP)


def rank(f):
    f = f64(f)
    o = np.zeros(len(f), np.int32)
    lib().orc_rank(_dp(f), len(f), _ip(o))
    return o


def de_ctpb_trials(seed, gen, X, fx, A, asize, F=0.5, CR=0.9, p=0.11, lb=-100.0, ub=100.0):
    X, fx = f64(X), f64(fx)
    NP, D = X.shape
    A = f64(A) if A is not None else np.zeros((1, D))
    U = np.zeros_like(X)
    part = np.zeros((NP, 4), np.int32)
    lib().orc_de_ctpb_trials(seed, gen, _dp(X), _dp(fx), NP, D, F, CR, p, _dp(A), asize, lb,
                             ub, _dp(U), _ip(part))
    return U, part


SHADE_H = 100


def shade_memory():
    """Initial SHADE memory: (M_F, M_CR, k) with every slot 0.5."""
    return np.full(SHADE_H, 0.5), np.full(SHADE_H, 0.5), 0


def shade_params(seed, gen, NP, MF, MCR):
    """Per-individual (F, CR, pbest pool size) drawn from the memory."""
    F, CR = np.zeros(NP), np.zeros(NP)
    kpb = np.zeros(NP, np.int32)
    MF, MCR = f64(MF), f64(MCR)
    lib().orc_shade_params(seed, gen, NP, len(MF), _dp(MF), _dp(MCR), _dp(F), _dp(CR), _ip(kpb))
    return F, CR, kpb


def shade_kmax(NP):
    return lib().orc_shade_kmax(NP)


def shade_trials(seed, gen, X, fx, F, CR, kpb, lb=-100.0, ub=100.0):
    X, fx, F, CR = f64(X), f64(fx), f64(F), f64(CR)
    kpb = np.ascontiguousarray(kpb, np.int32)
    NP, D = X.shape
    U = np.zeros_like(X)
    part = np.zeros((NP, 4), np.int32)
    lib().orc_shade_trials(seed, gen, _dp(X), _dp(fx), NP, D, _dp(F), _dp(CR), _ip(kpb), lb, ub,
                           _dp(U), _ip(part))
    return U, part


def shade_update(fx, fu, F, CR, MF, MCR, k):
    """Memory after one generation: returns (M_F', M_CR', k', improvements)."""
    fx, fu, F, CR = f64(fx), f64(fu), f64(F), f64(CR)
    MF, MCR = f64(MF).copy(), f64(MCR).copy()
    kk = C.c_int(k)
    n = lib().orc_shade_update(len(fx), len(MF), _dp(fx), _dp(fu), _dp(F), _dp(CR), _dp(MF),
                               _dp(MCR), C.byref(kk))
    return MF, MCR, kk.value, n


def cso_generation(seed, gen, X, V, fx, phi=0.1, lb=-100.0, ub=100.0):
    """One CSO generation: returns (X', V', pair) with pair[2k], pair[2k + 1]
    the winner and loser of pair k; the caller evaluates the losers."""
    X, V, fx = f64(X).copy(), f64(V).copy(), f64(fx)
    NP, D = X.shape
    pair = np.zeros(NP, np.int32)
    lib().orc_cso_generation(seed, gen, _dp(X), _dp(V), _dp(fx), NP, D, phi, lb, ub, _ip(pair))
    return X, V, pair


def de_select(seed, gen, X, fx, U, fu, A=None, asize=0):
    """Returns (X', fx', A', asize', accepted flags); inputs are not modified."""
    X, fx, U, fu = f64(X).copy(), f64(fx).copy(), f64(U), f64(fu)
    NP, D = X.shape
    acc = np.zeros(NP, np.uint8)
    if A is not None:
        A = f64(A).copy()
        asz = C.c_int(asize)
        lib().orc_de_select(seed, gen, _dp(X), _dp(fx), _dp(U), _dp(fu), NP, D, _dp(A),
                            C.byref(asz), acc.ctypes.data_as(C.POINTER(C.c_uint8)))
        return X, fx, A, asz.value, acc
    lib().orc_de_select(seed, gen, _dp(X), _dp(fx), _dp(U), _dp(fu), NP, D, None, None,
                        acc.ctypes.data_as(C.POINTER(C.c_uint8)))
    return X, fx, None, 0, acc


def pso_guides(fp, topology):
    fp = f64(fp)
    g = np.zeros(len(fp), np.int32)
    lib().orc_pso_guides(_dp(fp), len(fp), topology, _ip(g))
    return g


def pso_move(seed, gen, X, V, P, guide, w=0.7298, c1=1.49618, c2=1.49618, lb=-100.0,
             ub=100.0):
    X, V = f64(X).copy(), f64(V).copy()
    P = f64(P)
    NP, D = X.shape
    g = np.ascontiguousarray(guide, dtype=np.int32)
    lib().orc_pso_move(seed, gen, _dp(X), _dp(V), _dp(P), _ip(g), NP, D, w, c1, c2, lb, ub)
    return X, V


def pso_update(X, fx, P, fp):
    X, fx = f64(X), f64(fx)
    P, fp = f64(P).copy(), f64(fp).copy()
    NP, D = X.shape
    n = lib().orc_pso_update(_dp(X), _dp(fx), _dp(P), _dp(fp), NP, D)
    return P, fp, n


def psode_select(X, Y, fy, X3, f3):
    """PSODE's last two steps: returns (X', fx', V') -- V' = X3 - X, row i of
    X' is Y's where fy < f3, else X3's."""
    X, Y, fy, X3, f3 = f64(X), f64(Y), f64(fy), f64(X3), f64(f3)
    NP, D = X.shape
    Xn, fn, V = np.zeros((NP, D)), np.zeros(NP), np.zeros((NP, D))
    lib().orc_psode_select(_dp(X), _dp(Y), _dp(fy), _dp(X3), _dp(f3), NP, D, _dp(Xn), _dp(fn),
                           _dp(V))
    return Xn, fn, V


def psode_start(X, fx):
    """The PSO component's memory made from the initial population: zero
    velocity, personal bests = the population, ring guides."""
    X, fx = f64(X), f64(fx)
    return dict(V=np.zeros_like(X), P=X.copy(), fp=fx.copy(), guide=pso_guides(fx, 1))


def psode_generation(problem, seed, gen, X, fx, V, P, fp, guide, MF, MCR, k, w=0.7298,
                     c1=1.49618, c2=1.49618, lb=-100.0, ub=100.0):
    """One PSODE generation; inputs are not modified.  Returns a dict with the
    new X, fx, V, P, fp, guide, MF, MCR, k and the generation's evaluated rows
    Y, fy (PSO) and U, fu (SHADE)."""
    X, fx, V = f64(X).copy(), f64(fx).copy(), f64(V).copy()
    P, fp = f64(P).copy(), f64(fp).copy()
    g = np.ascontiguousarray(guide, dtype=np.int32).copy()
    MF, MCR = f64(MF).copy(), f64(MCR).copy()
    kk = C.c_int(k)
    NP, D = X.shape
    Y, fy, U, fu = np.zeros((NP, D)), np.zeros(NP), np.zeros((NP, D)), np.zeros(NP)
    lib().orc_psode_generation(problem.h, seed, gen, NP, _dp(X), _dp(fx), _dp(V), _dp(P),
                               _dp(fp), _ip(g), _dp(MF), _dp(MCR), C.byref(kk), w, c1, c2, lb,
                               ub, _dp(Y), _dp(fy), _dp(U), _dp(fu))
    return dict(X=X, fx=fx, V=V, P=P, fp=fp, guide=g, MF=MF, MCR=MCR, k=kk.value, Y=Y, fy=fy,
                U=U, fu=fu)


ALG_DE_RAND1, ALG_DE_CTPB, ALG_PSO_GBEST, ALG_PSO_RING, ALG_DE_SHADE, ALG_CSO = 0, 1, 2, 3, 4, 5
ALG_PSODE = 6


def make_alg(alg, NP, budget, F=0.5, CR=0.9, p=0.11, w=0.7298, c1=1.49618, c2=1.49618,
             lb=-100.0, ub=100.0):
    return Alg(alg, NP, F, CR, p, w, c1, c2, lb, ub, int(budget))


def run(problem: Problem, alg: Alg, seed: int, trace_cap: int = 0):
    r = Result()
    tf = np.zeros(max(trace_cap, 1), np.int64)
    tb = np.zeros(max(trace_cap, 1))
    lib().orc_run(problem.h, C.byref(alg), seed, C.byref(r),
                  tf.ctypes.data_as(C.POINTER(C.c_int64)) if trace_cap else None,
                  _dp(tb) if trace_cap else None, trace_cap)
    out = {"best": r.best, "fes": r.fes, "gens": r.gens, "success": bool(r.success)}
    if trace_cap:
        n = min(trace_cap, r.gens + 1)
        out["trace_fes"] = tf[:n].copy()
        out["trace_best"] = tb[:n].copy()
    return out


def run_many(problems, algs, seeds, nthreads=None):
    n = len(seeds)
    nthreads = nthreads or os.cpu_count() or 1
    ph = (C.c_void_p * n)(*[p.h for p in problems])
    aa = (Alg * n)(*algs)
    ss = (C.c_uint64 * n)(*[int(s) for s in seeds])
    rr = (Result * n)()
    lib().orc_run_many(ph, aa, ss, n, nthreads, rr)
    return [{"best": r.best, "fes": r.fes, "gens": r.gens, "success": bool(r.success)}
            for r in rr]
