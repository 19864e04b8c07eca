"""Observed error of every evaluation precision against the FP64 oracle,
per family and dimension (a measurement script, not a test; needs a GPU).

For each family and D it evaluates two row sets through the C ABI
(sevo_evaluate):
  uniform  X ~ U[-100, 100]^D (the batched-evaluation input),
  near     o + r * N(0, I) / sqrt(D), r = 1e-3 (||x - o|| ~ 1e-3),
in FP64, FP32 (CUDA cores), TF32 and split BF16 (tensor cores), and reports
the maximum absolute error, the maximum relative error |got - want| / |want|,
the largest fraction of the parity tolerance used (the rounding bound of
tests/gpu_util.py, on a subsample) -- for the mixed modes all of these of the
mixed values themselves (SEVO_POLICY_REFINE off) -- and, for the mixed modes,
how many rows FP64 refinement recomputes (value below 1e-4) and the largest
relative error of the refined output.

    python -m tests.mixed_error_table --out table.md --json table.json
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

import oracle as O
from tests import inputs
from tests.gpu_util import bound, tol64, tol_mixed

PRECS = ("FP64", "FP32", "TF32", "BF16X3")
NAMES = ["ellipsoid", "rosenbrock", "rastrigin", "schwefel", "ackley", "griewank", "hybrid",
         "composition", "comp-hybrid"]


def rows_for(D, n_small, n_1000, n_5000):
    return n_small if D <= 100 else (n_1000 if D <= 1000 else n_5000)


def one(S, fam, D, N, n_bound, seed):
    import torch
    p, q = S.Problem(seed, fam, D), O.Problem(seed, fam, D)
    o = q.shift(0)
    sets = {"uniform": inputs.uniform_pop(N, D, seed=seed),
            "near": inputs.near(o, N, 1e-3 / np.sqrt(D), seed=seed + 1)}
    res = {}
    for name, X in sets.items():
        want = q.eval(X)
        sub = np.arange(min(n_bound, N))
        bnd = bound(p, q, X[sub])
        xt = torch.as_tensor(X).cuda()
        for prec in PRECS:
            got, info = p.evaluate(xt, prec=getattr(S, prec), sync=True)
            got = got.cpu().numpy()
            raw = got
            if prec != "FP64":  # the mixed values themselves, refinement off
                lib = S.lib()
                assert lib.sevo_set_policy(S.POLICY_REFINE, 0) == 0
                try:
                    raw = p.evaluate(xt, prec=getattr(S, prec), sync=True)[0].cpu().numpy()
                finally:
                    lib.sevo_set_policy(S.POLICY_REFINE, 1)
            den = np.maximum(np.abs(want), 1e-300)
            err, err_out = np.abs(raw - want), np.abs(got - want)
            rel = err / den
            tol = tol64(want[sub], bnd) if prec == "FP64" else tol_mixed(prec, want[sub], bnd)
            res[(name, prec)] = {
                "max_abs": float(err.max()), "max_rel": float(rel.max()),
                "median_rel": float(np.median(rel)), "max_frac_of_tol": float((err[sub] / tol).max()),
                "out_max_rel": float((err_out / den).max()),
                "refined": int(info["refined"]), "n": int(N),
                "min_value": float(want.min()), "max_value": float(want.max())}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="10,30,50,100,1000,5000")
    ap.add_argument("--rows", type=int, default=10000)
    ap.add_argument("--rows-1000", type=int, default=2000)
    ap.add_argument("--rows-5000", type=int, default=200)
    ap.add_argument("--bound-rows", type=int, default=500)
    ap.add_argument("--out", default="")
    ap.add_argument("--json", default="")
    a = ap.parse_args(argv)
    import paper_2505_17430_gb300 as S
    S.build()
    table = []
    for D in (int(v) for v in a.dims.split(",")):
        fams = range(9) if D <= 1000 else range(7)
        for fam in fams:
            t0 = time.time()
            N = rows_for(D, a.rows, a.rows_1000, a.rows_5000)
            r = one(S, fam, D, N, a.bound_rows, 0x5EB00000 + 16 * fam + D)
            for (name, prec), v in r.items():
                table.append({"family": NAMES[fam], "D": D, "set": name, "prec": prec, **v})
            print(f"# D={D} {NAMES[fam]} {time.time() - t0:.1f}s", file=sys.stderr, flush=True)
    lines = ["| D | family | rows | prec | max abs err | max rel err | median rel err | "
             "max err / tolerance | rows refined | max rel err after refinement |",
             "|---|---|---|---|---|---|---|---|---|---|"]
    for t in table:
        lines.append(f"| {t['D']} | {t['family']} | {t['set']} ({t['n']}) | {t['prec']} | "
                     f"{t['max_abs']:.2e} | {t['max_rel']:.2e} | {t['median_rel']:.2e} | "
                     f"{t['max_frac_of_tol']:.3f} | {t['refined']} | {t['out_max_rel']:.2e} |")
    md = "\n".join(lines)
    print(md)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(md + "\n")
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(table, fh, indent=1)


if __name__ == "__main__":
    main()
