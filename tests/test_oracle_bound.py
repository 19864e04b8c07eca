"""The rounding bound behind every parity tolerance (orc_eval_bound), pinned
against exact arithmetic: rows of every family are evaluated with mpmath at
50 significant digits on the oracle's own (FP64) instance data, and the
oracle's FP64 error must stay within its share of the bound.  A second test
checks that the bound is not vacuous where the method decides success: on
rows 1e-7 from the optimum whose value is small it is below 1e-10 absolute
at D = 100.

The mpmath bodies below restate the textbook forms only to measure rounding;
what the forms are is pinned in test_oracle.py.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs
from tests.gpu_util import U64, tol64

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp


def _schwefel_s():
    # s = argmax_{t in [0,500]} t sin sqrt t: stationary point of u^2 sin u
    u = mp.findroot(lambda u: 2 * mpmath.sin(u) + u * mpmath.cos(u), mp.mpf("20.5"))
    return u * u


def _body(fam, z):
    n = len(z)
    if n == 0:
        return mp.mpf(0)
    if fam == O.ELLIPSOID:
        return mpmath.fsum((mp.mpf(10) ** (mp.mpf(6) * i / (n - 1)) if n > 1 else 1) * z[i] ** 2
                           for i in range(n))
    if fam == O.ROSENBROCK:
        return mpmath.fsum(100 * ((z[i] + 1) ** 2 - (z[i + 1] + 1)) ** 2 + z[i] ** 2
                           for i in range(n - 1))
    if fam == O.RASTRIGIN:
        return mpmath.fsum(t * t - 10 * mpmath.cos(2 * mp.pi * t) + 10 for t in z)
    if fam == O.SCHWEFEL:
        s = _schwefel_s()
        c = s * mpmath.sin(mpmath.sqrt(s))
        out = []
        for t in z:
            y = t + s
            if abs(y) <= 500:
                out.append(c - y * mpmath.sin(mpmath.sqrt(abs(y))))
            else:
                b = 500 if y > 0 else -500
                out.append(c - b * mpmath.sin(mpmath.sqrt(500)) + mp.mpf("1e-4") * (abs(y) - 500) ** 2)
        return mpmath.fsum(out)
    if fam == O.ACKLEY:
        sq = mpmath.fsum(t * t for t in z)
        sc = mpmath.fsum(mpmath.cos(2 * mp.pi * t) for t in z)
        return (20 - 20 * mpmath.exp(-mp.mpf("0.2") * mpmath.sqrt(sq / n))) + (mpmath.e - mpmath.exp(sc / n))
    if fam == O.GRIEWANK:
        pr = mp.mpf(1)
        for i, t in enumerate(z):
            pr *= mpmath.cos(t / mpmath.sqrt(i + 1))
        return mpmath.fsum(t * t for t in z) / 4000 + (1 - pr)
    raise ValueError(fam)


def _groups(fam, z, sizes, bodies):
    out, a = [], 0
    for n, b in zip(sizes, bodies):
        out.append(_body(int(b), z[a:a + int(n)]))
        a += int(n)
    return mpmath.fsum(out)


def _exact(q, x):
    """g(x) in 50-digit arithmetic on the oracle's FP64 shift and rotation."""
    D = q.D
    xs = [mp.mpf(float(v)) for v in x]

    def zc(c):
        o, M = q.shift(c), q.rotation(c)
        d = [xs[j] - mp.mpf(float(o[j])) for j in range(D)]
        return d, [mpmath.fsum(mp.mpf(float(M[i, j])) * d[j] for j in range(D)) for i in range(D)]

    if q.family <= O.GRIEWANK:
        return _body(q.family, zc(0)[1])
    if q.family == O.HYBRID:
        _, gs, gb = q.hybrid()
        return _groups(q.family, zc(0)[1], gs, gb)
    bodies, sigma, lam, bias = q.comp()
    h, s = [], []
    for c in range(q.K):
        d, z = zc(c)
        s.append(mpmath.fsum(t * t for t in d))
        if q.family == O.COMP_HYBRID:
            _, gs, gb = q.comp_hybrid(c)
            gc = _groups(q.family, z, gs, gb)
        else:
            gc = _body(int(bodies[c]), z)
        h.append(mp.mpf(float(lam[c])) * gc + mp.mpf(float(bias[c])))
    if any(v == 0 for v in s):
        return h[[v == 0 for v in s].index(True)]
    w = [1 / mpmath.sqrt(s[c]) * mpmath.exp(-s[c] / (2 * D * mp.mpf(float(sigma[c])) ** 2))
         for c in range(q.K)]
    W = mpmath.fsum(w)
    return mpmath.fsum(w[c] / W * h[c] for c in range(q.K))


FAMS = list(range(9))


@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("D", [10, 24])
def test_oracle_error_within_its_share_of_the_bound(fam, D):
    """|g_oracle - g_exact| <= u * (E/2 + D * G): the oracle's share of the
    body term (half of every weight) and its own D-term dot products for z.
    Rows: uniform, 1e-3 and 1e-7 from the optimum, and mixed distances."""
    mp.dps = 50
    seed = 313 + 7 * fam + D
    q = O.Problem(seed, fam, D)
    o = q.shift(0)
    X = np.vstack([inputs.uniform_pop(3, D, seed=seed), inputs.near(o, 3, 1e-3, seed=seed),
                   inputs.near(o, 3, 1e-7, seed=seed + 1), inputs.mixed_scales(o, 3, D, seed=seed)])
    got = q.eval(X)
    E, G, Gd = q.bound(X)
    share = U64 * (0.5 * E + D * G)
    for i in range(len(X)):
        err = abs(mp.mpf(float(got[i])) - _exact(q, X[i]))
        assert err <= share[i], (i, float(err), share[i])


@pytest.mark.parametrize("fam", FAMS)
def test_bound_resolves_success_near_the_optimum(fam):
    """At D = 100, on rows 1e-7 from the optimum whose value is below 1e-6,
    the rounding part of the FP64 parity tolerance (with the library's
    measured rotation difference) is below 1e-10 absolute,
    so the parity tests can tell a 1e-8 success from a failure.  For the six
    bodies every such row qualifies; a composition is not small there (a
    component with large values keeps a weight of order sqrt(s_1)), so only
    its optimum itself does."""
    D = 100
    q = O.Problem(0x5EB00000 + fam, fam, D)
    o = q.shift(0)
    X = np.vstack([inputs.near(o, 8, 1e-7, seed=fam), o[None, :]])
    want = q.eval(X)
    E, G, Gd = q.bound(X)
    import paper_2505_17430_gb300 as S
    from tests.gpu_util import rot_diff
    dM = rot_diff(S.Problem(0x5EB00000 + fam, fam, D), q)
    rnd = U64 * (E + 2.0 * D * G) + dM * Gd
    small = want < 1e-6
    if fam <= O.HYBRID:
        assert small.all(), want.max()
    assert small[-1] and want[-1] == 0.0
    assert (rnd[small] < 1e-10).all(), rnd[small].max()
    assert (tol64(want, (E, G, Gd, dM, D))[small] < 1e-10).all()


def test_bound_terms_vanish_where_the_derivative_does():
    """G and Gd carry the true derivative: at the optimum of every body it
    is zero (Schwefel and Rosenbrock included), so both vanish at x = o."""
    for fam in range(6):
        q = O.Problem(91 + fam, fam, 30)
        E, G, Gd = q.bound(q.shift(0)[None, :])
        assert G[0] == 0.0 and Gd[0] == 0.0, fam
        assert np.isfinite(E[0]) and E[0] >= 0.0
