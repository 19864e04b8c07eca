"""Pins of the FP64 oracle against what the definitions and mathematics fix
(no GPU).  Each test names what it pins and why a plausible mistake in the
oracle would fail it.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from tests import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SINGLE = [O.ELLIPSOID, O.ROSENBROCK, O.RASTRIGIN, O.SCHWEFEL, O.ACKLEY, O.GRIEWANK]
ALL = SINGLE + [O.HYBRID, O.COMPOSITION]


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    """Published Philox4x32-10 vectors (a wrong constant, round count, word
    order or key schedule changes every output word)."""
    for r in _rows("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_and_integer_maps():
    assert O.u53(0, 0) == 0.0
    assert O.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert O.u53(0x80000000, 0) == 0.5
    assert O.below(0, 7) == 0 and O.below(0xFFFFFFFF, 7) == 6
    assert O.below(0x80000000, 10) == 5


# ------------------------------------------------------------------ instances
def _gauss_numpy(seed, D, comp=0):
    """The seeded Gaussian matrix rebuilt from the oracle's Philox words with
    numpy's Box-Muller (an independent route to G)."""
    G = np.zeros(D * D)
    for e in range(D * D):
        pair = e >> 1
        w = O.philox([pair, pair >> 32, D, (17 << 24) | comp], [seed & 0xFFFFFFFF, seed >> 32])
        u1, u2 = O.u53(w[0], w[1]), O.u53(w[2], w[3])
        R = math.sqrt(-2.0 * math.log(1.0 - u1))
        th = 2.0 * math.pi * u2
        G[e] = R * (math.sin(th) if e & 1 else math.cos(th))
    return G.reshape(D, D)


@pytest.mark.parametrize("D", [2, 10, 30, 100])
def test_rotation_is_q_of_qr(D):
    """M is orthogonal to FP64 round-off, and M^T G is upper triangular with a
    positive diagonal, i.e. M is the Q of the QR of G (unique with diag R>0);
    it also equals LAPACK's Q after the same sign fix."""
    p = O.Problem(0x5EB00000 + D, O.ELLIPSOID, D)
    M = p.rotation()
    assert np.abs(M.T @ M - np.eye(D)).max() <= 10 * D * 2.0 ** -53
    G = _gauss_numpy(0x5EB00000 + D, D)
    R = M.T @ G
    assert np.abs(np.tril(R, -1)).max() <= 1e-12 * np.abs(G).max() * D
    assert (np.diag(R) > 0).all()
    Q2, R2 = np.linalg.qr(G)
    Q2 = Q2 * np.sign(np.diag(R2))[None, :]
    assert np.abs(Q2 - M).max() < 1e-11


def test_shift_range_and_determinism():
    p = O.Problem(3, O.RASTRIGIN, 500)
    o = p.shift()
    assert o.min() >= -80.0 and o.max() < 80.0
    assert abs(o.mean()) < 8.0 and 40.0 < o.std() < 52.0  # U[-80,80]: sd 46.2
    q = O.Problem(3, O.RASTRIGIN, 500)
    assert np.array_equal(o, q.shift()) and np.array_equal(p.rotation(), q.rotation())
    assert not np.array_equal(o[:100], O.Problem(3, O.RASTRIGIN, 100).shift())


def test_shift_from_pinned_draws():
    """o_j = -80 + 160 u, u = u53 of the known-answer-pinned Philox at
    counter (j >> 1, 0, D, SHIFT << 24 | component): words 0, 1 for even j and
    2, 3 for odd j.  Recomputed in exact rational arithmetic (within 2 u of
    80 + 160 u) for a plain instance and for two components of a composition,
    whose salt is the component index."""
    from fractions import Fraction as Fr
    u = Fr(1, 2 ** 53)
    for seed, fam, D, comps in ((0x51F7, O.RASTRIGIN, 9, (0,)),
                                (0x51F8, O.COMPOSITION, 6, (0, 1, 2))):
        p = O.Problem(seed, fam, D)
        for c in comps:
            o = p.shift(c)
            for j in range(D):
                w = O.philox([j >> 1, 0, D, (16 << 24) | c], [seed & 0xFFFFFFFF, seed >> 32])
                t = 160 * Fr(O.u53(w[2 * (j & 1)], w[2 * (j & 1) + 1]))
                assert abs(Fr(float(o[j])) - (t - 80)) <= 2 * u * (80 + t), (fam, c, j)


def test_plain_value_is_body_of_rotated_shift():
    """For the six plain families F - f* = body(M (x - o)) with M the exported
    rotation (the Q of the QR of the draw-pinned Gaussian matrix) applied as
    z_i = sum_j M_ij d_j, not its transpose (which would preserve norms and
    the optimum alike)."""
    for fam in range(6):
        D = 9
        q = O.Problem(0x7A00 + fam, fam, D)
        M, o = q.rotation(), q.shift()
        assert np.abs(M - M.T).max() > 1e-3  # the orientation is observable
        rng = np.random.default_rng(fam)
        for x in rng.uniform(-100, 100, (4, D)):
            z = M @ (x - o)
            assert np.allclose(q.transform(x), z, rtol=0, atol=1e-12)
            want = O.body(fam, z)
            assert q.eval(x[None, :])[0] == pytest.approx(want, rel=1e-12, abs=1e-12), fam
            assert abs(O.body(fam, M.T @ (x - o)) - want) > 1e-6 * abs(want), fam


def test_norm_preserved():
    p = O.Problem(9, O.GRIEWANK, 50)
    X = inputs.uniform_pop(20, 50, seed=1)
    for x in X:
        z = p.transform(x)
        d = x - p.shift()
        assert abs(np.linalg.norm(z) - np.linalg.norm(d)) <= 1e-14 * np.linalg.norm(d) * 10


# ------------------------------------------------------------------ bodies
@pytest.mark.parametrize("fam", ALL)
@pytest.mark.parametrize("D", [2, 10, 30, 100])
def test_value_at_optimum_is_exact_zero(fam, D):
    """f(o) = f* exactly: every body evaluates to exactly 0 at z = 0 (a stray
    constant, wrong offset or Schwefel shift would leave a residue)."""
    p = O.Problem(100 + D, fam, D)
    assert p.eval(p.shift()) == 0.0


def test_ellipsoid_closed_form():
    for D in (2, 10, 100):
        for k in range(D):
            z = np.zeros(D)
            z[k] = 1.0
            want = 10.0 ** (6.0 * k / (D - 1))
            assert O.body(O.ELLIPSOID, z) == pytest.approx(want, rel=1e-14)
    assert O.body(O.ELLIPSOID, np.array([3.0])) == 9.0


def test_rosenbrock_closed_form():
    for D in (2, 10, 100):
        assert O.body(O.ROSENBROCK, -np.ones(D)) == D - 1  # y = 0: each term 1
    # y = (2, 4): 100*(4-4)^2 + 1 = 1, and y=(2,0): 100*16+1
    assert O.body(O.ROSENBROCK, np.array([1.0, 3.0])) == 1.0
    assert O.body(O.ROSENBROCK, np.array([1.0, -1.0])) == 1601.0
    assert O.body(O.ROSENBROCK, np.array([0.3])) == 0.0


def test_rastrigin_integers():
    z = np.array([1.0, -2.0, 3.0, 0.0, 5.0])
    assert O.body(O.RASTRIGIN, z) == pytest.approx(float((z ** 2).sum()), abs=1e-12)
    assert O.body(O.RASTRIGIN, np.array([0.5])) == pytest.approx(0.25 + 20.0, abs=1e-12)


def test_ackley_constant_vector():
    for t in (0.25, 1.0, 3.7, -12.0):
        for D in (1, 5, 40):
            want = 20.0 - 20.0 * math.exp(-0.2 * abs(t)) + math.e - math.exp(math.cos(2 * math.pi * t))
            assert O.body(O.ACKLEY, np.full(D, t)) == pytest.approx(want, rel=1e-13, abs=1e-13)


def test_griewank_one_dimension():
    for t in (0.1, 2.0, -30.0, 400.0):
        want = t * t / 4000.0 + 1.0 - math.cos(t)
        assert O.body(O.GRIEWANK, np.array([t])) == pytest.approx(want, rel=1e-13, abs=1e-15)
    # second coordinate divides by sqrt(2)
    z = np.array([0.0, 2.0])
    assert O.body(O.GRIEWANK, z) == pytest.approx(4 / 4000 + 1 - math.cos(2 / math.sqrt(2)), rel=1e-13)


def test_schwefel_constants_and_nonnegativity():
    gold = {r[0]: (float(r[1]), float(r[2])) for r in _rows("schwefel_constants.txt")}
    # the body at z is c - (z+s) sin sqrt|z+s|: probe s and c through it
    ts = np.linspace(-2, 2, 40001)
    vals = np.array([O.body(O.SCHWEFEL, np.array([t])) for t in ts])
    assert vals.min() >= -1e-12 and vals[20000] == 0.0
    s_gold, tol = gold["argmax"]
    c_gold, tolc = gold["max_value"]
    # c - y sin sqrt y = 0 at y = s  =>  value at z = s_gold - s is ~0
    y = s_gold
    c_est = y * math.sin(math.sqrt(y))
    assert abs(c_est - c_gold) < tolc
    # value far away: outside [-500,500] the penalty makes it grow quadratically
    far = O.body(O.SCHWEFEL, np.array([2000.0]))
    assert far > 1e-4 * (2000 + s_gold - 500) ** 2
    # brute force on [-1000, 1000]: global minimum 0 at z = 0 only
    zs = np.linspace(-1000, 1000, 200001)
    v = np.array([O.body(O.SCHWEFEL, np.array([t])) for t in zs[::10]])
    assert v.min() >= 0.0
    assert abs(zs[::10][np.argmin(v)]) < 0.2


# ------------------------------------------------------------------ hybrid
def test_hybrid_structure():
    for D in (10, 30, 100, 1000):
        p = O.Problem(77, O.HYBRID, D)
        perm, gs, gb = p.hybrid()
        assert np.array_equal(np.sort(perm), np.arange(D))
        assert gs.sum() == D and 3 <= p.K <= 5 and (gs >= 1).all()
        assert ((gb >= 0) & (gb < 6)).all()
        assert (gs >= np.floor(0.1 * D) - 1).all()


def test_schwefel_outside_the_box_penalty():
    """Outside |y| <= 500 (y = z + s) the Schwefel term is its boundary value
    c - b sin sqrt|b| (b = 500 sign y) plus 1e-4 (|y| - 500)^2: continuous at
    |y| = 500 and checked at far points on both sides, with s found here by
    scipy's bracketing root finder on the stationarity condition
    sin u + (u / 2) cos u = 0, u = sqrt t, and c = s sin sqrt s."""
    opt = pytest.importorskip("scipy.optimize")
    u = opt.brentq(lambda v: math.sin(v) + 0.5 * v * math.cos(v), 20.0, 21.0, xtol=1e-15)
    s0 = u * u
    c = s0 * math.sin(u)
    edge = c - 500.0 * math.sin(math.sqrt(500.0))
    for z in (2000.0, 600.0, -2000.0, -1200.0):
        y = z + s0
        b = 500.0 if y > 0 else -500.0
        want = c - b * math.sin(math.sqrt(500.0)) + 1e-4 * (abs(y) - 500.0) ** 2
        assert O.body(O.SCHWEFEL, np.array([z])) == pytest.approx(want, rel=1e-10), z
    # continuity at y = 500: the two forms meet
    lo = O.body(O.SCHWEFEL, np.array([500.0 - s0 - 1e-9]))
    hi = O.body(O.SCHWEFEL, np.array([500.0 - s0 + 1e-9]))
    assert abs(lo - edge) < 1e-6 and abs(hi - edge) < 1e-6


def _hybrid_from_draws(seed, D, salt):
    """(K, bodies, E, permutation) of a hybrid structure from the
    known-answer-pinned Philox, salt 0 for a hybrid instance, 1 + c for
    component c of a composition of hybrids."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    K = 3 + O.below(O.philox([0, 0, D, (19 << 24) | salt], key)[0], 3)
    E, bodies = [], []
    for k in range(K):
        w = O.philox([1 + k, 0, D, (19 << 24) | salt], key)
        E.append(-math.log(1.0 - O.u53(w[0], w[1])))
        bodies.append(O.below(w[2], 6))
    perm = list(range(D))
    for i in range(D - 1, 0, -1):
        j = O.below(O.philox([i, 0, D, (18 << 24) | salt], key)[0], i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return K, bodies, E, perm


def _check_hybrid(got, want, D, what):
    perm, gs, gb = got
    K, bodies, E, wperm = want
    assert len(gs) == K and list(gb) == bodies, what
    for k in range(K - 1):
        t = (0.1 + (1.0 - 0.1 * K) * E[k] / sum(E)) * D
        if abs(t - round(t)) > 1e-9:  # away from a floor boundary
            assert gs[k] == math.floor(t), (what, k)
    assert gs.sum() == D and list(perm) == wperm, what


def test_hybrid_structure_from_pinned_draws():
    """A random hybrid instance from the known-answer-pinned Philox: K = 3 +
    below(w0, 3) of call (0, 0, D, HYB << 24 | salt); group k's body
    below(w2, 6) and E_k = -log(1 - u53(w0, w1)) of call (1 + k, 0, D,
    HYB << 24 | salt); sizes floor((0.1 + (1 - 0.1 K) E_k / sum E) D), the
    last group the remainder; the permutation by Fisher-Yates from the last
    index down, swapping i with below(w0, i + 1) of call (i, 0, D,
    PERM << 24 | salt).  Salt 0 for a hybrid instance; for component c of a
    composition of hybrids salt 1 + c, with N_c = 3 + below(w0, 3) of the
    composition call (0, 0, D, COMP << 24)."""
    for seed, D in ((0x4B1D, 50), (0x4B1E, 31), (0x4B1F, 100)):
        got = O.Problem(seed, O.HYBRID, D).hybrid()
        _check_hybrid(got, _hybrid_from_draws(seed, D, 0), D, seed)
    for seed, D in ((0x4C1D, 40), (0x4C1E, 23)):
        q = O.Problem(seed, O.COMP_HYBRID, D)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        Nc = 3 + O.below(O.philox([0, 0, D, 20 << 24], key)[0], 3)
        assert q.K == Nc, seed
        for c in range(Nc):
            _check_hybrid(q.comp_hybrid(c), _hybrid_from_draws(seed, D, 1 + c), D, (seed, c))


def test_hybrid_value_assembled_from_pinned_parts():
    """At generic points a random hybrid's value is sum_k body_k over group
    k's contiguous range of z' = M' (x - o), M' the rotation with its rows
    permuted (the exported rotation), assembled here from the exported parts
    and the pinned bodies: a group applied to the wrong range, the wrong body
    per group, or a body's index restarting at the wrong place fails."""
    for seed, D in ((0x4D1D, 20), (0x4D1E, 47)):
        q = O.Problem(seed, O.HYBRID, D)
        perm, gs, gb = q.hybrid()
        assert len(set(int(b) for b in gb)) > 1 or len(gb) == 1
        rng = np.random.default_rng(seed)
        X = np.vstack([rng.uniform(-100, 100, (4, D)), q.shift() + rng.standard_normal((3, D))])
        for x in X:
            z = q.rotation() @ (x - q.shift())
            want, start = 0.0, 0
            for n, b in zip(gs, gb):
                want += O.body(int(b), z[start:start + n]) if n > 0 else 0.0
                start += n
            assert q.eval(x[None, :])[0] == pytest.approx(want, rel=1e-10, abs=1e-12)


def test_hybrid_fixed_fractions():
    p = O.Problem(5, O.HYBRID, 100, hybrid=([0.3, 0.3, 0.4], [O.RASTRIGIN, O.ELLIPSOID, O.SCHWEFEL]))
    _, gs, gb = p.hybrid()
    assert list(gs) == [30, 30, 40] and list(gb) == [2, 0, 3]
    p = O.Problem(5, O.HYBRID, 10, hybrid=([0.3, 0.3, 0.4], [0, 1, 2]))
    assert list(p.hybrid()[1]) == [3, 3, 4]


@pytest.mark.parametrize("D", [10, 100])
def test_hybrid_of_separable_body_equals_plain(D):
    """All-Rastrigin hybrid == plain Rastrigin (same seed: same o and M;
    Rastrigin is separable and permutation-invariant).  A wrong group offset,
    size or permutation direction breaks it only if values are lost or
    duplicated, so it also checks every coordinate lands in exactly one group."""
    hy = O.Problem(42, O.HYBRID, D, hybrid=([0.2, 0.5, 0.3], [O.RASTRIGIN] * 3))
    pl = O.Problem(42, O.RASTRIGIN, D)
    X = inputs.uniform_pop(16, D, seed=3)
    assert np.allclose(hy.eval(X), pl.eval(X), rtol=1e-13, atol=0)


def test_hybrid_permutation_direction():
    """M' = P M: z'_t = z_{perm[t]}.  With an ellipsoid hybrid of one group
    the value equals the ellipsoid applied to z[perm] (not z[inv perm])."""
    D = 12
    hy = O.Problem(8, O.HYBRID, D, hybrid=([1.0], [O.ELLIPSOID]))
    pl = O.Problem(8, O.ELLIPSOID, D)
    perm = hy.hybrid()[0]
    x = inputs.uniform_pop(1, D, seed=4)[0]
    z = pl.transform(x)
    assert hy.eval(x) == pytest.approx(O.body(O.ELLIPSOID, z[perm]), rel=1e-13)
    inv = np.argsort(perm)
    if not np.array_equal(perm, inv):
        assert hy.eval(x) != pytest.approx(O.body(O.ELLIPSOID, z[inv]), rel=1e-6)


# ------------------------------------------------------------------ composition
@pytest.mark.parametrize("D", [2, 10, 50])
def test_composition_value_at_each_optimum(D):
    """F(o_c) = bias_c + f* exactly (weight collapses to e_c), and F >= f*."""
    p = O.Problem(0xC0 + D, O.COMPOSITION, D)
    body, sig, lam, bias = p.comp()
    assert 3 <= p.K <= 10
    assert list(bias) == [100.0 * c for c in range(p.K)]
    assert set(sig) <= {10.0, 20.0, 30.0, 40.0, 50.0, 60.0}
    assert ((lam >= 1e-6) & (lam <= 1.0)).all()
    for c in range(p.K):
        assert p.eval(p.shift(c)) == bias[c]
    X = inputs.uniform_pop(64, D, seed=5)
    assert (p.eval(X) >= 0.0).all()


def test_composition_parameters_from_pinned_draws():
    """A random composition from the known-answer-pinned Philox: N_c = 3 +
    below(w0, 8) of call (0, 0, D, COMP << 24); component c's sigma =
    10 (1 + below(w0, 6)), lambda = 10^(-6 + 6 u53(w1, w2)) and body
    below(w3, 6) of call (1 + c, 0, D, COMP << 24); bias = 100 c."""
    for seed, D in ((0xC0C0, 10), (0xC0C1, 30), (0xC0C2, 7), (0xC0C3, 64)):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        q = O.Problem(seed, O.COMPOSITION, D)
        body, sigma, lam, bias = q.comp()
        Nc = 3 + O.below(O.philox([0, 0, D, 20 << 24], key)[0], 8)
        assert len(body) == Nc, seed
        for c in range(Nc):
            w = O.philox([1 + c, 0, D, 20 << 24], key)
            assert sigma[c] == 10.0 * (1 + O.below(w[0], 6)), (seed, c)
            want = 10.0 ** (-6.0 + 6.0 * O.u53(w[1], w[2]))
            assert abs(lam[c] - want) <= 4e-16 * want, (seed, c)
            assert body[c] == O.below(w[3], 6), (seed, c)
            assert bias[c] == 100.0 * c


def test_composition_value_assembled_from_pinned_parts():
    """At generic points (uniform, and within a few units of one component's
    shift), F equals sum_c omega_c (lambda_c g_c(M_c (x - o_c)) + bias_c),
    omega = w / sum w with w_c = s_c^(-1/2) exp(-s_c / (2 D sigma_c^2)),
    s_c = |x - o_c|^2, assembled here from the exported shifts and rotations,
    the draw-pinned parameters and the closed-form-pinned bodies: a wrong
    weight exponent, a missing D or a swapped lambda/bias fails by far more
    than the tolerance."""
    for seed, D in ((0xA5A5, 12), (0xA5A6, 30)):
        q = O.Problem(seed, O.COMPOSITION, D)
        body, sig, lam, bias = q.comp()
        rng = np.random.default_rng(seed)
        X = np.vstack([rng.uniform(-100, 100, (5, D)),
                       q.shift(1) + 4.0 * rng.standard_normal((3, D)),
                       q.shift(2) + 0.5 * rng.standard_normal((2, D))])
        for x in X:
            g, sc = np.zeros(q.K), np.zeros(q.K)
            for c in range(q.K):
                d = x - q.shift(c)
                sc[c] = d @ d
                g[c] = O.body(int(body[c]), q.rotation(c) @ d)
            w = (1.0 / np.sqrt(sc)) * np.exp(-sc / (2.0 * D * sig * sig))
            om = w / w.sum() if w.sum() > 0 else np.full(q.K, 1.0 / q.K)
            want = float(om @ (lam * g + bias))
            assert q.eval(x[None, :])[0] == pytest.approx(want, rel=1e-10, abs=1e-12)


def test_composition_component_zero_is_the_single_instance():
    """Approaching o_1 along a ray x = o_1 + r u, the residual
    R(r) = (F(x) - f*) - lambda_1 g_1(x) vanishes linearly in r: component 1
    has the o, M and body of the single-family instance of the same seed,
    lambda_1 scales it, and the other weights decay as sqrt(s_1) (the
    s^{-1/2} factor).  A wrong lambda, body, component index or weight law
    leaves R(r)/r non-constant or R not vanishing."""
    D = 10
    p = O.Problem(0xBEEF, O.COMPOSITION, D)
    body, sig, lam, bias = p.comp()
    single = O.Problem(0xBEEF, int(body[0]), D)
    assert np.array_equal(single.shift(), p.shift(0))
    assert np.array_equal(single.rotation(), p.rotation(0))
    u = np.random.default_rng(1).standard_normal(D)
    u /= np.linalg.norm(u)
    ratios = []
    for r in (1e-5, 1e-6, 1e-7):
        x = p.shift(0) + r * u
        R = p.eval(x) - lam[0] * single.eval(x)
        assert R > 0
        ratios.append(R / r)
    assert abs(ratios[1] - ratios[0]) <= 1e-3 * ratios[1]
    assert abs(ratios[2] - ratios[1]) <= 1e-3 * ratios[2]


def test_composition_far_point_weights_finite():
    p = O.Problem(11, O.COMPOSITION, 30)
    x = np.full(30, 100.0)
    v = p.eval(x)
    assert np.isfinite(v) and v > 0


# ------------------------------------------------------------------ brute force D=2
@pytest.mark.parametrize("fam", ALL)
def test_bruteforce_grid_minimum_d2(fam):
    """2001 x 2001 grid over [-100,100]^2: every grid value is >= f*, and a
    local search (Nelder-Mead) started from the grid minimum ends at the
    optimum o (o_1 for a composition) with f - f* below 1e-8.  The grid is
    too coarse to resolve the 1e6-conditioned ellipsoid valley by itself, so
    the local search finishes what the brute force starts."""
    from scipy.optimize import minimize

    p = O.Problem(0x5EB00002 + fam, fam, 2)
    g = np.linspace(-100.0, 100.0, 2001)
    X = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    v = p.eval(X)
    assert v.min() >= 0.0
    best = X[np.argmin(v)]
    if fam == O.COMPOSITION:
        # unnormalised components leak through their weights (a cone of
        # slope ~ sum_c w_c (lambda_c g_c + bias_c) around o_1), so at D=2 the
        # global basin is narrower than one grid cell: the grid shows only
        # F >= f* = F(o_1); the local search starts from the cell next to o_1.
        assert p.eval(p.shift(0)) == 0.0 <= v.min()
        best = X[np.argmin(np.linalg.norm(X - p.shift(0), axis=1))]
    r = minimize(p.eval, best, method="Nelder-Mead",
                 options={"xatol": 1e-12, "fatol": 1e-16, "maxiter": 20000, "maxfev": 40000})
    # the plain Schwefel term c - y sin sqrt|y| rounds to within a few ulp of
    # c (~6e-14) of zero near its optimum, so allow that much below f*
    assert r.fun >= -1e-12 and r.fun <= 1e-8, (fam, r.fun)
    assert np.linalg.norm(r.x - p.shift(0)) <= 1e-3, (fam, r.x, p.shift(0))


# ------------------------------------------------------------------ DE operators
def test_de_rand1_partners_distinct_and_uniform():
    NP, D = 10, 6
    X = O.init_population(1, NP, D)
    counts = np.zeros((NP, NP))
    for g in range(1, 2001):
        U, part = O.de_rand1_trials(99, g, X)
        for i in range(NP):
            a, b, c, jr = part[i]
            assert len({i, a, b, c}) == 4 and 0 <= jr < D
            assert max(a, b, c) < NP
            counts[i, a] += 1
    # a uniform over the NP-1 others: chi-square with NP-2 dof per row
    for i in range(NP):
        row = np.delete(counts[i], i)
        exp = row.sum() / (NP - 1)
        chi2 = ((row - exp) ** 2 / exp).sum()
        assert chi2 < 30.0  # p ~ 1e-4 at 8 dof


def test_de_rand1_crossover_special_cases():
    NP, D = 12, 20
    X = O.init_population(2, NP, D, -1, 1)  # inside bounds, mutants stay inside mostly
    U, part = O.de_rand1_trials(5, 3, X, F=0.5, CR=0.0)
    for i in range(NP):
        diff = np.nonzero(U[i] != X[i])[0]
        assert set(diff) <= {part[i, 3]}          # CR=0: only j_rand crosses
    U1, part1 = O.de_rand1_trials(5, 3, X, F=0.0, CR=1.0)
    for i in range(NP):
        assert np.array_equal(U1[i], X[part1[i, 0]])  # F=0, CR=1: u = x_r1
    U2, part2 = O.de_rand1_trials(5, 3, X, F=0.5, CR=1.0)
    for i in range(NP):
        a, b, c, _ = part2[i]
        v = X[a] + 0.5 * (X[b] - X[c])
        assert np.allclose(U2[i], v, rtol=0, atol=1e-15)


def test_init_population_from_pinned_draws():
    """x_ij = lb + (ub - lb) u, u = u53 of the known-answer-pinned Philox at
    counter (j >> 1, i, 0, INIT << 24): words 0, 1 for even j and 2, 3 for odd
    j (an odd D uses half of its last call).  Recomputed in exact rational
    arithmetic: the oracle is within 2 u of |lb| + |(ub - lb) u|.  A swapped
    word pair, a counter per coordinate instead of per pair, or the row and
    column counters exchanged fail."""
    from fractions import Fraction as Fr
    NP, D, seed, lb, ub = 7, 11, 0x5EED0000ABCD, -3.5, 12.25
    X = O.init_population(seed, NP, D, lb, ub)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    u = Fr(1, 2 ** 53)
    for i in range(NP):
        for j in range(D):
            w = O.philox((j >> 1, i, 0, O.P_INIT << 24), key)
            r = Fr(O.u53(w[2 * (j & 1)], w[2 * (j & 1) + 1]))
            t = (Fr(ub) - Fr(lb)) * r
            assert abs(Fr(float(X[i, j])) - (Fr(lb) + t)) <= 2 * u * (abs(Fr(lb)) + t), (i, j)
            assert lb <= X[i, j] < ub


def test_de_rand1_crossover_from_pinned_draws():
    """Binomial crossover at an intermediate CR: coordinate j takes the mutant
    exactly when w_(j mod 4) 2^-32 < CR, w from the pinned Philox at counter
    (j >> 2, i, gen, CROSS << 24), or when j = j_rand = below(w3, D) of the
    partner call (0, i, gen, PART << 24); other coordinates keep the parent's
    bits.  The mutant is x_r1 + F (x_r2 - x_r3) within 2 u of its terms.  The
    population sits well inside the box, so no repair applies."""
    from fractions import Fraction as Fr
    NP, D, seed, gen, F, CR = 10, 13, 0xABCDEF12345, 4, 0.5, 0.5
    X = O.init_population(seed, NP, D, -1.0, 1.0)
    U, part = O.de_rand1_trials(seed, gen, X, F=F, CR=CR)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    u = Fr(1, 2 ** 53)
    crossed = kept = 0
    for i in range(NP):
        a, b, c, jr = (int(t) for t in part[i])
        wp = O.philox((0, i, gen, O.P_PART << 24), key)
        assert jr == O.below(wp[3], D)
        for j in range(D):
            w = O.philox((j >> 2, i, gen, O.P_CROSS << 24), key)
            if w[j & 3] / 2 ** 32 < CR or j == jr:
                crossed += 1
                t1, t2 = Fr(float(X[a, j])), Fr(F) * (Fr(float(X[b, j])) - Fr(float(X[c, j])))
                assert abs(Fr(float(U[i, j])) - (t1 + t2)) <= 2 * u * (abs(t1) + abs(t2)), (i, j)
            else:
                kept += 1
                assert U[i, j] == X[i, j], (i, j)
    assert crossed > 30 and kept > 30


def _kth_allowed(v, n, excluded):
    """The v-th smallest index of [0, n) not in `excluded` (v from 0)."""
    allowed = [t for t in range(n) if t not in excluded]
    return allowed[v]


def test_de_partners_from_pinned_draws():
    """Partners from the pinned Philox call (0, i, gen, PART << 24), w0..w3:
    rand/1 r1, r2, r3 are the below(w0, NP-1)-th, below(w1, NP-2)-th and
    below(w2, NP-3)-th index not yet excluded ({i}, then {i, r1}, then
    {i, r1, r2}); current-to-pbest takes pb = order[below(w0, k)] of the
    fitness ranking, r1 the below(w1, NP-1)-th index other than i and r2 the
    below(w2, NP + |A| - 2)-th index of population + archive other than i and
    r1; j_rand = below(w3, D) for both.  Recomputed here from that definition,
    not by the oracle's skip-over-sorted-exclusions loop."""
    NP, D, seed = 23, 5, 0x1234567890
    X = O.init_population(seed, NP, D)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for gen in range(1, 9):
        _, part = O.de_rand1_trials(seed, gen, X)
        for i in range(NP):
            w = O.philox((0, i, gen, O.P_PART << 24), key)
            a = _kth_allowed(O.below(w[0], NP - 1), NP, {i})
            b = _kth_allowed(O.below(w[1], NP - 2), NP, {i, a})
            c = _kth_allowed(O.below(w[2], NP - 3), NP, {i, a, b})
            assert list(part[i]) == [a, b, c, O.below(w[3], D)], (gen, i)
    fx = np.random.default_rng(3).permutation(NP).astype(float)
    A = O.init_population(seed + 1, NP, D)
    k = O.pbest_k(0.11, NP)
    order = list(np.argsort(fx, kind="stable"))
    for asize, gen in [(a, g) for a in (0, 6) for g in range(1, 9)]:
        _, part = O.de_ctpb_trials(seed, gen, X, fx, A, asize)
        for i in range(NP):
            w = O.philox((0, i, gen, O.P_PART << 24), key)
            pb = order[O.below(w[0], k)]
            r1 = _kth_allowed(O.below(w[1], NP - 1), NP, {i})
            r2 = _kth_allowed(O.below(w[2], NP + asize - 2), NP + asize, {i, r1})
            assert list(part[i]) == [pb, r1, r2, O.below(w[3], D)], (asize, i)


def test_de_midpoint_repair():
    NP, D = 8, 5
    X = np.full((NP, D), 99.0)
    X[:, 0] = -99.0
    X += np.arange(NP)[:, None] * 0.1 * np.sign(X) * -1
    U, part = O.de_rand1_trials(7, 1, X, F=5.0, CR=1.0)
    assert (U >= -100).all() and (U <= 100).all()
    for i in range(NP):
        a, b, c, _ = part[i]
        v = X[a] + 5.0 * (X[b] - X[c])
        for j in range(D):
            if v[j] > 100:
                assert U[i, j] == (100 + X[i, j]) * 0.5
            elif v[j] < -100:
                assert U[i, j] == (-100 + X[i, j]) * 0.5


def test_de_repair_order_parent_outside_box():
    """The repair tests u < lb first, then u > ub on the result, each once
    (Sec. 2.2's midpoint repair; the order is a reading where the paper is
    silent).  Parent 500 and a mutant below lb: (lb + 500)/2 = 200 is above ub,
    so the upper step follows, (ub + 500)/2 = 300.  Parent -500 and a mutant
    above ub: (ub - 500)/2 = -200 stays, below lb, as there is no second lower
    test."""
    NP, D = 6, 9
    for x0, rest, want in ((500.0, -150.0, 300.0), (-500.0, 150.0, -200.0)):
        X = np.full((NP, D), rest)
        X[0] = x0
        # row 0's partners all come from the other rows: v = rest + F (rest - rest)
        U, part = O.de_rand1_trials(11, 1, X, F=0.5, CR=1.0)
        assert 0 not in part[0, :3]
        assert np.array_equal(U[0], np.full(D, want))


def test_pbest_k_and_rank():
    assert O.pbest_k(0.11, 100) == 11 and O.pbest_k(0.11, 900) == 99
    assert O.pbest_k(0.11, 180) == 20 and O.pbest_k(0.11, 5) == 1
    f = np.array([3.0, 1.0, 2.0, 1.0, 0.5])
    assert list(O.rank(f)) == [4, 1, 3, 2, 0]


def test_de_ctpb_partners():
    NP, D = 40, 8
    X = O.init_population(3, NP, D)
    fx = np.random.default_rng(0).uniform(size=NP)
    A = O.init_population(4, NP, D)
    k = O.pbest_k(0.11, NP)
    top = set(O.rank(fx)[:k])
    for asize in (0, 7, NP):
        for g in range(1, 50):
            U, part = O.de_ctpb_trials(8, g, X, fx, A, asize)
            for i in range(NP):
                pb, r1, r2, jr = part[i]
                assert pb in top
                assert r1 != i and 0 <= r1 < NP
                assert r2 not in (i, r1) and 0 <= r2 < NP + asize
    # the formula with CR=1: v = x_i + F(x_pb - x_i) + F(x_r1 - x~_r2)
    U, part = O.de_ctpb_trials(8, 1, X, fx, A, NP, F=0.5, CR=1.0)
    XA = np.vstack([X, A])
    for i in range(NP):
        pb, r1, r2, _ = part[i]
        v = X[i] + 0.5 * (X[pb] - X[i]) + 0.5 * (X[r1] - XA[r2])
        v = np.where(v < -100, (-100 + X[i]) / 2, np.where(v > 100, (100 + X[i]) / 2, v))
        assert np.allclose(U[i], v, atol=1e-12, rtol=0)


def test_de_select_and_archive():
    NP, D = 30, 4
    X = O.init_population(1, NP, D)
    fx = np.arange(NP, dtype=float)
    U = O.init_population(2, NP, D)
    fu = fx.copy()
    fu[::3] -= 0.5   # better
    fu[1::3] += 0.5  # worse
    # fu[2::3] ties -> accepted
    A = np.zeros((NP, D))
    X2, fx2, A2, asz, acc = O.de_select(5, 1, X, fx, U, fu, A, 0)
    assert list(acc) == [1 if i % 3 != 1 else 0 for i in range(NP)]
    assert asz == acc.sum() == 20
    assert np.array_equal(A2[:20], X[acc.astype(bool)])
    assert np.array_equal(X2[acc.astype(bool)], U[acc.astype(bool)])
    # full archive: size stays NP and every slot holds a past parent row
    X3, fx3, A3, asz3, acc3 = O.de_select(5, 2, X, fx, U, fu, X.copy(), NP)
    assert asz3 == NP
    rows = {tuple(r) for r in X}
    assert all(tuple(r) in rows for r in A3)


def test_de_archive_eviction_from_pinned_draws():
    """An accepted parent (f_u <= f_x) enters the archive at the next free
    slot while it has fewer than NP rows, and once full replaces the slot
    below(w0, NP) of the pinned Philox call (0, i, gen, ARCH << 24), rows taken
    in index order.  Starting 3 rows short of full, the first three accepted
    parents fill it and the rest evict; a slot that no parent drew keeps its
    old row, and a slot drawn twice holds the later parent."""
    NP, D, seed, gen = 16, 3, 0xFEEDBEEF, 6
    X = O.init_population(seed, NP, D)
    U = O.init_population(seed + 7, NP, D)
    fx = np.ones(NP)
    fu = np.where(np.arange(NP) % 4 == 1, 2.0, 1.0)  # rows 1, 5, 9, 13 rejected; ties accepted
    A0 = O.init_population(seed + 9, NP, D)
    asize0 = NP - 3
    X2, fx2, A2, asz, acc = O.de_select(seed, gen, X, fx, U, fu, A0, asize0)
    assert list(acc) == [0 if i % 4 == 1 else 1 for i in range(NP)] and asz == NP
    key = (seed & 0xFFFFFFFF, seed >> 32)
    want = A0.copy()
    fill = asize0
    for i in np.nonzero(acc)[0]:
        if fill < NP:
            slot, fill = fill, fill + 1
        else:
            slot = O.below(O.philox((0, int(i), gen, O.P_ARCH << 24), key)[0], NP)
        want[slot] = X[i]
    assert np.array_equal(A2, want)
    assert np.array_equal(X2[acc == 1], U[acc == 1]) and np.array_equal(X2[acc == 0], X[acc == 0])


# ------------------------------------------------------------------ PSO operators
def test_pso_guides():
    fp = np.array([5.0, 1.0, 3.0, 1.0, 7.0, 0.5])
    assert list(O.pso_guides(fp, 0)) == [5] * 6
    # ring {i-1,i,i+1}: i=0 -> {5,0,1}: 0.5 at 5
    assert list(O.pso_guides(fp, 1)) == [5, 1, 1, 3, 5, 5]
    fp2 = np.array([1.0, 1.0, 2.0])
    assert list(O.pso_guides(fp2, 1)) == [0, 0, 0]  # ties -> lowest index


def test_pso_stationary_and_clamp():
    NP, D = 6, 7
    X = O.init_population(1, NP, D)
    V = np.random.default_rng(1).uniform(-5, 5, (NP, D))
    P = O.init_population(2, NP, D)
    g = np.zeros(NP, np.int32)
    X1, V1 = O.pso_move(3, 1, X, V, P, g, w=0.0, c1=0.0, c2=0.0)
    assert np.array_equal(X1, X) and (V1 == 0).all()
    # all at one point with p = g = x: stays put for any coefficients
    Xs = np.tile(X[:1], (NP, 1))
    Xs2, Vs2 = O.pso_move(3, 1, Xs, np.zeros_like(Xs), Xs, g)
    assert np.array_equal(Xs2, Xs)
    # clamp: huge velocity pushes out -> x on the bound and v = 0 there
    Vb = np.full((NP, D), 1e4)
    Xb, Vb2 = O.pso_move(3, 1, X, Vb, P, g, w=1.0)
    assert (Xb == 100.0).all() and (Vb2 == 0).all()


def test_pso_move_formula_from_pinned_draws():
    """v' = w v + c1 r1 (p_i - x) + c2 r2 (g_i - x), x' = x + v' (clamped),
    with r1 = u53(w0, w1) and r2 = u53(w2, w3) of one Philox call per
    coordinate at counter (j, i, gen, PSO << 24): recomputed here in exact
    rational arithmetic from the FP64 inputs and the known-answer-pinned
    generator, and the oracle must be within 4 u of the sum of the three
    terms' magnitudes.  c1 != c2, distinct personal bests and guides, and a
    non-zero velocity make a swapped pair of terms, one draw used twice, one
    draw per particle instead of per coordinate, or a dropped inertia term
    fail."""
    from fractions import Fraction as Fr
    NP, D, seed, gen = 9, 6, 0xC0FFEE1234, 7
    w, c1, c2 = 0.61, 1.3, 1.9
    X = O.init_population(seed, NP, D) * 0.3
    P = O.init_population(seed + 1, NP, D) * 0.3
    V = np.random.default_rng(5).uniform(-4, 4, (NP, D))
    guide = np.array([(3 * i + 2) % NP for i in range(NP)], np.int32)
    X2, V2 = O.pso_move(seed, gen, X, V, P, guide, w=w, c1=c1, c2=c2)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    u = Fr(1, 2 ** 53)
    for i in range(NP):
        for j in range(D):
            r = O.philox((j, i, gen, O.P_PSO << 24), key)
            r1, r2 = O.u53(r[0], r[1]), O.u53(r[2], r[3])
            x, p, g, v = (Fr(float(t)) for t in (X[i, j], P[i, j], P[guide[i], j], V[i, j]))
            t1, t2, t3 = Fr(w) * v, Fr(c1) * Fr(r1) * (p - x), Fr(c2) * Fr(r2) * (g - x)
            exact = t1 + t2 + t3
            mag = abs(t1) + abs(t2) + abs(t3)
            assert abs(Fr(float(V2[i, j])) - exact) <= 4 * u * mag, (i, j)
            xn = x + Fr(float(V2[i, j]))
            assert abs(Fr(float(X2[i, j])) - xn) <= u * abs(xn), (i, j)
    assert (np.abs(X2) < 100).all()  # no clamp in this case


def test_pso_control_run_reaches_success():
    """Control: global-best and ring PSO (NP = 40, w = 0.7298, c1 = c2 =
    1.49618) on the shifted-rotated Rastrigin and Griewank at D = 2 reach
    1e-8 within 1e5 evaluations.  (A rotated ellipsoid of condition 1e6 is
    no control for this PSO: its per-coordinate random coefficients are not
    rotation invariant, and it stalls there at 1e-6 .. 1e-2 even at D = 2.)"""
    for fam in (O.RASTRIGIN, O.GRIEWANK):
        q = O.Problem(2, fam, 2)
        for alg in (O.ALG_PSO_GBEST, O.ALG_PSO_RING):
            r = O.run(q, O.make_alg(alg, 40, 100000), 1)
            assert r["success"] and r["fes"] == 100000, (fam, alg, r["best"])


def test_pso_update_strict():
    NP, D = 4, 3
    X = O.init_population(1, NP, D)
    P = O.init_population(2, NP, D)
    fp = np.array([1.0, 2.0, 3.0, 4.0])
    fx = np.array([0.5, 2.0, 3.5, 1.0])
    P2, fp2, n = O.pso_update(X, fx, P, fp)
    assert n == 2 and list(fp2) == [0.5, 2.0, 3.0, 1.0]
    assert np.array_equal(P2[1], P[1]) and np.array_equal(P2[0], X[0])


# ------------------------------------------------------------------ whole runs
def test_run_budget_and_trace():
    p = O.Problem(1, O.RASTRIGIN, 10)
    a = O.make_alg(O.ALG_DE_RAND1, 50, 100000)
    r = O.run(p, a, 1, trace_cap=3000)
    assert r["fes"] == 100000 and r["gens"] == 1999
    assert r["trace_fes"][0] == 50 and r["trace_fes"][-1] == 100000
    assert (np.diff(r["trace_best"]) <= 0).all()
    # overshooting last generation counts only budget - fes rows
    a2 = O.make_alg(O.ALG_PSO_RING, 40, 1000 + 7)
    r2 = O.run(p, a2, 1, trace_cap=100)
    assert r2["fes"] == 1007 and r2["trace_fes"][-1] == 1007 and r2["gens"] == 25


def test_de_controls_reach_success_threshold():
    """Statistical controls: DE/rand/1/bin (NP=50, F=.5, CR=.9) reaches the
    1e-8 threshold on a unimodal shifted-rotated ellipsoid at D=5 within 1e5
    evaluations; DE/current-to-pbest/1/bin + archive does so on the
    shifted-rotated Ackley at D=10 for most seeds (it is the stronger
    operator).  A broken selection, crossover or partner draw stalls both."""
    p = O.Problem(2, O.ELLIPSOID, 5)
    r = O.run(p, O.make_alg(O.ALG_DE_RAND1, 50, 100000), 1)
    assert r["success"] and r["best"] <= 1e-8
    wins = sum(O.run(O.Problem(s, O.ACKLEY, 10), O.make_alg(O.ALG_DE_CTPB, 50, 100000), 1)["success"]
               for s in range(1, 6))
    assert wins >= 2


def test_run_many_equals_run():
    probs = [O.Problem(s, f, 10) for s, f in [(1, 2), (2, 4), (3, 6), (4, 7)]]
    algs = [O.make_alg(k, 40 if k >= 2 else 30, 3000) for k in range(4)]
    seeds = [11, 12, 13, 14]
    many = O.run_many(probs, algs, seeds, nthreads=3)
    for pr, al, sd, m in zip(probs, algs, seeds, many):
        one = O.run(pr, al, sd)
        assert one["best"] == m["best"] and one["fes"] == m["fes"]


# ---------------------------------------------------------------- SHADE
def _shade_samples(MF, MCR, NP=50, gens=200, seed=3):
    F, CR, K = [], [], []
    for g in range(1, gens + 1):
        f, c, k = O.shade_params(seed, g, NP, MF, MCR)
        F.append(f)
        CR.append(c)
        K.append(k)
    return np.concatenate(F), np.concatenate(CR), np.concatenate(K)


@pytest.mark.parametrize("loc", [0.3, 0.5, 0.7])
def test_shade_F_is_cauchy_resampled_positive_and_capped(loc):
    """F ~ Cauchy(M_F, 0.1) redrawn until > 0, capped at 1: the empirical
    median and the mass at F = 1 match the closed forms of that conditional
    Cauchy law (CDF G(x) = 1/2 + atan((x - loc)/0.1)/pi)."""
    H = O.SHADE_H
    F, _, _ = _shade_samples(np.full(H, loc), np.full(H, 0.5))
    assert (F > 0).all() and (F <= 1).all()
    G = lambda x: 0.5 + np.arctan((x - loc) / 0.1) / np.pi  # noqa: E731
    g0 = G(0.0)
    med = loc + 0.1 * np.tan(np.pi * (g0 + 0.5 * (1 - g0) - 0.5))
    assert abs(np.median(F) - med) < 0.006, (np.median(F), med)
    p_one = (1 - G(1.0)) / (1 - g0)
    assert abs(np.mean(F == 1.0) - p_one) < 0.01, (np.mean(F == 1.0), p_one)


def test_shade_CR_is_clipped_normal():
    """CR ~ N(M_CR, 0.1) clipped to [0, 1]: mean and spread at 0.5, and the
    mass at 1 for M_CR = 0.95 equals 1 - Phi(0.5)."""
    H = O.SHADE_H
    _, CR, _ = _shade_samples(np.full(H, 0.5), np.full(H, 0.5))
    assert abs(CR.mean() - 0.5) < 0.005 and abs(CR.std() - 0.1) < 0.005
    _, CR, _ = _shade_samples(np.full(H, 0.5), np.full(H, 0.95))
    from math import erf, sqrt
    p1 = 1 - 0.5 * (1 + erf(0.5 / sqrt(2)))
    assert abs(np.mean(CR == 1.0) - p1) < 0.015 and (CR >= 0).all() and (CR <= 1).all()


def test_shade_memory_slot_uniform_and_pool_range():
    """The memory slot is uniform over the H slots (mean of CR over slots
    holding M_CR[h] = h / H), and the pbest pool k = ceil(p NP) with
    p ~ U[2/NP, 0.2] spans 2 .. ceil(0.2 NP)."""
    H = O.SHADE_H
    _, CR, K = _shade_samples(np.full(H, 0.5), np.arange(H) / H, NP=100, gens=300)
    assert abs(CR.mean() - np.mean(np.clip(np.arange(H) / H, 0, 1))) < 0.01
    assert K.min() == 2 and K.max() == 20 and O.shade_kmax(100) == 20
    assert O.shade_kmax(8) == 2  # 2/NP > 0.2 for NP < 10


def test_shade_params_from_pinned_draws():
    """SHADE's per-row parameters from the known-answer-pinned Philox, call
    (t, i, gen, SHADE << 24): t = 0 gives the memory slot below(w0, H) and the
    pool fraction p = 2/NP + (0.2 - 2/NP) u53(w1, w2), k = floor(p NP + 0.5)
    in [1, NP]; t = 1 gives CR = M_CR + 0.1 z, z = sqrt(-2 ln(1 - u1))
    cos(2 pi u2) (u1 = u53(w0, w1), u2 = u53(w2, w3)), clipped to [0, 1];
    t = 2, 3, ... give Cauchy candidates M_F + 0.1 tan(pi (u53(w0, w1) - 0.5))
    until one is positive, capped at 1.  Distinct memory slots make the slot
    choice visible."""
    NP, H, seed, gen = 37, 6, 0x5AADE, 3
    MF = np.array([0.05, 0.2, 0.35, 0.5, 0.65, 0.8])
    MCR = np.array([0.9, 0.1, 0.7, 0.3, 0.5, 0.95])
    F, CR, kpb = O.shade_params(seed, gen, NP, MF, MCR)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    pmin = 2.0 / NP
    for i in range(NP):
        w = O.philox([0, i, gen, 6 << 24], key)
        h = O.below(w[0], H)
        t = (pmin + (0.2 - pmin) * O.u53(w[1], w[2])) * NP + 0.5
        if abs(t - round(t)) > 1e-9:
            assert kpb[i] == min(NP, max(1, math.floor(t))), i
        w = O.philox([1, i, gen, 6 << 24], key)
        u1, u2 = O.u53(w[0], w[1]), O.u53(w[2], w[3])
        cr = MCR[h] + 0.1 * math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)
        assert abs(CR[i] - min(1.0, max(0.0, cr))) <= 1e-13, i
        f = MF[h]
        for a in range(64):
            w = O.philox([2 + a, i, gen, 6 << 24], key)
            c = MF[h] + 0.1 * math.tan(math.pi * (O.u53(w[0], w[1]) - 0.5))
            if c > 0.0:
                f = c
                break
        assert abs(F[i] - min(1.0, f)) <= 1e-12 * max(1.0, abs(f)), i


def test_shade_memory_update_closed_form():
    """Weights proportional to the improvement fx - fu over strict
    improvements: M_F[k] = sum w F^2 / sum w F, M_CR[k] = sum w CR / sum w,
    then k advances (mod H); ties and non-improvements are ignored."""
    H = O.SHADE_H
    MF, MCR, k = O.shade_memory()
    fx = np.array([10.0, 10.0, 10.0, 5.0, 7.0, 3.0])
    fu = np.array([9.0, 8.0, 7.0, 5.0, 8.0, 3.0])  # improvements 1, 2, 3; a tie; worse; a tie
    F = np.array([0.5, 0.6, 0.7, 0.9, 0.9, 0.9])
    CR = np.array([0.1, 0.2, 0.3, 0.9, 0.9, 0.9])
    MF2, MCR2, k2, n = O.shade_update(fx, fu, F, CR, MF, MCR, 7 % H)
    assert n == 3 and k2 == 8
    assert MF2[7] == pytest.approx((0.25 + 2 * 0.36 + 3 * 0.49) / (0.5 + 2 * 0.6 + 3 * 0.7), rel=1e-15)
    assert MCR2[7] == pytest.approx((0.1 + 2 * 0.2 + 3 * 0.3) / 6, rel=1e-15)
    assert np.array_equal(np.delete(MF2, 7), np.delete(MF, 7))
    MF3, MCR3, k3, n = O.shade_update(fx, fx, F, CR, MF2, MCR2, H - 1)  # no improvement
    assert n == 0 and k3 == H - 1 and np.array_equal(MF3, MF2)
    _, _, k4, _ = O.shade_update(fx, fu, F, CR, MF2, MCR2, H - 1)  # wraps
    assert k4 == 0


def test_shade_trials_reduce_to_current_to_pbest_without_archive():
    """With F, CR and the pool size equal for every individual, the SHADE
    trial is the (pinned) current-to-pbest/1/bin trial with an empty
    archive."""
    NP, D = 40, 13
    X = O.init_population(11, NP, D)
    fx = O.Problem(5, O.RASTRIGIN, D).eval(X)
    k = O.pbest_k(0.11, NP)
    F, CR, kpb = np.full(NP, 0.5), np.full(NP, 0.9), np.full(NP, k, np.int32)
    U, part = O.shade_trials(11, 4, X, fx, F, CR, kpb)
    U2, part2 = O.de_ctpb_trials(11, 4, X, fx, np.zeros((1, D)), 0, F=0.5, CR=0.9, p=0.11)
    assert np.array_equal(U, U2) and np.array_equal(part, part2)


def test_shade_control_run_reaches_success():
    """Control: SHADE on the shifted-rotated ellipsoid (D = 10, NP = 50,
    6e4 evaluations) reaches the 1e-8 success threshold."""
    q = O.Problem(3, O.ELLIPSOID, 10)
    r = O.run(q, O.make_alg(O.ALG_DE_SHADE, 50, 60000), 1)
    assert r["success"] and r["fes"] == 60000


# ---------------------------------------------------------------- composition of hybrids
@pytest.mark.parametrize("D", [10, 37])
def test_comp_hybrid_structure_and_optima(D):
    """Each component carries a valid hybrid structure (a permutation, group
    sizes summing to D, bodies among the six); F(o_c) equals bias_c exactly
    and F >= 0 elsewhere (every component is a non-negative hybrid)."""
    q = O.Problem(0xF1 + D, O.COMP_HYBRID, D)
    assert 3 <= q.K <= 5 and q.ncomp == q.K
    _, sig, lam, bias = q.comp()
    for c in range(q.K):
        perm, gs, gb = q.comp_hybrid(c)
        assert sorted(perm) == list(range(D))
        assert gs.sum() == D and (gs >= 0).all() and 3 <= len(gs) <= 5
        assert ((gb >= 0) & (gb <= 5)).all()
        assert q.eval(q.shift(c)[None, :])[0] == bias[c]
    X = np.random.default_rng(D).uniform(-100, 100, (50, D))
    assert (q.eval(X) >= 0).all()


def test_comp_hybrid_component_reduces_to_its_hybrid():
    """Approaching o_c along a ray x = o_c + r u, the residual
    R(r) = F(x) - bias_c - lambda_c g_c(x) vanishes linearly in r (the other
    weights decay as sqrt(s_c)), with g_c assembled here from the pinned
    bodies over component c's permuted groups of z = M'_c (x - o_c).  A wrong
    group partition, body, permutation or lambda leaves R(r)/r non-constant."""
    D = 24
    q = O.Problem(0xF1F1, O.COMP_HYBRID, D)
    _, sig, lam, bias = q.comp()
    u = np.random.default_rng(2).standard_normal(D)
    u /= np.linalg.norm(u)
    for c in range(q.K):
        _, gs, gb = q.comp_hybrid(c)
        ratios = []
        for r in (1e-5, 1e-6, 1e-7):
            x = q.shift(c) + r * u
            z = q.rotation(c) @ (x - q.shift(c))
            g, start = 0.0, 0
            for n, b in zip(gs, gb):
                g += O.body(int(b), z[start:start + n]) if n > 0 else 0.0
                start += n
            R = q.eval(x[None, :])[0] - bias[c] - lam[c] * g
            ratios.append(R / r)
        assert abs(ratios[1] - ratios[0]) <= 1e-3 * abs(ratios[1]), (c, ratios)
        assert abs(ratios[2] - ratios[1]) <= 1e-3 * abs(ratios[2]), (c, ratios)


def test_comp_hybrid_value_assembled_from_pinned_parts():
    """At generic points, F equals the composition (weights as pinned for the
    plain composition family) of component values assembled here from the
    exported rotation and shift, the pinned bodies and each component's group
    partition: checks the per-component hybrid assembly, where an error would
    change g_c by O(1)."""
    D = 16
    q = O.Problem(0xF1F2, O.COMP_HYBRID, D)
    _, sig, lam, bias = q.comp()
    X = np.vstack([np.random.default_rng(4).uniform(-100, 100, (6, D)),
                   q.shift(1) + 3.0 * np.random.default_rng(5).standard_normal((4, D))])
    for x in X:
        g, s = np.zeros(q.K), np.zeros(q.K)
        for c in range(q.K):
            d = x - q.shift(c)
            s[c] = d @ d
            z = q.rotation(c) @ d
            _, gs, gb = q.comp_hybrid(c)
            start = 0
            for n, b in zip(gs, gb):
                g[c] += O.body(int(b), z[start:start + n]) if n > 0 else 0.0
                start += n
        w = (1.0 / np.sqrt(s)) * np.exp(-s / (2.0 * D * sig * sig))
        om = w / w.sum() if w.sum() > 0 else np.full(q.K, 1.0 / q.K)
        want = float(om @ (lam * g + bias))
        assert q.eval(x[None, :])[0] == pytest.approx(want, rel=1e-10)


# ---------------------------------------------------------------- CSO
def _cso_keys(seed, gen, NP):
    key = (seed & 0xFFFFFFFF, seed >> 32)
    return [O.philox((0, i, gen, (7 << 24)), key)[0] for i in range(NP)]


def test_cso_pairing_winners_and_unchanged_winners():
    """The pairs are the indices sorted by their Philox key (ties by index,
    counter (0, i, gen, CSO << 24), the KAT-pinned generator) taken two by
    two; the winner of each pair has the lower fitness (ties: the first) and
    passes unchanged; every particle appears exactly once."""
    NP, D, seed, gen = 40, 7, 0x1234_5678_9AB, 5
    X = O.init_population(seed, NP, D)
    fx = O.Problem(3, O.RASTRIGIN, D).eval(X)
    fx[3] = fx[11]  # a tie somewhere
    V = np.random.default_rng(1).uniform(-1, 1, (NP, D))
    X2, V2, pair = O.cso_generation(seed, gen, X, V, fx)
    keys = _cso_keys(seed, gen, NP)
    order = sorted(range(NP), key=lambda i: (keys[i], i))
    assert sorted(pair.tolist()) == list(range(NP))
    for k in range(NP // 2):
        a, b = order[2 * k], order[2 * k + 1]
        w, l = pair[2 * k], pair[2 * k + 1]
        assert {w, l} == {a, b}
        assert w == (a if fx[a] <= fx[b] else b)
        assert np.array_equal(X2[w], X[w]) and np.array_equal(V2[w], V[w])
        assert not np.array_equal(X2[l], X[l])


def test_cso_loser_update_formula():
    """Loser l: v' = R1 v + R2 (x_w - x_l) + phi R3 (xbar - x_l) with R1, R2
    from draw (1 + 2j, l, gen) and R3 from (2 + 2j, l, gen), xbar the mean
    position before the update, x' = x + v' clamped: recomputed here from
    the pinned generator to 1e-14 (the oracle fuses the multiply-adds)."""
    NP, D, seed, gen, phi = 12, 5, 77, 3, 0.1
    X = O.init_population(seed, NP, D) * 0.5
    fx = O.Problem(4, O.ELLIPSOID, D).eval(X)
    V = np.random.default_rng(2).uniform(-3, 3, (NP, D))
    X2, V2, pair = O.cso_generation(seed, gen, X, V, fx, phi=phi)
    xbar = X.mean(axis=0)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for k in range(NP // 2):
        w, l = pair[2 * k], pair[2 * k + 1]
        for j in range(D):
            r = O.philox((1 + 2 * j, l, gen, 7 << 24), key)
            R1, R2 = O.u53(r[0], r[1]), O.u53(r[2], r[3])
            r3 = O.philox((2 + 2 * j, l, gen, 7 << 24), key)
            R3 = O.u53(r3[0], r3[1])
            v = R1 * V[l, j] + R2 * (X[w, j] - X[l, j]) + phi * R3 * (xbar[j] - X[l, j])
            assert V2[l, j] == pytest.approx(v, rel=1e-13, abs=1e-12)
            assert X2[l, j] == pytest.approx(min(100.0, max(-100.0, X[l, j] + v)), rel=1e-13, abs=1e-12)


def test_cso_collapsed_swarm_is_stationary():
    """All particles at one point (dyadic coordinates, so the mean is exact)
    with zero velocity: x_w - x_l = 0 and xbar - x_l = 0, so nothing moves."""
    NP, D = 20, 6
    X = np.tile([-3.0, -1.5, -0.25, 0.5, 1.75, 3.0], (NP, 1))  # dyadic: exact mean
    fx = O.Problem(1, O.GRIEWANK, D).eval(X)
    X2, V2, _ = O.cso_generation(9, 1, X, np.zeros((NP, D)), fx)
    assert np.array_equal(X2, X) and not V2.any()


def test_cso_control_run_reaches_success():
    """Control: CSO (NP = 100, phi = 0.1) on the shifted-rotated Griewank at
    D = 30 reaches 1e-8 within 3e5 evaluations, NP/2 counted per generation."""
    q = O.Problem(3, O.GRIEWANK, 30)
    r = O.run(q, O.make_alg(O.ALG_CSO, 100, 300000, w=0.1), 1)
    assert r["success"] and r["fes"] == 300000 and r["gens"] == (300000 - 100) // 50


# ---------------------------------------------------------------- PSODE
def test_psode_select_worked_example():
    """Pairwise/3 selection by hand: row 0's PSO offspring is better and is
    taken; row 1 ties (the DE survivor stays); row 2's PSO offspring is
    worse.  V is the DE displacement X3 - X in every row."""
    X = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    Y = np.array([[0.5, 0.25], [7.0, 8.0], [9.0, 10.0]])
    fy = np.array([1.0, 2.0, 5.0])
    X3 = np.array([[1.5, 2.0], [3.0, 4.5], [5.0, 6.0]])
    f3 = np.array([1.5, 2.0, 3.0])
    Xn, fn, V = O.psode_select(X, Y, fy, X3, f3)
    assert Xn.tolist() == [[0.5, 0.25], [3.0, 4.5], [5.0, 6.0]]
    assert fn.tolist() == [1.0, 2.0, 3.0]
    assert V.tolist() == [[0.5, 0.0], [0.0, 0.5], [0.0, 0.0]]


@pytest.mark.parametrize("fam,D,NP", [(O.ELLIPSOID, 10, 20), (O.RASTRIGIN, 7, 16)])
def test_psode_without_pso_coefficients_is_shade(fam, D, NP):
    """With w = c1 = c2 = 0 the PSO offspring is the population itself, never
    strictly better than the DE survivor, so PSODE follows SHADE's
    trajectory exactly: the best-so-far after g generations (2 NP
    evaluations each) equals SHADE's after g generations (NP each)."""
    q, G = O.Problem(11, fam, D), 12
    r6 = O.run(q, O.make_alg(O.ALG_PSODE, NP, NP + 2 * NP * G, w=0, c1=0, c2=0), 5,
               trace_cap=G + 1)
    r4 = O.run(q, O.make_alg(O.ALG_DE_SHADE, NP, NP + NP * G), 5, trace_cap=G + 1)
    assert np.array_equal(r6["trace_best"], r4["trace_best"])
    assert r6["trace_fes"].tolist() == [NP + 2 * NP * g for g in range(G + 1)]


def _psode_parts(q, seed, gen, s, w=0.7298, c1=1.49618, c2=1.49618):
    """One generation assembled from the pinned PSO and SHADE operators."""
    Y, _ = O.pso_move(seed, gen, s["X"], s["V"], s["P"], s["guide"], w=w, c1=c1, c2=c2)
    fy = q.eval(Y)
    P, fp, _ = O.pso_update(Y, fy, s["P"], s["fp"])
    guide = O.pso_guides(fp, 1)
    F, CR, kpb = O.shade_params(seed, gen, len(s["fx"]), s["MF"], s["MCR"])
    U, _ = O.shade_trials(seed, gen, s["X"], s["fx"], F, CR, kpb)
    fu = q.eval(U)
    MF, MCR, k, _ = O.shade_update(s["fx"], fu, F, CR, s["MF"], s["MCR"], s["k"])
    X3, f3, _, _, _ = O.de_select(seed, gen, s["X"], s["fx"], U, fu)
    take = fy < f3
    return dict(X=np.where(take[:, None], Y, X3), fx=np.where(take, fy, f3), V=X3 - s["X"], P=P,
                fp=fp, guide=guide, MF=MF, MCR=MCR, k=k, Y=Y, fy=fy, U=U, fu=fu)


def test_psode_generation_assembles_pinned_parts():
    """Three generations of the oracle's PSODE equal the same generations
    assembled from the separately pinned PSO move, pbest update, ring
    guides, SHADE operators and one-to-one selection (same counters), bit
    for bit: the PSO offspring moves from the population with the carried
    velocity, the velocity becomes the DE displacement, and the better of
    the two offspring sets survives."""
    NP, D, seed = 24, 9, 4242
    q = O.Problem(21, O.ACKLEY, D)
    X = O.init_population(seed, NP, D)
    fx = q.eval(X)
    MF, MCR, k = O.shade_memory()
    s = dict(X=X, fx=fx, MF=MF, MCR=MCR, k=k, **O.psode_start(X, fx))
    assert not s["V"].any() and np.array_equal(s["guide"], O.pso_guides(fx, 1))
    for gen in range(1, 4):
        want = _psode_parts(q, seed, gen, s)
        got = O.psode_generation(q, seed, gen, s["X"], s["fx"], s["V"], s["P"], s["fp"],
                                 s["guide"], s["MF"], s["MCR"], s["k"])
        for key in ("X", "fx", "V", "P", "fp", "guide", "MF", "MCR", "Y", "fy", "U", "fu"):
            assert np.array_equal(got[key], want[key]), (gen, key)
        assert got["k"] == want["k"]
        s = got


def test_psode_invariants_and_budget_accounting():
    """Per generation: fitness never worsens row by row and is f of the row;
    each row is its PSO offspring, its DE trial or its old self; personal
    bests never
    worsen and are f of their rows.  A budget ending inside a generation
    counts the PSO rows first, then the DE rows: orc_run's best-so-far is
    the minimum over exactly those evaluations."""
    NP, D, seed = 16, 6, 99
    q = O.Problem(5, O.GRIEWANK, D)
    X = O.init_population(seed, NP, D)
    fx = q.eval(X)
    MF, MCR, k = O.shade_memory()
    s = dict(X=X, fx=fx, MF=MF, MCR=MCR, k=k, **O.psode_start(X, fx))
    evals = [fx]
    for gen in range(1, 5):
        g = O.psode_generation(q, seed, gen, s["X"], s["fx"], s["V"], s["P"], s["fp"],
                               s["guide"], s["MF"], s["MCR"], s["k"])
        assert (g["fx"] <= s["fx"]).all() and (g["fp"] <= s["fp"]).all()
        assert np.array_equal(q.eval(g["X"]), g["fx"]) and np.array_equal(q.eval(g["P"]), g["fp"])
        for i in range(NP):  # pairwise/3: one of the three candidates
            assert any(np.array_equal(g["X"][i], c[i]) for c in (g["Y"], g["U"], s["X"]))
        evals.append(np.concatenate([g["fy"], g["fu"]]))
        s = g
    for extra in (NP // 2 + 3, NP + 5):  # last generation ends in the PSO / DE rows
        budget = NP + 2 * NP * 3 + extra
        r = O.run(q, O.make_alg(O.ALG_PSODE, NP, budget), seed)
        want = min(np.min(e) for e in evals[:4])
        want = min(want, np.min(evals[4][:extra]))
        assert r["best"] == want and r["fes"] == budget and r["gens"] == 4


def test_psode_control_run_reaches_success():
    """Control: PSODE (NP = 50, ring PSO with w = 0.7298, c1 = c2 = 1.49618,
    and SHADE) solves the shifted-rotated Rosenbrock at D = 10 to 1e-8
    within 1e5 evaluations, 2 NP counted per generation."""
    q = O.Problem(3, O.ROSENBROCK, 10)
    r = O.run(q, O.make_alg(O.ALG_PSODE, 50, 100000), 1)
    assert r["success"] and r["fes"] == 100000 and r["gens"] == 1000
