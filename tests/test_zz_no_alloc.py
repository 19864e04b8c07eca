"""sevo_evaluate_noalloc: the evaluation entry point that allocates nothing.

For callers that cannot allocate device memory at the point of the call
(their memory manager owns the GPU's memory, or the call sits in a loop that
must not pay for an allocation), the library offers a variant of
sevo_evaluate whose scratch lives in a fixed device array.  This file runs
last so that, if it fails, a run that stops at the first failure has already
run every other test; it must pass alone in a fresh process too.
"""
import ctypes as C

import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu

# same tolerances as the evaluation parity tests: the variant runs the same
# kernels, so its output must agree with sevo_evaluate's within them
TOL = {0: 1e-12, 1: 2e-3, 2: 1e-4, 3: 1e-5}


@pytest.fixture(scope="module")
def S():
    import paper_2505_17430_gb300 as S
    S.build()
    return S


def _call_noalloc(S, p, X, out, prec):
    import torch
    return S.lib().sevo_evaluate_noalloc(p.h, C.c_void_p(X.data_ptr()), X.shape[0], p.D,
                                         X.stride(0), C.c_void_p(out.data_ptr()), prec,
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("fam", [2, 6, 7])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_noalloc_matches_evaluate_twice(S, fam, prec):
    import torch
    D, N = 30, 3000
    p = S.Problem(900 + fam, fam, D)
    X = torch.as_tensor(np.vstack([inputs.uniform_pop(N - 3, D, seed=fam),
                                   inputs.near(p.export()["o"], 3, 1e-4, seed=fam)])).cuda()
    ref = p.evaluate(X, prec=prec)          # also makes the problem's device copy
    torch.cuda.synchronize()
    for _ in range(2):                       # two calls in a row share the array
        out = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call_noalloc(S, p, X, out, prec) == 0
        torch.cuda.synchronize()
        a, b = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(b).all()
        assert (np.abs(a - b) <= TOL[prec] * np.maximum(np.abs(a), 1.0)).all()


def test_noalloc_rejects_oversize_and_missing_device_copy(S):
    import torch
    D = 10
    p = S.Problem(5, S.ACKLEY, D)
    N = 16384 + 1
    X = torch.zeros((N, D), dtype=torch.float64, device="cuda")
    out = torch.zeros(N, dtype=torch.float64, device="cuda")
    q = S.Problem(6, S.ACKLEY, D)            # never used on the device yet
    assert _call_noalloc(S, q, X[:10], out, 1) == -7
    p.evaluate(X[:10], prec=1)
    assert _call_noalloc(S, p, X, out, 1) == -6
    assert _call_noalloc(S, p, X[:16384], out, 1) == 0
