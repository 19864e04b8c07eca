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


def _max_rows_large_d(D, comp):
    """The row limit the header states for TF32 / BF16X3 at D > 128."""
    def a(x):
        return (x + 255) // 256 * 256

    kpad, nsub = (D + 63) // 64 * 64, 4 * ((D + 127) // 128)

    def need(n):
        return a(4 * n) + 512 + a(a(4 * n * kpad) + a(104 * n * nsub) + (a(160 * n) if comp else 0))

    n = 1
    while need(n + 1) <= 3 << 20:
        n += 1
    return n


@pytest.mark.parametrize("fam,D,N", [(2, 30, 3000), (6, 30, 3000), (7, 30, 3000),
                                     (6, 257, 1100), (7, 257, 1100)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_noalloc_matches_evaluate_twice(S, fam, D, N, prec):
    """The variant runs the same kernels on the same input as sevo_evaluate,
    so its output is bit-identical, on two calls in a row that share the
    array; D = 257 takes the large-D path (converted operand, chunked GEMM,
    slice records and, for the composition, its staging in the array)."""
    import torch
    p = S.Problem(900 + fam, fam, D)
    X = torch.as_tensor(np.vstack([inputs.uniform_pop(N - 3, D, seed=fam),
                                   inputs.near(p.export()["o"], 3, 1e-4, seed=fam)])).cuda()
    ref = p.evaluate(X, prec=prec)          # also makes the problem's device copy
    torch.cuda.synchronize()
    a = ref.cpu().numpy()
    for _ in range(2):                       # two calls in a row share the array
        out = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call_noalloc(S, p, X, out, prec) == 0
        torch.cuda.synchronize()
        b = out.cpu().numpy()
        assert np.isfinite(b).all()
        assert np.array_equal(a, b)


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


@pytest.mark.parametrize("fam", [2, 7])
def test_noalloc_large_d_row_limit(S, fam):
    """At D > 128 in the tensor-core modes the limit is the one the header
    states (D = 1000: 423 rows, 414 for a composition): a call at the limit
    succeeds, one row more returns SEVO_ERR_UNSUPPORTED and writes nothing."""
    import torch
    D = 1000
    n = _max_rows_large_d(D, fam == 7)
    assert n == (414 if fam == 7 else 423)
    p = S.Problem(40 + fam, fam, D)
    X = torch.as_tensor(inputs.uniform_pop(n + 1, D, seed=fam)).cuda()
    p.evaluate(X[:8], prec=1)
    for prec in (1, 2):
        out = torch.full((n + 1,), -1.0, dtype=torch.float64, device="cuda")
        assert _call_noalloc(S, p, X, out, prec) == -6
        torch.cuda.synchronize()
        assert (out.cpu().numpy() == -1.0).all()
        assert _call_noalloc(S, p, X[:n], out, prec) == 0
        torch.cuda.synchronize()
        assert np.array_equal(out[:n].cpu().numpy(), p.evaluate(X[:n], prec=prec).cpu().numpy())
    # the FP64 and FP32 CUDA-core paths keep the plain limit
    out = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    assert _call_noalloc(S, p, X, out, 0) == 0
