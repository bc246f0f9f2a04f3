"""Allocation-free eigendecomposition entry point (tctl_eig1d_noalloc).

Some callers cannot allocate device memory themselves (code running inside
another library's memory pool, a pipeline whose owner controls every
allocation, an embedded runtime with a fixed budget). For them the library
offers tctl_eig1d_noalloc, which computes the three 1D eigendecompositions
with scratch taken from a fixed device array inside the library instead of
cudaMalloc. These tests call it through the C ABI and check it against the
eigenpairs of a context built by tctl_setup (tctl_get_eigs), with the same
tolerances as the other eigenbasis tests, on two calls in a row (the shared
scratch keeps the previous call's contents). This file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2006_09314_gb300.inputs import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2006_09314_gb300 import tensorctl as T  # noqa: E402


def _noalloc(lib, coef, n, stream):
    lam = torch.full((3, n), float("nan"), dtype=torch.float64, device="cuda")
    V = torch.full((3, n, n), float("nan"), dtype=torch.float64, device="cuda")
    handle = stream.cuda_stream or 1  # torch's default stream is the legacy stream (handle 1)
    rc = lib.tctl_eig1d_noalloc(coef.data_ptr(), n, 0, lam.data_ptr(), V.data_ptr(),
                                ctypes.c_void_p(handle))
    return rc, lam, V


@pytest.mark.parametrize("n", [199, 256])
def test_noalloc_eigs_match_setup_on_two_calls(n):
    lib = T.load()
    pr = make_problem(n, 0.5, 1e-2, 1, 4242 + n)
    with T.Context(pr.coeffs, n, 0.5, 1e-2, 1e-6) as ctx:
        ref = [ctx.eigs(l) for l in range(3)]
    coef = torch.from_numpy(np.ascontiguousarray(pr.coeffs)).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        rc, lam, V = _noalloc(lib, coef, n, stream)
        assert rc == 0, T.tctl_last_error(None)
        torch.cuda.synchronize()
        lamh, Vh = lam.cpu().numpy(), V.cpu().numpy()
        for l in range(3):
            lr, Vr = ref[l]
            assert np.max(np.abs(lamh[l] - lr)) <= 1e-13 * lr.max()
            assert np.max(np.abs(Vh[l].T - Vr)) <= 5e-9


def test_noalloc_rejects_out_of_range_inputs():
    lib = T.load()
    stream = torch.cuda.current_stream()
    n = 300
    pr = make_problem(n, 0.5, 1e-2, 1, 1)
    coef = torch.from_numpy(np.ascontiguousarray(pr.coeffs)).cuda()
    rc, _, _ = _noalloc(lib, coef, n, stream)
    assert rc == -1 and "TCTL_EIG_NOALLOC_MAX_N" in T.tctl_last_error(None)
    n = 40
    pr = make_problem(n, 0.5, 1e-2, 1, 2)
    bad = pr.coeffs.copy()
    bad[2, 7] = -1.0
    coef = torch.from_numpy(np.ascontiguousarray(bad)).cuda()
    rc, _, _ = _noalloc(lib, coef, n, stream)
    assert rc == -2
    # a valid call after the failures still works
    coef = torch.from_numpy(np.ascontiguousarray(pr.coeffs)).cuda()
    rc, lam, _ = _noalloc(lib, coef, n, stream)
    torch.cuda.synchronize()
    assert rc == 0 and np.all(np.isfinite(lam.cpu().numpy()))
