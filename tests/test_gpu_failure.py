"""Failure detection on the device: a bounded wait that runs out becomes a status code.

Every mbarrier wait of the tensor-core kernels is bounded (1 s of global time,
with a poll-count backstop). tctl_inject_wait_timeout makes the next
tensor-core GEMM launch of a context withhold its operand copies, so the MMA
thread's wait for the first stage waits on a barrier nothing arrives on and
runs out after about 1 ms. The kernel then skips its epilogue, frees its
tensor memory and returns; the host reads the error flag. The call must
return TCTL_E_NUMERIC and the same context must keep working: nothing faults,
traps or hangs, and the data path of a solve is never fed the unwritten
output.
"""
import numpy as np
import pytest

from oracle import formats as F
from oracle import fullgrid as fg
from oracle import operator as op
from paper_2006_09314_gb300.inputs import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the marker deselects these on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2006_09314_gb300 import tensorctl as T  # noqa: E402


def _bound(A, B, digits):
    return 8.0 * 2.0 ** (-7 * digits) * A.shape[1] * np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :]


def test_gemm_wait_timeout_returns_status_and_context_stays_usable():
    n, alpha, beta = 40, 0.5, 1e-2
    pr = make_problem(n, alpha, beta, 3, 4141)
    rng = np.random.default_rng(4141)
    A = rng.standard_normal((300, 700))
    B = rng.standard_normal((700, 200))
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with T.Context(pr.coeffs, n, alpha, beta, 1e-6) as ctx:
        ctx.inject_wait_timeout(1)
        with pytest.raises(T.TctlError) as ei:
            ctx.gemm(6, At, Bt)
        assert ei.value.code == -8 and "timed out" in str(ei.value)
        # the injection was used up: the same GEMM now runs, twice in a row
        for _ in range(2):
            C = ctx.gemm(6, At, Bt).cpu().numpy()
            assert np.all(np.abs(C - A @ B) <= _bound(A, B, 6))
        # a cancelled injection starves nothing
        ctx.inject_wait_timeout(3)
        ctx.inject_wait_timeout(0)
        C = ctx.gemm(6, At, Bt).cpu().numpy()
        assert np.all(np.abs(C - A @ B) <= _bound(A, B, 6))
        # and a full solve on the same context matches the oracle's exact solution
        x, st, code = ctx.pcg_solve(T.CP.from_numpy(pr.yw, pr.yU))
    assert code == 0
    lams, Vs = zip(*[op.eig(*op.assemble(pr.coeffs[l])) for l in range(3)])
    ustar = fg.solve_exact(F.cp_full(pr.yw, pr.yU), lams, Vs, alpha, beta)
    w, U = x.to_numpy()
    assert np.linalg.norm(F.cp_full(w, U) - ustar) <= 1e-6 * np.linalg.norm(ustar)


def test_inject_argument_errors():
    pr = make_problem(16, 0.5, 1e-2, 1, 1)
    with T.Context(pr.coeffs, 16, 0.5, 1e-2, 1e-6) as ctx:
        with pytest.raises(T.TctlError) as ei:
            ctx.inject_wait_timeout(-1)
        assert ei.value.code == -1
