"""GPU parity of the digit-split tensor-core GEMM (tctl_gemm) against FP64 numpy.

The split represents each entry of op(A) (op(B)) by d signed 7-bit digits
below one binary exponent per row (column); the error of an entry of C is
bounded by about 2^-7d * K * max_k |A(i, k)| * max_k |B(k, j)| (truncation of
both operands plus the dropped digit products; the accumulation is exact in
the leading levels). Integers that fit the digits are exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the marker deselects these on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2006_09314_gb300 import tensorctl as T  # noqa: E402
from paper_2006_09314_gb300.inputs import make_problem  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    pr = make_problem(16, 0.5, 1e-2, 1, 1)
    c = T.Context(pr.coeffs, 16, 0.5, 1e-2, 1e-6)
    yield c
    c.close()


def _bound(A, B, digits, ta, tb):
    opA = A.T if ta else A
    opB = B.T if tb else B
    K = opA.shape[1]
    return 8.0 * 2.0 ** (-7 * digits) * K * np.abs(opA).max(1)[:, None] * np.abs(opB).max(0)[None, :]


@pytest.mark.parametrize("m,n,k,ta,tb", [(300, 77, 1000, False, False), (129, 65, 16, True, False),
                                         (64, 200, 2048, False, True), (1, 1, 5, True, True),
                                         (513, 33, 511, False, False), (40, 700, 37, True, True)])
@pytest.mark.parametrize("digits", [3, 4, 6])
def test_tc_gemm_error_bound(ctx, m, n, k, ta, tb, digits):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((k, m) if ta else (m, k)) * np.exp(rng.uniform(-8, 8, (k, 1) if ta else (m, 1)))
    B = rng.standard_normal((n, k) if tb else (k, n)) * np.exp(rng.uniform(-8, 8, (1, k) if tb else (1, n)))
    ref = (A.T if ta else A) @ (B.T if tb else B)
    C = ctx.gemm(digits, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), trans_a=ta, trans_b=tb)
    err = np.abs(C.cpu().numpy() - ref)
    assert np.all(err <= _bound(A, B, digits, ta, tb))


def test_tc_gemm_integers_exact_alpha_beta(ctx):
    rng = np.random.default_rng(3)
    A = rng.integers(-1000, 1001, (257, 700)).astype(np.float64)
    B = rng.integers(-1000, 1001, (700, 130)).astype(np.float64)
    C0 = rng.integers(-5, 6, (257, 130)).astype(np.float64)
    Ct = torch.from_numpy(C0.copy()).cuda()
    ctx.gemm(6, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C=Ct, alpha=2.0, beta=-0.5)
    assert np.array_equal(Ct.cpu().numpy(), 2.0 * (A @ B) - 0.5 * C0)


def test_tc_gemm_zero_rows_and_nan(ctx):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((200, 300))
    B = rng.standard_normal((300, 90))
    A[5] = 0.0
    B[:, 7] = 0.0
    A[9, 17] = np.nan
    C = ctx.gemm(6, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    assert np.all(C[5] == 0.0) and np.all(C[:, 7][np.arange(200) != 9] == 0.0)
    assert np.all(np.isnan(C[9]))
    ok = np.ones(200, bool)
    ok[9] = False
    ref = A[ok] @ B
    assert np.all(np.abs(C[ok] - ref) <= _bound(A[ok], B, 6, False, False))


@pytest.mark.parametrize("digits", [3, 6])
def test_tc_gemm_extreme_exponents(ctx, digits):
    """Rows of A scaled by 2^-1030 (subnormal), 2^-600, 1 and 2^600, columns of B
    by 1 and 2^400: the digit cut reads exponents and significands from the
    IEEE-754 fields and the epilogue assembles the result's fields (results
    from about 2^1000 down to subnormal ones, which take the FP64 route)."""
    rng = np.random.default_rng(11 + digits)
    m, n, k = 160, 70, 300
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((k, n))
    sa = np.array([-1030.0, -600.0, 0.0, 600.0])[np.arange(m) % 4]
    sb = np.array([0.0, 400.0])[np.arange(n) % 2]
    A = A * np.ldexp(1.0, sa.astype(int))[:, None]
    B = B * np.ldexp(1.0, sb.astype(int))[None, :]
    assert np.all(np.abs(A[0::4]) < 2.0 ** -1022)  # subnormal rows
    ref = A @ B
    C = ctx.gemm(digits, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    assert np.all(np.isfinite(C))
    assert np.all(np.abs(C - ref) <= _bound(A, B, digits, False, False))


@pytest.mark.parametrize("m,n,k", [(70, 30, 50), (2048, 5, 2048), (3000, 1, 126), (500, 16, 700),
                                   (257, 9, 33)])
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_fp64_path_digits0(ctx, m, n, k, ta, tb):
    """FP64 FMA kernels (exact-work 16 x 16 output tiles; skinny kernels for n <= 16) vs numpy."""
    rng = np.random.default_rng(m + 10 * n + 100 * k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C0 = rng.standard_normal((m, n))
    Ct = torch.from_numpy(C0.copy()).cuda()
    ctx.gemm(0, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C=Ct, trans_a=ta, trans_b=tb,
             alpha=1.5, beta=0.5)
    ref = 1.5 * ((A.T if ta else A) @ (B.T if tb else B)) + 0.5 * C0
    assert np.allclose(Ct.cpu().numpy(), ref, rtol=0, atol=1e-13 * k)


def test_tc_gemm_argument_errors(ctx):
    lib = T.load()
    assert lib.tctl_gemm(ctx.handle, 5, 0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4) == -1
    assert lib.tctl_gemm(ctx.handle, 6, 0, 0, 4, 4, 4, 1.0, None, 2, None, 4, 0.0, None, 4) == -1


@pytest.mark.parametrize("k,ra,rb,n", [(700, 5, 37, 70), (2048, 12, 36, 126), (33, 1, 1, 1),
                                       (257, 64, 3, 130)])
@pytest.mark.parametrize("digits", [4, 6])
def test_gemm_kr_equals_stored_product(ctx, k, ra, rb, n, digits):
    """The Khatri-Rao operand formed inside the digit split gives, bit for bit, what
    tctl_gemm gives on the stored product (same split, same kernel), and meets the
    digit-split error bound against FP64 numpy."""
    g = torch.Generator().manual_seed(k * 7 + ra * 3 + rb + digits)
    X = torch.randn(ra, k, generator=g, dtype=torch.float64).cuda()
    Y = torch.randn(rb, k, generator=g, dtype=torch.float64).cuda()
    B = torch.randn(n, k, generator=g, dtype=torch.float64).cuda()
    C0 = torch.randn(n, ra * rb, generator=g, dtype=torch.float64).cuda()
    C = ctx.gemm_kr(digits, X, Y, B, C=C0.clone(), alpha=0.75, beta=-0.5)
    KR = (Y[:, None, :] * X[None, :, :]).reshape(ra * rb, k).contiguous()  # row a + ra b
    Cs = C0.clone()
    # column-major: Cs^T (m x n) = 0.75 KR^T(k x m)^T B (k x n) - 0.5 Cs^T, trans_a = 1
    lib = T.load()
    assert lib.tctl_gemm(ctx.handle, digits, 1, 0, ra * rb, n, k, 0.75, KR.data_ptr(), k,
                         B.data_ptr(), k, -0.5, Cs.data_ptr(), ra * rb) == 0
    torch.cuda.synchronize()
    assert torch.equal(C, Cs)
    ref = 0.75 * (B.cpu().numpy() @ KR.cpu().numpy().T) - 0.5 * C0.cpu().numpy()
    bound = _bound(KR.cpu().numpy().T, B.cpu().numpy().T, digits, True, False).T
    assert np.all(np.abs(C.cpu().numpy() - ref) <= bound * 0.75 + 1e-15 * np.abs(C0.cpu().numpy()))


def test_gemm_kr_fp64_path_and_errors(ctx):
    g = torch.Generator().manual_seed(5)
    k, ra, rb, n = 300, 7, 9, 11
    X = torch.randn(ra, k, generator=g, dtype=torch.float64).cuda()
    Y = torch.randn(rb, k, generator=g, dtype=torch.float64).cuda()
    B = torch.randn(n, k, generator=g, dtype=torch.float64).cuda()
    C = ctx.gemm_kr(0, X, Y, B)
    KR = (Y[:, None, :] * X[None, :, :]).reshape(ra * rb, k)
    ref = B.cpu().numpy() @ KR.cpu().numpy().T
    assert np.abs(C.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    lib = T.load()
    assert lib.tctl_gemm_kr(ctx.handle, 5, 4, 2, 2, 4, 1.0, None, 4, None, 4, None, 4, 0.0, None, 4) == -1
    assert lib.tctl_gemm_kr(ctx.handle, 6, 4, 2, 2, 4, 1.0, X.data_ptr(), 2, Y.data_ptr(), 4,
                            B.data_ptr(), 4, 0.0, C.data_ptr(), 4) == -1


def test_autotuned_chunks_keep_the_error_bound():
    """The tile autotuner (opts.tune = 1) picks the contracted length per CTA
    of each shape class by timing 64, 128 and 256; every choice keeps the digit
    split's error bound and gives the fixed-chunk (tune = 0) result to within it."""
    pr = make_problem(16, 0.5, 1e-2, 1, 1)
    rng = np.random.default_rng(17)
    A = rng.standard_normal((700, 2048))
    B = rng.standard_normal((2048, 60))
    out = []
    for tune in (1, 0):
        with T.Context(pr.coeffs, 16, 0.5, 1e-2, 1e-6, opts=T.tctl_default_opts(tune=tune)) as c:
            out.append(c.gemm(6, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy())
    bound = _bound(A, B, 6, False, False)
    ref = A @ B
    for C in out:
        assert np.all(np.abs(C - ref) <= bound)
    assert np.all(np.abs(out[0] - out[1]) <= 2 * bound)
    table = T.tctl_tune_report()
    assert table and all(t["k_per_cta"] in (64, 128, 256) for t in table)
    mine = [t for t in table if t["digits"] == 6 and t["k_steps"] == 128]
    assert mine and all(len(t["ms"]) == 3 and min(x for x in t["ms"] if x > 0) > 0 for t in mine)
