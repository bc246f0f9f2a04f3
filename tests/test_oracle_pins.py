"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself or with the GPU library: every
expected value is a closed form, a brute-force computation on a tiny grid, an
invariant, or a special case the paper names.
"""
import math
import os

import numpy as np
import pytest

from oracle import expsum as es
from oracle import formats as F
from oracle import fullgrid as fg
from oracle import operator as op
from oracle import pcg as opcg
from oracle import truncation as tr
from paper_2006_09314_gb300.inputs import make_problem, coefficient_half_points

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _eig3(pr, driver="stemr"):
    lams, Vs = [], []
    for l in range(3):
        lam, V = op.eig(*op.assemble(pr.coeffs[l]), driver=driver)
        lams.append(lam)
        Vs.append(V)
    return lams, Vs


# ---------------------------------------------------------------- P1 closed form
@pytest.mark.parametrize("n", [8, 63, 200])
def test_P1_laplacian_closed_form(n):
    """a == 1: lambda_k = 4/h^2 sin^2(k pi h/2), v_k = sqrt(2h) sin(k pi x_i) (Section 3.5)."""
    h = 1.0 / (n + 1)
    d, e = op.assemble(np.ones(n + 1))
    lam, V = op.eig(d, e)
    k = np.arange(1, n + 1)
    lam_cf = 4.0 / h ** 2 * np.sin(k * math.pi * h / 2.0) ** 2
    # backward-stable eigensolvers: absolute error ~ eps * ||A||
    assert np.max(np.abs(lam - lam_cf)) < 1e-14 * lam_cf.max()
    x = np.arange(1, n + 1) * h
    Vcf = math.sqrt(2.0 * h) * np.sin(np.outer(x, k) * math.pi)
    Vcf = Vcf * np.where(op.sign_weights(n) @ Vcf < 0, -1.0, 1.0)[None, :]
    assert np.max(np.abs(V - Vcf)) < 1e-11


def test_P1_golden_printed_formula():
    vals = np.loadtxt(os.path.join(GOLDEN, "laplacian_eigs_n8.txt"))
    lam, _ = op.eig(*op.assemble(np.ones(9)))
    assert np.max(np.abs(lam - vals)) < 1e-14 * vals.max()


def test_paper_end_rows_coincide_for_unit_coefficient():
    d0, e0 = op.assemble(np.ones(17))
    d1, e1 = op.assemble(np.ones(17), paper_end_rows=True)
    assert np.array_equal(d0, d1) and np.array_equal(e0, e1)
    a = coefficient_half_points(16, 0.3)
    d1, _ = op.assemble(a, paper_end_rows=True)
    h2 = (1.0 / 17) ** 2
    assert d1[0] == pytest.approx(2 * a[1] / h2) and d1[-1] == pytest.approx(2 * a[15] / h2)


def test_assembly_matches_weak_form_stencil():
    """Diagonal (a_{i-1/2}+a_{i+1/2})/h^2, off-diagonal -a_{i+1/2}/h^2, SPD."""
    n = 12
    a = coefficient_half_points(n, 1.1)
    d, e = op.assemble(a)
    A = op.dense(d, e)
    h = 1.0 / (n + 1)
    y = np.random.default_rng(0).standard_normal(n)
    yp = np.concatenate([[0.0], y, [0.0]])
    flux = a * (yp[1:] - yp[:-1]) / h          # a_{i-1/2} (y_i - y_{i-1})/h, i=1..n+1
    Ay_ref = -(flux[1:] - flux[:-1]) / h
    assert np.allclose(A @ y, Ay_ref, rtol=1e-13, atol=1e-9)
    assert np.all(np.linalg.eigvalsh(A) > 0)


# ---------------------------------------------------------------- P2 alpha = 1
@pytest.mark.parametrize("n,beta", [(10, 1e-2), (16, 1.0)])
def test_P2_alpha_one_local_operator(n, beta):
    """alpha = 1: (A^-1 + beta A) u = y  <=>  u + beta A(A u) = A y, A by 7-point stencil."""
    pr = make_problem(n, 1.0, beta, 3, 11)
    lams, Vs = _eig3(pr)
    Y = F.cp_full(pr.yw, pr.yU)
    U = fg.solve_exact(Y, lams, Vs, 1.0, beta)
    Au = op.stencil_apply(pr.coeffs, U)
    lhs = U + beta * op.stencil_apply(pr.coeffs, Au)
    rhs = op.stencil_apply(pr.coeffs, Y)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-11


# ---------------------------------------------------------------- P3 brute force
@pytest.mark.parametrize("n,alpha,beta", [(4, 0.5, 1e-2), (5, 0.25, 1.0), (6, 0.75, 1e-4)])
def test_P3_dense_kronecker_sum(n, alpha, beta):
    pr = make_problem(n, alpha, beta, 2, 21)
    mats = [op.dense(*op.assemble(pr.coeffs[l])) for l in range(3)]
    K = op.kron_sum_dense(mats)
    mu, Q = np.linalg.eigh(K)
    F2K = (Q * (mu ** -alpha + beta * mu ** alpha)[None, :]) @ Q.T
    Y = F.cp_full(pr.yw, pr.yU)
    u_bf = np.linalg.solve(F2K, Y.reshape(-1)).reshape(Y.shape)
    lams, Vs = _eig3(pr)
    u = fg.solve_exact(Y, lams, Vs, alpha, beta)
    assert np.linalg.norm(u - u_bf) / np.linalg.norm(u_bf) < 1e-12
    # the stencil is the same operator
    X = np.random.default_rng(1).standard_normal(Y.shape)
    assert np.allclose(op.stencil_apply(pr.coeffs, X).reshape(-1), K @ X.reshape(-1), rtol=1e-12)


# ---------------------------------------------------------------- state equation pins
@pytest.mark.parametrize("n", [10, 16])
def test_state_alpha_one_inverts_the_stencil(n):
    """State equation (Section 3.1) at alpha = 1: y = A^-1 u, so the 7-point stencil of y is u."""
    pr = make_problem(n, 1.0, 1e-2, 3, 131)
    lams, Vs = _eig3(pr)
    U = F.cp_full(pr.yw, pr.yU)
    Y = fg.state_exact(U, lams, Vs, 1.0)
    assert np.linalg.norm(op.stencil_apply(pr.coeffs, Y) - U) / np.linalg.norm(U) < 1e-11
    # beta_p scales the state linearly
    Y3 = fg.state_exact(U, lams, Vs, 1.0, beta_state=3.0)
    assert np.linalg.norm(Y3 - 3.0 * Y) <= 1e-14 * np.linalg.norm(Y3)


def test_state_half_power_composes_to_the_inverse():
    """A^-1/2 applied twice is A^-1: the stencil of the twice-applied state returns u."""
    n = 12
    pr = make_problem(n, 0.5, 1e-2, 3, 132)
    lams, Vs = _eig3(pr)
    U = F.cp_full(pr.yw, pr.yU)
    Y2 = fg.state_exact(fg.state_exact(U, lams, Vs, 0.5), lams, Vs, 0.5)
    assert np.linalg.norm(op.stencil_apply(pr.coeffs, Y2) - U) / np.linalg.norm(U) < 1e-11
    # and the quarter power four times
    Y4 = U
    for _ in range(4):
        Y4 = fg.state_exact(Y4, lams, Vs, 0.25)
    assert np.linalg.norm(op.stencil_apply(pr.coeffs, Y4) - U) / np.linalg.norm(U) < 1e-11


@pytest.mark.parametrize("n,alpha", [(4, 0.5), (5, 0.25), (6, 0.75)])
def test_state_dense_kronecker_sum(n, alpha):
    """n <= 6: A^-alpha u by eigh of the dense n^3 x n^3 Kronecker sum, mu^-alpha."""
    pr = make_problem(n, alpha, 1e-2, 2, 133)
    mats = [op.dense(*op.assemble(pr.coeffs[l])) for l in range(3)]
    mu, Q = np.linalg.eigh(op.kron_sum_dense(mats))
    U = F.cp_full(pr.yw, pr.yU)
    ref = ((Q * (mu ** -alpha)[None, :]) @ (Q.T @ U.reshape(-1))).reshape(U.shape)
    lams, Vs = _eig3(pr)
    Y = fg.state_exact(U, lams, Vs, alpha)
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) < 1e-12


# ---------------------------------------------------------------- P4 invariants
def test_P4_invariants():
    n, alpha, beta = 12, 0.5, 1e-2
    pr = make_problem(n, alpha, beta, 3, 31)
    lams, Vs = _eig3(pr)
    for lam, V in zip(lams, Vs):
        assert np.all(lam > 0)
        assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-13
        assert np.all(op.sign_weights(n) @ V > 0)
    S = fg.spectral_sum(lams)
    f2 = fg.F2(S, alpha, beta)
    assert np.all(f2 >= 2 * math.sqrt(beta) * (1 - 1e-15))
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal((2, n, n, n))
    Fx = fg.apply_spectral(f2, x, Vs)
    Fy = fg.apply_spectral(f2, y, Vs)
    assert abs(np.sum(x * Fy) - np.sum(Fx * y)) < 1e-12 * np.linalg.norm(Fx) * np.linalg.norm(y)
    assert np.sum(x * Fx) > 0
    u1 = fg.solve_exact(x, lams, Vs, alpha, beta)
    u2 = fg.solve_exact(y, lams, Vs, alpha, beta)
    u12 = fg.solve_exact(2 * x - 3 * y, lams, Vs, alpha, beta)
    assert np.linalg.norm(u12 - (2 * u1 - 3 * u2)) < 1e-12 * np.linalg.norm(u12)
    # F2(A) u* = y
    assert np.linalg.norm(fg.apply_spectral(f2, u1, Vs) - x) < 1e-12 * np.linalg.norm(x)


# ---------------------------------------------------------------- P5 small alpha
def test_P5_small_alpha_limit():
    """alpha -> 0: F2 -> (1+beta) I, u* -> y/(1+beta) (remark after Table iternums_precond_3d)."""
    n, beta = 10, 0.3
    pr = make_problem(n, 1e-7, beta, 3, 41)
    lams, Vs = _eig3(pr)
    Y = F.cp_full(pr.yw, pr.yU)
    u = fg.solve_exact(Y, lams, Vs, 1e-7, beta)
    assert np.linalg.norm(u - Y / (1 + beta)) / np.linalg.norm(Y) < 1e-5


# ---------------------------------------------------------------- P6 second route
@pytest.mark.parametrize("n", [16, 100])
def test_P6_two_lapack_drivers(n):
    a = coefficient_half_points(n, 2.0)
    d, e = op.assemble(a)
    l1, V1 = op.eig(d, e, driver="stemr")
    l2, V2 = op.eig(d, e, driver="dense")
    assert np.max(np.abs(l1 - l2)) < 1e-13 * l2.max()
    assert np.max(np.abs(V1 - V2)) < 1e-9


# ---------------------------------------------------------------- formats (Appendix 1)
def _rand_cp(rng, n, R):
    return rng.standard_normal(R), [rng.standard_normal((n, R)) for _ in range(3)]


def test_canonical_inner_hadamard_axpy_brute_force():
    rng = np.random.default_rng(5)
    n = 7
    w1, U1 = _rand_cp(rng, n, 4)
    w2, U2 = _rand_cp(rng, n, 3)
    X1, X2 = F.cp_full(w1, U1), F.cp_full(w2, U2)
    # definition check of the expansion on one entry
    i, j, k = 2, 5, 1
    assert X1[i, j, k] == pytest.approx(sum(w1[t] * U1[0][i, t] * U1[1][j, t] * U1[2][k, t] for t in range(4)))
    assert F.cp_inner(w1, U1, w2, U2) == pytest.approx(np.sum(X1 * X2), rel=1e-12)
    hw, hU = F.cp_hadamard(w1, U1, w2, U2)
    assert len(hw) == 12
    assert np.allclose(F.cp_full(hw, hU), X1 * X2, rtol=1e-12, atol=1e-12)
    aw, aU = F.cp_axpby(2.0, w1, U1, -0.5, w2, U2)
    assert np.allclose(F.cp_full(aw, aU), 2 * X1 - 0.5 * X2, atol=1e-12)
    assert F.cp_norm(w1, U1) == pytest.approx(np.linalg.norm(X1), rel=1e-12)


def test_streamed_error_matches_full():
    rng = np.random.default_rng(6)
    n, alpha, beta = 9, 0.5, 1e-2
    pr = make_problem(n, alpha, beta, 3, 51)
    lams, Vs = _eig3(pr)
    Y = F.cp_full(pr.yw, pr.yU)
    ustar = fg.solve_exact(Y, lams, Vs, alpha, beta)
    uw, uU = _rand_cp(rng, n, 2)
    uw = 1e-3 * uw
    u = ustar + F.cp_full(uw, uU)
    # u as canonical: ustar is not canonical; instead compare a canonical u
    yw, yUh = F.cp_to_eigenbasis(pr.yw, pr.yU, Vs)
    vw, vUh = F.cp_to_eigenbasis(uw, uU, Vs)
    full = np.linalg.norm(F.cp_full(uw, uU) - ustar) / np.linalg.norm(ustar)
    streamed = fg.streamed_rel_error(lams, yw, yUh, vw, vUh, alpha, beta)
    assert streamed == pytest.approx(full, rel=1e-10)
    assert u.shape == Y.shape
    # several solutions in one pass: each against the error of its full expansion
    w2, U2 = _rand_cp(rng, n, 3)
    w2 = 3e-2 * w2
    vw2, vU2h = F.cp_to_eigenbasis(w2, U2, Vs)
    full2 = np.linalg.norm(F.cp_full(w2, U2) - ustar) / np.linalg.norm(ustar)
    many = fg.streamed_rel_errors(lams, yw, yUh, [(vw, vUh), (vw2, vU2h)], alpha, beta)
    assert many[0] == pytest.approx(full, rel=1e-10) and many[1] == pytest.approx(full2, rel=1e-10)


# ---------------------------------------------------------------- sinc exp-sums (Section 3.4)
def _spectrum(n, seed):
    pr = make_problem(n, 0.5, 1e-2, 1, seed)
    lams, _ = _eig3(pr)
    return lams


@pytest.mark.parametrize("alpha,beta", [(0.25, 1e-4), (0.5, 1e-2), (0.75, 1.0), (1.0, 1e-2)])
def test_sinc_F2_meets_target_on_spectrum(alpha, beta):
    lams = _spectrum(16, 61)
    S = fg.spectral_sum(lams).ravel()
    smin, smax = S.min(), S.max()
    for delta in (1e-6, 1e-8):
        rep = es.F2_expsum(alpha, beta, smin, smax, delta)
        err_all = es.measured_rel_error(rep, alpha, beta, S)
        err_dense = es.measured_rel_error(rep, alpha, beta, es.spectral_sample(smin, smax, 4000))
        assert err_all < delta and err_dense < delta


def test_sinc_single_power_exponential_convergence():
    """s^-g by the trapezoid rule: error decays exponentially in the number of terms."""
    smin, smax = 30.0, 3e6
    s = es.spectral_sample(smin, smax, 3000)
    errs, ranks = [], []
    for delta in (1e-3, 1e-5, 1e-7, 1e-9):
        tl, h, r = es.sinc_params(0.5, delta, smin, smax, left_gain=smax ** 0.5, right_q=delta * math.gamma(0.5) * smin ** 0.5 / 4)
        t, w = es.sinc_terms(0.5, tl, h, r)
        approx = (w[None, :] * np.exp(-np.outer(s, t))).sum(1)
        errs.append(np.max(np.abs(approx - s ** -0.5) * s ** 0.5))
        ranks.append(r)
    assert all(e < d for e, d in zip(errs, (1e-3, 1e-5, 1e-7, 1e-9)))
    # r grows roughly linearly in |log eps| (R <= C |log eps|, Section 3.4)
    inc = np.diff(ranks)
    assert np.all(inc > 0) and inc.max() < 3 * inc.min() + 4


def test_operator_factors_expand_to_expsum_and_rank_bound():
    """Canonical factors of D^-alpha + beta D*D^(alpha-1): rank r1 + 3 r2 (rank(D^alpha) <= 3R)."""
    n, alpha, beta = 6, 0.5, 1e-2
    lams = _spectrum(n, 71)
    S = fg.spectral_sum(lams)
    rep = es.F2_expsum(alpha, beta, S.min(), S.max(), 1e-7)
    w, U = es.operator_cp(rep, lams)
    assert len(w) == len(rep["t1"]) + 3 * len(rep["t2"])
    assert np.allclose(F.cp_full(w, U), es.F2_expsum_eval(rep, S.ravel()).reshape(S.shape), rtol=1e-12)
    rep1 = es.F2_expsum(1.0, beta, S.min(), S.max(), 1e-7)
    w1, U1 = es.operator_cp(rep1, lams)
    assert len(w1) == len(rep1["t1"]) + 3
    assert np.allclose(F.cp_full(w1, U1), es.F2_expsum_eval(rep1, S.ravel()).reshape(S.shape), rtol=1e-12)


def test_preconditioner_positive_and_spectrally_close():
    lams = _spectrum(24, 81)
    S = fg.spectral_sum(lams)
    for alpha, beta in [(0.5, 1e-2), (0.25, 1e-4), (0.75, 1.0)]:
        f2 = fg.F2(S, alpha, beta)
        th, p = es.precond_expsum(alpha, beta, S.min(), S.max(), 24)
        assert np.all(p >= 0)
        P = es.precond_eval(th, p, S.ravel()).reshape(S.shape)
        ratio = P * f2
        assert ratio.min() > 0.99 and ratio.max() < 1.01
        w, U = es.precond_cp(th, p, lams)
        if S.size <= 24 ** 3:
            assert np.allclose(F.cp_full(w, U), P, rtol=1e-10)


# ---------------------------------------------------------------- trunc (Appendix 1)
def _orth(rng, n, r):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def test_trunc_recovers_exact_low_tucker_rank():
    rng = np.random.default_rng(91)
    n = 10
    Q = [_orth(rng, n, r) for r in (2, 3, 2)]
    core = rng.standard_normal((2, 3, 2))
    X = F.tucker_full(core, Q)
    # canonical form with redundant, split terms: every core entry twice with halves
    w, U = [], [[], [], []]
    for a in range(2):
        for b in range(3):
            for c in range(2):
                for frac in (0.25, 0.75):
                    w.append(frac * core[a, b, c])
                    U[0].append(Q[0][:, a] * 3.0)
                    U[1].append(Q[1][:, b])
                    U[2].append(Q[2][:, c] / 3.0)
    U = [np.array(u).T for u in U]
    cw, cU = tr.trunc(np.array(w), U, 1e-10)
    assert np.linalg.norm(F.cp_full(cw, cU) - X) < 1e-12 * np.linalg.norm(X)
    assert len(cw) <= 2 * 2  # T2C: rank <= min(r1, r2) * r3
    tcore, tQ = tr.trunc(np.array(w), U, 1e-10, output="tucker")
    assert tcore.shape == (2, 3, 2)


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6])
def test_trunc_error_bound_and_reduction(eps):
    rng = np.random.default_rng(92)
    n, R = 20, 30
    w = np.exp(-1.0 * np.arange(R)) * rng.choice([-1, 1], R)
    U = [rng.standard_normal((n, R)) for _ in range(3)]
    X = F.cp_full(w, U)
    tw, tU = tr.trunc(w, U, eps)
    err = np.linalg.norm(F.cp_full(tw, tU) - X) / np.linalg.norm(X)
    assert err <= eps
    assert err > 1e-3 * eps  # it really truncated
    core, Q = tr.trunc(w, U, eps, output="tucker")
    errT = np.linalg.norm(F.tucker_full(core, Q) - X) / np.linalg.norm(X)
    assert errT <= eps
    for q in Q:
        assert np.max(np.abs(q.T @ q - np.eye(q.shape[1]))) < 1e-12


def test_trunc_with_cancellation_is_relative_to_result():
    """X - (X + d): the sum is small, trunc must keep eps relative to ||result||."""
    rng = np.random.default_rng(93)
    n, R = 8, 6
    w, U = _rand_cp(rng, n, R)
    w2, U2 = _rand_cp(rng, n, 2)
    aw, aU = F.cp_axpby(1.0, w, U, -1.0, w, U)
    dw, dU = F.cp_axpby(1.0, aw, aU, 1e-4, w2, U2)
    ref = F.cp_full(dw, dU)
    tw, tU = tr.trunc(dw, dU, 1e-6)
    assert np.linalg.norm(F.cp_full(tw, tU) - ref) <= 1e-6 * np.linalg.norm(ref)


# ---------------------------------------------------------------- Algorithm 1
@pytest.mark.parametrize("n,alpha,beta", [(8, 0.5, 1e-2), (12, 0.25, 1e-4), (10, 0.75, 1.0)])
def test_pcg_converges_to_exact_solution(n, alpha, beta):
    pr = make_problem(n, alpha, beta, 3, 101)
    lams, Vs = _eig3(pr)
    S = fg.spectral_sum(lams)
    rep = es.F2_expsum(alpha, beta, S.min(), S.max(), 1e-8)
    th, p = es.precond_expsum(alpha, beta, S.min(), S.max(), 24)
    xw, xU, info = opcg.pcg(es.operator_cp(rep, lams), es.precond_cp(th, p, lams), Vs,
                             pr.yw, pr.yU, 1e-6, rtol=1e-7)
    assert info["rel_res"] <= 1e-7 and info["iters"] <= 5
    ustar = fg.solve_exact(F.cp_full(pr.yw, pr.yU), lams, Vs, alpha, beta)
    err = np.linalg.norm(F.cp_full(xw, xU) - ustar) / np.linalg.norm(ustar)
    assert err < 2e-6


def _pcg_iters(n, alpha, beta, K, eps, rtol):
    pr = make_problem(n, alpha, beta, 2, 111)
    lams, Vs = _eig3(pr)
    S = fg.spectral_sum(lams)
    rep = es.F2_expsum(alpha, beta, S.min(), S.max(), 1e-8)
    th, p = es.precond_expsum(alpha, beta, S.min(), S.max(), K)
    _, _, info = opcg.pcg(es.operator_cp(rep, lams), es.precond_cp(th, p, lams), Vs,
                          pr.yw, pr.yU, eps, rtol=rtol, kmax=60)
    return info["iters"]


def test_pcg_iterations_bounded_independently_of_n():
    """A spectrally equivalent preconditioner keeps the count bounded in n (Tables iter_2d, iter_3d)."""
    its = [_pcg_iters(n, 0.5, 1e-2, 24, 1e-6, 1e-6) for n in (6, 10, 16)]
    assert max(its) <= 3, its


def test_pcg_iterations_fall_with_alpha():
    """Small alpha solves fastest: A^(+-alpha) -> I (remark after Table iternums_precond_3d)."""
    lo = _pcg_iters(10, 0.1, 1.0, 4, 1e-7, 1e-6)
    hi = _pcg_iters(10, 0.9, 1.0, 4, 1e-7, 1e-6)
    assert lo < hi, (lo, hi)
