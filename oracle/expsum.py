"""Separable (exponential-sum) representations of spectral functions (oracle).

Section 3.4 represents the negative power through the Laplace transform
("Laplace_transf") and a sinc quadrature on the real axis
("sinc_Laplace_tr_Dalpha"):

    s^-g = 1/Gamma(g) * int_0^inf t^(g-1) e^(-t s) dt
         = 1/Gamma(g) * int_R exp(g tau - e^tau s) dtau          (t = e^tau)
        ~= sum_k w_k exp(-t_k s),  tau_k = tau_lo + k h,  t_k = e^tau_k,
           w_k = h exp(g tau_k) / Gamma(g),                       k = 0..r-1,

and the positive power through the pointwise (Hadamard) split
D^alpha = D .* D^(alpha-1) with the rank-3 tensor D = lambda_i + lambda_j + lambda_k,
so rank(D^alpha) <= 3 R. Each exponential is separable,
exp(-t s) = exp(-t lambda_i) exp(-t lambda_j) exp(-t lambda_k).

The paper gives neither the quadrature parameters nor the meaning of the rank.
Reading used here (the same rule is implemented independently in the GPU
library): the trapezoid step is h = 2 pi d / ln(1/delta) with d = 1.2 (inside
the analyticity strip |Im tau| < pi/2 of the integrand); the left end is where
the omitted tail exp(g tau_a)/(g Gamma(g)) times max(m/F) falls below delta/4;
the right end is where the omitted tail t_b^(g-1) e^(-t_b s)/(s Gamma(g)) times
m/F falls below delta/4 at s = s_min; here F is the function whose relative
error is controlled (F2 for the operator) and m the multiplier of the term
(1 for s^-alpha, beta*s for s^(alpha-1)). delta is the target maximal relative
error of F2 on the spectral interval; the achieved error is measured, not
assumed (measured_rel_error).

Preconditioner (Section 3.5, case (B): a direct low Kronecker-rank
approximation of F3 = 1/F2 in the same eigenbasis): 1/F2 is not completely
monotone, so it is written as P(s) = s * sum_k p_k exp(-theta_k s) with
p_k >= 0 (which keeps P positive, hence the preconditioner SPD). The nodes are
K geometric points in [0.05/s_max, 20/s_min]; the weights solve the
non-negative least-squares problem min sum_j (P(s_j) F2(s_j) - 1)^2 over 256
geometric sample points s_j in [s_min, s_max] (columns scaled to unit norm).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import nnls
from scipy.special import gamma as Gamma

__all__ = [
    "sinc_params",
    "sinc_terms",
    "F2_expsum",
    "F2_expsum_eval",
    "precond_expsum",
    "precond_eval",
    "operator_cp",
    "precond_cp",
    "measured_rel_error",
    "spectral_sample",
]

SINC_D = 1.2
PRE_SAMPLES = 256


def _F2(s, alpha, beta):
    return s ** (-alpha) + beta * s ** alpha


def _min_F2(alpha, beta, s_min, s_max):
    if alpha >= 1.0:
        star = 1.0 / math.sqrt(beta)
    else:
        star = beta ** (-1.0 / (2.0 * alpha))
    if s_min <= star <= s_max:
        return 2.0 * math.sqrt(beta)
    return min(_F2(s_min, alpha, beta), _F2(s_max, alpha, beta))


def _solve_right_end(g, q):
    """Smallest-ish x > 0 with x^(g-1) e^-x <= q (fixed point x = -ln q + (g-1) ln x)."""
    x = max(1.0, -math.log(q))
    for _ in range(60):
        x = max(1e-300, -math.log(q) + (g - 1.0) * math.log(x))
    return x


def sinc_params(g, delta, s_min, s_max, left_gain, right_q):
    """(tau_lo, h, r) of the trapezoid rule for s^-g.

    left_gain = max over the interval of m(s)/F(s); right_q = the value q such
    that the right tail is small enough when x^(g-1) e^-x <= q, x = t_b s_min.
    """
    h = 2.0 * math.pi * SINC_D / math.log(1.0 / delta)
    # left: exp(g tau_a) / (g Gamma(g)) * left_gain <= delta/4
    tau_a = math.log(0.25 * delta * g * Gamma(g) / left_gain) / g
    x = _solve_right_end(g, right_q)
    tau_b = math.log(x / s_min)
    tau_lo = tau_a + 0.5 * h
    tau_hi = tau_b - 0.5 * h
    r = int(math.ceil((tau_hi - tau_lo) / h)) + 1
    tau_lo = tau_hi - (r - 1) * h
    return tau_lo, h, r


def sinc_terms(g, tau_lo, h, r):
    """Nodes t_k and weights w_k of s^-g ~= sum_k w_k exp(-t_k s)."""
    tau = tau_lo + h * np.arange(r, dtype=np.float64)
    return np.exp(tau), h * np.exp(g * tau) / Gamma(g)


def F2_expsum(alpha, beta, s_min, s_max, delta):
    """Exp-sum pieces of F2(s) = s^-alpha + beta s * s^(alpha-1).

    Returns dict(t1, w1, t2, w2, alpha, beta): F2 ~= sum w1 e^-t1 s
    + beta s sum w2 e^-t2 s. For alpha = 1 the positive part is exactly beta*s
    (t2, w2 empty, exact_linear=True).
    """
    F2min = _min_F2(alpha, beta, s_min, s_max)
    F2lo = _F2(s_min, alpha, beta)
    F2hi = _F2(s_max, alpha, beta)
    # term 1: s^-alpha, multiplier 1
    tl, h, r = sinc_params(alpha, 0.5 * delta, s_min, s_max,
                           left_gain=1.0 / F2min,
                           right_q=0.25 * 0.5 * delta * Gamma(alpha) * F2lo * s_min ** alpha)
    t1, w1 = sinc_terms(alpha, tl, h, r)
    out = dict(alpha=alpha, beta=beta, t1=t1, w1=w1, exact_linear=False,
               t2=np.zeros(0), w2=np.zeros(0))
    if alpha >= 1.0:
        out["exact_linear"] = True
        return out
    g = 1.0 - alpha
    tl, h, r = sinc_params(g, 0.5 * delta, s_min, s_max,
                           left_gain=beta * s_max / F2hi,
                           right_q=0.25 * 0.5 * delta * Gamma(g) * F2lo * s_min ** g / (beta * s_min))
    out["t2"], out["w2"] = sinc_terms(g, tl, h, r)
    return out


def F2_expsum_eval(rep, s):
    s = np.asarray(s, dtype=np.float64)
    v = (rep["w1"][None, :] * np.exp(-np.outer(s, rep["t1"]))).sum(1)
    if rep["exact_linear"]:
        return v + rep["beta"] * s
    v2 = (rep["w2"][None, :] * np.exp(-np.outer(s, rep["t2"]))).sum(1)
    return v + rep["beta"] * s * v2


def spectral_sample(s_min, s_max, m):
    return np.exp(np.linspace(math.log(s_min), math.log(s_max), m))


def measured_rel_error(rep, alpha, beta, s_values):
    s = np.asarray(s_values, dtype=np.float64)
    ex = _F2(s, alpha, beta)
    return float(np.max(np.abs(F2_expsum_eval(rep, s) - ex) / ex))


def precond_expsum(alpha, beta, s_min, s_max, K):
    """Nodes theta (K,) and NNLS weights p (K,) of P(s) = s sum_k p_k exp(-theta_k s)."""
    theta = np.exp(np.linspace(math.log(0.05 / s_max), math.log(20.0 / s_min), K))
    s = spectral_sample(s_min, s_max, PRE_SAMPLES)
    A = np.exp(-np.outer(s, theta)) * (s * _F2(s, alpha, beta))[:, None]
    cs = np.linalg.norm(A, axis=0)
    p, _ = nnls(A / cs[None, :], np.ones_like(s), maxiter=50 * K * K + 1000)
    return theta, p / cs


def precond_eval(theta, p, s):
    s = np.asarray(s, dtype=np.float64)
    return s * (p[None, :] * np.exp(-np.outer(s, theta))).sum(1)


def operator_cp(rep, lams):
    """Canonical factors (in the eigenbasis) of the separable F2 representation.

    Term order: the r1 terms of s^-alpha; then for every node of s^(alpha-1)
    the three terms m = 1, 2, 3 whose mode-m factor carries lambda^(m)
    (for alpha = 1: the three terms of beta*s).
    """
    w, U = [], [[], [], []]
    for t, c in zip(rep["t1"], rep["w1"]):
        w.append(c)
        for l in range(3):
            U[l].append(np.exp(-t * lams[l]))
    if rep["exact_linear"]:
        for m in range(3):
            w.append(rep["beta"])
            for l in range(3):
                U[l].append(lams[l].copy() if l == m else np.ones_like(lams[l]))
    else:
        for t, c in zip(rep["t2"], rep["w2"]):
            for m in range(3):
                w.append(rep["beta"] * c)
                for l in range(3):
                    e = np.exp(-t * lams[l])
                    U[l].append(lams[l] * e if l == m else e)
    return np.array(w), [np.array(u).T for u in U]


def precond_cp(theta, p, lams):
    """Canonical factors of P(s) = (lambda_i+lambda_j+lambda_k) sum_k p_k e^(-theta_k s); zero weights dropped."""
    w, U = [], [[], [], []]
    for t, c in zip(theta, p):
        if c <= 0.0:
            continue
        for m in range(3):
            w.append(c)
            for l in range(3):
                e = np.exp(-t * lams[l])
                U[l].append(lams[l] * e if l == m else e)
    return np.array(w), [np.array(u).T for u in U]
