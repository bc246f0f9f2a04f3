"""Exact full-grid solve of the discrete control equation (oracle, FP64, CPU).

The control equation ("Lagrange_cont", Section 3.1) with the paper's
beta_p = 1 and gamma = beta reads

    F2(A) u = y_Omega,   F2(s) = s^-alpha + beta s^alpha,

where A = A_1 (+) A_2 (+) A_3 is the Kronecker-sum FD operator. With the 1D
eigenbasis A_l = V_l diag(lambda^(l)) V_l^T, every spectral function of A is
diagonal in the tensor eigenbasis ("DiagGen", "DiagFGen2D", "DiagKron3D"):

    F(A) x = (V1 x V2 x V3) [ F(lambda_i + lambda_j + lambda_k) .* ((V1^T x V2^T x V3^T) x) ],

so the exact solution is u* = (xV) [ ((xV^T) y) ./ F2(S) ] with
S[i,j,k] = lambda^(1)_i + lambda^(2)_j + lambda^(3)_k. The mode products are
plain matmuls (BLAS dgemm through numpy).

Arrays are (n, n, n) indexed [i1, i2, i3].
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "F2",
    "spectral_sum",
    "mode_product",
    "to_eigenbasis",
    "from_eigenbasis",
    "apply_spectral",
    "solve_exact",
    "state_exact",
    "streamed_rel_error",
    "streamed_rel_errors",
]


def F2(s, alpha: float, beta: float):
    """F2(s) = s^-alpha + beta s^alpha (the symbol of the control equation).

    s^alpha is evaluated once and s^-alpha as its reciprocal."""
    t = np.asarray(s, dtype=np.float64) ** alpha
    return 1.0 / t + beta * t


def spectral_sum(lams) -> np.ndarray:
    """S[i,j,k] = lambda^(1)_i + lambda^(2)_j + lambda^(3)_k."""
    l1, l2, l3 = lams
    return l1[:, None, None] + l2[None, :, None] + l3[None, None, :]


def mode_product(X: np.ndarray, M: np.ndarray, mode: int) -> np.ndarray:
    """(X x_mode M)[.., a, ..] = sum_i M[a, i] X[.., i, ..]."""
    Xm = np.moveaxis(X, mode, 0)
    sh = Xm.shape
    Y = (M @ Xm.reshape(sh[0], -1)).reshape((M.shape[0],) + sh[1:])
    return np.moveaxis(Y, 0, mode)


def to_eigenbasis(X, Vs):
    """(V1^T x V2^T x V3^T) X."""
    for l in range(3):
        X = mode_product(X, Vs[l].T, l)
    return X


def from_eigenbasis(Xh, Vs):
    """(V1 x V2 x V3) Xh."""
    for l in range(3):
        Xh = mode_product(Xh, Vs[l], l)
    return Xh


def apply_spectral(f_of_S: np.ndarray, X: np.ndarray, Vs) -> np.ndarray:
    """F(A) X given the diagonal F(S) in the eigenbasis."""
    return from_eigenbasis(f_of_S * to_eigenbasis(X, Vs), Vs)


def solve_exact(Y: np.ndarray, lams, Vs, alpha: float, beta: float) -> np.ndarray:
    """u* = F2(A)^-1 y by full-grid diagonalization."""
    S = spectral_sum(lams)
    return from_eigenbasis(to_eigenbasis(Y, Vs) / F2(S, alpha, beta), Vs)


def state_exact(U: np.ndarray, lams, Vs, alpha: float, beta_state: float = 1.0) -> np.ndarray:
    """State equation ("State"): y = beta_p A^-alpha u."""
    S = spectral_sum(lams)
    return beta_state * from_eigenbasis(to_eigenbasis(U, Vs) * S ** (-alpha), Vs)


def _slab_range_terms(args):
    """||u*_hat||^2 and ||u*_hat - u_hat_m||^2 summed over the i3-slabs c0 <= c < c1."""
    (l1, l2, l3, c0, c1, Yh1, Yh2, y3, sols, alpha, beta) = args
    n1, blk = l1.shape[0], 256  # rows of a slab at a time (cache-sized temporaries)
    den = 0.0
    num = [0.0] * len(sols)
    for c in range(c0, c1):
        Yw = Yh1 * y3[c][None, :]
        Us = [(Uh1 * u3[c][None, :], Uh2) for Uh1, Uh2, u3 in sols]
        for i0 in range(0, n1, blk):
            S = l1[i0:i0 + blk, None] + l2[None, :] + l3[c]
            ystar = Yw[i0:i0 + blk] @ Yh2.T
            np.divide(ystar, F2(S, alpha, beta), out=ystar)
            yv = ystar.ravel()
            den += float(yv @ yv)
            for m, (A1, Uh2) in enumerate(Us):
                d = A1[i0:i0 + blk] @ Uh2.T
                np.subtract(ystar, d, out=d)
                dv = d.ravel()
                num[m] += float(dv @ dv)
    return den, num


def streamed_rel_errors(lams, yw, yU_hat, sols, alpha, beta, pool=None):
    """||u* - u_m|| / ||u*|| for several canonical u_m of one problem, one pass.

    Both tensors are given in the eigenbasis as canonical factors:
    y_hat = sum_j yw_j (x_l yU_hat[l][:, j]), u_hat = sum_k uw_k (x_l uU_hat[l][:, k]);
    sols is a list of (uw, uU_hat). The tensor eigenbasis is orthogonal, so the
    error there equals the error on the grid. u*_hat = y_hat ./ F2(S) is formed
    one i3-slab at a time (never the n^3 array), once for all the solutions;
    a pool, if given, takes contiguous ranges of slabs.
    """
    l1, l2, l3 = lams
    n3 = l3.shape[0]
    y3 = yU_hat[2] * yw[None, :]
    s3 = [(uU[0], uU[1], uU[2] * uw[None, :]) for uw, uU in sols]
    parts = 1 if pool is None else min(n3, 4 * getattr(pool, "_processes", 4))
    bounds = [round(i * n3 / parts) for i in range(parts + 1)]
    jobs = [(l1, l2, l3, bounds[i], bounds[i + 1], yU_hat[0], yU_hat[1], y3, s3, alpha, beta)
            for i in range(parts) if bounds[i + 1] > bounds[i]]
    res = pool.map(_slab_range_terms, jobs, chunksize=1) if pool is not None else map(_slab_range_terms, jobs)
    den = 0.0
    num = [0.0] * len(sols)
    for d, nm in res:
        den += d
        for m in range(len(sols)):
            num[m] += nm[m]
    return [float(np.sqrt(v / den)) for v in num]


def streamed_rel_error(lams, yw, yU_hat, uw, uU_hat, alpha, beta, pool=None):
    """||u* - u|| / ||u*|| without forming n^3 arrays (one solution of streamed_rel_errors)."""
    return streamed_rel_errors(lams, yw, yU_hat, [(uw, uU_hat)], alpha, beta, pool=pool)[0]
