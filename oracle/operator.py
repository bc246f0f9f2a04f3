"""1D Sturm-Liouville matrices and their eigenbasis (oracle, FP64, CPU).

Section 3.2 discretizes -(a(x) y')' = lambda y, y(0) = y(1) = 0 with
one-sided difference quotients and the coefficient a evaluated at the
half-points a_{i+-1/2}. Read as the standard symmetric Dirichlet stencil
(h = 1/(n+1), x_i = i h):

    (A y)_i = [ (a_{i-1/2} + a_{i+1/2}) y_i - a_{i-1/2} y_{i-1} - a_{i+1/2} y_{i+1} ] / h^2,

i.e. diagonal (a_{i-1/2} + a_{i+1/2})/h^2 and off-diagonal -a_{i+1/2}/h^2.
The paper's printed end rows (diagonal 2 a_{3/2} in row 1 and 2 a_{n-1/2} in
row n, overall factor -1/h^2) are available with paper_end_rows=True; both
readings coincide for a == 1. A is symmetric positive definite.

Section 3.3 ("eigs_1D") factorizes A_l = V_l diag(lambda^(l)) V_l^T with the
eigenvectors as the columns of the orthogonal V_l; the 3D operator is the
Kronecker sum A = A_1 (+) A_2 (+) A_3 ("eqn_low_rank_lap").
Eigenvector signs are arbitrary; the oracle fixes each column v so that
sum_i v_i g_i > 0 with the fixed weights g_i = 2 frac(i * 0.6180339887498949) - 1
(i = 1..n, a Weyl sequence). The first entry is not used because high modes
of a variable-coefficient operator localize and their first entry can
underflow; the weighted sum is of order one for every column.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

__all__ = [
    "assemble",
    "dense",
    "eig",
    "normalise_signs",
    "sign_weights",
    "stencil_apply",
    "kron_sum_dense",
]


def assemble(a_half: np.ndarray, paper_end_rows: bool = False):
    """Tridiagonal A_(l) from a(x_{i-1/2}), i = 1..n+1 (Section 3.2).

    Returns (d, e): diagonal (n,) and off-diagonal (n-1,), float64.
    """
    a_half = np.asarray(a_half, dtype=np.float64)
    n = a_half.shape[0] - 1
    h = 1.0 / (n + 1)
    inv_h2 = 1.0 / (h * h)
    d = (a_half[:-1] + a_half[1:]) * inv_h2
    e = -a_half[1:-1] * inv_h2
    if paper_end_rows:
        # printed end rows: a_{1,1} = -2 a_{3/2}, a_{n,n} = -2 a_{n-1/2}, times -1/h^2
        d = d.copy()
        d[0] = 2.0 * a_half[1] * inv_h2
        d[-1] = 2.0 * a_half[n - 1] * inv_h2
    return d, e


def dense(d: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Dense symmetric tridiagonal matrix with diagonal d and off-diagonal e."""
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def sign_weights(n: int) -> np.ndarray:
    """g_i = 2 frac(i * 0.6180339887498949) - 1, i = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return 2.0 * np.mod(i * 0.6180339887498949, 1.0) - 1.0


def normalise_signs(V: np.ndarray) -> np.ndarray:
    """Flip columns so that sum_i V[i, k] g_i > 0 for every k."""
    d = sign_weights(V.shape[0]) @ V
    s = np.where(d < 0.0, -1.0, 1.0)
    return V * s[None, :]


def eig(d: np.ndarray, e: np.ndarray, driver: str = "stemr"):
    """Eigenpairs of the symmetric tridiagonal A_(l) by LAPACK (Section 3.3).

    Returns (lam ascending (n,), V (n, n) with eigenvectors as columns).
    driver: 'stemr' (MRRR), 'stev' or 'dense' (full symmetric eigh, a second
    independent route used as a pin).
    """
    if driver == "dense":
        lam, V = np.linalg.eigh(dense(d, e))
    else:
        lam, V = sla.eigh_tridiagonal(d, e, lapack_driver=driver)
    order = np.argsort(lam)
    return lam[order], normalise_signs(V[:, order])


def stencil_apply(a_halves, Y: np.ndarray) -> np.ndarray:
    """A Y for the 3D Kronecker-sum operator as a 7-point stencil.

    Y is an (n, n, n) array indexed [i1, i2, i3]; zero Dirichlet values are
    used outside the grid. a_halves[l] holds a_l(x_{i-1/2}), i = 1..n+1.
    No eigenvectors are involved (used to pin the alpha = 1 case).
    """
    n = Y.shape[0]
    h2 = (1.0 / (n + 1)) ** 2
    out = np.zeros_like(Y)
    for l in range(3):
        a = np.asarray(a_halves[l], dtype=np.float64)
        Ym = np.moveaxis(Y, l, 0)
        Yp = np.zeros((n + 2,) + Ym.shape[1:])
        Yp[1:-1] = Ym
        am = a[:-1].reshape((n,) + (1,) * (Y.ndim - 1))   # a_{i-1/2}
        ap = a[1:].reshape((n,) + (1,) * (Y.ndim - 1))    # a_{i+1/2}
        r = (am + ap) * Yp[1:-1] - am * Yp[:-2] - ap * Yp[2:]
        out += np.moveaxis(r / h2, 0, l)
    return out


def kron_sum_dense(mats) -> np.ndarray:
    """Dense A_1 (+) A_2 (+) A_3 acting on vec(Y) with i1 slowest (C order of [i1,i2,i3])."""
    A1, A2, A3 = mats
    I1, I2, I3 = (np.eye(A.shape[0]) for A in mats)
    return (np.kron(np.kron(A1, I2), I3) + np.kron(np.kron(I1, A2), I3)
            + np.kron(np.kron(I1, I2), A3))
