"""Sketched rank-constrained least-squares solves (Sec. 4, Alg. 5), FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Both solvers return (C_(n)^T, A^(n)) for the subproblem
    min || Z B - Y ||_F  s.t.  rank(B) <= R,  B = C_(n)^T A^(n)T
with Z = S P^(n) (m x r) and Y = S T_(n)^T (m x s).

Gauge reading: singular vectors are defined up to sign.  Both the oracle and the
CUDA library fix it the same way: each column of A^(n) is flipped so that its
entry of largest magnitude (first such index on ties) is positive, and the
matching column of C_(n)^T is flipped with it, which leaves B unchanged.
"""

from __future__ import annotations

import numpy as np


def canonical_signs(Cn: np.ndarray, V: np.ndarray):
    """Flip paired columns so that the largest-|.| entry of each column of V is positive."""
    idx = np.argmax(np.abs(V), axis=0)
    flip = np.where(V[idx, np.arange(V.shape[1])] < 0, -1.0, 1.0)
    return Cn * flip[None, :], V * flip[None, :]


def rsvd_oversampled_rank(R: int, oversample: int, r: int, s: int) -> int:
    """Number of columns of the Gaussian test matrix in Alg. 5 (reading: R + p, clipped)."""
    return max(R, min(R + oversample, r, s))


def lrls_exact(Z: np.ndarray, Y: np.ndarray, R: int):
    """Best rank-R approximation of argmin_X ||Z X - Y|| (the solution defined in Theorem 4.1).

    X_opt by a LAPACK least-squares solve, then its truncated SVD
    X_opt ~= U_R Sigma_R V_R^T; C_(n)^T = U_R Sigma_R and A^(n) = V_R.
    """
    X = np.linalg.lstsq(Z, Y, rcond=None)[0]
    U, sig, Vh = np.linalg.svd(X, full_matrices=False)
    Cn = U[:, :R] * sig[None, :R]
    return canonical_signs(Cn, Vh[:R].T)


def rsvd_lrls(Z: np.ndarray, Y: np.ndarray, R: int, Omega: np.ndarray):
    """RSVD-LRLS, Alg. 5, step by step with a given Gaussian test matrix Omega (s x k).

    B = (Z^T Z)^{-1};  C = B Z^T Y Omega;  Q, _ = qr(C);  D = Q^T B Z^T Y;
    U, Sigma, V = svd(D);  return Q U(:, :R) Sigma(:R, :R) and V(:, :R).
    """
    B = np.linalg.inv(Z.T @ Z)
    C = B @ (Z.T @ Y) @ Omega
    Q, _ = np.linalg.qr(C)
    D = Q.T @ B @ (Z.T @ Y)
    U, sig, Vh = np.linalg.svd(D, full_matrices=False)
    Cn = Q @ (U[:, :R] * sig[None, :R])
    return canonical_signs(Cn, Vh[:R].T)
