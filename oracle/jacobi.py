"""Oracle: a hand-written cyclic Jacobi eigensolver for tiny symmetric pencils.

Test infrastructure only (see ``oracle/__init__``).  It exists to pin the
LAPACK call of ``oracle.eigen`` on 64-particle inputs with a route that shares
nothing with it: the pencil (H, M) is reduced to a standard problem with a
hand-written Cholesky factor L (M = L L^T), A = L^{-1} H L^{-T}, and A is
diagonalised by cyclic Jacobi rotations (the classical method; each rotation
zeroes one off-diagonal pair).  Pure Python loops: small inputs only.
"""
from __future__ import annotations

import math

import numpy as np


def cholesky(M):
    n = M.shape[0]
    L = np.zeros_like(M, dtype=np.float64)
    for j in range(n):
        s = M[j, j] - sum(L[j, p] * L[j, p] for p in range(j))
        if s <= 0.0:
            raise ValueError("matrix is not positive definite")
        L[j, j] = math.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (M[i, j] - sum(L[i, p] * L[j, p] for p in range(j))) / L[j, j]
    return L


def forward_solve(L, B):
    n = L.shape[0]
    X = np.zeros_like(B, dtype=np.float64)
    for i in range(n):
        X[i] = (B[i] - L[i, :i] @ X[:i]) / L[i, i]
    return X


def jacobi_eigh(A, sweeps=60, tol=1e-15):
    """Eigenvalues (ascending) and vectors of a symmetric A by cyclic Jacobi."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(sweeps):
        off = math.sqrt(sum(A[p, q] ** 2 for p in range(n) for q in range(n) if p != q))
        if off <= tol * math.sqrt(sum(A[p, p] ** 2 for p in range(n))):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p, q] == 0.0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * A[p, q])
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                # A <- J^T A J with the rotation in the (p, q) plane
                ap = A[:, p].copy()
                aq = A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap = A[p, :].copy()
                aq = A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    w = np.diag(A).copy()
    order = np.argsort(w)
    return w[order], V[:, order]


def generalized_jacobi(H, M):
    """All eigenpairs of H c = lam M c (dense, tiny): C is M-orthonormal."""
    L = cholesky(np.asarray(M, dtype=np.float64))
    Y = forward_solve(L, np.asarray(H, dtype=np.float64))        # L^{-1} H
    A = forward_solve(L, Y.T).T                                  # L^{-1} H L^{-T}
    A = 0.5 * (A + A.T)
    w, V = jacobi_eigh(A)
    # c = L^{-T} v  (back substitution with L^T)
    n = L.shape[0]
    C = np.zeros_like(V)
    for i in range(n - 1, -1, -1):
        C[i] = (V[i] - L[i + 1:, i] @ C[i + 1:]) / L[i, i]
    return w, C
