"""Oracle: lowest-k generalized eigenpairs of H_w c = lambda M c, and checks.

Test infrastructure only (see ``oracle/__init__``).

Sec. 3.2, Eq. 15: minimise tr(c^T H_w c) subject to c^T M c = I, solved by the
lowest generalized eigenvectors.  Supp. Sec. B "Eigenanalysis": the spectrum
always contains the constant mode with eigenvalue zero.  Convention here: the
k returned pairs are the k lowest, ascending, the constant mode included at
index 0 (the paper's m counts the non-constant ones, m = k - 1).

Tiers: dense LAPACK (scipy.linalg.eigh, Cholesky + symmetric solve) up to a
few thousand particles; sparse shift-invert Lanczos (scipy eigsh with a sparse
LU of H - sigma M) beyond.  Residuals and M-principal angles judge any
candidate eigenpairs against an FP64 H, M; where the exact eigenvectors are
too costly to form, ``subspace_angle_bound`` bounds the angle from the exact
eigenvalues alone.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

F64 = np.float64


def eigh_dense(H, M, k):
    """k lowest generalized eigenpairs by LAPACK (dense).  Returns (lam, C),
    C M-orthonormal, columns ascending in lam."""
    H = H.toarray() if sp.issparse(H) else np.asarray(H, F64)
    M = M.toarray() if sp.issparse(M) else np.asarray(M, F64)
    lam, C = sla.eigh(H, M, subset_by_index=[0, k - 1])
    return lam, C


def eigsh_sparse(H, M, k, sigma=None):
    """k lowest generalized eigenpairs by shift-invert Lanczos around sigma < 0
    (H - sigma M is then positive definite).  Returns (lam, C) ascending."""
    H = sp.csc_matrix(H, dtype=F64)
    M = sp.csc_matrix(M, dtype=F64)
    if sigma is None:
        # a negative shift of the order of the smallest non-zero eigenvalues
        sigma = -1e-3 * float(H.diagonal().mean() / M.diagonal().mean())
    lam, C = spla.eigsh(H, k=k, M=M, sigma=sigma, which="LM", tol=1e-12)
    order = np.argsort(lam)
    lam, C = lam[order], C[:, order]
    # M-normalise (eigsh already returns M-orthonormal vectors; enforce it)
    nrm = np.sqrt(np.einsum("ij,ij->j", C, M @ C))
    return lam, C / nrm


def residuals(H, M, lam, C):
    """||H c_j - lam_j M c_j||_2 / (|lam_j| ||M c_j||_2) per column (FP64)."""
    C = np.asarray(C, dtype=F64)
    HC = H @ C
    MC = M @ C
    R = HC - MC * np.asarray(lam, F64)[None, :]
    num = np.linalg.norm(R, axis=0)
    den = np.abs(np.asarray(lam, F64)) * np.linalg.norm(MC, axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        return num / den


def absolute_residuals(H, M, lam, C):
    """||H c_j - lam_j M c_j||_2 / ||M c_j||_2 (for the zero eigenvalue)."""
    C = np.asarray(C, dtype=F64)
    MC = M @ C
    R = H @ C - MC * np.asarray(lam, F64)[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(MC, axis=0)


def m_orthonormalise(M, C):
    """C (M-orthonormal basis of the same span) via Cholesky of C^T M C."""
    C = np.asarray(C, dtype=F64)
    G = C.T @ (M @ C)
    L = np.linalg.cholesky(0.5 * (G + G.T))
    return np.linalg.solve(L, C.T).T


def max_principal_angle(M, A, B):
    """Largest M-principal angle (radians) between span(A) and span(B).
    sin(theta_max) = || (I - Qb Qb^T M) Qa ||_M  with Qa, Qb M-orthonormal."""
    Qa = m_orthonormalise(M, A)
    Qb = m_orthonormalise(M, B)
    S = Qa - Qb @ (Qb.T @ (M @ Qa))
    G = S.T @ (M @ S)
    s2 = max(float(np.linalg.eigvalsh(0.5 * (G + G.T)).max()), 0.0)
    return float(np.arcsin(min(1.0, np.sqrt(s2))))


def rayleigh_ritz(H, M, C):
    """FP64 Rayleigh-Ritz of H, M on span(C): (theta, Y) ascending."""
    C = np.asarray(C, dtype=F64)
    A = C.T @ (H @ C)
    B = C.T @ (M @ C)
    th, Z = sla.eigh(0.5 * (A + A.T), 0.5 * (B + B.T))
    return th, C @ Z


def subspace_angle_bound(H, M, C, lam):
    """Upper bound on the largest M-principal angle between span(C) (k
    columns) and the exact eigenspace of the k lowest eigenvalues, from the
    exact eigenvalues lam (ascending, at least k + 1 of them) alone.

    With Y an M-orthonormal basis of span(C), written Y = U_k A + U_perp B in
    the exact M-orthonormal eigenvectors, A^T A + B^T B = I and
    ||B||_F = ||sin Theta||_F.  Then
        tr(Y^T H Y) = tr(A^T L_k A) + tr(B^T L_perp B)
                   >= sum_{j<k} lam_j - lam_{k-1} ||B||_F^2 + lam_k ||B||_F^2,
    since the diagonal of A A^T is at most 1 and its trace is k - ||B||_F^2.
    Hence sin(theta_max) <= ||sin Theta||_F
                         <= sqrt((tr(Y^T H Y) - sum_{j<k} lam_j) / (lam_k - lam_{k-1})).
    Returns the angle (radians); 0 when the excess trace rounds below zero."""
    Y = m_orthonormalise(M, C)
    k = Y.shape[1]
    lam = np.asarray(lam, F64)
    excess = float(np.trace(Y.T @ (H @ Y))) - float(lam[:k].sum())
    gap = float(lam[k] - lam[k - 1])
    s2 = max(excess, 0.0) / gap
    return float(np.arcsin(min(1.0, np.sqrt(s2))))
