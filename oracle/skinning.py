"""Oracle: skinning weight fields and linear blend skinning, plain FP64.

Test infrastructure only (see ``oracle/__init__``).

Paper: Sec. 3.2 discretises each skinning weight field with RKPM,
    W^j(X) = sum_k phi_k(X) c_k^j,
with phi_k the corrected shape functions of the particle cloud (Eqs. 6-11, here
``rkpm.shape_functions_at``) and c the nodal values (the eigenmodes); Eq. 1 is
linear blend skinning with m affine transforms Z_j in R^{3x4}:
    x = X + sum_j W^j(X) Z_j [X; 1].
"""
import numpy as np

from . import rkpm


def weights(Q, P, a, C, scale=None):
    """W (nq x m): W[q, j] = sum_k phi_k(Q_q) C[k, j] (Sec. 3.2)."""
    phi, _ = rkpm.shape_functions_at(Q, P, a, scale=scale)
    return phi @ np.asarray(C, dtype=np.float64)


def lbs(X, W, Z):
    """x (nq x 3) = X + sum_j W[:, j] Z_j [X; 1] (Eq. 1); Z is (m, 3, 4)."""
    X = np.asarray(X, dtype=np.float64)
    Xh = np.concatenate([X, np.ones((X.shape[0], 1))], axis=1)       # [X; 1] per point
    ZX = np.einsum("jrc,qc->qjr", np.asarray(Z, dtype=np.float64), Xh)  # Z_j [X; 1]
    return X + np.einsum("qj,qjr->qr", np.asarray(W, dtype=np.float64), ZX)
