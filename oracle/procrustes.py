"""Energy-norm Procrustes phase corrector: Sec. 3.2-3.3 and Alg. 1 (UpdateSVD), FP64.

Test infrastructure only (see the package docstring).

The corrector Omega minimises ||F - Omega G||_F over orthogonal Omega
(eq. OPP / procurstesform); with M = F G^T = X Sigma Y^T the minimiser is
Omega = X Y^T (eq. correlationmatrixM and below).  M grows by F^k G^k^T per
iteration and its truncated SVD is updated with Alg. 1.  numpy's reduced
(Householder) QR and its SVD serve as the library steps `truncatedqr` and
`svd` of Alg. 1.
"""
from __future__ import annotations

from typing import Optional

import numpy as np


def truncated_qr(A: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """`truncatedqr` of Alg. 1, read as the reduced QR factorisation of Sec. 3.3.1
    (Q has as many columns as A, R is square)."""
    Q, R = np.linalg.qr(A, mode="reduced")
    return Q, R


def rank_cut(sigma: np.ndarray, tol: float) -> int:
    """rankM = number of singular values with sigma_i / max sigma > tol (Alg. 1)."""
    if sigma.size == 0 or sigma.max() <= 0:
        return 0
    return int(np.sum(sigma / sigma.max() > tol))


def update_svd(U: Optional[np.ndarray], S: Optional[np.ndarray], V: Optional[np.ndarray],
               F: np.ndarray, G: np.ndarray, tol: float):
    """Alg. 1: the truncated SVD of U S V^T + F G^T.

    Returns (U~, S~, V~) with U~ S~ V~^T ~= M^{k+1}, S~ a 1-D array of the
    retained singular values.  U, S, V = None stands for "S is empty".
    """
    if S is None or S.size == 0:
        QF, RF = truncated_qr(F)
        QG, RG = truncated_qr(G)
        Xr, sig, YrT = np.linalg.svd(RF @ RG.T)
        r = rank_cut(sig, tol)
        return QF @ Xr[:, :r], sig[:r].copy(), QG @ YrT.T[:, :r]
    UF = U.T @ F
    VG = V.T @ G
    QF, RF = truncated_qr(F - U @ UF)
    QG, RG = truncated_qr(G - V @ VG)
    s = S.size
    H = np.vstack([UF, RF]) @ np.vstack([VG, RG]).T
    H[:s, :s] += np.diag(S)
    Xh, sig, YhT = np.linalg.svd(H)
    r = rank_cut(sig, tol)
    U_new = np.hstack([U, QF]) @ Xh[:, :r]
    V_new = np.hstack([V, QG]) @ YhT.T[:, :r]
    return U_new, sig[:r].copy(), V_new


def apply_corrector(X: np.ndarray, Y: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Omega g with Omega = X Y^T (Alg. 3: [q, p] = X Y^T [nabla_h w, c^-1 w_t])."""
    return X @ (Y.T @ g)


def procrustes(F: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Omega_* = X Y^T from the full SVD of M = F G^T (Sec. 3.3)."""
    X, _, YT = np.linalg.svd(F @ G.T)
    return X @ YT
