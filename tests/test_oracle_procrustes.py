"""Pins of the Procrustes corrector and of UpdateSVD (Sec. 3.2-3.3, Alg. 1):
brute-force optimality on 2x2 and 3x3 problems, orthogonality, the minimum
residual formula, the rank statement, and incremental = batch SVD."""
import math

import numpy as np
import pytest

from oracle import procrustes


def _omega_from_update(F, G, tol=1e-15):
    X, S, Y = procrustes.update_svd(None, None, None, F, G, tol)
    return X @ Y.T


def _rot(a, reflect=False):
    R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    return R @ np.diag([1.0, -1.0]) if reflect else R


def test_procrustes_2x2_brute_force():
    rng = np.random.default_rng(0)
    for _ in range(20):
        F, G = rng.standard_normal((2, 2, 5))
        for Om in (procrustes.procrustes(F, G), _omega_from_update(F, G)):
            best = np.linalg.norm(F - Om @ G)
            for a in np.linspace(0, 2 * math.pi, 3601):
                for refl in (False, True):
                    assert np.linalg.norm(F - _rot(a, refl) @ G) >= best - 1e-9
            np.testing.assert_allclose(Om @ Om.T, np.eye(2), atol=1e-12)


def test_procrustes_3x3_random_search():
    rng = np.random.default_rng(1)
    for _ in range(5):
        F, G = rng.standard_normal((2, 3, 7))
        Om = _omega_from_update(F, G)
        best = np.linalg.norm(F - Om @ G)
        for _ in range(4000):
            Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
            assert np.linalg.norm(F - Q @ G) >= best - 1e-9
        # local search around the optimum never improves it
        for _ in range(500):
            A = rng.standard_normal((3, 3)) * 1e-3
            Q = Om @ (np.eye(3) + (A - A.T)) @ np.linalg.inv(np.eye(3) - (A - A.T))   # Cayley step
            assert np.linalg.norm(F - Q @ G) >= best - 1e-12


def test_minimum_residual_formula():
    # r_min^2 = ||F||^2 + ||G||^2 - 2 trace(Sigma) (Sec. 3.3), full-rank M
    rng = np.random.default_rng(2)
    F, G = rng.standard_normal((2, 6, 9))
    X, S, Y = procrustes.update_svd(None, None, None, F, G, 1e-15)
    assert S.size == 6
    r2 = np.linalg.norm(F - X @ Y.T @ G) ** 2
    assert abs(r2 - (np.linalg.norm(F) ** 2 + np.linalg.norm(G) ** 2 - 2 * S.sum())) < 1e-9 * r2


def test_rank_of_M_is_min_rank():
    # rank M = min(rank F, rank G) (Sec. 3.3.1) when the column spaces are generic
    rng = np.random.default_rng(3)
    F = rng.standard_normal((12, 2)) @ rng.standard_normal((2, 6))   # rank 2
    G = rng.standard_normal((12, 3)) @ rng.standard_normal((3, 6))   # rank 3
    _, S, _ = procrustes.update_svd(None, None, None, F, G, 1e-10)
    assert S.size == 2


def test_rank_cut_is_strict():
    assert procrustes.rank_cut(np.array([1.0, 1e-3, 1e-3 - 1e-12]), 1e-3) == 1
    assert procrustes.rank_cut(np.array([2.0, 1.0]), 0.5) == 1
    assert procrustes.rank_cut(np.zeros(3), 1e-3) == 0


def test_incremental_update_equals_batch_svd():
    # Alg. 1 caption: U~ S~ V~^T = U S V^T + F G^T; with tol -> 0 the sum of
    # the products is recovered and the singular values match the batch SVD
    rng = np.random.default_rng(4)
    rows = 40
    U = S = V = None
    M = np.zeros((rows, rows))
    for k in range(4):
        F, G = rng.standard_normal((2, rows, 5))
        U, S, V = procrustes.update_svd(U, S, V, F, G, 1e-15)
        M += F @ G.T
        np.testing.assert_allclose(U @ np.diag(S) @ V.T, M, atol=1e-10 * np.abs(M).max())
        np.testing.assert_allclose(S, np.linalg.svd(M, compute_uv=False)[: S.size], rtol=1e-10)
        np.testing.assert_allclose(U.T @ U, np.eye(S.size), atol=1e-10)
        np.testing.assert_allclose(V.T @ V, np.eye(S.size), atol=1e-10)


def test_planted_mistakes_are_caught():
    rng = np.random.default_rng(5)
    F, G = rng.standard_normal((2, 3, 7))
    good = np.linalg.norm(F - _omega_from_update(F, G) @ G)
    X, S, Y = procrustes.update_svd(None, None, None, F, G, 1e-15)
    # Omega = X Y (missing transpose) or Y X^T (roles swapped) is not optimal
    for bad in (X @ Y, Y @ X.T):
        assert np.linalg.norm(F - bad @ G) > good + 1e-6
    # dropping the diag(S) block of H breaks the incremental identity
    F2, G2 = rng.standard_normal((2, 3, 7))
    UF, VG = X.T @ F2, Y.T @ G2
    H_bad = UF @ VG.T
    Xh, sig, _ = np.linalg.svd(H_bad)
    M = F @ G.T + F2 @ G2.T
    assert abs(np.sum(sig) - np.sum(np.linalg.svd(M, compute_uv=False))) > 1e-3
