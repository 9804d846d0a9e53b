"""Pins of the registration oracle: the weighted Procrustes fit against
closed forms (identity matching of a rotated copy, a reflection that the
determinant correction must refuse, invariance to the plan's scale) and the
whole alternation on a small misaligned partial cloud."""
import numpy as np
import pytest

import pot_workloads as W
from oracle import registration as RG


def test_fit_recovers_a_rigid_motion_from_an_exact_matching():
    g = np.random.default_rng(0)
    Y0 = g.normal(size=(20, 3))
    R0 = RG.rotation([1.0, 2.0, -0.5], 0.7)
    t0 = np.array([0.3, -0.1, 0.2])
    X = RG.transform(Y0, R0, t0)
    P = np.diag(g.uniform(0.5, 1.5, size=20))     # any positive weights on the true pairs
    R, t, mass = RG.rigid_fit(X, Y0, P)
    np.testing.assert_allclose(R, R0, atol=1e-12)
    np.testing.assert_allclose(t, t0, atol=1e-12)
    assert mass == pytest.approx(P.sum())
    # the fit does not depend on the plan's total mass
    R2, t2, _ = RG.rigid_fit(X, Y0, 3.7 * P)
    np.testing.assert_allclose(R2, R, atol=1e-12)
    np.testing.assert_allclose(t2, t, atol=1e-12)


def test_fit_returns_a_rotation_not_a_reflection():
    g = np.random.default_rng(1)
    Y0 = g.normal(size=(15, 3))
    F = np.diag([1.0, 1.0, -1.0])                  # a mirror image: the best orthogonal map is F itself
    X = Y0 @ F.T
    R, t, _ = RG.rigid_fit(X, Y0, np.eye(15))
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    assert np.linalg.det(R) == pytest.approx(1.0)
    # and it is the best proper rotation: no random rotation does better
    P = np.eye(15)
    best = ((X - RG.transform(Y0, R, t)) ** 2).sum()
    for k in range(200):
        Rk = RG.rotation(g.normal(size=3), g.uniform(0, np.pi))
        tk = (X - Y0 @ Rk.T).mean(axis=0)
        assert ((X - RG.transform(Y0, Rk, tk)) ** 2).sum() >= best - 1e-9


def test_printed_rotation_is_the_transpose_for_the_stated_model():
    """Reading N19: with x = R0 y the SVD of sum x y^T gives U V^T = R0; the
    printed V U^T is R0^T."""
    g = np.random.default_rng(2)
    Y0 = g.normal(size=(30, 3))
    R0 = RG.rotation([0.2, -1.0, 0.4], 0.9)
    X = Y0 @ R0.T
    U, S, Vt = np.linalg.svd(X.T @ Y0)
    np.testing.assert_allclose(U @ Vt, R0, atol=1e-12)
    np.testing.assert_allclose(Vt.T @ U.T, R0.T, atol=1e-12)


def test_alternation_aligns_a_partial_misaligned_cloud():
    X, Y0, R_true, t_true = W.registration_3d(0, n=120, frac=0.5, max_angle=0.4, max_shift=0.08)
    m = Y0.shape[0]
    s = 0.6 * min(m, X.shape[0]) / max(m, X.shape[0])
    R, t, k, hist = RG.register(X, Y0, s, gamma0=0.02, anneal=0.83, gamma_min=0.002, eps=1e-3, max_reg=40,
                                tol=1e-6)
    # the source maps back onto the target points it was cut from
    np.testing.assert_allclose(R, R_true, atol=2e-2)
    np.testing.assert_allclose(t, t_true, atol=2e-2)
    assert hist[-1] < hist[0]
