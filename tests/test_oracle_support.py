"""Pins the oracle's support-reduction iteration (Sec. 5.3: proximal gradient
descent on L(beta) + lam |beta|_1 with L the squared RKHS distance of the
weighted kernel mean embeddings) to what the mathematics fixes: the closed
form with an identity Gram, the minimiser without penalty, the optimality
(KKT) conditions of the lasso at convergence on a real signature-kernel Gram,
and a loss that never increases at a step size below 1 / (2 |K|)."""
import numpy as np
import pytest

import oracle
from paper_2006_14794_gb300 import inputs


def test_soft_threshold_is_the_papers_operator():
    v = np.array([-2.0, -0.5, 0.0, 0.3, 0.5, 1.7])
    np.testing.assert_array_equal(oracle.soft_threshold(v, 0.5), [-1.5, 0.0, 0.0, 0.0, 0.0, 1.2])


def test_identity_gram_closed_form():
    # K = I: min |alpha - beta|^2 + lam |beta|_1 separates per coordinate, with
    # minimiser beta_i = sign(alpha_i) max(|alpha_i| - lam/2, 0)
    rng = np.random.default_rng(400)
    a = rng.normal(size=40)
    lam = 0.6
    beta, hist = oracle.support_reduction(np.eye(40), a, np.zeros(40), 0.2, lam, 200)
    want = np.sign(a) * np.maximum(np.abs(a) - lam / 2, 0.0)
    np.testing.assert_allclose(beta, want, atol=1e-12)
    assert hist[-1] == pytest.approx(float(np.sum((a - want) ** 2) + lam * np.abs(want).sum()), rel=1e-12)


def _spd(n=12, seed=401):
    # a seeded symmetric positive definite Gram: the pins below are about the
    # iteration, and need a convex L (Grams of the discrete scheme can be
    # indefinite at the level of its discretisation error)
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, 2 * n)) / np.sqrt(2 * n)
    return A @ A.T + 0.05 * np.eye(n)


def test_no_penalty_recovers_the_weights():
    # lam = 0: L >= 0 with L(alpha) = 0 and K positive definite, so the
    # iteration converges to beta = alpha
    K = _spd()
    n = K.shape[0]
    a = np.full(n, 1.0 / n)
    gamma = 0.5 / np.linalg.eigvalsh(K).max()
    beta, hist = oracle.support_reduction(K, a, np.zeros(n), gamma, 0.0, 5000)
    np.testing.assert_allclose(beta, a, atol=1e-10)
    assert hist[-1] < 1e-18


def test_kkt_conditions_and_monotone_loss():
    # at the lasso's minimiser: grad_i L + lam sign(beta_i) = 0 where beta_i != 0,
    # |grad_i L| <= lam where beta_i = 0 (grad L = -2 K (alpha - beta))
    K = _spd()
    n = K.shape[0]
    a = np.random.default_rng(402).uniform(0.5, 1.5, size=n) / n
    lam = 0.02
    gamma = 0.5 / np.linalg.eigvalsh(K).max()
    beta, hist = oracle.support_reduction(K, a, a.copy(), gamma, lam, 20000)
    grad = -2.0 * K @ (a - beta)
    nz = beta != 0
    assert 0 < nz.sum() < n   # a genuinely reduced support
    np.testing.assert_allclose(grad[nz] + lam * np.sign(beta[nz]), 0.0, atol=1e-10)
    assert np.all(np.abs(grad[~nz]) <= lam + 1e-10)
    assert np.all(np.diff(hist) <= 1e-15)   # proximal gradient with gamma <= 1/(2|K|) never ascends
