"""Pins of the REML / derivative oracle: finite differences, closed forms, stationarity."""
import math

import numpy as np
import pytest

import synth
from oracle import gls as G
from oracle import reml as R


@pytest.fixture(scope="module")
def cohort():
    return synth.make_cohort(41, 300, h=0.4, sigma2=1.0, n_markers=400)


def fd(f, x, step=1e-5):
    return (f(x + step) - f(x - step)) / (2 * step)


@pytest.mark.parametrize("h", [0.1, 0.25])
def test_gradient_matches_central_differences(cohort, h):
    c = cohort
    s2 = 1.3
    g = R.reml_grad(c.phi, h, s2, c.XL, c.Y)
    g0 = np.linalg.norm(R.reml_grad(c.phi, 0.1, s2, c.XL, c.Y))
    g_h = fd(lambda v: R.reml_loglik(c.phi, v, s2, c.XL, c.Y), h)
    g_s = fd(lambda v: R.reml_loglik(c.phi, h, v, c.XL, c.Y), s2)
    assert abs(g_h - g[0]) <= 1e-6 * max(abs(g[0]), g0)
    assert abs(g_s - g[1]) <= 1e-6 * max(abs(g[1]), g0)


def test_h0_closed_form(cohort):
    """At h = 0 (M = s2 I) l has a closed form in the OLS residuals."""
    c = cohort
    s2 = 0.7
    n, q = c.XL.shape
    y = c.Y[:, 0]
    beta, *_ = np.linalg.lstsq(c.XL, y, rcond=None)
    rss = float(np.sum((y - c.XL @ beta) ** 2))
    _, logdet_xtx = np.linalg.slogdet(c.XL.T @ c.XL)
    ref = -0.5 * ((n - q) * math.log(2 * math.pi) + n * math.log(s2)
                  + logdet_xtx - q * math.log(s2) + rss / s2)
    assert abs(R.reml_loglik(c.phi, 0.0, s2, c.XL, y) - ref) <= 1e-9 * abs(ref)


def test_profiled_sigma2_is_stationary(cohort):
    c = cohort
    for h in (0.2, 0.6):
        s2 = R.profiled_sigma2(c.phi, h, c.XL, c.Y)
        g = R.reml_grad(c.phi, h, s2, c.XL, c.Y)
        assert abs(g[1]) <= 1e-9 * max(1.0, abs(g[0]))


def test_reml_fit_is_a_maximum(cohort):
    c = cohort
    h_hat = R.fit_h(c.phi, c.XL, c.Y)
    assert 0.0 < h_hat < 1.0

    def prof(h):
        return R.reml_loglik(c.phi, h, R.profiled_sigma2(c.phi, h, c.XL, c.Y), c.XL, c.Y)

    assert prof(h_hat) >= prof(h_hat - 1e-3) and prof(h_hat) >= prof(h_hat + 1e-3)
    s2 = R.profiled_sigma2(c.phi, h_hat, c.XL, c.Y)
    assert abs(R.reml_grad(c.phi, h_hat, s2, c.XL, c.Y)[0]) <= 1e-4


def test_db_dh_closed_form_and_finite_differences(cohort):
    c = synth.make_cohort(42, 200, t=2, h=0.35, sigma2=1.7, n_markers=300)
    X = c.snps(12)
    gen = R.db_dh(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    closed = R.db_dh(c.phi, c.h, c.sigma2, c.XL, c.Y, X, closed_form=True)
    scale = np.max(np.abs(gen), axis=-1, keepdims=True)
    assert np.max(np.abs(gen - closed) / scale) <= 1e-9

    def b_of(h):
        return G.gls(c.phi, h, c.sigma2, c.XL, c.Y, X)[0]

    num = (b_of(c.h + 1e-5) - b_of(c.h - 1e-5)) / 2e-5
    assert np.max(np.abs(num - gen) / scale) <= 1e-6


def test_planted_sign_error_is_caught(cohort):
    """The FD pin rejects a gradient with the trace term's sign flipped."""
    c = cohort
    h, s2 = 0.25, 1.3
    M, _, P, _, _, _ = R.reml_parts(c.phi, h, s2, c.XL, c.Y)
    y = c.Y[:, 0]
    Py = P @ y
    dM = s2 * (c.phi - np.eye(c.n))
    wrong = -0.5 * (-np.sum(P * dM) - Py @ dM @ Py)
    g_h = fd(lambda v: R.reml_loglik(c.phi, v, s2, c.XL, c.Y), h)
    assert abs(g_h - wrong) > 1e-3 * abs(g_h)
