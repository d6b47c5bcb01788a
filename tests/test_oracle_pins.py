"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against a hand-derived
value, exact rational arithmetic, a textbook closed form, an invariance of Eq. (1),
or a different algorithm (explicit inverse, QR, numpy least squares).
"""
import numpy as np
import pytest

import synth
from oracle import exact as E
from oracle import gls as G
from tests.golden.load import load

EPS = np.finfo(np.float64).eps


def rel_b(b, ref):
    """max over SNPs/phenotypes/coefficients of |b - ref| / max(|ref_i|_inf)."""
    scale = np.maximum(np.max(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.max(np.abs(b - ref) / scale))


def small_case(seed, n, m, t=1, h=0.4, sigma2=1.0, n_markers=200):
    c = synth.make_cohort(seed, n, t=t, h=h, sigma2=sigma2, n_markers=n_markers)
    return c, c.snps(m)


# ---------------------------------------------------------------- golden -----
@pytest.mark.parametrize("route", ["hoisted", "per_snp", "explicit"])
def test_hand_example_correlated_M(route):
    g = load("hand_gls_n3.txt")
    b, w, s = G.gls(g["M"], None, None, g["XL"], g["y"], g["x"], is_phi=False, route=route)
    assert s[0] == 0
    np.testing.assert_allclose(b[0, 0], g["b"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(w[0, 0], g["wald"], rtol=1e-14)
    # the same M written as sigma^2 (h Phi + (1-h) I)
    b2, w2, _ = G.gls(g["phi"], g["h"], g["sigma2"], g["XL"], g["y"], g["x"], route=route)
    np.testing.assert_allclose(b2[0, 0], g["b"], rtol=1e-14, atol=1e-14)


def test_hand_example_diagonal_M():
    g = load("hand_wls_n3.txt")
    for route in ("hoisted", "per_snp", "explicit"):
        b, w, _ = G.gls(g["M"], None, None, g["XL"], g["y"], g["x"], is_phi=False, route=route)
        np.testing.assert_allclose(b[0, 0], g["b"], rtol=1e-14)
        np.testing.assert_allclose(w[0, 0], g["wald"], rtol=1e-14)


def test_exact_oracle_on_hand_example():
    g = load("hand_gls_n3.txt")
    X = np.hstack([g["XL"], g["x"].astype(float)])
    b, wald = E.gls_exact(g["M"].astype(int).tolist(), X.astype(int).tolist(),
                          g["y"].astype(int).tolist())
    assert [float(v) for v in b] == [1.0, 1.5]
    assert float(wald) == 2.25


# -------------------------------------------------------------- cholesky -----
def test_cholesky_by_hand():
    np.testing.assert_array_equal(G.cholesky_plain(np.array([[9.0]])), [[3.0]])
    L = G.cholesky_plain(np.array([[4.0, 2.0], [2.0, 5.0]]))
    np.testing.assert_array_equal(L, [[2.0, 0.0], [1.0, 2.0]])


@pytest.mark.parametrize("n", [1, 7, 64, 300])
def test_cholesky_reconstruction(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    M = A @ A.T + n * np.eye(n)
    L = G.cholesky_plain(M)
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.all(np.diag(L) > 0)
    err = np.linalg.norm(L @ L.T - M) / np.linalg.norm(M)
    assert err <= 10 * n * EPS
    np.testing.assert_allclose(L, G.cholesky(M, "lapack"), rtol=1e-12, atol=1e-12 * np.abs(L).max())


def test_cholesky_not_spd_reports_pivot():
    M = np.eye(5)
    M[3, 3] = -1.0
    with pytest.raises(G.NotSPDError) as ei:
        G.cholesky_plain(M)
    assert ei.value.pivot == 3


def test_forward_substitution():
    rng = np.random.default_rng(3)
    n = 200
    A = rng.standard_normal((n, n))
    L = np.linalg.cholesky(A @ A.T + n * np.eye(n))
    B = rng.integers(0, 3, size=(n, 5)).astype(float)
    X1 = G.forward_substitution_plain(L, B)
    assert np.max(np.abs(L @ X1 - B)) <= 50 * n * EPS * np.max(np.abs(B))
    np.testing.assert_allclose(X1, G.forward_substitution(L, B, "lapack"), rtol=1e-12, atol=1e-13)


# ----------------------------------------------------- exact arithmetic ------
@pytest.mark.parametrize("seed,n,q", [(0, 5, 1), (1, 6, 2), (2, 8, 3), (3, 7, 3)])
def test_fp64_routes_match_exact_rational(seed, n, q):
    rng = np.random.default_rng(seed)
    A = rng.integers(-3, 4, size=(n, n))
    M = (A @ A.T + 2 * np.eye(n, dtype=int)).astype(int)
    XL = np.ones((n, q), dtype=int)
    if q > 1:
        XL[:, 1:] = rng.integers(-4, 5, size=(n, q - 1))
    x = rng.integers(0, 3, size=(n, 1))
    y = rng.integers(-9, 10, size=n)
    X = np.hstack([XL, x])
    bx, wx = E.gls_exact(M.tolist(), X.tolist(), y.tolist())
    bx = np.array([float(v) for v in bx])
    for route in ("hoisted", "per_snp", "explicit"):
        b, w, s = G.gls(M.astype(float), None, None, XL.astype(float), y.astype(float),
                        x.astype(np.int8), is_phi=False, route=route)
        assert s[0] == 0
        assert rel_b(b[0, 0], bx) <= 1e-11
        assert abs(w[0, 0] - float(wx)) <= 1e-10 * max(1.0, float(wx))


# -------------------------------------------------- textbook closed forms ----
@pytest.mark.parametrize("sigma2", [1.0, 0.37, 5.0])
def test_h0_is_ols(sigma2):
    c, X = small_case(11, 150, 40, h=0.0, sigma2=sigma2)
    b, w, s = G.gls(c.phi, 0.0, sigma2, c.XL, c.Y, X)
    assert np.all(s == 0)
    for i in range(X.shape[1]):
        Xi = np.hstack([c.XL, X[:, i:i + 1].astype(float)])
        ref, *_ = np.linalg.lstsq(Xi, c.Y[:, 0], rcond=None)
        assert rel_b(b[i, 0], ref) <= 1e-11
        # Wald with known variance sigma^2: b_p^2 / (sigma^2 [(X^T X)^{-1}]_pp)
        wref = ref[-1] ** 2 / (sigma2 * np.linalg.inv(Xi.T @ Xi)[-1, -1])
        assert abs(w[i, 0] - wref) <= 1e-9 * max(1.0, wref)


def test_qr_cross_check():
    c, X = small_case(5, 120, 30)
    L = G.factor(c.phi, c.h, c.sigma2)
    b, _, _ = G.gls_per_snp(L, c.XL, c.Y, X)
    bq = G.gls_qr(L, c.XL, c.Y, X)
    assert rel_b(b, bq) <= 1e-11


def test_hoisted_equals_eq1_explicit():
    c, X = small_case(6, 64, 50, t=3)
    b1, w1, _ = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X, route="hoisted")
    b2, w2, _ = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X, route="per_snp")
    b3, w3, _ = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X, route="explicit")
    assert rel_b(b1, b2) <= 1e-12
    assert rel_b(b1, b3) <= 1e-11
    assert np.max(np.abs(w1 - w3) / np.maximum(w3, 1.0)) <= 1e-10


# ------------------------------------------------------------ invariances ----
def test_scaling_invariance():
    c, X = small_case(7, 100, 25)
    b1, w1, _ = G.gls(c.phi, c.h, 1.0, c.XL, c.Y, X)
    b2, w2, _ = G.gls(c.phi, c.h, 3.7, c.XL, c.Y, X)
    assert rel_b(b2, b1) <= 1e-12
    # S scales 1/c and b stays: the Wald statistic scales by 1/c
    np.testing.assert_allclose(w2 * 3.7, w1, rtol=1e-10)


def test_permuting_individuals():
    c, X = small_case(8, 90, 20, t=2)
    perm = np.random.default_rng(0).permutation(c.n)
    M = G.build_M(c.phi, c.h, c.sigma2)
    b1, w1, _ = G.gls(M, None, None, c.XL, c.Y, X, is_phi=False)
    b2, w2, _ = G.gls(M[np.ix_(perm, perm)], None, None, c.XL[perm], c.Y[perm],
                      X[perm], is_phi=False)
    assert rel_b(b2, b1) <= 1e-11
    np.testing.assert_allclose(w2, w1, rtol=1e-9, atol=1e-12)


def test_snp_order_and_block_size():
    c, X = small_case(9, 80, 37)
    L = G.factor(c.phi, c.h, c.sigma2)
    b, w, s = G.gls_hoisted(L, c.XL, c.Y, X)
    perm = np.random.default_rng(1).permutation(X.shape[1])
    bp, wp, _ = G.gls_hoisted(L, c.XL, c.Y, X[:, perm])
    assert rel_b(bp, b[perm]) <= 1e-13
    parts = [G.gls_hoisted(L, c.XL, c.Y, X[:, a:a + 10])[0] for a in range(0, 37, 10)]
    assert rel_b(np.concatenate(parts), b) <= 1e-13


def test_S_formed_symmetric():
    c, X = small_case(10, 70, 15)
    L = G.factor(c.phi, c.h, c.sigma2)
    S, R, _ = G.normal_equations_per_snp(L, c.XL, c.Y, X)
    assert np.array_equal(S, np.transpose(S, (0, 2, 1)))
    assert np.all(np.linalg.eigvalsh(S) > 0)


# ------------------------------------------------ multi-trait (Section 5) ---
def test_multitrait_matches_exact_rational_per_trait():
    """Two traits with M_1 = Phi + I (h = 1/2, sigma^2 = 2) and M_2 = Phi + 3 I
    (h = 1/4, sigma^2 = 4), integer Phi: each b_ij against exact rational Eq. (1)."""
    rng = np.random.default_rng(7)
    n, q = 7, 2
    A = rng.integers(-2, 3, size=(n, n))
    phi = (A @ A.T).astype(float)
    XL = np.ones((n, q))
    XL[:, 1] = rng.integers(-3, 4, size=n)
    X = rng.integers(0, 3, size=(n, 3)).astype(np.int8)
    Y = rng.integers(-5, 6, size=(n, 2)).astype(float)
    b, w, s = G.gls_multitrait(phi, [0.5, 0.25], [2.0, 4.0], XL, Y, X)
    assert b.shape == (3, 2, q + 1) and s.shape == (3, 2)
    for j, shift in enumerate((1, 3)):
        Mj = (phi + shift * np.eye(n)).astype(int).tolist()
        for i in range(3):
            Xi = np.hstack([XL, X[:, i:i + 1]]).astype(int).tolist()
            bx, wx = E.gls_exact(Mj, Xi, Y[:, j].astype(int).tolist())
            assert s[i, j] == 0
            assert rel_b(b[i, j], np.array([float(v) for v in bx])) <= 1e-11
            assert abs(w[i, j] - float(wx)) <= 1e-10 * max(1.0, float(wx))


def test_multitrait_with_one_M_is_the_multi_phenotype_solve():
    """Equal (h, sigma^2) for every trait: one shared M, i.e. t phenotype columns."""
    c, X = small_case(13, 90, 12, t=3)
    b, w, s = G.gls_multitrait(c.phi, [c.h] * 3, [c.sigma2] * 3, c.XL, c.Y, X)
    rb, rw, rs = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X, route="explicit")
    assert rel_b(b, rb) <= 1e-11
    assert np.all(s == rs[:, None])


def test_multitrait_trait_order():
    c, X = small_case(14, 80, 9, t=3)
    hs, s2 = [0.1, 0.5, 0.8], [1.0, 0.6, 2.0]
    b, w, s = G.gls_multitrait(c.phi, hs, s2, c.XL, c.Y, X)
    perm = [2, 0, 1]
    bp, wp, sp = G.gls_multitrait(c.phi, [hs[k] for k in perm], [s2[k] for k in perm],
                                  c.XL, c.Y[:, perm], X)
    assert np.array_equal(bp, b[:, perm]) and np.array_equal(wp, w[:, perm])


# ------------------------------------- the p x p matrix S_i^-1 (Section 3) ---
def test_cov_matches_exact_rational_inverse():
    """S_i^-1 = (X_i^T M^-1 X_i)^-1 of both oracle routes against exact rationals."""
    rng = np.random.default_rng(8)
    n, q = 7, 2
    A = rng.integers(-2, 3, size=(n, n))
    M = (A @ A.T + 2 * np.eye(n, dtype=int)).astype(int)
    XL = np.ones((n, q), dtype=int)
    XL[:, 1] = rng.integers(-3, 4, size=n)
    X = rng.integers(0, 3, size=(n, 4)).astype(np.int8)
    Minv = E.inverse(M.tolist())
    for route in ("hoisted", "explicit"):
        cov, st = G.gls_cov(M.astype(float), None, None, XL.astype(float), X, is_phi=False,
                            route=route)
        assert np.all(st == 0)
        for i in range(X.shape[1]):
            Xi = np.hstack([XL, X[:, i:i + 1]]).astype(int).tolist()
            XiT = [list(r) for r in zip(*Xi)]
            Ai = E.matmul(E.matmul(XiT, Minv), Xi)
            ref = np.array([[float(v) for v in row] for row in E.inverse(Ai)])
            assert np.max(np.abs(cov[i] - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_cov_is_consistent_with_wald_and_spd():
    c, X = small_case(15, 120, 20, t=2)
    X = X.copy(order="F")
    X[:, 4] = 1
    cov, st = G.gls_cov(c.phi, c.h, c.sigma2, c.XL, X)
    b, w, s = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    np.testing.assert_array_equal(st, s)
    ok = s == 0
    assert st[4] == 1 and np.all(np.isnan(cov[4]))
    # Wald = b_p^2 / (S^-1)_pp for every phenotype (the oracle's Wald comes from C_pp^2)
    pp = cov[ok][:, -1, -1]
    assert np.max(np.abs(b[ok][:, :, -1] ** 2 / pp[:, None] - w[ok]) / np.maximum(w[ok], 1)) <= 1e-10
    assert np.max(np.abs(cov[ok] - np.transpose(cov[ok], (0, 2, 1)))) <= 1e-12 * np.max(np.abs(cov[ok]))
    assert np.all(np.linalg.eigvalsh(cov[ok]) > 0)


# ------------------------------------------------------- degenerate SNPs -----
def test_degenerate_and_bad_snps():
    c, X = small_case(12, 60, 6)
    X = X.copy(order="F")
    X[:, 1] = 1          # constant column: collinear with the intercept
    X[:, 2] = 0          # all-zero column: S_BR = 0
    X[5, 3] = 3          # dosage outside {0,1,2}
    X[0, 4] = -1
    for route in ("hoisted", "per_snp"):
        b, w, s = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X, route=route)
        assert list(s) == [0, 1, 1, 2, 2, 0]
        assert np.all(np.isnan(b[1:5])) and np.all(np.isnan(w[1:5]))
        assert np.all(np.isfinite(b[[0, 5]]))


# --------------------------------------------- the pins catch planted bugs ---
def _planted(kind, c, X):
    """The hoisted route with one plausible mistake planted in it."""
    L = G.factor(c.phi, c.h, c.sigma2)
    XLbar, ybar, S_TL, bbar_T = G.setup_hoisted(L, c.XL, c.Y)
    if kind == "raw_y_in_bbar_T":       # the typo of Section 2.1 taken literally
        bbar_T = XLbar.T @ c.Y
    elif kind == "transposed_L":        # solve with L^T instead of L
        XLbar = np.linalg.solve(L.T, c.XL)
        ybar = np.linalg.solve(L.T, c.Y)
        S_TL, bbar_T = XLbar.T @ XLbar, XLbar.T @ ybar
    elif kind == "dropped_identity_term":
        L = G.cholesky(c.sigma2 * (c.h * c.phi + np.eye(c.n)))
        XLbar, ybar, S_TL, bbar_T = G.setup_hoisted(L, c.XL, c.Y)
    return G.gls_hoisted(L, c.XL, c.Y, X, setup=(XLbar, ybar, S_TL, bbar_T))


@pytest.mark.parametrize("kind", ["raw_y_in_bbar_T", "transposed_L", "dropped_identity_term"])
def test_planted_mistakes_are_caught(kind):
    c, X = small_case(13, 40, 8)
    ref, _, _ = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X, route="explicit")
    good, _, _ = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    bad, _, _ = _planted(kind, c, X)
    assert rel_b(good, ref) <= 1e-11
    assert rel_b(bad, ref) > 1e-6
