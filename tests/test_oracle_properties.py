"""Property checks of the CPU oracle over random small problems (hypothesis, CPU only):
the three routes to Eq. (1) agree, b is invariant to scaling M and to permuting
individuals, and S_i^-1 agrees with the Wald statistic."""
import numpy as np
import pytest

from oracle import gls as G

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")


def problem(seed, n, q, t, m):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    M = A @ A.T / n + np.eye(n)
    XL = np.column_stack([np.ones(n)] + [rng.standard_normal(n) for _ in range(q - 1)])
    Y = rng.standard_normal((n, t))
    X = rng.integers(0, 3, size=(n, m)).astype(np.int8)
    return M, XL, Y, X


def rel(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


@hyp.settings(max_examples=40, deadline=None)
@hyp.given(seed=st.integers(0, 10**6), n=st.integers(8, 40), q=st.integers(1, 4),
           t=st.integers(1, 3), m=st.integers(1, 6))
def test_routes_scaling_and_permutation(seed, n, q, t, m):
    M, XL, Y, X = problem(seed, n, q, t, m)
    b1, w1, s1 = G.gls(M, None, None, XL, Y, X, is_phi=False)
    b2, w2, s2 = G.gls(M, None, None, XL, Y, X, is_phi=False, route="per_snp")
    b3, w3, s3 = G.gls(M, None, None, XL, Y, X, is_phi=False, route="explicit")
    ok = (s1 == 0) & (s2 == 0) & (s3 == 0)
    if not ok.any():
        return
    assert rel(b1[ok], b3[ok]) <= 1e-8 and rel(b2[ok], b3[ok]) <= 1e-8
    bs, _, _ = G.gls(3.7 * M, None, None, XL, Y, X, is_phi=False)
    assert rel(bs[ok], b1[ok]) <= 1e-9
    perm = np.random.default_rng(seed + 1).permutation(n)
    bp, _, _ = G.gls(M[np.ix_(perm, perm)], None, None, XL[perm], Y[perm], X[perm], is_phi=False)
    assert rel(bp[ok], b1[ok]) <= 1e-8
    cov, sc = G.gls_cov(M, None, None, XL, X, is_phi=False)
    good = ok & (sc == 0)
    pp = cov[good][:, -1, -1]
    wald = b1[good][:, :, -1] ** 2 / pp[:, None]
    assert np.max(np.abs(wald - w1[good]) / np.maximum(w1[good], 1.0)) <= 1e-8
