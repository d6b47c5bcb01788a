"""FP64 CUDA path vs the CPU oracle, through the C ABI (GPU tests).

Tolerance (FP64 path): every coefficient of b_i within 1e-10 of the oracle, relative
to max_c |b_ic| of the same SNP (the intercept included). The Wald statistic is
derived from b_i: to first order its error is 2 sqrt(W) C_pp |db_p| (C_pp =
1/sqrt((S^{-1})_pp), max|b| C_pp below 1e3 here) plus W times the relative error of
(S^{-1})_pp. The FP64 path's b is within a few n u (u = 2^-53) of the oracle's, about
1e-12 at n = 10^4, so the tests hold |dW| <= 1e-10 max(W, 1) (2e3 times that). Status
codes must match exactly.
"""
import numpy as np
import pytest

import synth
from oracle import gls as G
from tests.golden.load import load

pytestmark = pytest.mark.gpu

B_TOL = 1e-10
W_TOL = 1e-10


def rel_b(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


def assert_parity(out, ref):
    b, w, s = out
    rb, rw, rs = ref
    np.testing.assert_array_equal(s, rs)
    ok = rs == 0
    assert np.all(np.isnan(b[~ok])) and np.all(np.isnan(w[~ok]))
    if ok.any():
        eb = rel_b(b[ok], rb[ok])
        ew = float(np.max(np.abs(w[ok] - rw[ok]) / np.maximum(rw[ok], 1.0)))
        print(f"[errors] fp64 {b.shape}: b {eb:.3e} wald {ew:.3e}")
        assert eb <= B_TOL
        assert ew <= W_TOL


@pytest.fixture(scope="module")
def gwas(gpu):
    from paper_1304_2272_gb300 import gwas as g
    g.load()
    return g


def run(gwas, c, X, **opts):
    with gwas.GLS(c.n, c.q + 1, c.t, **opts) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        return e.solve(X)


def oracle(c, X):
    return G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)


def test_small_workload_full_parity(gwas):
    # n = 1000, p = 4, m = 10,000, h = 0.4, sigma^2 = 1, Phi from 5000 markers
    c = synth.make_cohort(0, 1000)
    X = c.snps(10000)
    out = run(gwas, c, X, m_blk=4096)  # 2 full blocks + a ragged one
    assert_parity(out, oracle(c, X))


@pytest.mark.parametrize("n,m,p,t,mblk", [
    (2, 5, 2, 1, 4), (17, 9, 3, 2, 4), (64, 65, 4, 1, 64), (65, 130, 4, 3, 100),
    (257, 300, 5, 1, 128), (1003, 333, 4, 1, 128), (130, 70, 20, 1, 64), (200, 50, 4, 16, 32),
    (150, 40, 4, 64, 64), (140, 33, 20, 64, 32),   # the largest t (64) and p (20)
])
def test_ragged_shapes(gwas, n, m, p, t, mblk):
    c = synth.make_cohort(100 + n, n, q=p - 1, t=t, n_markers=300)
    X = c.snps(m)
    assert_parity(run(gwas, c, X, m_blk=mblk), oracle(c, X))


@pytest.mark.parametrize("name", ["hand_gls_n3.txt", "hand_wls_n3.txt"])
def test_hand_examples(gwas, name):
    g = load(name)
    with gwas.GLS(3, 2, 1) as e:
        e.factor(g["M"], XL=g["XL"], Y=g["y"], is_phi=False)
        b, w, s = e.solve(g["x"])
    assert s[0] == 0
    np.testing.assert_allclose(b[0, 0], g["b"], rtol=1e-13)
    np.testing.assert_allclose(w[0, 0], g["wald"], rtol=1e-12)


def test_degenerate_and_bad_snps(gwas):
    c = synth.make_cohort(12, 300, n_markers=400)
    X = c.snps(70).copy(order="F")
    X[:, 1] = 1
    X[:, 2] = 0
    X[5, 3] = 3
    X[0, 4] = -1
    X[:, 69] = 2
    out = run(gwas, c, X, m_blk=64)
    ref = oracle(c, X)
    assert list(out[2][:6]) == [0, 1, 1, 2, 2, 0] and out[2][69] == 1
    assert_parity(out, ref)


def test_not_spd_reports_pivot(gwas):
    n = 150
    rng = np.random.default_rng(0)
    A = rng.standard_normal((n, n))
    M = A @ A.T / n + np.eye(n)
    M[97, 97] = -5.0
    with pytest.raises(G.NotSPDError) as ei:
        G.cholesky_plain(M)
    with gwas.GLS(n, 4, 1) as e:
        with pytest.raises(gwas.GwasError) as ge:
            e.factor(M, XL=np.ones((n, 3)), Y=np.ones(n), is_phi=False)
        assert ge.value.status == gwas.GWAS_ERR_NOT_SPD
        assert ge.value.index == ei.value.pivot
        # no solve without a successful factorisation
        with pytest.raises(gwas.GwasError) as se:
            e.solve(np.zeros((n, 3), dtype=np.int8))
        assert se.value.status == gwas.GWAS_ERR_STATE


def test_block_size_and_snp_order_bitwise(gwas):
    c = synth.make_cohort(21, 500, n_markers=600)
    X = c.snps(400)
    b1, w1, s1 = run(gwas, c, X, m_blk=64)
    b2, w2, s2 = run(gwas, c, X, m_blk=4096)
    np.testing.assert_array_equal(b1, b2)
    np.testing.assert_array_equal(w1, w2)
    perm = np.random.default_rng(3).permutation(400)
    b3, _, _ = run(gwas, c, np.asfortranarray(X[:, perm]), m_blk=128)
    np.testing.assert_array_equal(b3, b1[perm])


def test_device_entry_point_matches_host(gwas):
    import torch
    c = synth.make_cohort(31, 700, n_markers=800)
    X = c.snps(1000)
    ref = run(gwas, c, X, m_blk=1000)
    e = gwas.GLS(c.n, 4, 1, m_blk=1000)
    e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()  # SNP-major = column-major n x m
    bd = torch.empty((1000, 1, 4), dtype=torch.float64, device="cuda")
    wd = torch.empty((1000, 1), dtype=torch.float64, device="cuda")
    sd = torch.empty(1000, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    gwas.gwas_solve_block_device(e.ctx, Xd, 1000, bd, wd, sd)
    gwas.gwas_sync(e.ctx)
    np.testing.assert_array_equal(bd.cpu().numpy(), ref[0])
    np.testing.assert_array_equal(wd.cpu().numpy(), ref[1])
    np.testing.assert_array_equal(sd.cpu().numpy(), ref[2])
    st = e.stats()
    assert st["trsm_launches"] >= 1 and st["kernel_launches"] >= 2
    e.close()


def test_sync_with_timeout_never_hangs(gwas):
    c = synth.make_cohort(41, 2000, n_markers=500)
    X = c.snps(4096)
    e = gwas.GLS(c.n, 4, 1, m_blk=4096)
    e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
    b = np.empty((4096, 1, 4))
    w = np.empty((4096, 1))
    s = np.empty(4096, dtype=np.uint8)
    gwas.gwas_solve_block(e.ctx, X, 4096, b, w, s)
    try:
        gwas.gwas_sync(e.ctx, 0)
    except gwas.GwasError as err:
        assert err.status == gwas.GWAS_ERR_TIMEOUT
    gwas.gwas_sync(e.ctx, -1)
    assert_parity((b, w, s), oracle(c, X))
    e.close()


def test_multi_phenotype(gwas):
    c = synth.make_cohort(51, 800, t=16, n_markers=900)
    X = c.snps(500)
    assert_parity(run(gwas, c, X, m_blk=256), oracle(c, X))


def test_sigma_scaling_and_h0(gwas):
    c = synth.make_cohort(61, 400, h=0.0, sigma2=2.5, n_markers=500)
    X = c.snps(200)
    b, w, s = run(gwas, c, X, m_blk=256)
    for i in range(0, 200, 37):
        Xi = np.hstack([c.XL, X[:, i:i + 1].astype(float)])
        ref, *_ = np.linalg.lstsq(Xi, c.Y[:, 0], rcond=None)
        assert rel_b(b[i, 0], ref) <= B_TOL


def test_full_size_sampled(gwas):
    """n = 10,000 in the benchmark's launch shape (one block of 16,384 SNPs)."""
    import torch
    n, mb = 10000, 16384
    c = synth.make_cohort(0, n, device="cuda")
    Xd = synth.genotypes_torch(5, n, mb, "cuda")
    e = gwas.GLS(n, 4, 1, m_blk=mb)
    e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
    bd = torch.empty((mb, 1, 4), dtype=torch.float64, device="cuda")
    wd = torch.empty((mb, 1), dtype=torch.float64, device="cuda")
    sd = torch.empty(mb, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    gwas.gwas_solve_block_device(e.ctx, Xd, mb, bd, wd, sd)
    gwas.gwas_sync(e.ctx)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, mb - 1], rng.choice(mb, 254, replace=False)]))
    Xs = np.asfortranarray(Xd[idx].cpu().numpy().T)
    L = G.factor(c.phi, c.h, c.sigma2)
    ref = G.gls_hoisted(L, c.XL, c.Y, Xs)
    out = (bd.cpu().numpy()[idx], wd.cpu().numpy()[idx], sd.cpu().numpy()[idx])
    assert_parity(out, ref)
    e.close()


def test_timing_over_many_blocks(gwas):
    """With timing on, the event times of a long run are folded as launches complete:
    every launch is counted once."""
    c = synth.make_cohort(60, 128, n_markers=200)
    X = c.snps(64 * 150)
    with gwas.GLS(c.n, 4, 1, m_blk=64, timing=1) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        out = e.solve(X)
        st = e.stats()
    assert st["trsm_launches"] == 150 and st["blocks"] == 150 and st["trsm_ms"] > 0
    assert_parity(out, oracle(c, X))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_cov_output_matches_oracle(gwas, precision, tol):
    """S_i^-1 (the p x p matrix beside b_i) against the oracle, NaN where status != 0."""
    import torch
    c = synth.make_cohort(91, 400, t=2, n_markers=300)
    X = c.snps(300).copy(order="F")
    X[:, 5] = 2
    X[0, 6] = 5
    mb, p = X.shape[1], 4
    prec = gwas.GWAS_PREC_FP64 if precision == "fp64" else gwas.GWAS_PREC_MIXED
    with gwas.GLS(c.n, p, 2, m_blk=512, precision=prec) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
        bd = torch.empty((mb, 2, p), dtype=torch.float64, device="cuda")
        wd = torch.empty((mb, 2), dtype=torch.float64, device="cuda")
        sd = torch.empty(mb, dtype=torch.uint8, device="cuda")
        cd = torch.empty((mb, p, p), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        gwas.gwas_solve_block_cov_device(e.ctx, Xd, mb, bd, wd, sd, cd)
        gwas.gwas_sync(e.ctx)
        with pytest.raises(gwas.GwasError):
            gwas.gwas_solve_block_cov_device(e.ctx, Xd, mb, bd, wd, sd, None)
    cov = cd.cpu().numpy().transpose(0, 2, 1)      # each matrix column-major
    st = sd.cpu().numpy()
    ref, rs = G.gls_cov(c.phi, c.h, c.sigma2, c.XL, X)
    np.testing.assert_array_equal(st, rs)
    assert st[5] == 1 and st[6] == 2 and np.all(np.isnan(cov[st != 0]))
    ok = rs == 0
    scale = np.max(np.abs(ref[ok]), axis=(1, 2), keepdims=True)
    assert np.max(np.abs(cov[ok] - ref[ok]) / scale) <= tol
    # the Wald statistic is b_p^2 / (S^-1)_pp
    w = wd.cpu().numpy()[ok]
    b = bd.cpu().numpy()[ok]
    assert np.max(np.abs(b[:, :, -1] ** 2 / cov[ok][:, -1, -1][:, None] - w) / np.maximum(w, 1)) <= 1e-9
