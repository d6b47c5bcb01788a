"""REML likelihood, its adjoint gradient, db_i/dh and the REML fit on the GPU vs the oracle.

Tolerances: l within 1e-10 relative; gradients within 1e-8 of max(|g|, 1) against the
oracle's trace formula and within 1e-6 of central finite differences (step 1e-5) of
the GPU's own l; db_i/dh within 1e-8 relative to max |db_i/dh| of the SNP against the
oracle's generic form; the fitted h within 1e-6 of the oracle's REML maximiser.
"""
import numpy as np
import pytest

import synth
from oracle import gls as G
from oracle import reml as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw(gpu):
    from paper_1304_2272_gb300 import gwas as g
    g.load()
    return g


@pytest.fixture(scope="module")
def cohort():
    return synth.make_cohort(51, 400, t=2, h=0.4, sigma2=1.0, n_markers=500)


def engine(gw, c):
    from paper_1304_2272_gb300.reml import REMLEngine
    return REMLEngine(c.phi, c.XL, c.Y)


# h >= 1e-2 takes the trace identities (no Phi product, no M^-1); 0 <= h < 1e-2 the
# direct route with Phi and M^-1
@pytest.mark.parametrize("h,s2", [(0.1, 1.0), (0.25, 1.3), (0.7, 0.6), (0.01, 0.9),
                                  (0.005, 1.1), (0.0, 0.8)])
def test_reml_matches_oracle(gw, cohort, h, s2):
    c = cohort
    e = engine(gw, c)
    r = e.eval(h, s2)
    ref = R.reml_loglik(c.phi, h, s2, c.XL, c.Y[:, 0])
    gref = R.reml_grad(c.phi, h, s2, c.XL, c.Y[:, 0])
    assert abs(r["loglik"] - ref) <= 1e-10 * abs(ref)
    assert abs(r["dl_dh"] - gref[0]) <= 1e-8 * max(abs(gref[0]), 1.0)
    assert abs(r["dl_dsigma2"] - gref[1]) <= 1e-8 * max(abs(gref[1]), 1.0)
    s2_hat = R.profiled_sigma2(c.phi, h, c.XL, c.Y[:, 0])
    assert abs(r["sigma2_hat"] - s2_hat) <= 1e-10 * s2_hat
    # profiled: everything at sigma2_hat
    rp = e.eval(h, s2, profile=True)
    refp = R.reml_loglik(c.phi, h, s2_hat, c.XL, c.Y[:, 0])
    gp = R.reml_grad(c.phi, h, s2_hat, c.XL, c.Y[:, 0])
    assert abs(rp["loglik"] - refp) <= 1e-10 * abs(refp)
    assert abs(rp["dl_dh"] - gp[0]) <= 1e-8 * max(abs(gp[0]), 1.0)
    assert abs(rp["dl_dsigma2"]) <= 1e-8
    e.close()


@pytest.mark.parametrize("h", [0.1, 0.25])
def test_gpu_gradient_matches_central_differences(gw, cohort, h):
    c = cohort
    e = engine(gw, c)
    s2 = 1.1
    r = e.eval(h, s2)
    step = 1e-5
    fh = (e.eval(h + step, s2)["loglik"] - e.eval(h - step, s2)["loglik"]) / (2 * step)
    fs = (e.eval(h, s2 + step)["loglik"] - e.eval(h, s2 - step)["loglik"]) / (2 * step)
    g0 = abs(e.eval(0.1, s2)["dl_dh"])
    assert abs(fh - r["dl_dh"]) <= 1e-6 * max(abs(r["dl_dh"]), g0)
    assert abs(fs - r["dl_dsigma2"]) <= 1e-6 * max(abs(r["dl_dsigma2"]), g0)
    e.close()


def test_autograd_function(gw, cohort):
    import torch
    from paper_1304_2272_gb300.reml import reml_loglik
    c = cohort
    e = engine(gw, c)
    h = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    s2 = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    l = reml_loglik(h, s2, e)
    l.backward()
    gref = R.reml_grad(c.phi, 0.3, 0.9, c.XL, c.Y[:, 0])
    assert abs(h.grad.item() - gref[0]) <= 1e-8 * max(abs(gref[0]), 1.0)
    assert abs(s2.grad.item() - gref[1]) <= 1e-8 * max(abs(gref[1]), 1.0)
    e.close()


def test_db_dh_matches_oracle_and_finite_differences(gw):
    import torch
    c = synth.make_cohort(52, 300, t=2, h=0.35, sigma2=1.7, n_markers=400)
    X = c.snps(150).copy(order="F")
    X[:, 7] = 1  # degenerate: NaN and status 1
    m = X.shape[1]
    ctx = gw.gwas_init(c.n, 4, 2, m_blk=256)
    try:
        gw.gwas_reml(ctx, np.asfortranarray(c.phi), c.h, c.sigma2, c.XL, c.Y)
        Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
        bd = torch.empty((m, 2, 4), dtype=torch.float64, device="cuda")
        sd = torch.empty(m, dtype=torch.uint8, device="cuda")
        dd = torch.empty((m, 2, 4), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        gw.gwas_solve_block_grad_device(ctx, Xd, m, bd, None, sd, dd)
        gw.gwas_sync(ctx)
        dbdh = dd.cpu().numpy()
        status = sd.cpu().numpy()

        def b_at(h):
            gw.gwas_factor(ctx, np.asfortranarray(c.phi), True, h, c.sigma2, c.XL, c.Y)
            gw.gwas_solve_block_device(ctx, Xd, m, bd, None, sd)
            gw.gwas_sync(ctx)
            return bd.cpu().numpy()

        num = (b_at(c.h + 1e-5) - b_at(c.h - 1e-5)) / 2e-5
    finally:
        gw.gwas_finalize(ctx)
    ref = R.db_dh(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    ok = status == 0
    assert status[7] == 1 and np.all(np.isnan(dbdh[7]))
    scale = np.max(np.abs(ref[ok]), axis=-1, keepdims=True)
    assert np.max(np.abs(dbdh[ok] - ref[ok]) / scale) <= 1e-8
    assert np.max(np.abs(num[ok] - dbdh[ok]) / scale) <= 1e-6


def test_db_dh_needs_reml_state(gw):
    """db/dh without a preceding gwas_reml is refused. The buffers are real device tensors
    of the call's sizes, so even a call that got past the check would only compute."""
    import torch
    c = synth.make_cohort(53, 100, n_markers=200)
    ctx = gw.gwas_init(c.n, 4, 1, m_blk=64)
    try:
        gw.gwas_factor(ctx, np.asfortranarray(c.phi), True, c.h, c.sigma2, c.XL, c.Y)
        Xd = torch.from_numpy(np.ascontiguousarray(c.snps(8).T)).cuda()
        bd = torch.empty((8, 1, 4), dtype=torch.float64, device="cuda")
        sd = torch.empty(8, dtype=torch.uint8, device="cuda")
        dd = torch.empty((8, 1, 4), dtype=torch.float64, device="cuda")
        with pytest.raises(gw.GwasError) as ei:
            gw.gwas_solve_block_grad_device(ctx, Xd, 8, bd, None, sd, dd)
        assert ei.value.status == gw.GWAS_ERR_STATE
    finally:
        gw.gwas_finalize(ctx)


def test_gls_autograd_gives_db_dh(gw):
    """A loss on b_i back-propagates to h through GLSFunction: torch.autograd gives
    sum_i <w_i, db_i/dh>, which must match the oracle's generic db/dh (1e-8) and central
    differences of the loss on the GPU (step 1e-5, 1e-6); the sigma^2 gradient is exactly
    zero (b_i does not change when M is scaled) and so is its central difference (1e-6)."""
    import torch
    from paper_1304_2272_gb300.reml import REMLEngine, gls_b
    c = synth.make_cohort(55, 300, t=2, h=0.35, sigma2=1.7, n_markers=400)
    X = c.snps(150).copy(order="F")
    X[:, 7] = 1      # singular: NaN in b, no contribution to the gradient
    X[4, 11] = 5     # bad dosage: the same
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    wts = torch.from_numpy(np.random.default_rng(3).standard_normal((150, 2, 4))).cuda()
    e = REMLEngine(c.phi, c.XL, c.Y, m_blk=256)

    def loss(hv, s2v, grad=False):
        h = torch.tensor(hv, dtype=torch.float64, requires_grad=grad)
        s2 = torch.tensor(s2v, dtype=torch.float64, requires_grad=grad)
        return (torch.nan_to_num(gls_b(h, s2, Xd, e)) * wts).sum(), h, s2

    try:
        val, h, s2 = loss(c.h, c.sigma2, True)
        e.eval(0.6, 0.9)     # move the context away: backward must return to (h, sigma2)
        val.backward()
        step = 1e-5
        fd_h = (loss(c.h + step, c.sigma2)[0] - loss(c.h - step, c.sigma2)[0]).item() / (2 * step)
        fd_s = (loss(c.h, c.sigma2 + step)[0] - loss(c.h, c.sigma2 - step)[0]).item() / (2 * step)
    finally:
        e.close()
    ref = R.db_dh(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    w = wts.cpu().numpy()
    ok = ~np.isnan(ref)
    assert not ok[7].any() and not ok[11].any()
    expected = float(np.sum(ref[ok] * w[ok]))
    scale = float(np.sum(np.abs(ref[ok] * w[ok])))
    g = h.grad.item()
    print(f"[errors] GLSFunction dL/dh {g:.12e} oracle {expected:.12e} FD {fd_h:.12e}")
    assert abs(g - expected) <= 1e-8 * scale
    assert abs(fd_h - g) <= 1e-6 * scale
    assert s2.grad.item() == 0.0
    assert abs(fd_s) <= 1e-6 * scale


def test_reml_fit_from_h0(gw):
    from paper_1304_2272_gb300.reml import REMLEngine, fit_h
    c = synth.make_cohort(54, 800, h=0.4, sigma2=1.0, n_markers=800)
    e = REMLEngine(c.phi, c.XL, c.Y)
    fit = fit_h(e, h0=0.1)
    e.close()
    h_ref = R.fit_h(c.phi, c.XL, c.Y[:, 0])
    assert abs(fit["h"] - h_ref) <= 1e-6
    assert abs(fit["dl_dh"]) <= 1e-6
    print(f"REML fit: h = {fit['h']:.8f} (oracle {h_ref:.8f}, true 0.4), "
          f"{fit['evals']} evaluations")


@pytest.fixture(scope="module")
def cohort_10k():
    return synth.make_cohort(0, 10000, h=0.4, sigma2=1.0, device="cuda")


@pytest.mark.parametrize("h,s2", [(0.1, 1.0), (0.4, 1.2)])
def test_reml_full_size_matches_oracle(gw, cohort_10k, h, s2):
    """n = 10,000 (the workload the benchmark fits h on): the GPU's trace-identity route
    (h >= 1e-2: Phi from M, tr M^-1 = |L^-1|_F^2) against the oracle's explicit M^-1 and
    Phi, at the small-case bounds (l 1e-10 relative, gradients 1e-8 of max(|g|, 1))."""
    from paper_1304_2272_gb300.reml import REMLEngine
    c = cohort_10k
    e = REMLEngine(c.phi, c.XL, c.Y)
    try:
        r = e.eval(h, s2)
    finally:
        e.close()
    ref = R.reml_loglik(c.phi, h, s2, c.XL, c.Y[:, 0])
    gref = R.reml_grad(c.phi, h, s2, c.XL, c.Y[:, 0])
    print(f"[errors] REML n=10000 h={h}: l {abs(r['loglik'] - ref) / abs(ref):.2e}, "
          f"dl/dh {abs(r['dl_dh'] - gref[0]) / max(abs(gref[0]), 1.0):.2e}, "
          f"dl/ds2 {abs(r['dl_dsigma2'] - gref[1]) / max(abs(gref[1]), 1.0):.2e}")
    assert abs(r["loglik"] - ref) <= 1e-10 * abs(ref)
    assert abs(r["dl_dh"] - gref[0]) <= 1e-8 * max(abs(gref[0]), 1.0)
    assert abs(r["dl_dsigma2"] - gref[1]) <= 1e-8 * max(abs(gref[1]), 1.0)
