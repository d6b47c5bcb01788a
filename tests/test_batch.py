"""Batched cohorts (uneven n, several phenotypes) in one grouped launch, vs the oracle.

Each cohort of a batch is an independent instance of Eq. (1) with its own M, X_L and
Y (t phenotype columns sharing one M); the grouped launch must give every cohort the
results of a single-cohort solve: bitwise for the same kernel arithmetic, and within
the FP64 (1e-10) or mixed (1e-6) tolerance of the oracle.
"""
import numpy as np
import pytest

import synth
from oracle import gls as G

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}
# |dW| / max(W, 1): 3 limbs of 9 bits, 2e3 * 2^-27 (the derivation is in test_parity_mixed.py)
WALD_TOL = {"fp64": 1e-10, "mixed": 1.5e-5}


def rel_b(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


@pytest.fixture(scope="module")
def gw(gpu):
    from paper_1304_2272_gb300 import gwas as g
    g.load()
    return g


def make_batch(seeds_n, t, m_of, n_markers=400, h_of=None):
    cohorts, Xs = [], []
    for k, (seed, n) in enumerate(seeds_n):
        h = 0.4 if h_of is None else h_of(k)
        c = synth.make_cohort(seed, n, t=t, h=h, n_markers=n_markers)
        cohorts.append(c)
        Xs.append(c.snps(m_of(k)))
    return cohorts, Xs


def run_batch(gw, cohorts, Xs, precision, solves=1, **opts):
    import torch
    prec = gw.GWAS_PREC_FP64 if precision == "fp64" else gw.GWAS_PREC_MIXED
    t = cohorts[0].t
    m_blk = max(X.shape[1] for X in Xs)
    b = gw.gwas_batch_init([c.n for c in cohorts], 4, t, precision=prec, m_blk=m_blk, **opts)
    try:
        for k, c in enumerate(cohorts):
            gw.gwas_batch_factor(b, k, np.asfortranarray(c.phi), True, c.h, c.sigma2, c.XL, c.Y)
        Xd = [torch.from_numpy(np.ascontiguousarray(X.T)).cuda() for X in Xs]
        outs = []
        for _ in range(solves):
            bd = [torch.full((X.shape[1], t, 4), -1.0, dtype=torch.float64, device="cuda") for X in Xs]
            wd = [torch.full((X.shape[1], t), -1.0, dtype=torch.float64, device="cuda") for X in Xs]
            sd = [torch.full((X.shape[1],), 9, dtype=torch.uint8, device="cuda") for X in Xs]
            torch.cuda.synchronize()
            gw.gwas_batch_solve_device(b, Xd, [X.shape[1] for X in Xs], bd, wd, sd)
            gw.gwas_batch_sync(b)
            outs.append([(x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy())
                         for x, y, z in zip(bd, wd, sd)])
        stats = gw.gwas_batch_get_stats(b)
    finally:
        gw.gwas_batch_finalize(b)
    return outs, stats


# mixed batches: the CTA-pair kernel (default) or one CTA per 128-SNP tile (tile_cfg bit 12);
# a separate linear tile (default) or linear rows fused into the limb tiles (bit 17)
VARIANTS = {"pair": -1, "single": 1 << 12, "pair_fused": 1 << 17,
            "single_fused": (1 << 17) | (1 << 12),
            # the linear rows as the last rows of the last limb tile (bit 21)
            "pair_ztail": 1 << 21, "single_ztail": (1 << 21) | (1 << 12)}


@pytest.mark.parametrize("precision,variant", [("fp64", "pair"), ("mixed", "pair"),
                                               ("mixed", "single"), ("mixed", "pair_ztail")])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_batch_uneven_cohorts_vs_oracle(gw, precision, variant, use_graph):
    seeds_n = [(1, 129), (2, 300), (3, 64), (4, 1003), (5, 517)]
    cohorts, Xs = make_batch(seeds_n, t=3, m_of=lambda k: [70, 257, 1, 300, 128][k],
                             h_of=lambda k: 0.2 + 0.15 * k)
    outs, stats = run_batch(gw, cohorts, Xs, precision, solves=2, use_graph=use_graph,
                            tile_cfg=VARIANTS[variant])
    assert stats["trsm_launches"] == 2
    for (b1, w1, s1), (b2, w2, s2) in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(b1, b2)   # a replayed graph gives the same bits
        np.testing.assert_array_equal(s1, s2)
    for c, X, (b, w, s) in zip(cohorts, Xs, outs[0]):
        rb, rw, rs = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
        np.testing.assert_array_equal(s, rs)
        ok = rs == 0
        assert rel_b(b[ok], rb[ok]) <= TOL[precision]
        assert float(np.max(np.abs(w[ok] - rw[ok]) / np.maximum(rw[ok], 1.0))) <= WALD_TOL[precision]


@pytest.mark.parametrize("precision,variant,t", [("fp64", "pair", 2), ("mixed", "pair", 2),
                                                 ("mixed", "single", 3), ("mixed", "pair_fused", 2),
                                                 ("mixed", "single_fused", 3),
                                                 ("mixed", "pair_ztail", 2),
                                                 ("mixed", "single_ztail", 3)])
def test_batch_matches_single_cohort_bitwise(gw, precision, variant, t):
    seeds_n = [(11, 250), (12, 700), (13, 90)]
    cohorts, Xs = make_batch(seeds_n, t=t, m_of=lambda k: [333, 129, 64][k])
    cfg = VARIANTS[variant]
    outs, _ = run_batch(gw, cohorts, Xs, precision, tile_cfg=cfg)
    prec = gw.GWAS_PREC_FP64 if precision == "fp64" else gw.GWAS_PREC_MIXED
    for c, X, (b, w, s) in zip(cohorts, Xs, outs[0]):
        # a single context with the batch's tile configuration runs the same kernel variant
        with gw.GLS(c.n, 4, c.t, precision=prec, m_blk=X.shape[1], tile_cfg=cfg) as e:
            e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
            rb, rw, rs = e.solve(X)
        np.testing.assert_array_equal(b, rb)
        np.testing.assert_array_equal(w, rw)
        np.testing.assert_array_equal(s, rs)


def test_batch_repointing_rebuilds_the_graph(gw):
    import torch
    seeds_n = [(21, 200), (22, 350)]
    cohorts, Xs = make_batch(seeds_n, t=1, m_of=lambda k: 200)
    b = gw.gwas_batch_init([c.n for c in cohorts], 4, 1, precision=gw.GWAS_PREC_MIXED, m_blk=256)
    try:
        for k, c in enumerate(cohorts):
            gw.gwas_batch_factor(b, k, np.asfortranarray(c.phi), True, c.h, c.sigma2, c.XL, c.Y)
        refs = [G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X) for c, X in zip(cohorts, Xs)]
        for mbs in ([200, 200], [150, 37], [200, 200]):
            Xd = [torch.from_numpy(np.ascontiguousarray(X[:, :m].T)).cuda() for X, m in zip(Xs, mbs)]
            bd = [torch.empty((m, 1, 4), dtype=torch.float64, device="cuda") for m in mbs]
            sd = [torch.empty((m,), dtype=torch.uint8, device="cuda") for m in mbs]
            torch.cuda.synchronize()
            gw.gwas_batch_solve_device(b, Xd, mbs, bd, None, sd)
            gw.gwas_batch_sync(b)
            for (rb, _, rs), x, m in zip(refs, bd, mbs):
                assert rel_b(x.cpu().numpy(), rb[:m]) <= 1e-6
    finally:
        gw.gwas_batch_finalize(b)


def test_batch_sampled_cohorts_like_the_batched_workload(gw):
    """8 cohorts, n ~ U[1000, 8000], 16 phenotypes, h ~ U(0.2, 0.8), mixed, sampled SNPs."""
    import torch
    rng = np.random.default_rng(7)
    ns = sorted(rng.integers(1000, 8001, size=8).tolist())
    hs = rng.uniform(0.2, 0.8, size=8)
    cohorts = [synth.make_cohort(100 + k, n, t=16, h=float(hs[k]), device="cuda")
               for k, n in enumerate(ns)]
    mb = 2048
    Xd = [synth.genotypes_torch(500 + k, c.n, mb, "cuda") for k, c in enumerate(cohorts)]
    b = gw.gwas_batch_init(ns, 4, 16, precision=gw.GWAS_PREC_MIXED, m_blk=mb)
    try:
        for k, c in enumerate(cohorts):
            gw.gwas_batch_factor(b, k, np.asfortranarray(c.phi), True, c.h, c.sigma2, c.XL, c.Y)
        bd = [torch.empty((mb, 16, 4), dtype=torch.float64, device="cuda") for _ in ns]
        sd = [torch.empty((mb,), dtype=torch.uint8, device="cuda") for _ in ns]
        torch.cuda.synchronize()
        gw.gwas_batch_solve_device(b, Xd, [mb] * 8, bd, None, sd)
        gw.gwas_batch_sync(b)
    finally:
        gw.gwas_batch_finalize(b)
    for k, c in enumerate(cohorts):
        idx = np.unique(np.r_[0, mb - 1, rng.choice(mb, 30, replace=False)])
        Xs = np.asfortranarray(Xd[k][idx].cpu().numpy().T)
        L = G.factor(c.phi, c.h, c.sigma2)
        rb, _, rs = G.gls_hoisted(L, c.XL, c.Y, Xs)
        s = sd[k].cpu().numpy()[idx]
        np.testing.assert_array_equal(s, rs)
        assert rel_b(bd[k].cpu().numpy()[idx], rb) <= 1e-6
