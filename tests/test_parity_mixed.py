"""Mixed-precision CUDA path (BF16 limbs of L^{-1} on tcgen05) vs the FP64 oracle.

Tolerance: every coefficient of b_i within 1e-6 of the FP64 oracle, relative to
max_c |b_ic| of the same SNP, for 3 limbs (the contract of the mixed path). Each limb
adds 9 bits: the limb truncation is 2^-9S of the tile maximum of L^{-1} per element.
With 2 limbs (2^-18) the tests hold b to 1e-4; with 4 limbs (2^-36) to 1e-9 (measured
~2e-11); with 5 limbs (2^-45) to the FP64 path's own 1e-10 (measured ~6e-14).

The Wald statistic W = b_p^2 / (S^{-1})_pp has, to first order, the error
2 sqrt(W) C_pp |db_p| (C_pp = (S^{-1})_pp^{-1/2}, the inverse standard error of the SNP
effect) plus W times the relative error of (S^{-1})_pp. With |db_p| about 2^-BS max|b|
for S limbs of B bits and max|b| C_pp below 1e3 in these workloads, |dW| / max(W, 1) is
held to 2e3 * 2^-BS (at least 1e-10): 7.6e-3 for 2 limbs, 1.5e-5 for 3, 2.9e-8 for 4 and
1e-10 for 5 (9-bit limbs).
"""
import numpy as np
import pytest

import synth
from oracle import gls as G

pytestmark = pytest.mark.gpu

TOL = {2: 1e-4, 3: 1e-6, 4: 1e-9, 5: 1e-10}


def wald_tol(limbs, bits=9):
    """Bound on |dW| / max(W, 1) for `limbs` limbs of `bits` bits (module docstring)."""
    return max(2e3 * 2.0 ** (-bits * limbs), 1e-10)


WALD_TOL = {s: wald_tol(s) for s in (2, 3, 4, 5)}
# tile_cfg bits: 12 forces one CTA per 128-SNP tile, 13 forces CTA pairs (cta_group::2),
# 17 fuses the linear rows into the limb tiles (a separate linear tile by default)
VARIANTS = {"default": -1, "single": 1 << 12, "pair": 1 << 13,
            "single_fused": (1 << 17) | (1 << 12), "pair_fused": (1 << 17) | (1 << 13),
            # the linear rows as the last rows of the last limb tile (bit 21)
            "single_ztail": (1 << 21) | (1 << 12), "pair_ztail": (1 << 21) | (1 << 13)}


def rel_b(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


def wald_err(w, rw):
    return float(np.max(np.abs(w - rw) / np.maximum(rw, 1.0)))


@pytest.fixture(scope="module")
def gwas(gpu):
    from paper_1304_2272_gb300 import gwas as g
    g.load()
    return g


def run(gwas, c, X, limbs=3, **opts):
    with gwas.GLS(c.n, c.q + 1, c.t, precision=gwas.GWAS_PREC_MIXED, n_limbs=limbs,
                  **opts) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        return e.solve(X)


def check(out, ref, limbs):
    b, w, s = out
    rb, rw, rs = ref
    np.testing.assert_array_equal(s, rs)
    ok = rs == 0
    assert np.all(np.isnan(b[~ok])) and np.all(np.isnan(w[~ok]))
    eb = rel_b(b[ok], rb[ok]) if ok.any() else 0.0
    ew = wald_err(w[ok], rw[ok]) if ok.any() else 0.0
    print(f"[errors] limbs={limbs} n={b.shape} b {eb:.3e} wald {ew:.3e}")
    assert eb <= TOL[limbs], f"b error {eb:.3e}"
    assert ew <= WALD_TOL[limbs], f"Wald error {ew:.3e}"
    return eb, ew


def oracle(c, X):
    return G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)


@pytest.mark.parametrize("variant", ["single_fused", "single", "pair", "pair_fused", "default",
                                     "pair_ztail", "single_ztail"])
def test_mixed_small_first(gwas, variant):
    c = synth.make_cohort(3, 128, n_markers=200)
    X = c.snps(130)
    check(run(gwas, c, X, m_blk=256, tile_cfg=VARIANTS[variant]), oracle(c, X), 3)


@pytest.mark.parametrize("variant", ["default", "pair", "single", "pair_fused", "single_fused",
                                     "pair_ztail", "single_ztail"])
def test_mixed_small_workload_full(gwas, variant):
    # n = 1000, p = 4, m = 10,000 (the oracle-sized workload), 3 limbs
    c = synth.make_cohort(0, 1000)
    X = c.snps(10000)
    eb, ew = check(run(gwas, c, X, m_blk=4096, tile_cfg=VARIANTS[variant]), oracle(c, X), 3)
    print(f"n=1000 mixed x3 ({variant}): max rel b err {eb:.2e}, Wald err {ew:.2e}")


def tol_bits(bits_per_limb, limbs):
    """b tolerance for limbs of B bits: 2^6 times the truncation 2^-BS of the tile maximum
    (the 9-bit limbs measure 1.3x-2.3x of 2^-BS at n = 1000)."""
    return max(2.0 ** (6 - bits_per_limb * limbs), 1e-13)


@pytest.mark.parametrize("cap,bits", [(1, 8), (2, 7)])
@pytest.mark.parametrize("limbs", [3, 4, 5])
def test_smaller_limb_radix(gwas, cap, bits, limbs):
    """8- and 7-bit limbs (the radix taken for n >= 32768 and n >= 65536), forced at
    n = 1000 through tile_cfg bits 15-16; the separate, fused and last-tile linear layouts."""
    c = synth.make_cohort(0, 1000)
    X = c.snps(3000)
    ref = oracle(c, X)
    for extra in (0, 1 << 17, 1 << 21):
        out = run(gwas, c, X, limbs=limbs, m_blk=1024, tile_cfg=(cap << 15) | extra)
        b, w, s = out
        np.testing.assert_array_equal(s, ref[2])
        ok = ref[2] == 0
        eb = rel_b(b[ok], ref[0][ok])
        ew = wald_err(w[ok], ref[1][ok])
        print(f"[errors] n=1000 mixed x{limbs} of {bits} bits (layout bits {extra:#x}): max rel b "
              f"err {eb:.2e}, Wald err {ew:.2e}")
        assert eb <= tol_bits(bits, limbs)
        assert ew <= wald_tol(limbs, bits)


@pytest.mark.parametrize("limbs", [4, 5])
@pytest.mark.parametrize("variant", ["default", "pair"])
def test_mixed_more_limbs_full(gwas, limbs, variant):
    # n = 1000, m = 10,000 with 4 and 5 limbs (5: the FP64 tolerance)
    c = synth.make_cohort(0, 1000)
    X = c.snps(10000)
    eb, ew = check(run(gwas, c, X, limbs=limbs, m_blk=4096, tile_cfg=VARIANTS[variant]),
                   oracle(c, X), limbs)
    print(f"n=1000 mixed x{limbs} ({variant}): max rel b err {eb:.2e}, Wald err {ew:.2e}")


@pytest.mark.parametrize("layout", ["", "_fused", "_ztail"])
@pytest.mark.parametrize("limbs", [2, 3, 4, 5])
def test_pair_and_single_cta_bitwise(gwas, limbs, layout):
    # both variants use the same tile height and N = 256 tile (limb rows, fused linear
    # rows, zero rows), hence the same limbs and the same partial sums
    c = synth.make_cohort(23, 700, n_markers=700)
    X = c.snps(777)
    v1, v2 = "pair" + layout, "single" + layout
    b1, w1, _ = run(gwas, c, X, limbs=limbs, m_blk=1024, tile_cfg=VARIANTS[v1])
    b2, w2, _ = run(gwas, c, X, limbs=limbs, m_blk=1024, tile_cfg=VARIANTS[v2])
    np.testing.assert_array_equal(b1, b2)
    np.testing.assert_array_equal(w1, w2)


@pytest.mark.parametrize("variant", ["pair", "single", "pair_fused", "single_fused", "pair_ztail",
                                     "single_ztail"])
@pytest.mark.parametrize("limbs", [2, 3, 4, 5])
@pytest.mark.parametrize("n,m,p,t,mblk", [
    (64, 1, 4, 1, 64), (65, 127, 4, 1, 128), (130, 129, 3, 2, 128), (1003, 300, 4, 3, 512),
    (200, 257, 6, 1, 256),
])
def test_mixed_ragged(gwas, variant, limbs, n, m, p, t, mblk):
    c = synth.make_cohort(200 + n + limbs, n, q=p - 1, t=t, n_markers=300)
    X = c.snps(m)
    check(run(gwas, c, X, limbs=limbs, m_blk=mblk, tile_cfg=VARIANTS[variant]), oracle(c, X),
          limbs)


@pytest.mark.parametrize("limbs", [2, 3, 5])
@pytest.mark.parametrize("n,t", [(1000, 2), (257, 1)])
def test_constant_snps_are_singular_with_an_intercept(gwas, limbs, n, t):
    """A SNP with every dosage equal is exactly collinear with the intercept column: the
    oracle's pivot test flags it; the limb arithmetic decides it exactly (integer test
    of the dosages, FP64 test of the all-ones column at factor time)."""
    c = synth.make_cohort(300 + n, n, t=t, n_markers=400)
    X = c.snps(40).copy(order="F")
    X[:, 3] = 1
    X[:, 7] = 2
    X[:, 9] = 0
    out = run(gwas, c, X, limbs=limbs, m_blk=64)
    ref = oracle(c, X)
    assert list(ref[2][[3, 7, 9]]) == [1, 1, 1]
    check(out, ref, limbs)


@pytest.mark.parametrize("limbs", [3, 5])
def test_constant_snp_without_intercept_is_solved(gwas, limbs):
    """Without an intercept in X_L a constant SNP is an ordinary regressor."""
    c = synth.make_cohort(41, 600, n_markers=400)
    XL = np.asfortranarray(c.XL[:, 1:])
    X = c.snps(30).copy(order="F")
    X[:, 2] = 1
    X[:, 5] = 2
    X[:, 8] = 0
    with gwas.GLS(c.n, XL.shape[1] + 1, 1, precision=gwas.GWAS_PREC_MIXED, n_limbs=limbs,
                  m_blk=64) as e:
        e.factor(c.phi, c.h, c.sigma2, XL, c.Y)
        out = e.solve(X)
    ref = G.gls(c.phi, c.h, c.sigma2, XL, c.Y, X)
    assert list(ref[2][[2, 5, 8]]) == [0, 0, 1]
    check(out, ref, limbs)


@pytest.mark.parametrize("p,t", [(20, 1), (4, 64), (20, 64)])
def test_mixed_largest_p_and_t(gwas, p, t):
    """p = 20 (the generic p x p solve) and t = 64 phenotypes: the linear rows fill a whole
    N = 256 linear tile (3 x 83 = 249 rows)."""
    c = synth.make_cohort(400 + p + t, 300, q=p - 1, t=t, n_markers=300)
    X = c.snps(150)
    check(run(gwas, c, X, m_blk=128), oracle(c, X), 3)


def test_mixed_linear_rows_beyond_one_tile_are_unsupported(gwas):
    """4 limbs x (19 + 64) linear rows exceed one UMMA (N <= 256): refused at init."""
    with pytest.raises(gwas.GwasError) as ei:
        gwas.GLS(300, 20, 64, precision=gwas.GWAS_PREC_MIXED, n_limbs=4, m_blk=128)
    assert ei.value.status == gwas.GWAS_ERR_UNSUPPORTED


def test_mixed_degenerate_and_bad(gwas):
    c = synth.make_cohort(12, 300, n_markers=400)
    X = c.snps(70).copy(order="F")
    X[:, 1] = 1
    X[:, 2] = 0
    X[5, 3] = 3
    X[0, 4] = -1
    out = run(gwas, c, X, m_blk=128)
    assert list(out[2][:6]) == [0, 1, 1, 2, 2, 0]
    check(out, oracle(c, X), 3)


def test_mixed_multi_phenotype(gwas):
    c = synth.make_cohort(52, 900, t=16, n_markers=900)
    X = c.snps(400)
    check(run(gwas, c, X, m_blk=512), oracle(c, X), 3)


def test_mixed_block_size_and_order_bitwise(gwas):
    # blocks of 128 SNPs run whole; a block of 2,500 runs as two launches over its halves
    # (SNPs 0-1279 and 1280-2499) with the second half's conversion and the first half's
    # solves on a second stream; blocks of 1,100 split at 768; all give the same bits
    c = synth.make_cohort(22, 600, n_markers=700)
    X = c.snps(2500)
    b1, w1, s1 = run(gwas, c, X, m_blk=128)
    b2, w2, s2 = run(gwas, c, X, m_blk=4096)
    np.testing.assert_array_equal(b1, b2)
    np.testing.assert_array_equal(w1, w2)
    np.testing.assert_array_equal(s1, s2)
    b4, _, _ = run(gwas, c, X, m_blk=1100)
    np.testing.assert_array_equal(b1, b4)
    perm = np.random.default_rng(4).permutation(2500)
    b3, _, _ = run(gwas, c, np.asfortranarray(X[:, perm]), m_blk=256)
    np.testing.assert_array_equal(b3, b1[perm])


@pytest.fixture(scope="module")
def full_size():
    """The n = 10,000 cohort and the oracle's Cholesky factor of its M."""
    c = synth.make_cohort(0, 10000, device="cuda")
    return c, G.factor(c.phi, c.h, c.sigma2)


@pytest.mark.parametrize("limbs,cfg", [(3, -1), (4, -1), (5, -1), (3, (1 << 21) | (1 << 13)),
                                       (5, (1 << 21) | (1 << 13))])
def test_mixed_full_size_sampled(gwas, full_size, limbs, cfg):
    """n = 10,000, one block of 16,384 SNPs in the benchmark's launch shape (the default
    layout, and the linear rows in the last limb tile)."""
    import torch
    n, mb = 10000, 16384
    c, L = full_size
    Xd = synth.genotypes_torch(5, n, mb, "cuda")
    e = gwas.GLS(n, 4, 1, m_blk=mb, precision=gwas.GWAS_PREC_MIXED, n_limbs=limbs, tile_cfg=cfg)
    e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
    bd = torch.empty((mb, 1, 4), dtype=torch.float64, device="cuda")
    wd = torch.empty((mb, 1), dtype=torch.float64, device="cuda")
    sd = torch.empty(mb, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    gwas.gwas_solve_block_device(e.ctx, Xd, mb, bd, wd, sd)
    gwas.gwas_sync(e.ctx)
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([[0, 127, 128, mb - 1], rng.choice(mb, 252, replace=False)]))
    Xs = np.asfortranarray(Xd[idx].cpu().numpy().T)
    ref = G.gls_hoisted(L, c.XL, c.Y, Xs)
    out = (bd.cpu().numpy()[idx], wd.cpu().numpy()[idx], sd.cpu().numpy()[idx])
    eb, ew = check(out, ref, limbs)
    print(f"n=10000 mixed x{limbs} (tile_cfg {cfg}): max rel b err {eb:.2e}, Wald err {ew:.2e}")
    e.close()
