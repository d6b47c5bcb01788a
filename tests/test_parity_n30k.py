"""Large cohorts: n = 30,000 (the mixed-precision workload's n) in the benchmark's launch
shapes, FP64 (1e-10), 3-limb mixed (1e-6) and 5-limb mixed (1e-10); n = 32,767, the last
n with 9-bit limbs; n = 33,000 with 8-bit limbs. Sampled SNPs against the oracle. Exercises
the 64-bit index arithmetic of the limb buffers (rows x n_pad > 2^31) and the 2^24
exactness bound at its n limits."""
import numpy as np
import pytest

import synth
from oracle import gls as G

pytestmark = pytest.mark.gpu

N = 30000


def rel_b(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


def wald_err(w, rw):
    return float(np.max(np.abs(w - rw) / np.maximum(rw, 1.0)))


def wald_tol(limbs, bits):
    """|dW| / max(W, 1) bound of the mixed path: 2e3 * 2^-(bits * limbs), at least 1e-10
    (the derivation is in test_parity_mixed.py); FP64 is held to 1e-10."""
    return 1e-10 if limbs is None else max(2e3 * 2.0 ** (-bits * limbs), 1e-10)


@pytest.fixture(scope="module")
def gw(gpu):
    from paper_1304_2272_gb300 import gwas as g
    g.load()
    return g


@pytest.fixture(scope="module")
def big():
    c = synth.make_cohort(30, N, device="cuda")
    return c, G.factor(c.phi, c.h, c.sigma2)


@pytest.mark.parametrize("limbs", [3])   # 5 limbs of 8 bits: forced at n = 1000 elsewhere
def test_beyond_32767_takes_8_bit_limbs(gw, limbs):
    """n = 33,000: beyond 32767 the limbs carry 8 bits so that the FP32 sums stay exact
    (measured at n = 40,000 as well: 9.0e-8); sampled SNPs of one block."""
    import torch
    n, mb = 33000, 2048
    c, L = big33k()
    Xd = synth.genotypes_torch(41, n, mb, "cuda")
    with gw.GLS(n, 4, 1, m_blk=mb, precision=gw.GWAS_PREC_MIXED, n_limbs=limbs) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        bd = torch.empty((mb, 1, 4), dtype=torch.float64, device="cuda")
        wd = torch.empty((mb, 1), dtype=torch.float64, device="cuda")
        sd = torch.empty(mb, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        gw.gwas_solve_block_device(e.ctx, Xd, mb, bd, wd, sd)
        gw.gwas_sync(e.ctx)
    idx = np.unique(np.concatenate([[0, mb - 1], np.random.default_rng(7).choice(mb, 40, replace=False)]))
    Xs = np.asfortranarray(Xd[idx].cpu().numpy().T)
    rb, rw, rs = G.gls_hoisted(L, c.XL, c.Y, Xs)
    b, s = bd.cpu().numpy()[idx], sd.cpu().numpy()[idx]
    w = wd.cpu().numpy()[idx]
    np.testing.assert_array_equal(s, rs)
    ok = rs == 0
    err = rel_b(b[ok], rb[ok])
    ew = wald_err(w[ok], rw[ok])
    print(f"[errors] n=33000 mixed x{limbs} (8-bit limbs): max rel b err {err:.2e}, "
          f"Wald err {ew:.2e}")
    assert err <= (1e-6 if limbs == 3 else 1e-10)
    assert ew <= wald_tol(limbs, 8)


def big33k():
    c = synth.make_cohort(40, 33000, device="cuda")
    return c, G.factor(c.phi, c.h, c.sigma2)


def test_mixed_at_the_exactness_limit(gw):
    """n = 32,767, the largest n for which the FP32 sums of 9-bit limb products
    (|A_l| <= 256, dosages <= 2) stay exact (512 n < 2^24); sampled SNPs of one block."""
    import torch
    n, mb = 32767, 2048
    c = synth.make_cohort(32, n, device="cuda")
    Xd = synth.genotypes_torch(33, n, mb, "cuda")
    Xd[:, :100] = 2          # large dosages in the first rows of L^-1's columns
    with gw.GLS(n, 4, 1, m_blk=mb, precision=gw.GWAS_PREC_MIXED, n_limbs=3) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        bd = torch.empty((mb, 1, 4), dtype=torch.float64, device="cuda")
        wd = torch.empty((mb, 1), dtype=torch.float64, device="cuda")
        sd = torch.empty(mb, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        gw.gwas_solve_block_device(e.ctx, Xd, mb, bd, wd, sd)
        gw.gwas_sync(e.ctx)
    idx = np.unique(np.concatenate([[0, mb - 1], np.random.default_rng(6).choice(mb, 40, replace=False)]))
    Xs = np.asfortranarray(Xd[idx].cpu().numpy().T)
    L = G.factor(c.phi, c.h, c.sigma2)
    rb, rw, rs = G.gls_hoisted(L, c.XL, c.Y, Xs)
    b, s = bd.cpu().numpy()[idx], sd.cpu().numpy()[idx]
    w = wd.cpu().numpy()[idx]
    np.testing.assert_array_equal(s, rs)
    ok = rs == 0
    err = rel_b(b[ok], rb[ok])
    ew = wald_err(w[ok], rw[ok])
    print(f"[errors] n=32767 mixed x3: max rel b err {err:.2e}, Wald err {ew:.2e}")
    assert err <= 1e-6
    assert ew <= wald_tol(3, 9)


@pytest.mark.parametrize("precision,limbs,mb,tol", [
    ("fp64", 3, 1024, 1e-10), ("mixed", 3, 4096, 1e-6), ("mixed", 5, 4096, 1e-10)])
def test_n30k_sampled(gw, big, precision, limbs, mb, tol):
    import torch
    c, L = big
    prec = gw.GWAS_PREC_FP64 if precision == "fp64" else gw.GWAS_PREC_MIXED
    Xd = synth.genotypes_torch(31, N, mb, "cuda")
    Xd[17] = 1                      # constant: singular with the intercept
    with gw.GLS(N, 4, 1, m_blk=mb, precision=prec, n_limbs=limbs) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        bd = torch.empty((mb, 1, 4), dtype=torch.float64, device="cuda")
        wd = torch.empty((mb, 1), dtype=torch.float64, device="cuda")
        sd = torch.empty(mb, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        gw.gwas_solve_block_device(e.ctx, Xd, mb, bd, wd, sd)
        gw.gwas_sync(e.ctx)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, 17, 127, 128, mb - 1], rng.choice(mb, 60, replace=False)]))
    Xs = np.asfortranarray(Xd[idx].cpu().numpy().T)
    rb, rw, rs = G.gls_hoisted(L, c.XL, c.Y, Xs)
    b, s = bd.cpu().numpy()[idx], sd.cpu().numpy()[idx]
    w = wd.cpu().numpy()[idx]
    np.testing.assert_array_equal(s, rs)
    assert s[list(idx).index(17)] == 1
    ok = rs == 0
    err = rel_b(b[ok], rb[ok])
    ew = wald_err(w[ok], rw[ok])
    print(f"[errors] n=30000 {precision} x{limbs}: max rel b err {err:.2e}, Wald err {ew:.2e}")
    assert err <= tol
    assert ew <= wald_tol(None if precision == "fp64" else limbs, 9)


def test_mixed_refuses_n_beyond_7_bit_limbs(gw):
    with pytest.raises(gw.GwasError) as ei:
        gw.GLS(131072, 4, 1, m_blk=64, precision=gw.GWAS_PREC_MIXED)
    assert ei.value.status == gw.GWAS_ERR_UNSUPPORTED
