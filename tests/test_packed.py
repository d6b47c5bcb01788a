"""2-bit packed genotype calls: unpacked on the GPU into the int8 layout, so the results
equal the int8 path's bit for bit; missing calls give status 2; against the oracle."""
import numpy as np
import pytest

import synth
from oracle import gls as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw(gpu):
    from paper_1304_2272_gb300 import gwas as g
    g.load()
    return g


def solve_int8(gw, e, X, mb):
    m = X.shape[1]
    b = np.empty((m, e.t, e.p)); w = np.empty((m, e.t)); s = np.empty(m, dtype=np.uint8)
    gw.gwas_solve_all(e.ctx, np.asfortranarray(X), m, b, w, s)
    return b, w, s


def solve_packed(gw, e, P, m, mb, code):
    b = np.empty((m, e.t, e.p)); w = np.empty((m, e.t)); s = np.empty(m, dtype=np.uint8)
    for i0 in range(0, m, mb):
        k = min(mb, m - i0)
        gw.gwas_solve_block_packed(e.ctx, np.asfortranarray(P[:, i0:i0 + k]), k, code,
                                   b[i0:i0 + k], w[i0:i0 + k], s[i0:i0 + k])
    gw.gwas_sync(e.ctx)
    return b, w, s


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,m,mb", [(1000, 700, 256), (1003, 300, 128), (7, 9, 4)])
@pytest.mark.parametrize("table", ["dosage", "plink"])
def test_packed_equals_int8_path(gw, precision, n, m, mb, table):
    c = synth.make_cohort(90 + n, n, t=2, n_markers=max(50, n // 2))
    X = c.snps(m).copy(order="F")
    X[min(2, n - 1), 1] = -1          # missing call
    if m > 4:
        X[:, 4] = 1                   # constant: singular
    if table == "dosage":
        code, P = gw.CODE_DOSAGE, synth.pack_2bit(X)
    else:
        code, P = gw.CODE_PLINK_BED, synth.pack_2bit(X, call_of=(3, 2, 0), missing_call=1)
    assert P.shape == (-(-n // 4), m)
    prec = gw.GWAS_PREC_FP64 if precision == "fp64" else gw.GWAS_PREC_MIXED
    with gw.GLS(n, 4, 2, m_blk=mb, precision=prec) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        ref8 = solve_int8(gw, e, X, mb)
        got = solve_packed(gw, e, P, m, mb, code)
        st = e.stats()
    for a, r in zip(got, ref8):
        np.testing.assert_array_equal(a, r)
    assert got[2][1] == 2
    assert st["h2d_bytes"] == n * m + P.shape[0] * m
    rb, rw, rs = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    np.testing.assert_array_equal(got[2], rs)


def test_packed_device_entry(gw):
    import torch
    c = synth.make_cohort(95, 640, n_markers=500)
    X = c.snps(333)
    P = synth.pack_2bit(X)
    mb = X.shape[1]
    with gw.GLS(c.n, 4, 1, m_blk=512) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        ref = solve_int8(gw, e, X, 512)
        Pd = torch.from_numpy(np.ascontiguousarray(P.T)).cuda()      # SNP-major columns
        bd = torch.empty((mb, 1, 4), dtype=torch.float64, device="cuda")
        wd = torch.empty((mb, 1), dtype=torch.float64, device="cuda")
        sd = torch.empty(mb, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        gw.gwas_solve_block_packed_device(e.ctx, Pd, mb, gw.CODE_DOSAGE, bd, wd, sd)
        gw.gwas_sync(e.ctx)
        np.testing.assert_array_equal(bd.cpu().numpy(), ref[0])
        np.testing.assert_array_equal(sd.cpu().numpy(), ref[2])
        with pytest.raises(ValueError):
            gw.gwas_solve_block_packed_device(e.ctx, Pd, mb, [0, 1, 2], bd, wd, sd)
        with pytest.raises(gw.GwasError):
            gw.gwas_solve_block_packed_device(e.ctx, Pd, 0, gw.CODE_DOSAGE, bd, wd, sd)
