"""Failure detection without a GPU fault: bounded device waits, host-side errors.

A pipeline kernel whose partner never signals must give up after its time limit and
report it, with the device still usable; host-side failures come back as status codes.
"""
import numpy as np
import pytest

import synth
from oracle import gls as G


@pytest.mark.gpu
def test_device_wait_gives_up_and_device_stays_usable(gpu):
    from paper_1304_2272_gb300 import gwas
    st, waited = gwas.gwas_selftest_wait(0, 200)
    assert st == gwas.GWAS_ERR_TIMEOUT
    assert 150.0 <= waited <= 5000.0
    # the same process and device still solve correctly
    c = synth.make_cohort(61, 200, n_markers=300)
    X = c.snps(65)
    for prec in (gwas.GWAS_PREC_FP64, gwas.GWAS_PREC_MIXED):
        with gwas.GLS(c.n, 4, 1, m_blk=128, precision=prec) as e:
            e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
            b, w, s = e.solve(X)
        rb, _, rs = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
        np.testing.assert_array_equal(s, rs)
        assert np.nanmax(np.abs(b - rb)) <= 1e-6 * np.nanmax(np.abs(rb))


def test_selftest_rejects_bad_arguments():
    from paper_1304_2272_gb300 import gwas
    st, _ = gwas.gwas_selftest_wait(0, 0)
    assert st == gwas.GWAS_ERR_ARG


@pytest.mark.gpu
def test_host_side_errors_are_status_codes(gpu):
    from paper_1304_2272_gb300 import gwas
    with pytest.raises(gwas.GwasError) as ei:
        gwas.gwas_init(0, 4, 1)
    assert ei.value.status == gwas.GWAS_ERR_ARG
    with pytest.raises(gwas.GwasError) as ei:
        gwas.gwas_init(100, 4, 1, precision=gwas.GWAS_PREC_MIXED, n_limbs=9)
    assert ei.value.status == gwas.GWAS_ERR_UNSUPPORTED
    c = synth.make_cohort(62, 100, n_markers=200)
    with gwas.GLS(c.n, 4, 1, m_blk=64) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        X = np.asfortranarray(c.snps(65))
        with pytest.raises(gwas.GwasError) as ei:       # mb > m_blk
            gwas.gwas_solve_block(e.ctx, X, 65, np.empty((65, 1, 4)), None,
                                  np.empty(65, np.uint8))
        assert ei.value.status == gwas.GWAS_ERR_ARG
        # a corrupt block (dosage 7) is reported per SNP, the rest is solved
        X2 = c.snps(40).copy(order="F")
        X2[3, 5] = 7
        b, w, s = e.solve(X2)
        assert s[5] == 2 and np.all(np.isnan(b[5])) and np.all(s[np.arange(40) != 5] == 0)


@pytest.mark.gpu
def test_wait_block_and_pinned_host_buffers(gpu):
    """Host-path blocks in page-locked buffers from gwas_host_alloc: gwas_wait_block(k)
    returns once block k's outputs are in host memory; a block not yet submitted is an
    argument error; the results equal those of gwas_solve_all."""
    import ctypes
    from paper_1304_2272_gb300 import gwas as gw
    c = synth.make_cohort(81, 200, n_markers=200)
    X = c.snps(3 * 64)
    n, mb, p = c.n, 64, 4
    with gw.GLS(n, p, 1, m_blk=mb) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        ref = e.solve(X)
        xs = gw.gwas_host_alloc(n * mb * 3)
        bs = gw.gwas_host_alloc(mb * p * 8 * 3)
        ss = gw.gwas_host_alloc(mb * 3)
        try:
            ctypes.memmove(xs, np.ascontiguousarray(X.T).ctypes.data, n * mb * 3)
            first = gw.gwas_get_stats(e.ctx)["blocks"]
            for k in range(3):
                gw.gwas_solve_block(e.ctx, xs + k * n * mb, mb, bs + k * mb * p * 8, None,
                                    ss + k * mb)
            base = 3  # e.solve above ran 3 host-path blocks through gwas_solve_all
            for k in range(3):
                gw.gwas_wait_block(e.ctx, base + k, 5000)
            with pytest.raises(gw.GwasError) as ei:
                gw.gwas_wait_block(e.ctx, base + 3, 10)
            assert ei.value.status == gw.GWAS_ERR_ARG
            b = np.frombuffer((ctypes.c_double * (3 * mb * p)).from_address(bs), dtype=np.float64)
            s = np.frombuffer((ctypes.c_uint8 * (3 * mb)).from_address(ss), dtype=np.uint8)
            np.testing.assert_array_equal(b.reshape(3 * mb, 1, p), ref[0])
            np.testing.assert_array_equal(s, ref[2])
            assert gw.gwas_get_stats(e.ctx)["blocks"] == first + 3
        finally:
            gw.gwas_host_free(xs)
            gw.gwas_host_free(bs)
            gw.gwas_host_free(ss)
