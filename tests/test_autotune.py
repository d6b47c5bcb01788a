"""Autotuner and tile-configuration switching keep the results of the mixed path."""
import numpy as np
import pytest

import synth
from oracle import gls as G

pytestmark = pytest.mark.gpu


def rel_b(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


@pytest.fixture(scope="module")
def gw(gpu):
    from paper_1304_2272_gb300 import gwas as g
    g.load()
    return g


def test_set_tile_cfg_resplits_and_keeps_parity(gw):
    c = synth.make_cohort(31, 900, n_markers=900)
    X = c.snps(600)
    ref = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    with gw.GLS(c.n, 4, 1, precision=gw.GWAS_PREC_MIXED, n_limbs=3, m_blk=1024) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        # pair <-> single, separate <-> fused linear rows (85 <-> 81 rows per tile) <->
        # linear rows in the last tile (one more row tile)
        for cfg in (1 << 13, 1 << 12, (1 << 12) | (20 << 4) | 3, (1 << 17) | (1 << 13),
                    (1 << 21) | (1 << 13), (1 << 21) | (1 << 12), -1):
            gw.gwas_set_tile_cfg(e.ctx, cfg)
            b, w, s = e.solve(X)
            np.testing.assert_array_equal(s, ref[2])
            assert rel_b(b, ref[0]) <= 1e-6


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotune_picks_a_valid_config(gw, precision):
    c = synth.make_cohort(32, 1500, n_markers=900)
    X = c.snps(700)
    prec = gw.GWAS_PREC_MIXED if precision == "mixed" else gw.GWAS_PREC_FP64
    with gw.GLS(c.n, 4, 1, precision=prec, m_blk=8192) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        before = e.stats()
        res = gw.gwas_autotune(e.ctx, None, 8192, 2)
        assert res["candidates"] >= 1 and res["snps_per_s"] > 0
        assert res["m_blk"] in (4096, 8192)
        assert e.stats()["snps"] == before["snps"]   # tuning runs are not counted
        b, w, s = e.solve(X)
    ref = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    np.testing.assert_array_equal(s, ref[2])
    assert rel_b(b, ref[0]) <= (1e-6 if precision == "mixed" else 1e-10)


def test_tuning_cache_roundtrip(gw, tmp_path, monkeypatch):
    from paper_1304_2272_gb300 import autotune
    monkeypatch.setenv("GWAS_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    c = synth.make_cohort(33, 700, n_markers=500)
    with gw.GLS(c.n, 4, 1, precision=gw.GWAS_PREC_MIXED, m_blk=4096) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        r1 = autotune.tuned_tile_cfg(e.ctx, c.n, 4, 1, 1, 3, 4096)
        r2 = autotune.tuned_tile_cfg(e.ctx, c.n, 4, 1, 1, 3, 4096)
    assert not r1["cached"] and r2["cached"] and r1["tile_cfg"] == r2["tile_cfg"]
