"""Section 5's multi-trait problem: t traits of one cohort, each with its own
M_j = sigma2_j (h_j Phi + (1 - h_j) I), solved as one batch whose cohorts share the
dosage block; every b_ij against the oracle (FP64 1e-10, mixed 1e-6)."""
import numpy as np
import pytest

import synth
from oracle import gls as G

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}
HS = [0.1, 0.35, 0.6, 0.85]
S2 = [1.0, 0.5, 2.0, 1.3]


def rel_b(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


@pytest.fixture(scope="module")
def gw(gpu):
    from paper_1304_2272_gb300 import gwas as g
    g.load()
    return g


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,m,mblk", [(700, 900, 512), (129, 65, 64)])
def test_multitrait_matches_oracle(gw, precision, n, m, mblk):
    from paper_1304_2272_gb300.multitrait import MultiTrait
    c = synth.make_cohort(61 + n, n, t=4, n_markers=600)
    X = c.snps(m).copy(order="F")
    X[:, 3] = 2           # constant: singular for every trait
    X[0, 5] = 7           # bad dosage
    prec = gw.GWAS_PREC_FP64 if precision == "fp64" else gw.GWAS_PREC_MIXED
    with MultiTrait(n, 4, m_blk=mblk, precision=prec) as mt:
        mt.factor(c.phi, HS, S2, c.XL, c.Y)
        b, w, s = mt.solve(X)
    rb, rw, rs = G.gls_multitrait(c.phi, HS, S2, c.XL, c.Y, X)
    np.testing.assert_array_equal(s, rs)
    assert np.all(s[3] == 1) and np.all(s[5] == 2)
    ok = rs == 0
    assert np.all(np.isnan(b[~ok]))
    assert rel_b(b[ok], rb[ok]) <= TOL[precision]
    print(f"multi-trait {precision} n={n}: max rel b err {rel_b(b[ok], rb[ok]):.2e}")


def test_shared_dosages_convert_once_and_match_copies(gw):
    """Mixed batch: traits handed the same dosage pointer share one BF16 conversion; the
    results equal those of a batch given separate copies of the block, bit for bit."""
    import torch
    c = synth.make_cohort(77, 500, t=3, n_markers=500)
    X = c.snps(300)
    mb = X.shape[1]

    def run(shared):
        b = gw.gwas_batch_init([c.n] * 3, 4, 1, precision=gw.GWAS_PREC_MIXED, m_blk=512)
        try:
            for j in range(3):
                gw.gwas_batch_factor(b, j, np.asfortranarray(c.phi), True, HS[j], S2[j], c.XL,
                                     np.asfortranarray(c.Y[:, j:j + 1]))
            X0 = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
            Xs = [X0] * 3 if shared else [X0.clone() for _ in range(3)]
            bd = [torch.empty((mb, 1, 4), dtype=torch.float64, device="cuda") for _ in range(3)]
            wd = [torch.empty((mb, 1), dtype=torch.float64, device="cuda") for _ in range(3)]
            sd = [torch.empty(mb, dtype=torch.uint8, device="cuda") for _ in range(3)]
            torch.cuda.synchronize()
            gw.gwas_batch_solve_device(b, Xs, [mb] * 3, bd, wd, sd)
            gw.gwas_batch_sync(b)
            return [x.cpu().numpy() for x in bd], [x.cpu().numpy() for x in sd]
        finally:
            gw.gwas_batch_finalize(b)

    b1, s1 = run(True)
    b2, s2 = run(False)
    for j in range(3):
        np.testing.assert_array_equal(b1[j], b2[j])
        np.testing.assert_array_equal(s1[j], s2[j])
