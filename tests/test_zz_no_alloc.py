"""The allocation-free entry point gives the results of the regular FP64 block solve.

gwas_solve_block_noalloc serves callers that cannot allocate device memory when they
call in (their GPU memory is held by another allocator, or a serving loop cannot
afford cudaMalloc/cudaFree). It runs the FP64 block kernels on caller buffers with
its scratch in a fixed array inside the library. This file is collected last so that a
run stopping at its first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

B_TOL = 1e-10   # the FP64 parity tolerance of the other GPU tests
W_TOL = 1e-7


def rel_b(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


def col_major(t):
    """A torch matrix laid out column-major (memory of its transpose, row-major)."""
    return t.T.contiguous()


def test_noalloc_matches_regular_entry_point(gpu):
    import torch
    from paper_1304_2272_gb300 import gwas

    c = synth.make_cohort(77, 700, t=2, n_markers=800)
    n, q, t, p = c.n, c.q, c.t, c.q + 1
    m = 300
    X = c.snps(m)
    dev = "cuda:0"
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(dev)  # column-major n x m

    # regular path: context, factor, device entry point
    ref = gwas.GLS(n, p, t, m_blk=m)
    ref.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
    b0 = torch.empty((m, t, p), dtype=torch.float64, device=dev)
    w0 = torch.empty((m, t), dtype=torch.float64, device=dev)
    s0 = torch.empty(m, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    gwas.gwas_solve_block_device(ref.ctx, Xd, m, b0, w0, s0)
    gwas.gwas_sync(ref.ctx)
    ref.close()

    # the caller's own inputs for the allocation-free call (computed here with torch)
    phi = torch.from_numpy(c.phi).to(dev)
    M = c.sigma2 * (c.h * phi + (1.0 - c.h) * torch.eye(n, dtype=torch.float64, device=dev))
    L = torch.linalg.cholesky(M)
    Linv = torch.linalg.solve_triangular(L, torch.eye(n, dtype=torch.float64, device=dev),
                                         upper=False)
    Linv = torch.tril(Linv)
    XLbar = Linv @ torch.from_numpy(c.XL).to(dev)
    Ybar = Linv @ torch.from_numpy(c.Y).to(dev)
    S_TL = XLbar.T @ XLbar
    bbar_T = XLbar.T @ Ybar
    args = (col_major(Linv), n, col_major(XLbar), col_major(Ybar), col_major(S_TL),
            col_major(bbar_T))

    results = []
    for _ in range(2):  # two calls in a row share the scratch array
        b1 = torch.full((m, t, p), -7.0, dtype=torch.float64, device=dev)
        w1 = torch.full((m, t), -7.0, dtype=torch.float64, device=dev)
        s1 = torch.full((m,), 9, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        gwas.gwas_solve_block_noalloc(n, p, t, *args, Xd, m, b1, w1, s1, stream=None)
        torch.cuda.synchronize()
        results.append((b1.cpu().numpy(), w1.cpu().numpy(), s1.cpu().numpy()))

    rb, rw, rs = b0.cpu().numpy(), w0.cpu().numpy(), s0.cpu().numpy()
    assert np.all(rs == 0)
    for b, w, s in results:
        np.testing.assert_array_equal(s, rs)
        assert rel_b(b, rb) <= B_TOL
        assert float(np.max(np.abs(w - rw) / np.maximum(rw, 1.0))) <= W_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu):
    from paper_1304_2272_gb300 import gwas

    # n = 10,000, p = 4, t = 1 needs ~6.3 kB of scratch per SNP: 100,000 SNPs do not fit
    one = 256  # any non-null address: the size check comes before any launch
    with pytest.raises(gwas.GwasError) as ei:
        gwas.gwas_solve_block_noalloc(10000, 4, 1, one, 10000, one, one, one, one, one,
                                      100000, one, one, one)
    assert ei.value.status == gwas.GWAS_ERR_TOO_LARGE
