"""The allocation-free entry point gives the results of the regular FP64 block solve.

gwas_solve_block_noalloc serves callers that cannot allocate device memory when they
call in (their GPU memory is held by another allocator, or a serving loop cannot
afford cudaMalloc/cudaFree). It runs the FP64 block kernels on caller buffers with
its scratch in a fixed array inside the library. These tests compare it with the
regular device entry point and with the CPU oracle (Eq. (1)), including a singular and a
bad-dosage SNP, a strided L^{-1}, no Wald output and a side stream. This file is
collected last so that a run stopping at its first failure has already run every other
test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest
from scipy.linalg import solve_triangular

import synth
from oracle import gls as G

pytestmark = pytest.mark.gpu

B_TOL = 1e-10   # the FP64 parity tolerance of the other GPU tests
W_TOL = 1e-10   # the FP64 Wald tolerance of the other GPU tests


def rel_b(b, ref):
    scale = np.maximum(np.nanmax(np.abs(ref), axis=-1, keepdims=True), 1e-300)
    return float(np.nanmax(np.abs(b - ref) / scale))


def col_major(a, dev, ld=None):
    """A device tensor holding the matrix `a` column-major, with leading dimension ld
    (the rows beyond a's in every column are NaN, so a kernel that read them would
    spoil its results)."""
    import torch
    rows, cols = a.shape
    ld = rows if ld is None else ld
    buf = np.full((cols, ld), np.nan)
    buf[:, :rows] = a.T
    return torch.from_numpy(buf).to(dev)


def planted_cohort():
    c = synth.make_cohort(77, 700, t=2, n_markers=800)
    X = c.snps(300).copy(order="F")
    X[:, 5] = 1      # constant: collinear with the intercept -> status 1
    X[3, 9] = 3      # a dosage outside {0, 1, 2} -> status 2
    return c, X


def caller_inputs(c, dev, ld=None):
    """What a caller computes once per cohort (here with the CPU oracle): L^{-1},
    Xbar_L, Ybar, S_TL and bbar_T, as device tensors laid out as the C ABI wants."""
    L = G.factor(c.phi, c.h, c.sigma2)
    Linv = np.tril(solve_triangular(L, np.eye(c.n), lower=True))
    XLbar, Ybar, S_TL, bbar_T = G.setup_hoisted(L, c.XL, c.Y)
    ld = c.n if ld is None else ld
    return (col_major(Linv, dev, ld), ld, col_major(XLbar, dev), col_major(Ybar, dev),
            col_major(S_TL, dev), col_major(bbar_T, dev))


def regular_solve(gwas, c, Xd, m):
    import torch
    dev = Xd.device
    t, p = c.t, c.q + 1
    ref = gwas.GLS(c.n, p, t, m_blk=m)
    ref.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
    b0 = torch.empty((m, t, p), dtype=torch.float64, device=dev)
    w0 = torch.empty((m, t), dtype=torch.float64, device=dev)
    s0 = torch.empty(m, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    gwas.gwas_solve_block_device(ref.ctx, Xd, m, b0, w0, s0)
    gwas.gwas_sync(ref.ctx)
    ref.close()
    return b0.cpu().numpy(), w0.cpu().numpy(), s0.cpu().numpy()


def check_against(out, ref):
    b, w, s = out
    rb, rw, rs = ref
    np.testing.assert_array_equal(s, rs)
    ok = rs == 0
    assert np.all(np.isnan(b[~ok]))
    assert rel_b(b[ok], rb[ok]) <= B_TOL
    if w is not None:
        assert np.all(np.isnan(w[~ok]))
        assert float(np.max(np.abs(w[ok] - rw[ok]) / np.maximum(rw[ok], 1.0))) <= W_TOL


def test_noalloc_matches_regular_entry_point_and_oracle(gpu):
    import torch
    from paper_1304_2272_gb300 import gwas

    c, X = planted_cohort()
    n, t, p, m = c.n, c.t, c.q + 1, X.shape[1]
    dev = "cuda:0"
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(dev)  # column-major n x m
    regular = regular_solve(gwas, c, Xd, m)
    oracle = G.gls(c.phi, c.h, c.sigma2, c.XL, c.Y, X)
    assert list(oracle[2][[5, 9]]) == [1, 2]
    args = caller_inputs(c, dev)

    for _ in range(2):  # two calls in a row share the scratch array
        b1 = torch.full((m, t, p), -7.0, dtype=torch.float64, device=dev)
        w1 = torch.full((m, t), -7.0, dtype=torch.float64, device=dev)
        s1 = torch.full((m,), 9, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        gwas.gwas_solve_block_noalloc(n, p, t, *args, Xd, m, b1, w1, s1, stream=None)
        torch.cuda.synchronize()
        out = (b1.cpu().numpy(), w1.cpu().numpy(), s1.cpu().numpy())
        check_against(out, regular)
        check_against(out, oracle)


def test_noalloc_strided_linv_without_wald_on_a_side_stream(gpu):
    """L^{-1} a column slice of a wider buffer (ld = n + 64, the extra rows NaN), no Wald
    output, the work queued on a torch side stream."""
    import torch
    from paper_1304_2272_gb300 import gwas

    c, X = planted_cohort()
    n, t, p, m = c.n, c.t, c.q + 1, X.shape[1]
    dev = "cuda:0"
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(dev)
    rb, _, rs = regular_solve(gwas, c, Xd, m)
    args = caller_inputs(c, dev, ld=n + 64)
    side = torch.cuda.Stream(device=dev)
    for _ in range(2):
        b1 = torch.full((m, t, p), -7.0, dtype=torch.float64, device=dev)
        s1 = torch.full((m,), 9, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        gwas.gwas_solve_block_noalloc(n, p, t, *args, Xd, m, b1, None, s1, stream=side)
        side.synchronize()
        check_against((b1.cpu().numpy(), None, s1.cpu().numpy()), (rb, None, rs))


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu):
    """n = 4096, p = 4, t = 1 and 7000 SNPs need 17.9 MB of row-tile partials, more than the
    16 MiB array: refused before any launch. The buffers are real device tensors of the
    call's sizes, so even a call that got past the check would only compute."""
    import torch
    from paper_1304_2272_gb300 import gwas

    n, p, t, mb = 4096, 4, 1, 7000
    dev = "cuda:0"
    f64 = dict(dtype=torch.float64, device=dev)
    Linv = torch.eye(n, **f64)
    XLbar = torch.zeros((p - 1, n), **f64)
    Ybar = torch.zeros((t, n), **f64)
    S_TL = torch.eye(p - 1, **f64)
    bbar_T = torch.zeros((t, p - 1), **f64)
    X = torch.ones((mb, n), dtype=torch.int8, device=dev)
    b = torch.empty((mb, t, p), **f64)
    w = torch.empty((mb, t), **f64)
    st = torch.empty(mb, dtype=torch.uint8, device=dev)
    with pytest.raises(gwas.GwasError) as ei:
        gwas.gwas_solve_block_noalloc(n, p, t, Linv, n, XLbar, Ybar, S_TL, bbar_T, X, mb, b, w,
                                      st)
    assert ei.value.status == gwas.GWAS_ERR_TOO_LARGE


def test_noalloc_refuses_host_buffers(gpu):
    """A host array is refused by the binding (TypeError); a page-locked host buffer passed
    as a raw address gets past the binding and is refused by the C entry point
    (GWAS_ERR_ARG, no launch). That buffer is reachable from the GPU, so even a call that
    got past the check would only read host memory."""
    import torch
    from paper_1304_2272_gb300 import gwas

    c, X = planted_cohort()
    n, t, p, m = c.n, c.t, c.q + 1, X.shape[1]
    dev = "cuda:0"
    args = caller_inputs(c, dev)
    b = torch.empty((m, t, p), dtype=torch.float64, device=dev)
    st = torch.empty(m, dtype=torch.uint8, device=dev)
    with pytest.raises(TypeError):
        gwas.gwas_solve_block_noalloc(n, p, t, *args, np.asfortranarray(X), m, b, None, st)
    Xh = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory()
    with pytest.raises(gwas.GwasError) as ei:
        gwas.gwas_solve_block_noalloc(n, p, t, *args, int(Xh.data_ptr()), m, b, None, st)
    assert ei.value.status == gwas.GWAS_ERR_ARG
