"""The FP64 fma rate probe, the denominator of the FP64 block kernel's roofline.

gwas_fp64_fma_rate times the block kernel's own inner loop (4 x 4 register tiles of fma
on shared-memory operands) without any global memory traffic. It must report a rate
below the unit-count bound (152 SMs x 2 FP64 fma per clock x 2 flop x the maximum clock,
1.259 TFLOP/s at 2070 MHz) and at or above the algorithmic rate the FP64 block kernel
reaches on the same device, so that the kernel's roofline fraction is at most 1.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_bounds_the_block_kernel(gpu):
    import torch
    from paper_1304_2272_gb300 import gwas
    r = gwas.gwas_fp64_fma_rate(0)
    print(f"[probe] FP64 fma rate {r:.4f} TFLOP/s")
    assert 0.5 < r < 1.3

    n, mb = 4096, 8192
    c = synth.make_cohort(81, n, device="cuda")
    Xd = synth.genotypes_torch(82, n, mb, "cuda")
    with gwas.GLS(n, 4, 1, m_blk=mb, timing=1) as e:
        e.factor(c.phi, c.h, c.sigma2, c.XL, c.Y)
        b = torch.empty((mb, 1, 4), dtype=torch.float64, device="cuda")
        s = torch.empty(mb, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        gwas.gwas_solve_block_device(e.ctx, Xd, mb, b, None, s)   # warm-up
        gwas.gwas_sync(e.ctx)
        gwas.gwas_reset_stats(e.ctx)
        for _ in range(3):
            gwas.gwas_solve_block_device(e.ctx, Xd, mb, b, None, s)
        st = e.stats()
    launch_s = st["trsm_ms"] / st["trsm_launches"] / 1e3
    achieved = (n * (n + 1) + 2.0 * n * 5) * mb / launch_s / 1e12
    print(f"[probe] FP64 block kernel {achieved:.4f} TFLOP/s (algorithmic), "
          f"{achieved / r:.3f} of the probe")
    assert np.all(s.cpu().numpy() == 0)
    assert achieved <= 1.02 * r   # 2 % for clock changes between the two timings
