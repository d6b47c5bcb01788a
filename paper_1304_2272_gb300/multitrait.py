"""Several traits of one cohort, each with its own covariance M_j (Section 5).

For t traits y_j with M_j = sigma2_j (h_j Phi + (1 - h_j) I), the SNP loop of Eq. (1)
gains a trait dimension: b_ij = (X_i^T M_j^-1 X_i)^-1 X_i^T M_j^-1 y_j. Every trait is a
cohort of one batch (its own factor, L_j^-1 and, on the mixed path, limbs); each solve
hands every trait the same dosage block, which the mixed path converts to BF16 once.
This module only marshals arguments: the factorisations and every step of the solve
run in the CUDA library through the batch entry points of ``include/gwas.h``.
"""
from __future__ import annotations

import numpy as np

from . import gwas


class MultiTrait:
    """``MultiTrait(n, t).factor(phi, hs, sigma2s, XL, Y).solve(X)``."""

    def __init__(self, n: int, t: int, p: int = 4, m_blk: int = 16384, device: int = 0,
                 **opts):
        self.n, self.t, self.p, self.m_blk = int(n), int(t), int(p), int(m_blk)
        self.device = int(device)
        self.batch = gwas.gwas_batch_init([self.n] * self.t, self.p, 1, m_blk=self.m_blk,
                                          device=self.device, **opts)

    def factor(self, phi, hs, sigma2s, XL, Y):
        """Factor M_j for every trait j (phi n x n, XL n x (p-1), Y n x t)."""
        if len(hs) != self.t or len(sigma2s) != self.t:
            raise ValueError("one h and one sigma2 per trait")
        phi = np.asfortranarray(np.asarray(phi, dtype=np.float64))
        XL = np.asfortranarray(np.asarray(XL, dtype=np.float64).reshape(self.n, -1))
        Y = np.asarray(Y, dtype=np.float64).reshape(self.n, self.t)
        for j in range(self.t):
            gwas.gwas_batch_factor(self.batch, j, phi, True, float(hs[j]), float(sigma2s[j]),
                                   XL, np.asfortranarray(Y[:, j:j + 1]))
        return self

    def solve_device(self, X, mb: int, b, wald, status):
        """One block of mb SNPs: X is a device (mb x n) int8 tensor (each SNP contiguous);
        b (t x mb x p), wald (t x mb) and status (t x mb) are device tensors, trait-major."""
        gwas.gwas_batch_solve_device(self.batch, [X] * self.t, [mb] * self.t,
                                     [b[j] for j in range(self.t)],
                                     [wald[j] for j in range(self.t)],
                                     [status[j] for j in range(self.t)])

    def solve(self, X):
        """b (m x t x p), wald (m x t), status (m x t) for host dosages X (n x m int8)."""
        import torch
        X = np.asarray(X, dtype=np.int8)
        m = X.shape[1]
        dev = f"cuda:{self.device}"
        b = np.empty((m, self.t, self.p))
        wald = np.empty((m, self.t))
        status = np.empty((m, self.t), dtype=np.uint8)
        bd = torch.empty((self.t, self.m_blk, self.p), dtype=torch.float64, device=dev)
        wd = torch.empty((self.t, self.m_blk), dtype=torch.float64, device=dev)
        sd = torch.empty((self.t, self.m_blk), dtype=torch.uint8, device=dev)
        Xd = torch.empty((self.m_blk, self.n), dtype=torch.int8, device=dev)
        for i0 in range(0, m, self.m_blk):
            mb = min(self.m_blk, m - i0)
            Xd[:mb].copy_(torch.from_numpy(np.ascontiguousarray(X[:, i0:i0 + mb].T)))
            torch.cuda.synchronize(dev)
            self.solve_device(Xd, mb, bd[:, :mb], wd[:, :mb], sd[:, :mb])
            gwas.gwas_batch_sync(self.batch)
            b[i0:i0 + mb] = bd[:, :mb].permute(1, 0, 2).cpu().numpy()
            wald[i0:i0 + mb] = wd[:, :mb].T.cpu().numpy()
            status[i0:i0 + mb] = sd[:, :mb].T.cpu().numpy()
        return b, wald, status

    def stats(self) -> dict:
        return gwas.gwas_batch_get_stats(self.batch)

    def close(self):
        if self.batch:
            gwas.gwas_batch_finalize(self.batch)
            self.batch = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
