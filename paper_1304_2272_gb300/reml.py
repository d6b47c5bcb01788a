"""REML fitting of h through the library's hand-written adjoint (marshalling only).

``REMLFunction`` is a ``torch.autograd.Function`` whose forward calls ``gwas_reml`` (FP64
Cholesky and L^-1 on the GPU) and whose backward returns the adjoint gradient the
library computed with it, so the REML log-likelihood can be used like any other torch
objective. ``GLSFunction`` does the same for the per-SNP estimates: its forward returns
b_i of Eq. (1) for a block of SNPs at (h, sigma^2), its backward forms the
vector-Jacobian product sum_i <g_i, db_i/dh> from the library's db_i/dh pass (which
recomputes M^-1 x_i from the dosages instead of storing Xbar). ``fit_h`` maximises the
profiled likelihood (sigma^2 profiled out) by a safeguarded secant iteration on its
derivative dl/dh, starting from h0.
"""
from __future__ import annotations

import numpy as np

from . import gwas


class REMLEngine:
    """Holds a context and the cohort's inputs for repeated REML evaluations."""

    def __init__(self, Phi, XL, Y, pheno: int = 0, **opts):
        self.Phi = np.asfortranarray(np.asarray(Phi, dtype=np.float64))
        self.XL = np.asfortranarray(np.asarray(XL, dtype=np.float64))
        n = self.Phi.shape[0]
        self.Y = np.asfortranarray(np.asarray(Y, dtype=np.float64).reshape(n, -1))
        self.n, self.q, self.t = n, self.XL.shape[1], self.Y.shape[1]
        self.pheno = pheno
        self.ctx = gwas.gwas_init(n, self.q + 1, self.t, **opts)
        self.evals = 0
        # Phi is read by every evaluation: keep one copy in device memory (Phi is
        # symmetric, so its storage order does not matter)
        import torch
        dev = f"cuda:{int(opts.get('device', 0))}"
        self.Phi_dev = torch.from_numpy(np.ascontiguousarray(self.Phi)).to(dev)
        torch.cuda.synchronize(dev)

    def eval(self, h: float, sigma2: float, profile: bool = False) -> dict:
        self.evals += 1
        r = gwas.gwas_reml(self.ctx, self.Phi_dev, h, sigma2, self.XL, self.Y, self.pheno,
                           profile)
        self.state = (float(h), float(sigma2))  # the (h, sigma2) the context is factored at
        return r

    def at(self, h: float, sigma2: float) -> None:
        """Make the context hold the factor (and db/dh state) of (h, sigma2)."""
        if getattr(self, "state", None) != (float(h), float(sigma2)):
            self.eval(h, sigma2)

    def close(self):
        if self.ctx:
            gwas.gwas_finalize(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_function():
    import torch

    class REMLFunction(torch.autograd.Function):
        """l(h, sigma^2) with its analytic gradient from the library."""

        @staticmethod
        def forward(ctx, h, sigma2, engine):
            r = engine.eval(float(h), float(sigma2))
            ctx.save_for_backward(torch.tensor([r["dl_dh"], r["dl_dsigma2"]], dtype=torch.float64))
            return torch.tensor(r["loglik"], dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g[0], grad_out * g[1], None

    return REMLFunction


REMLFunction = None


def reml_loglik(h, sigma2, engine):
    """Differentiable REML log-likelihood (torch tensors h, sigma2 of dtype float64)."""
    global REMLFunction
    if REMLFunction is None:
        REMLFunction = _make_function()
    return REMLFunction.apply(h, sigma2, engine)


def _make_gls_function():
    import torch

    def solve(engine, X, with_grad):
        m = int(X.shape[0])
        dev = X.device
        b = torch.empty((m, engine.t, engine.q + 1), dtype=torch.float64, device=dev)
        st = torch.empty(m, dtype=torch.uint8, device=dev)
        if with_grad:
            d = torch.empty_like(b)
            gwas.gwas_solve_block_grad_device(engine.ctx, X, m, b, None, st, d)
        else:
            d = None
            gwas.gwas_solve_block_device(engine.ctx, X, m, b, None, st)
        gwas.gwas_sync(engine.ctx)
        return b, st, d

    class GLSFunction(torch.autograd.Function):
        """b_i(h, sigma^2) of a block of SNPs (m x t x p, NaN where status != 0), with
        db_i/dh from the library's adjoint pass. b does not depend on sigma^2 (scaling M
        scales S_i^-1 and bbar_i inversely), so its sigma^2 gradient is exactly zero."""

        @staticmethod
        def forward(ctx, h, sigma2, X, engine):
            engine.at(float(h), float(sigma2))
            b, st, _ = solve(engine, X, False)
            ctx.engine, ctx.hs = engine, (float(h), float(sigma2))
            ctx.save_for_backward(h, sigma2, X)
            return b

        @staticmethod
        def backward(ctx, grad_b):
            h, sigma2, X = ctx.saved_tensors
            engine = ctx.engine
            engine.at(*ctx.hs)  # another evaluation may have moved the context since
            _, st, d = solve(engine, X, True)
            ok = (st == 0).view(-1, 1, 1)
            # chain rule: dL/dh = sum_i <dL/db_i, db_i/dh> over the solved SNPs
            gh = torch.where(ok, grad_b * d, torch.zeros_like(d)).sum()
            return (gh.to(device=h.device, dtype=h.dtype).reshape(h.shape),
                    torch.zeros_like(sigma2), None, None)

    return GLSFunction


GLSFunction = None


def gls_b(h, sigma2, X, engine):
    """Differentiable b_i of Eq. (1) for the SNPs of X (a device int8 tensor of shape
    (m, n), i.e. n x m column-major dosages, m <= the engine's m_blk) at heritability h and
    scale sigma2 (float64 torch scalars); returns an m x t x p device tensor."""
    global GLSFunction
    if GLSFunction is None:
        GLSFunction = _make_gls_function()
    return GLSFunction.apply(h, sigma2, X, engine)


def fit_h(engine: REMLEngine, h0: float = 0.1, lo: float = 1e-4, hi: float = 1 - 1e-4,
          tol: float = 1e-10, max_iter: int = 60) -> dict:
    """Maximise the profiled REML likelihood in h from h0 using dl/dh (gradient-based).

    Secant steps on g(h) = dl_p/dh, kept inside a bracket [a, b] with g(a) > 0 > g(b)
    once one is found (bisection when a secant step leaves it)."""
    def g(h):
        return engine.eval(h, 1.0, profile=True)["dl_dh"]

    h_prev, g_prev = h0, g(h0)
    a, b = (lo, hi)
    ga, gb = None, None
    if g_prev > 0:
        a, ga = h0, g_prev
    else:
        b, gb = h0, g_prev
    # first step: move along the gradient until the sign changes (bracket)
    step = 0.05 if g_prev > 0 else -0.05
    h = min(max(h0 + step, lo), hi)
    history = [(h0, g_prev)]
    for _ in range(max_iter):
        gh = g(h)
        history.append((h, gh))
        if gh > 0:
            a, ga = h, gh
        else:
            b, gb = h, gh
        if abs(h - h_prev) < tol or gh == 0.0:
            break
        if ga is not None and gb is not None:
            cand = h - gh * (h - h_prev) / (gh - g_prev) if gh != g_prev else 0.5 * (a + b)
            if not (min(a, b) < cand < max(a, b)):
                cand = 0.5 * (a + b)
        else:
            cand = h + (h - h_prev) * 2.0  # still looking for a sign change
            cand = min(max(cand, lo), hi)
        h_prev, g_prev = h, gh
        h = cand
    r = engine.eval(h, 1.0, profile=True)
    return {"h": h, "sigma2": r["sigma2_hat"], "loglik": r["loglik"], "dl_dh": r["dl_dh"],
            "evals": engine.evals, "history": history}
