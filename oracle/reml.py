"""REML log-likelihood, its gradient and db_i/dh in plain FP64 -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module.

The paper takes M as given (Section 1: "M is SPD"); these are the quantities of the
variance-component model behind it, M(h, sigma^2) = sigma^2 (h Phi + (1-h) I), for the
null model y = X_L beta + e, e ~ N(0, M):

  l(h, s2) = -1/2 [ (n-q) log 2 pi + log|M| + log|X_L^T M^-1 X_L| + y^T P y ],
  P = M^-1 - M^-1 X_L (X_L^T M^-1 X_L)^-1 X_L^T M^-1,
  dl/dtheta = -1/2 [ tr(P dM/dtheta) - y^T P (dM/dtheta) P y ],
  dM/dh = s2 (Phi - I),   dM/ds2 = M / s2.

For the per-SNP GLS estimates of Eq. (1), differentiating the normal equations
X_i^T M^-1 (y - X_i b_i) = 0 gives
  db_i/dh = -S_i^-1 X_i^T M^-1 (dM/dh) M^-1 r_i,   r_i = y - X_i b_i,  S_i = X_i^T M^-1 X_i,
and, for h > 0 (dM/dh = (M - s2 I)/h and X_i^T M^-1 r_i = 0),
  db_i/dh = (s2/h) S_i^-1 (M^-1 X_i)^T (M^-1 r_i).
The explicit-inverse routes below are the definitions written out (small n only).
"""
from __future__ import annotations

import math

import numpy as np

from .gls import build_M, genotype_status, spd_solve


def _inv_spd(M: np.ndarray) -> np.ndarray:
    """M^-1 for SPD M through its Cholesky factor (LAPACK)."""
    from scipy.linalg import cho_factor, cho_solve
    c = cho_factor(M, lower=True)
    return cho_solve(c, np.eye(M.shape[0]))


def reml_parts(phi, h: float, sigma2: float, XL, y):
    """(M, M^-1, P, logdet M, logdet X_L^T M^-1 X_L, y^T P y) of the null model."""
    M = build_M(phi, h, sigma2)
    L = np.linalg.cholesky(M)
    logdet_M = 2.0 * float(np.sum(np.log(np.diag(L))))
    Minv = _inv_spd(M)
    XL = np.asarray(XL, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    A = XL.T @ Minv @ XL
    sign, logdet_A = np.linalg.slogdet(A)
    MX = Minv @ XL
    P = Minv - MX @ np.linalg.solve(A, MX.T)
    return M, Minv, P, logdet_M, float(logdet_A), float(y @ P @ y)


def reml_loglik(phi, h: float, sigma2: float, XL, y) -> float:
    n, q = np.asarray(XL).shape
    _, _, _, ldM, ldA, yPy = reml_parts(phi, h, sigma2, XL, y)
    return -0.5 * ((n - q) * math.log(2.0 * math.pi) + ldM + ldA + yPy)


def reml_grad(phi, h: float, sigma2: float, XL, y) -> np.ndarray:
    """(dl/dh, dl/dsigma2) from the trace formula with explicit dM."""
    phi = np.asarray(phi, dtype=np.float64)
    n = phi.shape[0]
    M, _, P, _, _, _ = reml_parts(phi, h, sigma2, XL, y)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    Py = P @ y
    out = []
    for dM in (sigma2 * (phi - np.eye(n)), M / sigma2):
        out.append(-0.5 * (np.sum(P * dM) - Py @ dM @ Py))
    return np.array(out)


def profiled_sigma2(phi, h: float, XL, y) -> float:
    """sigma^2 maximising l at fixed h: y^T P_1 y / (n - q), P_1 = P at sigma^2 = 1."""
    n, q = np.asarray(XL).shape
    return reml_parts(phi, h, 1.0, XL, y)[5] / (n - q)


def fit_h(phi, XL, y, lo: float = 1e-6, hi: float = 1.0 - 1e-6, xtol: float = 1e-12) -> float:
    """The REML estimate of h with sigma^2 profiled out (bounded 1-D search)."""
    from scipy.optimize import minimize_scalar

    def negl(h):
        return -reml_loglik(phi, h, profiled_sigma2(phi, h, XL, y), XL, y)

    r = minimize_scalar(negl, bounds=(lo, hi), method="bounded", options={"xatol": xtol})
    return float(r.x)


def db_dh(phi, h: float, sigma2: float, XL, Y, X, closed_form: bool = False) -> np.ndarray:
    """db_i/dh for every SNP column of X (m x t x p); NaN where the SNP is degenerate."""
    phi = np.asarray(phi, dtype=np.float64)
    n = phi.shape[0]
    M = build_M(phi, h, sigma2)
    Minv = _inv_spd(M)
    dM = sigma2 * (phi - np.eye(n))
    XL = np.asarray(XL, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64).reshape(n, -1)
    Xg = np.asarray(X)
    status = genotype_status(Xg)
    m, t, p = Xg.shape[1], Y.shape[1], XL.shape[1] + 1
    out = np.full((m, t, p), np.nan)
    for i in range(m):
        if status[i]:
            continue
        Xi = np.hstack([XL, Xg[:, i:i + 1].astype(np.float64)])
        S = Xi.T @ Minv @ Xi
        if not spd_solve(S[None], (Xi.T @ Minv @ Y)[None])[2][0]:
            continue  # singular S_i: the SNP's outputs stay NaN, as for b_i
        B = np.linalg.solve(S, Xi.T @ Minv @ Y)          # p x t
        R = Y - Xi @ B
        if closed_form:
            G = (sigma2 / h) * np.linalg.solve(S, (Minv @ Xi).T @ (Minv @ R))
        else:
            G = -np.linalg.solve(S, Xi.T @ Minv @ dM @ Minv @ R)
        out[i] = G.T
    return out
