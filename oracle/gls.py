"""Plain FP64 CPU oracle of the GLS hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module. The product (the CUDA library and its Python binding) never
calls it, and this module imports nothing from the product.

What it computes (Peise, Fabregat, Aulchenko, Bientinesi, "Algorithms for
Large-scale Whole Genome Association Analysis"):

* Eq. (1): for each SNP i, b_i = (X_i^T M^{-1} X_i)^{-1} X_i^T M^{-1} y with
  X_i = [X_L | x_i] (Section 1).
* Section 2: the GLS is reduced to an OLS by L L^T := M, Xbar_i := L^{-1} X_i,
  ybar := L^{-1} y, then S_i := Xbar_i^T Xbar_i, bbar_i := Xbar_i^T ybar,
  b_i := S_i^{-1} bbar_i through a Cholesky factorisation of S_i.
* Section 2.1 / Algorithm 1: the i-independent pieces (Xbar_L, ybar, S_TL, bbar_T)
  are hoisted out of the SNP loop.

Three independent routes are provided so that each can check the others:
``gls_per_snp`` (the six steps of Section 2 applied to each full X_i),
``gls_hoisted`` (Algorithm 1) and ``gls_explicit_inverse`` (Eq. (1) written out with
an explicit M^{-1} from Gauss-Jordan elimination, no Cholesky, no triangular solve).

Readings of the paper that this oracle takes (the paper is silent or garbled there):

* The OLS formula of Section 2 omits Xbar_i^T in front of ybar; the oracle uses
  b_i = (Xbar_i^T Xbar_i)^{-1} Xbar_i^T ybar, as the six-step listing does.
* Section 2.1 writes S_BLi and S_BRi with stray transposes; read as Xbar_Ri^T Xbar_L
  (1 x (p-1)) and Xbar_Ri^T Xbar_Ri (scalar), as in Algorithm 1.
* Section 2.1 and Algorithms 1-3 write bbar_T := Xbar_L^T y (raw y); the algebra of
  the six steps needs ybar = L^{-1} y there, and Algorithm 1's SNP loop itself uses
  ybar. The oracle uses ybar everywhere.
* M = sigma^2 (h Phi + (1-h) I) is the variance-component covariance of this
  project's workloads; the paper only states that M is SPD (Section 1).
* The p x p output of Section 3 (a symmetric matrix produced next to b_i) is read as
  S_i^{-1}; the oracle exposes its (p,p) entry through the Wald statistic
  W_i = b_{i,p}^2 / (S_i^{-1})_{pp}.
* A SNP whose p x p system is singular (Cholesky pivot <= 1e-12 * max diag S_i)
  gets status 1 and NaN outputs; a dosage outside {0,1,2} gets status 2 and NaN.

Several phenotype columns Y (n x t) share one M (the one-M special case of the
multi-trait extension in Section 5): S_i is shared, bbar_i has t columns.

Output layout (matches the C ABI): b[i, j, c] = coefficient c of SNP i for phenotype
j (shape m x t x p), wald[i, j] (m x t), status[i] (m, uint8).
"""
from __future__ import annotations

import math

import numpy as np

PLAIN_MAX_N = 2048       # above this the Cholesky step uses LAPACK (same definition)
PLAIN_TRSV_MAX_N = 512   # above this forward substitution uses LAPACK dtrsm
SINGULAR_RTOL = 1e-12

STATUS_OK = 0
STATUS_SINGULAR = 1
STATUS_BAD_GENOTYPE = 2


class NotSPDError(ValueError):
    """M is not symmetric positive definite; ``pivot`` is the failing column."""

    def __init__(self, pivot: int):
        super().__init__(f"matrix not SPD: Cholesky pivot {pivot} is not positive")
        self.pivot = pivot


# ---------------------------------------------------------------------------
# Step a1: the covariance matrix.
# ---------------------------------------------------------------------------
def build_M(phi: np.ndarray, h: float, sigma2: float) -> np.ndarray:
    """M = sigma^2 (h Phi + (1 - h) I), n x n float64."""
    phi = np.asarray(phi, dtype=np.float64)
    n = phi.shape[0]
    return sigma2 * (h * phi + (1.0 - h) * np.eye(n))


# ---------------------------------------------------------------------------
# Step a2: Cholesky factorisation L L^T := M (Section 2, first operation).
# ---------------------------------------------------------------------------
def cholesky_plain(M: np.ndarray) -> np.ndarray:
    """Textbook column-by-column Cholesky, no blocking.

    Column j: L_jj = sqrt(M_jj - sum_k<j L_jk^2),
    L_ij = (M_ij - sum_k<j L_ik L_jk) / L_jj for i > j.
    Raises NotSPDError with the failing column if a pivot is not positive.
    """
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    L = np.zeros((n, n), dtype=np.float64)
    for j in range(n):
        d = M[j, j] - np.dot(L[j, :j], L[j, :j])
        if not d > 0.0:
            raise NotSPDError(j)
        L[j, j] = math.sqrt(d)
        if j + 1 < n:
            L[j + 1:, j] = (M[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def cholesky(M: np.ndarray, method: str = "auto") -> np.ndarray:
    """L with L L^T = M. ``plain`` = the loop above; ``lapack`` = numpy's dpotrf."""
    n = np.asarray(M).shape[0]
    if method == "plain" or (method == "auto" and n <= PLAIN_MAX_N):
        return cholesky_plain(M)
    try:
        return np.linalg.cholesky(np.asarray(M, dtype=np.float64))
    except np.linalg.LinAlgError:
        # locate the failing pivot with the plain definition
        return cholesky_plain(M)


# ---------------------------------------------------------------------------
# Triangular solves Xbar := L^{-1} X (Section 2, second and third operations).
# ---------------------------------------------------------------------------
def forward_substitution_plain(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve L X = B row by row: X_i = (B_i - sum_k<i L_ik X_k) / L_ii."""
    L = np.asarray(L, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    B2 = B.reshape(B.shape[0], -1)
    n = L.shape[0]
    X = np.zeros_like(B2, dtype=np.float64)
    for i in range(n):
        X[i] = (B2[i] - L[i, :i] @ X[:i]) / L[i, i]
    return X[:, 0] if vec else X


def forward_substitution(L: np.ndarray, B: np.ndarray, method: str = "auto") -> np.ndarray:
    """L^{-1} B. ``plain`` = the loop above; ``lapack`` = scipy's triangular solve."""
    n = np.asarray(L).shape[0]
    if method == "plain" or (method == "auto" and n <= PLAIN_TRSV_MAX_N):
        return forward_substitution_plain(L, B)
    from scipy.linalg import solve_triangular
    return solve_triangular(np.asarray(L, dtype=np.float64),
                            np.asarray(B, dtype=np.float64), lower=True,
                            check_finite=False)


# ---------------------------------------------------------------------------
# Small helpers shared by the routes below.
# ---------------------------------------------------------------------------
def dot_cols(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Column-wise dot products sum_r U[r, c] V[r, c] (symmetric in U and V)."""
    return np.sum(U * V, axis=0)


def genotype_status(X: np.ndarray) -> np.ndarray:
    """Status 2 for every SNP column holding a dosage outside {0, 1, 2}."""
    X = np.asarray(X)
    bad = np.any((X < 0) | (X > 2), axis=0)
    return np.where(bad, STATUS_BAD_GENOTYPE, STATUS_OK).astype(np.uint8)


def spd_solve(S: np.ndarray, R: np.ndarray, rtol: float = SINGULAR_RTOL):
    """Batched p x p SPD solve by Cholesky (Section 2, sixth operation).

    S: (m, p, p), R: (m, p, t). Returns (b (m, p, t), Sinv_pp (m,), ok (m,)).
    A SNP whose pivot falls to <= rtol * max_j S_jj is marked not ok.
    """
    S = np.asarray(S, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    m, p, _ = S.shape
    C = np.zeros_like(S)
    scale = np.max(np.diagonal(S, axis1=1, axis2=2), axis=1)
    ok = np.ones(m, dtype=bool)
    for j in range(p):
        d = S[:, j, j] - np.sum(C[:, j, :j] ** 2, axis=1)
        ok &= d > rtol * scale
        C[:, j, j] = np.sqrt(np.where(ok, d, 1.0))
        for i in range(j + 1, p):
            C[:, i, j] = (S[:, i, j] - np.sum(C[:, i, :j] * C[:, j, :j], axis=1)) / C[:, j, j]
    # forward: C z = R
    Zs = np.zeros_like(R)
    for i in range(p):
        Zs[:, i, :] = (R[:, i, :] - np.einsum("mk,mkt->mt", C[:, i, :i], Zs[:, :i, :])) / C[:, i, i][:, None]
    # backward: C^T b = z
    bsol = np.zeros_like(R)
    for i in reversed(range(p)):
        bsol[:, i, :] = (Zs[:, i, :] - np.einsum("mk,mkt->mt", C[:, i + 1:, i], bsol[:, i + 1:, :])) / C[:, i, i][:, None]
    sinv_pp = 1.0 / C[:, p - 1, p - 1] ** 2
    return bsol, sinv_pp, ok


def _finish(b_mpt: np.ndarray, sinv_pp: np.ndarray, ok: np.ndarray, status: np.ndarray):
    """Wald statistic and NaN/status conventions; returns (b m x t x p, wald m x t, status)."""
    b = np.transpose(b_mpt, (0, 2, 1)).copy()              # m x t x p
    wald = b[:, :, -1] ** 2 / sinv_pp[:, None]
    status = status.copy()
    status[(status == STATUS_OK) & ~ok] = STATUS_SINGULAR
    bad = status != STATUS_OK
    b[bad] = np.nan
    wald[bad] = np.nan
    return b, wald, status


# ---------------------------------------------------------------------------
# Route 1: the six steps of Section 2 applied to each full design matrix X_i.
# ---------------------------------------------------------------------------
def normal_equations_per_snp(L: np.ndarray, XL: np.ndarray, Y: np.ndarray,
                             X: np.ndarray, trsv: str = "auto"):
    """S_i = Xbar_i^T Xbar_i and bbar_i = Xbar_i^T ybar for every SNP (Section 2).

    Xbar_i = L^{-1}[X_L | x_i]; S_i is formed in full, both triangles, from column
    dot products. Returns (S m x p x p, bbar m x p x t, genotype status)."""
    XL = np.asarray(XL, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64).reshape(XL.shape[0], -1)
    Xg = np.asarray(X)
    m = Xg.shape[1]
    q = XL.shape[1]
    t = Y.shape[1]
    p = q + 1
    status = genotype_status(Xg)
    XLbar = forward_substitution(L, XL, trsv)
    ybar = forward_substitution(L, Y, trsv)
    xbar = forward_substitution(L, Xg.astype(np.float64), trsv)
    S = np.empty((m, p, p))
    Rr = np.empty((m, p, t))
    cols = [np.broadcast_to(XLbar[:, j:j + 1], xbar.shape) for j in range(q)] + [xbar]
    for a in range(p):
        for c in range(p):
            S[:, a, c] = dot_cols(cols[a], cols[c])
        for j in range(t):
            Rr[:, a, j] = dot_cols(cols[a], np.broadcast_to(ybar[:, j:j + 1], xbar.shape))
    return S, Rr, status


def gls_per_snp(L: np.ndarray, XL: np.ndarray, Y: np.ndarray, X: np.ndarray,
                trsv: str = "auto"):
    """b_i for every SNP column of X via the six steps of Section 2 on X_i = [X_L | x_i]."""
    S, Rr, status = normal_equations_per_snp(L, XL, Y, X, trsv)
    b, sinv_pp, ok = spd_solve(S, Rr)
    return _finish(b, sinv_pp, ok, status)


# ---------------------------------------------------------------------------
# Route 2: Algorithm 1 (Section 2.1), i-independent work hoisted out of the loop.
# ---------------------------------------------------------------------------
def setup_hoisted(L: np.ndarray, XL: np.ndarray, Y: np.ndarray, trsv: str = "auto"):
    """Algorithm 1 before the loop: Xbar_L, ybar, S_TL = Xbar_L^T Xbar_L, bbar_T = Xbar_L^T ybar."""
    XL = np.asarray(XL, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64).reshape(XL.shape[0], -1)
    XLbar = forward_substitution(L, XL, trsv)
    ybar = forward_substitution(L, Y, trsv)
    S_TL = XLbar.T @ XLbar
    bbar_T = XLbar.T @ ybar
    return XLbar, ybar, S_TL, bbar_T


def gls_hoisted(L: np.ndarray, XL: np.ndarray, Y: np.ndarray, X: np.ndarray,
                trsv: str = "auto", setup=None):
    """Algorithm 1: per SNP, xbar = L^{-1} x_i, S_BLi = xbar^T Xbar_L,
    S_BRi = xbar^T xbar, bbar_Bi = xbar^T ybar, then the p x p solve."""
    XLbar, ybar, S_TL, bbar_T = setup if setup is not None else setup_hoisted(L, XL, Y, trsv)
    Xg = np.asarray(X)
    m = Xg.shape[1]
    q = XLbar.shape[1]
    t = ybar.shape[1]
    p = q + 1
    status = genotype_status(Xg)
    xbar = forward_substitution(L, Xg.astype(np.float64), trsv)
    S_BL = xbar.T @ XLbar                     # m x q
    S_BR = np.sum(xbar * xbar, axis=0)        # m
    bbar_B = xbar.T @ ybar                    # m x t
    S = np.empty((m, p, p))
    S[:, :q, :q] = S_TL
    S[:, q, :q] = S_BL
    S[:, :q, q] = S_BL
    S[:, q, q] = S_BR
    Rr = np.empty((m, p, t))
    Rr[:, :q, :] = bbar_T
    Rr[:, q, :] = bbar_B
    b, sinv_pp, ok = spd_solve(S, Rr)
    return _finish(b, sinv_pp, ok, status)


# ---------------------------------------------------------------------------
# Route 3: Eq. (1) written out with an explicit inverse (no Cholesky at all).
# ---------------------------------------------------------------------------
def gauss_jordan_inverse(A: np.ndarray) -> np.ndarray:
    """Inverse by Gauss-Jordan elimination with partial pivoting."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    aug = np.hstack([A, np.eye(n)])
    for col in range(n):
        piv = col + int(np.argmax(np.abs(aug[col:, col])))
        if aug[piv, col] == 0.0:
            raise np.linalg.LinAlgError("singular matrix")
        if piv != col:
            aug[[col, piv]] = aug[[piv, col]]
        aug[col] /= aug[col, col]
        f = aug[:, col].copy()
        f[col] = 0.0
        aug -= np.outer(f, aug[col])
    return aug[:, n:]


def gls_explicit_inverse(M: np.ndarray, XL: np.ndarray, Y: np.ndarray, X: np.ndarray):
    """Eq. (1) literally: A_i = X_i^T M^{-1} X_i, r_i = X_i^T M^{-1} Y,
    b_i = A_i^{-1} r_i, Wald = b_p^2 / (A_i^{-1})_pp. Small n only."""
    Minv = gauss_jordan_inverse(M)
    XL = np.asarray(XL, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64).reshape(XL.shape[0], -1)
    Xg = np.asarray(X)
    m = Xg.shape[1]
    t = Y.shape[1]
    status = genotype_status(Xg)
    b = np.full((m, t, XL.shape[1] + 1), np.nan)
    wald = np.full((m, t), np.nan)
    for i in range(m):
        if status[i] != STATUS_OK:
            continue
        Xi = np.hstack([XL, Xg[:, i:i + 1].astype(np.float64)])
        A = Xi.T @ Minv @ Xi
        r = Xi.T @ Minv @ Y
        try:
            Ainv = gauss_jordan_inverse(A)
        except np.linalg.LinAlgError:
            status[i] = STATUS_SINGULAR
            continue
        bi = Ainv @ r
        b[i] = bi.T
        wald[i] = bi[-1] ** 2 / Ainv[-1, -1]
    return b, wald, status


# ---------------------------------------------------------------------------
# OLS by Householder QR of Xbar_i (the alternative named in Section 2).
# ---------------------------------------------------------------------------
def gls_qr(L: np.ndarray, XL: np.ndarray, Y: np.ndarray, X: np.ndarray):
    """b_i from the QR factorisation of Xbar_i: R b_i = Q^T ybar (b only)."""
    XLbar = forward_substitution(L, np.asarray(XL, dtype=np.float64))
    Y = np.asarray(Y, dtype=np.float64).reshape(XLbar.shape[0], -1)
    ybar = forward_substitution(L, Y)
    Xg = np.asarray(X)
    xbar = forward_substitution(L, Xg.astype(np.float64))
    m = Xg.shape[1]
    out = np.empty((m, Y.shape[1], XLbar.shape[1] + 1))
    for i in range(m):
        Q, R = np.linalg.qr(np.hstack([XLbar, xbar[:, i:i + 1]]))
        out[i] = np.linalg.solve(R, Q.T @ ybar).T
    return out


# ---------------------------------------------------------------------------
# Top level.
# ---------------------------------------------------------------------------
def factor(phi_or_M: np.ndarray, h: float | None, sigma2: float | None,
           is_phi: bool = True, method: str = "auto") -> np.ndarray:
    """Steps a1 + a2: the Cholesky factor L of M (built from Phi when ``is_phi``)."""
    M = build_M(phi_or_M, h, sigma2) if is_phi else np.asarray(phi_or_M, dtype=np.float64)
    return cholesky(M, method)


def gls(phi_or_M, h, sigma2, XL, Y, X, is_phi: bool = True, route: str = "hoisted"):
    """b, Wald and status for every SNP column of X (m x t x p, m x t, m)."""
    if route == "explicit":
        M = build_M(phi_or_M, h, sigma2) if is_phi else np.asarray(phi_or_M, dtype=np.float64)
        return gls_explicit_inverse(M, XL, Y, X)
    L = factor(phi_or_M, h, sigma2, is_phi)
    if route == "per_snp":
        return gls_per_snp(L, XL, Y, X)
    return gls_hoisted(L, XL, Y, X)


def gls_multitrait(phi, hs, sigma2s, XL, Y, X, route: str = "hoisted"):
    """Section 5's multi-trait problem, b_ij = (X_i^T M_j^-1 X_i)^-1 X_i^T M_j^-1 y_j with
    M_j = sigma2_j (h_j Phi + (1 - h_j) I): every trait j is Eq. (1) with its own M_j and
    phenotype column y_j, for the same SNPs. Returns b (m x t x p), wald (m x t) and
    status (m x t), one column per trait."""
    Y = np.asarray(Y, dtype=np.float64).reshape(np.asarray(XL).shape[0], -1)
    outs = [gls(phi, h, s2, XL, Y[:, j:j + 1], X, route=route)
            for j, (h, s2) in enumerate(zip(hs, sigma2s))]
    b = np.concatenate([o[0] for o in outs], axis=1)
    wald = np.concatenate([o[1] for o in outs], axis=1)
    status = np.stack([o[2] for o in outs], axis=1)
    return b, wald, status


def gls_cov(phi_or_M, h, sigma2, XL, X, is_phi: bool = True, route: str = "hoisted"):
    """S_i^{-1} = (X_i^T M^{-1} X_i)^{-1} for every SNP (m x p x p, NaN unless status 0):
    the covariance of b_i (sigma^2 is inside M), read as the p x p matrix the method
    generates beside b_i (Section 3). ``hoisted``: S_i from Algorithm 1's Xbar_i, inverted
    by its p x p Cholesky; ``explicit``: Eq. (1)'s X_i^T M^{-1} X_i with a Gauss-Jordan
    M^{-1} and A_i^{-1} (small n only). Also returns the status (as ``gls``)."""
    XL = np.asarray(XL, dtype=np.float64)
    n = XL.shape[0]
    Xg = np.asarray(X)
    m, p = Xg.shape[1], XL.shape[1] + 1
    out = np.full((m, p, p), np.nan)
    if route == "explicit":
        M = build_M(phi_or_M, h, sigma2) if is_phi else np.asarray(phi_or_M, dtype=np.float64)
        Minv = gauss_jordan_inverse(M)
        status = genotype_status(Xg)
        for i in range(m):
            if status[i] != STATUS_OK:
                continue
            Xi = np.hstack([XL, Xg[:, i:i + 1].astype(np.float64)])
            try:
                out[i] = gauss_jordan_inverse(Xi.T @ Minv @ Xi)
            except np.linalg.LinAlgError:
                status[i] = STATUS_SINGULAR
        return out, status
    L = factor(phi_or_M, h, sigma2, is_phi)
    S, _, status = normal_equations_per_snp(L, XL, np.zeros((n, 1)), Xg)
    eye = np.broadcast_to(np.eye(p), S.shape)
    Sinv, _, ok = spd_solve(S, eye)
    status = np.where(status != STATUS_OK, status, np.where(ok, STATUS_OK, STATUS_SINGULAR))
    good = status == STATUS_OK
    out[good] = Sinv[good]
    return out, status.astype(np.uint8)
