"""Seeded generators for the GLS workloads (no method arithmetic here).

Workload shape, from the paper's problem statement (Section 1, Eq. 1) and its
experiments (Sections 3.1 and 4.3): n individuals, p = 4 columns per design matrix
(intercept + 2 covariates + 1 SNP), m SNPs. The relatedness model behind M and the
distributions below are this project's synthetic recipe:

* SNP columns: int8 dosages x ~ Binomial(2, f_j), f_j ~ U(0.05, 0.5), one f per SNP,
  stored column-major (each SNP's n dosages contiguous), like the paper's blocks of
  contiguous vectors X_blk.
* Relatedness: Phi = Z Z^T / K from K = 5000 simulated markers, each marker
  standardised by its empirical allele frequency; monomorphic markers are redrawn.
* Covariates: X_L = [1, N(0,1), N(0,1)] (n x 3).
* Phenotypes: y = X_L beta + sigma * (sqrt(h) Z u / sqrt(K) + sqrt(1-h) e), with
  beta, u, e standard normal. The random part has covariance
  sigma^2 (h Phi + (1-h) I), so y ~ N(X_L beta, M) without factoring M.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

N_MARKERS = 5000
FREQ_LO, FREQ_HI = 0.05, 0.5


def allele_freqs(rng: np.random.Generator, count: int,
                 lo: float = FREQ_LO, hi: float = FREQ_HI) -> np.ndarray:
    """Allele frequencies f ~ U(lo, hi), float64 vector of length ``count``."""
    return rng.uniform(lo, hi, size=count)


def genotypes(rng: np.random.Generator, n: int, freqs: np.ndarray) -> np.ndarray:
    """Dosages Binomial(2, f_j) as an n x m int8 array in column-major order."""
    freqs = np.asarray(freqs, dtype=np.float64)
    m = freqs.shape[0]
    g = (rng.random((n, m)) < freqs).astype(np.int8)
    g += (rng.random((n, m)) < freqs).astype(np.int8)
    return np.asfortranarray(g)


def relatedness(rng: np.random.Generator, n: int, n_markers: int = N_MARKERS,
                device: str | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Relatedness Phi = Z Z^T / K and the standardised markers Z (n x K, float64).

    Markers with an empirical frequency of 0 or 1 (monomorphic) are redrawn until
    every marker is polymorphic. ``device`` (e.g. "cuda:0") only moves the Z Z^T
    product onto a torch device for large n; the result is returned on the host.
    """
    freqs = allele_freqs(rng, n_markers)
    G = genotypes(rng, n, freqs)
    while True:
        fhat = G.mean(axis=0, dtype=np.float64) / 2.0
        bad = np.flatnonzero((fhat <= 0.0) | (fhat >= 1.0))
        if bad.size == 0:
            break
        G[:, bad] = genotypes(rng, n, allele_freqs(rng, bad.size))
    Z = (G.astype(np.float64) - 2.0 * fhat) / np.sqrt(2.0 * fhat * (1.0 - fhat))
    if device is None:
        phi = (Z @ Z.T) / float(n_markers)
    else:
        import torch
        Zt = torch.from_numpy(Z).to(device)
        phi = (Zt @ Zt.T / float(n_markers)).cpu().numpy()
    phi = np.ascontiguousarray(0.5 * (phi + phi.T))  # exact symmetry of the input
    return phi, Z


def covariates(rng: np.random.Generator, n: int, q: int = 3) -> np.ndarray:
    """Fixed covariates X_L = [1, N(0,1), ...] as an n x q float64 column-major array."""
    XL = np.empty((n, q), dtype=np.float64, order="F")
    XL[:, 0] = 1.0
    if q > 1:
        XL[:, 1:] = rng.standard_normal((n, q - 1))
    return XL


def phenotypes(rng: np.random.Generator, XL: np.ndarray, Z: np.ndarray, h: float,
               sigma2: float, t: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """t phenotype columns y = X_L beta + N(0, sigma^2 (h Phi + (1-h) I)).

    Returns (Y n x t column-major, beta q x t)."""
    n, q = XL.shape
    K = Z.shape[1]
    beta = rng.standard_normal((q, t))
    u = rng.standard_normal((K, t))
    e = rng.standard_normal((n, t))
    g = (Z @ u) / np.sqrt(float(K))
    Y = XL @ beta + np.sqrt(sigma2) * (np.sqrt(h) * g + np.sqrt(1.0 - h) * e)
    return np.asfortranarray(Y), beta


@dataclass
class Cohort:
    """One cohort's inputs: relatedness, covariates, phenotypes and model parameters."""
    n: int
    q: int
    t: int
    h: float
    sigma2: float
    phi: np.ndarray      # n x n float64, symmetric
    XL: np.ndarray       # n x q float64, column-major
    Y: np.ndarray        # n x t float64, column-major
    beta: np.ndarray     # q x t true fixed effects
    seed: int

    def snps(self, m: int, stream: int = 0) -> np.ndarray:
        """m seeded SNP columns (n x m int8, column-major); ``stream`` picks a block."""
        ss = np.random.SeedSequence([self.seed, 7, stream])
        rng = np.random.default_rng(ss)
        return genotypes(rng, self.n, allele_freqs(rng, m))


def make_cohort(seed: int, n: int, q: int = 3, t: int = 1, h: float = 0.4,
                sigma2: float = 1.0, n_markers: int = N_MARKERS,
                device: str | None = None) -> Cohort:
    """Draw one cohort with the recipe in the module docstring."""
    s_markers, s_cov, s_phen = np.random.SeedSequence([seed, 1]).spawn(3)
    phi, Z = relatedness(np.random.default_rng(s_markers), n, n_markers, device=device)
    XL = covariates(np.random.default_rng(s_cov), n, q)
    Y, beta = phenotypes(np.random.default_rng(s_phen), XL, Z, h, sigma2, t)
    return Cohort(n=n, q=q, t=t, h=h, sigma2=sigma2, phi=phi, XL=XL, Y=Y,
                  beta=beta, seed=seed)


def genotypes_torch(seed: int, n: int, m: int, device, freqs=None):
    """Large SNP blocks drawn directly on a torch device (n x m int8, column-major).

    Returned as a torch tensor of shape (m, n) in row-major order, i.e. the same
    memory as an n x m column-major matrix: SNP j's dosages are row j.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    if freqs is None:
        f = torch.rand((m, 1), generator=g, device=device, dtype=torch.float32)
        f = FREQ_LO + (FREQ_HI - FREQ_LO) * f
    else:
        f = torch.as_tensor(freqs, dtype=torch.float32, device=device).reshape(m, 1)
    a = (torch.rand((m, n), generator=g, device=device) < f).to(torch.int8)
    a += (torch.rand((m, n), generator=g, device=device) < f).to(torch.int8)
    return a


def pack_2bit(X: np.ndarray, call_of=(0, 1, 2), missing_call: int = 3) -> np.ndarray:
    """Pack int8 dosages (n x m) into 2-bit calls, four individuals per byte: column j
    becomes ceil(n/4) bytes, individual k in bits 2(k%4), 2(k%4)+1 of byte k/4. Dosage d
    in {0,1,2} becomes call ``call_of[d]``; any other value becomes ``missing_call``.
    Returns a (ceil(n/4) x m) uint8 array in F-order."""
    X = np.asarray(X)
    n, m = X.shape
    calls = np.full(X.shape, missing_call, dtype=np.uint8)
    for d in range(3):
        calls[X == d] = call_of[d]
    nb = -(-n // 4)
    padded = np.zeros((4 * nb, m), dtype=np.uint8)
    padded[:n] = calls
    q = padded.reshape(nb, 4, m)
    out = q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)
    return np.asfortranarray(out.astype(np.uint8))
