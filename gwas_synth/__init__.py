"""Seeded synthetic GWAS inputs shaped like the paper's workloads.

This module is the ONLY code shared by the oracle side and the CUDA side.
It draws inputs and nothing else: it holds none of the GLS arithmetic
(no M, no Cholesky, no solves).  Every draw comes from a counter-based
Philox generator keyed by (seed, stream, study) with the chunk index in the
counter, so any range of SNP columns can be regenerated on its own.

Recipe (the shapes of Sec. 1.3-1.4 of the paper: n ~ 1e4 samples, p = 4,
millions of SNPs):

* kinship  Phi = Z Z^T / k + 1e-3 I, Z (n x k) genotypes drawn Binomial(2, f_l),
  f_l ~ U(0.05, 0.5), each column standardised with its sample mean and
  population SD (a constant column is redrawn, up to 64 times, then zeroed);
* covariates X_L (n x (p-1)): an intercept column of ones, then N(0,1) columns;
* SNP dosages x_j ~ Binomial(2, f_j), f_j ~ U(0.05, 0.5), stored int8
  (or float64 for the small FP64-dosage workload);
* phenotype y = X_L beta + 0.05 x_4 + e with e ~ N(0, M),
  M = sigma2 (h Phi + (1-h) I).  e is drawn without factoring M:
  e = sqrt(sigma2) (sqrt(h) (Z u / sqrt(k) + sqrt(1e-3) v) + sqrt(1-h) w)
  with u ~ N(0, I_k), v, w ~ N(0, I_n), whose covariance is exactly M.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20130218
CHUNK = 256            # SNP columns per generator chunk (fixed: independent of bs)
KINSHIP_RIDGE = 1e-3

# generator streams
_S_KINSHIP = 1
_S_COVAR = 2
_S_NOISE = 3
_S_DOSAGE = 4
_S_FREQ = 5


def _rng(seed: int, stream: int, study: int, index: int = 0) -> np.random.Generator:
    key = [int(seed) & 0xFFFFFFFFFFFFFFFF, (int(stream) << 32) | (int(study) & 0xFFFFFFFF)]
    return np.random.Generator(np.random.Philox(key=key, counter=[0, 0, 0, int(index)]))


def default_beta(q: int) -> np.ndarray:
    """Fixed-covariate effects: (1.0, 0.5, -0.5, 0.25, -0.25, ...)."""
    base = [1.0, 0.5, -0.5]
    out = []
    for i in range(q):
        if i < 3:
            out.append(base[i])
        else:
            out.append(0.25 * (1 if i % 2 else -1) / (1 + (i - 3) // 2))
    return np.asarray(out, dtype=np.float64)


def _binomial2(rng: np.random.Generator, freqs: np.ndarray, n: int) -> np.ndarray:
    """n x len(freqs) matrix of Binomial(2, f) draws (column-major, int8)."""
    u = rng.random((len(freqs), 2, n))
    d = (u[:, 0, :] < freqs[:, None]).astype(np.int8) + (u[:, 1, :] < freqs[:, None]).astype(np.int8)
    return np.asfortranarray(d.T)


def kinship_genotypes(n: int, k: int, seed: int = DEFAULT_SEED, study: int = 0) -> np.ndarray:
    """Standardised kinship genotypes Z (n x k, float64, column-major)."""
    rng = _rng(seed, _S_KINSHIP, study)
    freqs = rng.uniform(0.05, 0.5, size=k)
    Z = np.empty((n, k), dtype=np.float64, order="F")
    for c0 in range(0, k, CHUNK):
        c1 = min(k, c0 + CHUNK)
        crng = _rng(seed, _S_KINSHIP, study, 1 + c0 // CHUNK)
        block = _binomial2(crng, freqs[c0:c1], n).astype(np.float64)
        for j in range(block.shape[1]):
            col = block[:, j]
            redraw = 0
            while col.std() == 0.0 and redraw < 64:  # constant column: redraw from the chunk stream
                redraw += 1
                col = _binomial2(crng, freqs[c0 + j:c0 + j + 1], n)[:, 0].astype(np.float64)
            sd = col.std()
            # a column that stays constant (always so when n = 1) carries no kinship
            block[:, j] = (col - col.mean()) / sd if sd > 0.0 else 0.0
        Z[:, c0:c1] = block
    return Z


def kinship(Z: np.ndarray) -> np.ndarray:
    """Phi = Z Z^T / k + 1e-3 I (float64, symmetric, n x n)."""
    n, k = Z.shape
    Phi = Z @ Z.T
    Phi /= k
    Phi[np.diag_indices(n)] += KINSHIP_RIDGE
    return np.asfortranarray(Phi)


def covariates(n: int, q: int, seed: int = DEFAULT_SEED, study: int = 0) -> np.ndarray:
    """X_L (n x q): intercept then N(0,1) columns (float64, column-major)."""
    rng = _rng(seed, _S_COVAR, study)
    XL = np.empty((n, q), dtype=np.float64, order="F")
    if q > 0:
        XL[:, 0] = 1.0
    for j in range(1, q):
        XL[:, j] = rng.standard_normal(n)
    return XL


def snp_frequencies(c0: int, c1: int, seed: int = DEFAULT_SEED, study: int = 0) -> np.ndarray:
    """Allele frequencies f_j ~ U(0.05, 0.5) of SNP columns c0..c1-1."""
    out = np.empty(max(0, c1 - c0), dtype=np.float64)
    if c1 <= c0:
        return out
    for ch in range(c0 // CHUNK, (c1 - 1) // CHUNK + 1):
        f = _rng(seed, _S_FREQ, study, ch).uniform(0.05, 0.5, size=CHUNK)
        a, b = max(c0, ch * CHUNK), min(c1, (ch + 1) * CHUNK)
        out[a - c0:b - c0] = f[a - ch * CHUNK:b - ch * CHUNK]
    return out


def dosages(n: int, c0: int, c1: int, seed: int = DEFAULT_SEED, study: int = 0) -> np.ndarray:
    """SNP dosage columns c0..c1-1 (n x (c1-c0) int8, column-major, values 0/1/2)."""
    out = np.empty((n, c1 - c0), dtype=np.int8, order="F")
    if c1 <= c0:
        return out
    for ch in range(c0 // CHUNK, (c1 - 1) // CHUNK + 1):
        a, b = max(c0, ch * CHUNK), min(c1, (ch + 1) * CHUNK)
        f = snp_frequencies(ch * CHUNK, (ch + 1) * CHUNK, seed, study)
        rng = _rng(seed, _S_DOSAGE, study, ch)
        u = rng.random((CHUNK, 2, n))
        sel = slice(a - ch * CHUNK, b - ch * CHUNK)
        d = (u[sel, 0, :] < f[sel, None]).astype(np.int8) + (u[sel, 1, :] < f[sel, None]).astype(np.int8)
        out[:, a - c0:b - c0] = d.T
    return out


def phenotype(Z: np.ndarray, XL: np.ndarray, x_causal: np.ndarray, h: float, sigma2: float,
              seed: int = DEFAULT_SEED, study: int = 0, snp_effect: float = 0.05) -> np.ndarray:
    """y = X_L beta + snp_effect * x_causal + e,  e ~ N(0, sigma2 (h Phi + (1-h) I))."""
    n, k = Z.shape
    rng = _rng(seed, _S_NOISE, study)
    u = rng.standard_normal(k)
    v = rng.standard_normal(n)
    w = rng.standard_normal(n)
    e = np.sqrt(sigma2) * (np.sqrt(h) * (Z @ u / np.sqrt(k) + np.sqrt(KINSHIP_RIDGE) * v)
                           + np.sqrt(1.0 - h) * w)
    beta = default_beta(XL.shape[1])
    return XL @ beta + snp_effect * np.asarray(x_causal, dtype=np.float64) + e


def study(n: int, p: int, k: int, h: float, sigma2: float = 1.0,
          seed: int = DEFAULT_SEED, study_id: int = 0) -> dict:
    """One synthetic study: Phi, X_L, y and the generator parameters.

    The phenotype carries a small effect of SNP column 4 (the fifth SNP).
    """
    if p < 1 or n < 1:
        raise ValueError("need n >= 1 and p >= 1")
    Z = kinship_genotypes(n, k, seed, study_id)
    Phi = kinship(Z)
    XL = covariates(n, p - 1, seed, study_id)
    x4 = dosages(n, 4, 5, seed, study_id)[:, 0]
    y = phenotype(Z, XL, x4, h, sigma2, seed, study_id)
    return dict(n=n, p=p, k=k, h=float(h), sigma2=float(sigma2), seed=seed, study=study_id,
                Phi=Phi, XL=XL, y=y)


# The workloads (names say what they are, with their sizes).
WORKLOADS = {
    # plain FP64 GLS, small: dosages stored as float64
    "n1000_p4_m10k_f64": dict(n=1000, p=4, m=10_000, k=2000, h=0.6, sigma2=1.0, bs=4096, storage="f64"),
    # paper scale: n = 1e4, int8 dosages streamed in blocks of 4096 SNPs
    "n10k_p4_m1M_int8": dict(n=10_000, p=4, m=1_000_000, k=5000, h=0.5, sigma2=1.0, bs=4096, storage="int8"),
}
