"""Seeded generators for the synthetic GWAS workloads.

The paper characterises its experiments only by the sizes (n, p, m, t)
(Section 6); it names no dataset.  These generators stand in for real cohorts
with the structure of the paper's workload (Section 2, Fig. 1):

* genotypes X_R: int8 in {0, 1, 2}, one allele frequency f_i ~ U(0.05, 0.5)
  per SNP and Hardy-Weinberg proportions (each individual carries two
  independent Bernoulli(f_i) alleles);
* kinship Phi: G_s G_s^T / 5000 + 1e-3 I, where G_s holds 5000 extra SNPs with
  every column standardised by its sample mean and its sample standard
  deviation (ddof = 0; monomorphic columns are redrawn);
* covariates X_L = [1 | N(0,1) | N(0,1) | ...] (n x (p-1));
* heritabilities h_j^2 ~ U(0.1, 0.9);
* phenotypes Y ~ N(0, 1), i.i.d.

Memory layouts are those of the C interface (column-major), written as C-order
numpy arrays: ``XR`` has shape (m, n) (SNP-major), ``Y`` (t, n) (trait-major),
``XL`` (p-1, n) and ``phi`` (n, n).

Genotypes and phenotypes are drawn in fixed chunks, each from its own child
seed, so any sub-range [i0, i1) of SNPs (or of traits) can be regenerated on
its own and matches the same range of a full draw.  Nothing here computes any
part of the GLS method.
"""
from __future__ import annotations

import concurrent.futures as _cf
import dataclasses
import math
import os

import numpy as np

BASE_SEED = 20121029

# sub-seed offsets
_GENO, _KIN, _COV, _H2, _PHENO, _REQ = 0, 1, 2, 3, 4, 5

SNP_CHUNK = 8192
TRAIT_CHUNK = 1024
KINSHIP_SNPS = 5000


def _chunk_rng(seed: int, stream: int, chunk: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream, chunk])))


def _hwe_draw(rng: np.random.Generator, f: np.ndarray, n: int) -> np.ndarray:
    """Genotype counts for len(f) SNPs x n individuals, int8 (SNP-major).

    One uniform per genotype: count = [u >= (1-f)^2] + [u >= 1 - f^2], which
    gives P(0) = (1-f)^2, P(1) = 2f(1-f), P(2) = f^2 (Hardy-Weinberg).
    """
    u = rng.random((f.shape[0], n), dtype=np.float64)
    lo = ((1.0 - f) ** 2)[:, None]
    hi = (1.0 - f * f)[:, None]
    out = (u >= lo).astype(np.int8)
    out += (u >= hi).astype(np.int8)
    return out


def _geno_chunk(n: int, seed: int, c: int):
    rng = _chunk_rng(seed, _GENO, c)
    f = rng.uniform(0.05, 0.5, size=SNP_CHUNK)
    return f, _hwe_draw(rng, f, n)


def allele_freqs(m: int, seed: int = BASE_SEED, i0: int = 0, i1: int | None = None) -> np.ndarray:
    """Allele frequency of SNPs [i0, i1)."""
    i1 = m if i1 is None else i1
    out = np.empty(i1 - i0)
    for c in range(i0 // SNP_CHUNK, (i1 + SNP_CHUNK - 1) // SNP_CHUNK if i1 > i0 else 0):
        rng = _chunk_rng(seed, _GENO, c)
        f = rng.uniform(0.05, 0.5, size=SNP_CHUNK)
        a, b = max(i0, c * SNP_CHUNK), min(i1, (c + 1) * SNP_CHUNK)
        out[a - i0:b - i0] = f[a - c * SNP_CHUNK:b - c * SNP_CHUNK]
    return out


def genotypes(n: int, m: int, seed: int = BASE_SEED, i0: int = 0, i1: int | None = None,
              threads: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """SNPs [i0, i1) of an n x m genotype matrix: int8 array of shape (i1-i0, n)."""
    i1 = m if i1 is None else i1
    if not (0 <= i0 <= i1 <= m):
        raise ValueError("bad SNP range")
    rows = i1 - i0
    if out is None:
        out = np.empty((rows, n), dtype=np.int8)
    if rows == 0:
        return out
    chunks = range(i0 // SNP_CHUNK, (i1 + SNP_CHUNK - 1) // SNP_CHUNK)

    def work(c):
        _, g = _geno_chunk(n, seed, c)
        a, b = max(i0, c * SNP_CHUNK), min(i1, (c + 1) * SNP_CHUNK)
        out[a - i0:b - i0] = g[a - c * SNP_CHUNK:b - c * SNP_CHUNK]

    threads = threads or min(16, os.cpu_count() or 1)
    if threads > 1 and len(chunks) > 1:
        with _cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, chunks))
    else:
        for c in chunks:
            work(c)
    return out


def kinship(n: int, seed: int = BASE_SEED, snps: int = KINSHIP_SNPS, ridge: float = 1e-3) -> np.ndarray:
    """Kinship-like SPD matrix Phi (n x n) from `snps` standardised extra SNPs."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, _KIN])))
    f = rng.uniform(0.05, 0.5, size=snps)
    g = _hwe_draw(rng, f, n).astype(np.float64)  # (snps, n)
    while True:
        sd = g.std(axis=1)
        bad = np.flatnonzero(sd == 0.0)
        if bad.size == 0:
            break
        fb = rng.uniform(0.05, 0.5, size=bad.size)
        g[bad] = _hwe_draw(rng, fb, n)
    gs = (g - g.mean(axis=1, keepdims=True)) / g.std(axis=1, keepdims=True)
    phi = gs.T @ gs / snps
    phi = 0.5 * (phi + phi.T)
    phi[np.diag_indices(n)] += ridge
    return phi


def covariates(n: int, pm1: int = 3, seed: int = BASE_SEED) -> np.ndarray:
    """X_L as a (p-1, n) array: an intercept row of ones, then N(0,1) rows."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, _COV])))
    xl = np.empty((pm1, n))
    if pm1 > 0:
        xl[0] = 1.0
        if pm1 > 1:
            xl[1:] = rng.standard_normal((pm1 - 1, n))
    return xl


def heritabilities(t: int, seed: int = BASE_SEED, lo: float = 0.1, hi: float = 0.9) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, _H2])))
    return rng.uniform(lo, hi, size=t)


def phenotypes(n: int, t: int, seed: int = BASE_SEED, j0: int = 0, j1: int | None = None) -> np.ndarray:
    """Traits [j0, j1) of Y: float64 array of shape (j1-j0, n), i.i.d. N(0,1)."""
    j1 = t if j1 is None else j1
    if not (0 <= j0 <= j1 <= t):
        raise ValueError("bad trait range")
    out = np.empty((j1 - j0, n))
    for c in range(j0 // TRAIT_CHUNK, (j1 + TRAIT_CHUNK - 1) // TRAIT_CHUNK if j1 > j0 else 0):
        rng = _chunk_rng(seed, _PHENO, c)
        y = rng.standard_normal((TRAIT_CHUNK, n))
        a, b = max(j0, c * TRAIT_CHUNK), min(j1, (c + 1) * TRAIT_CHUNK)
        out[a - j0:b - j0] = y[a - c * TRAIT_CHUNK:b - c * TRAIT_CHUNK]
    return out


@dataclasses.dataclass
class Problem:
    n: int
    m: int
    t: int
    pm1: int
    phi: np.ndarray   # (n, n) float64
    XL: np.ndarray    # (p-1, n) float64
    XR: np.ndarray    # (m, n) int8
    Y: np.ndarray     # (t, n) float64
    h2: np.ndarray    # (t,) float64

    @property
    def p(self) -> int:
        return self.pm1 + 1


def make_problem(n: int, m: int, t: int, pm1: int = 3, seed: int = BASE_SEED,
                 with_snps: bool = True) -> Problem:
    xr = genotypes(n, m, seed) if with_snps else np.empty((0, n), np.int8)
    return Problem(n=n, m=m, t=t, pm1=pm1, phi=kinship(n, seed), XL=covariates(n, pm1, seed),
                   XR=xr, Y=phenotypes(n, t, seed), h2=heritabilities(t, seed))


def serving_requests(count: int, m: int, seed: int = BASE_SEED, t_max: int = 2000,
                     len_lo: int = 10_000, len_hi: int = 1_000_000, rate: float = 1.0):
    """A Poisson stream of requests: (arrival, t_k, i0, i1, h2 seed key, Y seed key).

    t_k = round(exp U(ln 1, ln t_max)); the SNP-range length is log-uniform on
    [len_lo, min(len_hi, m)] with a uniform start; inter-arrival times are
    exponential with the given rate (requests per second).
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, _REQ])))
    hi = min(len_hi, m)
    lo = min(len_lo, hi)
    reqs = []
    now = 0.0
    for k in range(count):
        now += rng.exponential(1.0 / rate)
        tk = int(round(math.exp(rng.uniform(0.0, math.log(t_max)))))
        tk = max(1, min(t_max, tk))
        ln = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        ln = max(1, min(m, ln))
        i0 = int(rng.integers(0, m - ln + 1))
        reqs.append({"id": k, "arrival": now, "t": tk, "i0": i0, "i1": i0 + ln,
                     "seed": int(rng.integers(0, 2**62))})
    return reqs
