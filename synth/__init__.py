"""Seeded synthetic inputs for the multi-trait GWAS grid of GLS problems.

This package is shared by the CPU oracle, the tests and the benchmark.  It
draws random numbers only: it holds none of the method's arithmetic.
"""
from .generators import (  # noqa: F401
    BASE_SEED,
    Problem,
    allele_freqs,
    covariates,
    genotypes,
    heritabilities,
    kinship,
    make_problem,
    phenotypes,
    serving_requests,
)
