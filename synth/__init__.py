"""Seeded synthetic inputs shaped like the paper's GWAS workloads.

This package only draws random inputs (genotypes, relatedness matrix, covariates,
phenotypes) and packs dosages into the 2-bit input format. It holds none of the GLS method's arithmetic and is shared by the CPU
oracle, the tests and the benchmark; nothing here imports the CUDA path or the oracle.
"""
from .generators import (  # noqa: F401
    Cohort,
    allele_freqs,
    covariates,
    genotypes,
    genotypes_torch,
    make_cohort,
    pack_2bit,
    relatedness,
)
