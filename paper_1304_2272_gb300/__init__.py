"""GB300 (sm_103a) engine for the mixed-model GWAS GLS hot path.

The compute path lives in the CUDA library ``libgwas_gb300.so`` (sources in
``csrc/``, C ABI in ``include/gwas.h``); ``gwas`` is its ctypes binding. Importing
this package loads nothing; the library is loaded on first use and fails loudly
when it cannot be built or loaded. There is no CPU fallback.
"""
from .gwas import (  # noqa: F401
    GLS,
    GWAS_PREC_FP64,
    GWAS_PREC_MIXED,
    GwasError,
    gwas_autotune,
    gwas_batch_factor,
    gwas_batch_finalize,
    gwas_batch_get_stats,
    gwas_batch_init,
    gwas_batch_last_error,
    gwas_batch_reset_stats,
    gwas_batch_solve_device,
    gwas_batch_stream,
    gwas_batch_sync,
    gwas_default_opts,
    gwas_error_index,
    gwas_factor,
    gwas_finalize,
    gwas_get_stats,
    gwas_init,
    gwas_last_error,
    gwas_reset_stats,
    gwas_solve_all,
    gwas_solve_block,
    gwas_solve_block_cov_device,
    gwas_solve_block_device,
    gwas_solve_block_noalloc,
    gwas_solve_block_packed,
    gwas_solve_block_packed_device,
    gwas_reml,
    gwas_set_tile_cfg,
    gwas_solve_block_grad_device,
    gwas_stream,
    gwas_sync,
    load,
)
