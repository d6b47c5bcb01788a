"""CPU oracle of the GLS hot path -- TEST INFRASTRUCTURE ONLY.

Plain FP64 (and exact rational) restatements of the paper's method, written to be
checked by eye against the paper. Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the CUDA library and
its binding never do, and this package imports nothing from them.
"""
from . import exact, gls, reml  # noqa: F401
