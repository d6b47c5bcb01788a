"""Cache of autotuned tile configurations (the timing itself runs in the library).

``tuned_tile_cfg`` returns the fastest tile configuration for a problem shape on this
GPU, running ``gwas_autotune`` once per (device, n, p, t, precision, limbs, m_blk) key
and remembering the answer in a JSON file (``$GWAS_AUTOTUNE_CACHE``, default
``~/.cache/gwas_gb300/autotune.json``).
"""
from __future__ import annotations

import json
import os
from pathlib import Path

from . import gwas


def cache_path() -> Path:
    p = os.environ.get("GWAS_AUTOTUNE_CACHE")
    return Path(p) if p else Path.home() / ".cache" / "gwas_gb300" / "autotune.json"


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def _load() -> dict:
    try:
        return json.loads(cache_path().read_text())
    except (OSError, ValueError):
        return {}


def _store(db: dict) -> None:
    path = cache_path()
    try:
        path.parent.mkdir(parents=True, exist_ok=True)
        tmp = path.with_suffix(".tmp")
        tmp.write_text(json.dumps(db, indent=1, sort_keys=True))
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home: tuning still applies to the context


def key_for(n: int, p: int, t: int, precision: int, limbs: int, m_blk: int) -> str:
    return f"{_device_name()}|n={n}|p={p}|t={t}|prec={precision}|limbs={limbs}|mblk={m_blk}"


def tuned_tile_cfg(ctx, n: int, p: int, t: int, precision: int, limbs: int, m_blk: int,
                   X=None, retune: bool = False) -> dict:
    """Apply the cached (or freshly measured) best tile configuration to ``ctx``."""
    key = key_for(n, p, t, precision, limbs, m_blk)
    db = _load()
    if not retune and key in db:
        gwas.gwas_set_tile_cfg(ctx, db[key]["tile_cfg"])
        return dict(db[key], cached=True)
    res = gwas.gwas_autotune(ctx, X, m_blk)
    db[key] = res
    _store(db)
    return dict(res, cached=False)
