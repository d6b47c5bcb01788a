"""Reader for the hand-derived fixtures in this folder (whitespace key/value lines)."""
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent


def load(name: str) -> dict:
    out = {}
    for line in (HERE / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        arr = np.array([float(v) for v in vals])
        out[key] = arr if arr.size > 1 else arr[0]
    n = int(out["n"])
    out["n"] = n
    for k in ("M", "phi"):
        if k in out:
            out[k] = out[k].reshape(n, n)
    out["XL"] = out["XL"].reshape(n, -1, order="F")
    out["x"] = out["x"].astype(np.int8).reshape(n, 1)
    out["b"] = np.atleast_1d(out["b"])
    return out
