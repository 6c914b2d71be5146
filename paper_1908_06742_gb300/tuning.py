"""JSON cache of autotuner choices (tile shapes, block shapes, residency).

Keyed by device name, the kind of launch, storage precision and a digest of
the instance sizes, so a tuning found once is reused on the same GPU model for
the same workload shape.  File: $DDFLB_TUNE_CACHE or ~/.cache/ddflb/tuning.json.
"""
from __future__ import annotations

import hashlib
import json
import os


def path() -> str:
    return os.environ.get("DDFLB_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ddflb", "tuning.json"))


def _device() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def key(kind: str, cfgs) -> str:
    sizes = ",".join(f"{c.nx}x{c.ny}:{c.bc}" for c in cfgs)
    digest = hashlib.sha256(sizes.encode()).hexdigest()[:16]
    return f"{_device()}|{kind}|{cfgs[0].storage}|n={len(cfgs)}|{digest}"


def _load() -> dict:
    try:
        with open(path()) as f:
            return json.load(f)
    except Exception:
        return {}


def lookup(k: str):
    return _load().get(k)


def store(k: str, rec: dict) -> None:
    d = _load()
    d[k] = rec
    p = path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)
