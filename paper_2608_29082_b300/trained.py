"""Stored parameter sets (checkpoints of Theta) and their loading.

A checkpoint is a small JSON file: {"J": ..., "nu_pre": ..., "nu_post": ...,
"theta": [...], "eta": [...], "wB": [[w1, w2], ...], "wR": ..., "wP": ...,
"trained_on": "..."}.  Loading into a hierarchy with more levels copies the
deepest trained level (the paper's transfer rule, Sec. 4.2).
"""
from __future__ import annotations

import json
import os

import numpy as np

from .solver import LMGParams

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT = os.path.join(HERE, "params", "checker513_learned.json")
LOGNORMAL1025 = os.path.join(HERE, "params", "lognormal1025_learned.json")


def save(params: LMGParams, path: str, **meta) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    d = {"J": params.J, "nu_pre": int(params.nu_pre), "nu_post": int(params.nu_post),
         "theta": params.theta.tolist(), "eta": params.eta.tolist(), "wB": params.wB.tolist(),
         "wR": params.wR.tolist(), "wP": params.wP.tolist()}
    d.update(meta)
    with open(path, "w") as fh:
        json.dump(d, fh, indent=1)


def read(path: str) -> LMGParams:
    d = json.load(open(path))
    return LMGParams(np.asarray(d["theta"], float), np.asarray(d["eta"], float),
                     np.asarray(d["wB"], float), np.asarray(d["wR"], float),
                     np.asarray(d["wP"], float), int(d["nu_pre"]), int(d["nu_post"]))


def load(path: str | None, J: int) -> LMGParams:
    """The parameter set at path (default: the packaged trained set if present,
    else the identity initialisation), adapted to J levels."""
    p = path or (DEFAULT if os.path.exists(DEFAULT) else None)
    if p is None:
        return LMGParams.identity(J)
    return read(p).with_levels(J)


def describe(path: str | None) -> str:
    p = path or (DEFAULT if os.path.exists(DEFAULT) else None)
    if p is None:
        return "identity initialisation (Sec. 3.4), no trained set present"
    d = json.load(open(p))
    return f"{os.path.basename(p)}: {d.get('trained_on', 'trained')}"
