"""Tile-shape autotuning with a JSON cache.

The library keeps a table variant[kind][radius bucket][order bucket] of
compiled tile shapes (bf_tuning_get / bf_tuning_set).  ``autotune_grid``
times every variant on a synthetic image for each (kind, radius, N) of a
grid (bf_autotune, CUDA events) and records the winners; ``save`` / ``load``
keep the table in a JSON file so a later process can reuse it without
re-timing.
"""
from __future__ import annotations

import json
import os
from typing import Iterable

from . import api

DEFAULT_GRID = {
    "kinds": (api.BOX, api.GAUSS),
    "radii": (3, 5, 9, 15, 20, 30, 45, 60),
    "orders": (3, 8, 24, 48, 100, 200),
}


def autotune_grid(height: int = 1024, width: int = 1024, kinds: Iterable[int] = None,
                  radii: Iterable[int] = None, orders: Iterable[int] = None, sigma_r: float = 30.0,
                  reps: int = 3, seed: int = 0):
    """Time every tile variant for each grid point; return the table entries."""
    import torch

    from . import synth
    kinds = DEFAULT_GRID["kinds"] if kinds is None else kinds
    radii = DEFAULT_GRID["radii"] if radii is None else radii
    orders = DEFAULT_GRID["orders"] if orders is None else orders
    img = torch.from_numpy(synth.blocks_image(height, width, 32, 15.0, seed=seed)).cuda()
    entries = {}
    for kind in kinds:
        for r in radii:
            for N in orders:
                sr = max(sigma_r, 128.0 / 12.8)
                ss = r / 3.0
                key = (kind, api.radius_bucket(r), api.order_bucket(N))
                try:
                    v, ms = api.autotune(img, kind, sr, N, radius=r, sigma_s=ss, reps=reps)
                except api._lib.BFError:
                    continue
                entries[key] = {"kind": kind, "radius_bucket": key[1], "order_bucket": key[2],
                                "variant": v, "ms": ms, "radius": r, "N": N,
                                "shape": [height, width]}
    return list(entries.values())


def save(entries, path: str) -> None:
    import torch
    dev = torch.cuda.get_device_name(0) if torch.cuda.is_available() else "unknown"
    with open(path, "w") as fh:
        json.dump({"device": dev, "entries": entries}, fh, indent=1)


def load(path: str) -> int:
    """Install the entries of a JSON cache into the library's table."""
    if not os.path.exists(path):
        return 0
    with open(path) as fh:
        data = json.load(fh)
    n = 0
    for e in data.get("entries", []):
        api.tuning_set(int(e["kind"]), int(e["radius_bucket"]), int(e["order_bucket"]),
                       int(e["variant"]))
        n += 1
    return n
