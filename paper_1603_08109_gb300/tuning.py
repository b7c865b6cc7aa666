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


def _bucket(spec):
    return (int(spec["kind"]), api.radius_bucket(spec["radius"]), api.order_bucket(spec["N"]))


def autotune_batch(images, outs, specs, reps: int = 3, margin: float = 0.01,
                   coverage: float = 0.95):
    """Tune the table for a batch plan on the batch's own time.

    Isolated single-image timings miss what a batch does to a variant (the
    persistent launches share the GPU with the per-image and banded launches
    on the plan's side streams), so each (kind, radius bucket, order bucket)
    that the batch occupies is tuned on the graph time of the whole batch:
    greedily, buckets in decreasing order of estimated work until `coverage`
    of it is covered, each bucket trying every variant that its images can
    run while the other entries stay fixed.  A variant replaces the bucket's
    current entry only if the batch gets faster by more than `margin` (timing
    noise must not move the table).  Returns (entries, ms before, ms after)."""
    import torch

    dev = images[0].device
    stream = torch.cuda.current_stream(dev)

    def timed(plan):
        plan.replay()
        torch.cuda.synchronize(dev)
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.replay()
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None or t < best else best
        return best

    def measure():
        plan = api.BatchPlan(images, outs, specs)
        try:
            return timed(plan), plan.variants()
        finally:
            plan.close()

    work = {}
    members = {}
    for k, sp in enumerate(specs):
        key = _bucket(sp)
        work[key] = work.get(key, 0.0) + (sp["N"] + 1.0) * (2 * sp["radius"] + 1) * \
            sp["height"] * sp["width"]
        members.setdefault(key, []).append(k)
    order = sorted(work, key=lambda k: -work[k])
    total = sum(work.values())
    t0, _ = measure()
    best = t0
    entries = []
    done = 0.0
    for key in order:
        if done >= coverage * total:
            break
        done += work[key]
        cur = api.tuning_get(*key)
        choice = cur
        for v in range(-1, api.variant_count(key[0])):
            if v == cur:
                continue
            api.tuning_set(*key, v)
            plan = api.BatchPlan(images, outs, specs)
            try:
                got = plan.variants()
                if v >= 0 and not any(got[k] == v for k in members[key]):
                    continue  # no image of the bucket can run v
                t = timed(plan)
            finally:
                plan.close()
            if t < best * (1.0 - margin):
                best, choice = t, v
        api.tuning_set(*key, choice)
        entries.append({"kind": key[0], "radius_bucket": key[1], "order_bucket": key[2],
                        "variant": choice, "ms": best, "batch": True})
    return entries, t0, best
