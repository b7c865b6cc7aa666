"""Host-side work partitioning across ranks (one process per GPU).

The filter shards without any data exchange: independent images go to
different ranks, and one large image splits into row bands.  An output row
depends on input rows within the radius W, so a rank that outputs rows
[y0, y1) reads input rows [y0 - W, y1 + W) (clipped to the image) once; the
image-gradient needs input rows within 2W and output cotangents within W of
the band.  The only cross-rank reduction is the scalar sigma_r gradient.
"""
from __future__ import annotations

__all__ = ["assign_images", "row_bands", "Band"]


class Band:
    """Rows [y0, y1) that a rank outputs, and the input window it needs."""

    def __init__(self, y0: int, y1: int, height: int, radius: int, grad: bool = False):
        self.y0, self.y1 = y0, y1
        halo = 2 * radius if grad else radius
        self.in0 = max(0, y0 - halo)
        self.in1 = min(height, y1 + halo)
        # rows of the output cotangent that influence the band's image gradient
        self.g0 = max(0, y0 - radius)
        self.g1 = min(height, y1 + radius)

    @property
    def rows(self) -> int:
        return self.y1 - self.y0

    def __repr__(self):  # pragma: no cover
        return "Band(out=[%d,%d), in=[%d,%d))" % (self.y0, self.y1, self.in0, self.in1)


def row_bands(height: int, world: int, radius: int, grad: bool = False):
    """Split `height` rows into `world` contiguous bands of near-equal size."""
    if world < 1 or height < 1:
        raise ValueError("height and world must be positive")
    base, extra = divmod(height, world)
    bands, y = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        bands.append(Band(y, y + n, height, radius, grad))
        y += n
    return bands


def assign_images(costs, world: int):
    """Longest-processing-time-first assignment of independent images to
    ranks; returns one list of image indices per rank."""
    loads = [0.0] * world
    out = [[] for _ in range(world)]
    for k in sorted(range(len(costs)), key=lambda i: -costs[i]):
        r = min(range(world), key=lambda j: loads[j])
        out[r].append(k)
        loads[r] += costs[k]
    return out
