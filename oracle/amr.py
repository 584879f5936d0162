"""Oracle for the AMR refinement rule of the 3D EBIT method (arxiv 2509.26361,
Sec. 2.5) and the narrow-band brick set built on it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.5: EBIT keeps one marker per edge, so cells on different refinement
levels must never share the interface.  The paper's rule: every cell inside the
3x3x3 block of cells centred on an interfacial cell is refined to the finest
level.  An interfacial cell is one that the interface crosses.  With the
colour-vertex field, that is a cell whose eight corner colours are not all
equal: an edge carries a marker exactly when its two end colours differ, and a
cell whose corners agree has no marker on any of its twelve edges.

Layout as in the package: ``cb`` is indexed [k, j, i] (x fastest), bit 0 the
node colour; node (i, j, k) is the lowest corner of cell (i, j, k); periodic.
"""
from __future__ import annotations

import numpy as np


def interfacial_cells(cb):
    """Boolean [nz, ny, nx]: cell (i, j, k) has corner colours that differ."""
    c = np.asarray(cb) & 1
    lo = np.ones(c.shape, dtype=bool)
    hi = np.zeros(c.shape, dtype=bool)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                corner = np.roll(c, (-dk, -dj, -di), axis=(0, 1, 2)).astype(bool)
                lo &= corner
                hi |= corner
    return hi & ~lo  # some corner is 1 and some corner is 0


def refine_mask(cb):
    """Boolean [nz, ny, nx]: cells within the 3x3x3 block around an interfacial
    cell (the cells that the rule of Sec. 2.5 refines to the finest level)."""
    f = interfacial_cells(cb)
    out = np.zeros_like(f)
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                out |= np.roll(f, (dk, dj, di), axis=(0, 1, 2))
    return out


def brick_tiles(cb, tile=8):
    """Ascending ids (x fastest) of the tile x tile x tile bricks that hold at
    least one refined cell; partial bricks at the upper ends count their cells
    inside the grid only."""
    m = refine_mask(cb)
    nz, ny, nx = m.shape
    tz, ty, tx = -(-nz // tile), -(-ny // tile), -(-nx // tile)
    ids = []
    for bz in range(tz):
        for by in range(ty):
            for bx in range(tx):
                if m[bz * tile:(bz + 1) * tile, by * tile:(by + 1) * tile, bx * tile:(bx + 1) * tile].any():
                    ids.append((bz * ty + by) * tx + bx)
    return np.array(ids, dtype=np.int64)
