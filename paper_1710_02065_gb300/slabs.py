"""Slab decomposition of one lattice along x (host-side plan).

One solve split over R ranks gives each rank the x range [x0, x1) of every
row (the direction-major layout keeps each slab a set of contiguous row
segments).  A step needs, besides the rank's own cells, the populations that
stream into the slab across its two x faces: the ones with xi_x > 0 of the
column just left of the slab (x0 - 1) and the ones with xi_x < 0 of the
column just right of it (x1), with wrap-around on a periodic x axis.  Those
are the halo: 3 populations per face cell on D2Q9, 5 on D3Q19, 9 on D3Q27.
This module computes the slabs and the crossing directions; the exchange
itself is the caller's (host memory or a collective library).
"""
from __future__ import annotations

import numpy as np


def slab_ranges(nx: int, nranks: int) -> list[tuple[int, int]]:
    """Near-equal [x0, x1) ranges covering 0..nx-1 in rank order."""
    if nranks < 1 or nranks > nx:
        raise ValueError(f"cannot split {nx} columns over {nranks} ranks")
    edges = [(nx * r) // nranks for r in range(nranks + 1)]
    return [(edges[r], edges[r + 1]) for r in range(nranks)]


def crossing_directions(xi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Indices of the directions that leave a slab through its +x face
    (xi_x > 0, received by the right neighbour) and through its -x face
    (xi_x < 0, received by the left neighbour)."""
    xi = np.asarray(xi)
    return np.flatnonzero(xi[:, 0] > 0), np.flatnonzero(xi[:, 0] < 0)


def halo_bytes_per_step(n: tuple[int, int, int], xi: np.ndarray, elem_bytes: int) -> int:
    """Bytes one slab receives per step: the crossing populations of both
    faces (ny nz cells each)."""
    right, left = crossing_directions(xi)
    return (len(right) + len(left)) * n[1] * n[2] * elem_bytes
