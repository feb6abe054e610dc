"""Virtual-processor (VP) layouts: rectangular blocks of grid columns.

A VP is (grid, x0, y0, w, h): columns x0 <= i < x0+w, y0 <= j < y0+h of one
grid.  The layouts here tile each grid exactly (no gap, no overlap).
"""
import heapq

import numpy as np

from .rng import splitmix64


def regular_blocks(nx, ny, bw, bh, grid=0):
    """Row-major blocks of bw x bh columns; partial blocks at the far edges."""
    vps = []
    for y0 in range(0, ny, bh):
        for x0 in range(0, nx, bw):
            vps.append((grid, x0, y0, min(bw, nx - x0), min(bh, ny - y0)))
    return vps


def guillotine(nx, ny, nleaves, min_side, seed, grid=0, x_align=1):
    """Seeded guillotine partition into `nleaves` uneven rectangles.

    Repeatedly take the region of largest area (ties: lowest creation id),
    cut it across its longer side (ties: cut across x, i.e. split the width)
    at a position drawn uniformly among those that leave both parts at least
    `min_side` long -- for cuts across x, among the positions on multiples of
    `x_align` columns (min_side and nx multiples of x_align keep every x
    extent a multiple of it).  Split number s draws its position from output
    s of SplitMix64(seed).  The two parts get the next two creation ids.
    Leaves are returned in row-major order of their (y0, x0) corners.
    """
    heap = [(-nx * ny, 0, 0, 0, nx, ny)]
    next_id = 1
    leaves = 1
    s = 0
    while leaves < nleaves:
        negarea, rid, x0, y0, w, h = heapq.heappop(heap)
        split_w = w >= h
        length = w if split_w else h
        step = x_align if split_w else 1
        npos = (length - 2 * min_side) // step + 1
        if npos <= 0:
            raise ValueError("cannot split region %r further" % ((x0, y0, w, h),))
        cut = min_side + step * int(splitmix64(seed, s) % np.uint64(npos))
        s += 1
        if split_w:
            a = (x0, y0, cut, h)
            b = (x0 + cut, y0, w - cut, h)
        else:
            a = (x0, y0, w, cut)
            b = (x0, y0 + cut, w, h - cut)
        for part in (a, b):
            heapq.heappush(heap, (-part[2] * part[3], next_id) + part)
            next_id += 1
        leaves += 1
    rects = sorted((e[3], e[2], e[4], e[5]) for e in heap)   # (y0, x0, w, h)
    return [(grid, x0, y0, w, h) for (y0, x0, w, h) in rects]


def layout_stats(vps):
    """Realised side and area distribution of a layout (for reports)."""
    w = np.array([v[3] for v in vps])
    h = np.array([v[4] for v in vps])
    a = w * h
    return {"n": len(vps), "w_min": int(w.min()), "w_max": int(w.max()),
            "h_min": int(h.min()), "h_max": int(h.max()),
            "area_min": int(a.min()), "area_max": int(a.max()),
            "area_mean": float(a.mean())}
