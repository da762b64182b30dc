"""Brute-force definitions used to pin the oracle.

Each helper restates a definition of Sec. 2 of the paper directly, by
enumeration or by global connected-component labelling (scipy), so that a
mistake in the oracle's faster formulations shows up as a disagreement.
Nothing here is used by the CUDA library or by the oracle.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

S8 = np.ones((3, 3), dtype=int)
S4 = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]])


def _structs(conn: int):
    return (S8, S4) if conn == 8 else (S4, S8)


def component_counts(X: np.ndarray, conn: int = 8) -> tuple[int, int]:
    """(# n-components of X, # nbar-components of the complement of X), with
    everything outside the box counted as background (a one-pixel frame
    joins the outside into one component)."""
    so, sb = _structs(conn)
    P = np.pad(X != 0, 1)
    return ndimage.label(P, structure=so)[1], ndimage.label(~P, structure=sb)[1]


def globally_simple(X: np.ndarray, y: int, x: int, conn: int = 8) -> bool:
    """Definition of a simple point (Sec. 2) tested on the whole image: x in X is
    simple iff removing it neither deletes nor splits its n-component and
    neither creates nor merges nbar-components of the complement.  For x not in
    X the question is whether x may be added, i.e. whether x is simple for
    X cup {x}.  Both reduce to unchanged component counts."""
    A = (X != 0).copy()
    A[y, x] = True
    B = A.copy()
    B[y, x] = False
    return component_counts(A, conn) == component_counts(B, conn)


def edt_brute(F: np.ndarray, outside_is_feature: bool = False) -> np.ndarray:
    """min over feature points q of |p - q|^2 for every pixel p, by enumeration;
    INF (1 << 62) when there is no feature."""
    h, w = F.shape
    pts = np.argwhere(F != 0)
    if outside_is_feature:
        ring = [(-1, x) for x in range(-1, w + 1)] + [(h, x) for x in range(-1, w + 1)]
        ring += [(y, -1) for y in range(h)] + [(y, w) for y in range(h)]
        pts = np.concatenate([pts.reshape(-1, 2), np.array(ring)]) if ring else pts
    if len(pts) == 0:
        return np.full((h, w), 1 << 62, np.int64)
    yy, xx = np.mgrid[0:h, 0:w]
    best = np.full((h, w), 1 << 62, np.int64)
    for qy, qx in pts:
        d = (yy - qy) ** 2 + (xx - qx) ** 2
        np.minimum(best, d, out=best)
    return best


def disc_offsets(r: int):
    return [(dy, dx) for dy in range(-r, r + 1) for dx in range(-r, r + 1) if dx * dx + dy * dy <= r * r]


def _shift(S: np.ndarray, dy: int, dx: int, fill: bool) -> np.ndarray:
    """out[y, x] = S[y + dy, x + dx], `fill` outside the box."""
    h, w = S.shape
    out = np.full((h, w), fill, bool)
    ys0, ys1 = max(0, -dy), min(h, h - dy)
    xs0, xs1 = max(0, -dx), min(w, w - dx)
    if ys0 < ys1 and xs0 < xs1:
        out[ys0:ys1, xs0:xs1] = S[ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
    return out


def dilate_union(S: np.ndarray, r: int) -> np.ndarray:
    """delta_r(S): union of the balls B_r(x), x in S, kept inside the box."""
    S = S != 0
    out = np.zeros_like(S)
    for dy, dx in disc_offsets(r):
        out |= _shift(S, dy, dx, False)
    return out.astype(np.uint8)


def erode_union(S: np.ndarray, r: int) -> np.ndarray:
    """eps_r(S): points whose whole ball B_r lies in S (outside = background)."""
    S = S != 0
    out = np.ones_like(S)
    for dy, dx in disc_offsets(r):
        out &= _shift(S, dy, dx, False)
    return out.astype(np.uint8)


def opening(S, r):
    return dilate_union(erode_union(S, r), r)


def closing(S, r):
    return erode_union(dilate_union(S, r), r)


def is_simply_connected(S: np.ndarray, conn: int = 8) -> bool:
    """One n-component and a complement (outside included) that is one
    nbar-component."""
    return component_counts(S, conn) == (1, 1)
