"""Topology-preserving smoothing of marching-squares contours (the paper
smooths its marching-squares boundaries, without creating intersections,
before it writes tool paths, Sec. 4; the method it cites is not restated
there, so this operator is our own, written from the grid structure of
marching squares).

TEST INFRASTRUCTURE ONLY: used by the tests, never by the product package.

Every contour vertex lies on a grid edge e of the padded sample grid (width
W = nx + 2): horizontal edge 2 (J W + I) from sample (I, J) to (I + 1, J),
vertical edge 2 (J W + I) + 1 from (I, J) to (I, J + 1); padded sample (I, J)
sits at (x0 + (I - 1/2) px, y0 + (J - 1/2) px). A vertex moves only along its
own edge:
  M1 K Jacobi iterations. In each, from the positions of the previous one
     (float32), the vertex's free coordinate a (x on a horizontal edge, y on a
     vertical one) becomes a + lam (m - a) with m = (a_p + a_s) / 2, a_p and
     a_s the same coordinate of its loop predecessor and successor, clamped to
     [lo + mu px, lo + (1 - mu) px], lo the coordinate of the edge's first
     sample. The arithmetic is float32, every operation rounded on its own
     (no fused multiply-add), in this order: m = 0.5 (a_p + a_s); a + lam (m
     - a); lo = c0 + I px (I or J the sample's column or row, c0 = x0 - px / 2
     or y0 - px / 2, and lam, mu px, (1 - mu) px rounded once from FP64);
     the bounds lo + mu px and lo + (1 - mu) px. The other coordinate is never
     changed.
  M2 loops of fewer than 3 vertices are left as they are.
Why no crossing can appear: each segment joins two vertices on two edges of
one cell (after the simplification of oracle/simplify.py, of the convex 1 x 2
block of a dropped vertex), and every vertex stays strictly inside its edge,
so the segment stays inside that cell (block); the two segments of a saddle
cell each cut off one corner and lie strictly on the two sides of the
diagonal through the other two corners. With mu = 1/2 every vertex sits at
its edge's midpoint: the marching squares of a binary image, as the paper
traces it.
"""
from __future__ import annotations

import numpy as np


def edge_axis_and_lo(eid: int, W: int, x0: float, y0: float, px: float):
    """(axis, lo) of grid edge eid: axis 0 (x free) for a horizontal edge,
    1 (y free) for a vertical one; lo = the free coordinate of its first
    sample, x0 + (I - 1/2) px or y0 + (J - 1/2) px, in FP64."""
    base, vert = divmod(int(eid), 2)
    J, I = divmod(base, W)
    if vert:
        return 1, y0 + (float(J) - 0.5) * px
    return 0, x0 + (float(I) - 0.5) * px


def edge_axis_and_lo32(eid: int, W: int, x0: float, y0: float, px: float):
    """(axis, lo) as edge_axis_and_lo, with lo in float32: c0 + I px (or
    c0 + J px), c0 = x0 - px / 2 (or y0 - px / 2) rounded from FP64, the
    product and the sum each rounded to float32 (M1)."""
    base, vert = divmod(int(eid), 2)
    J, I = divmod(base, W)
    f = np.float32
    if vert:
        return 1, f(f(y0 - 0.5 * px) + f(f(J) * f(px)))
    return 0, f(f(x0 - 0.5 * px) + f(f(I) * f(px)))


def smooth_loops(loop_off, edge_id, xy, *, x0: float, y0: float, pixel: float, nx: int,
                 lam: float, margin: float, iterations: int):
    """All loops of one contour set (loop_off[n_loops + 1] into edge_id / xy);
    returns the smoothed positions (float32 [n, 2]); edge ids and offsets are
    unchanged."""
    f = np.float32
    W = int(nx) + 2
    cur = np.asarray(xy, dtype=np.float32).copy()
    n_all = cur.shape[0]
    axis = np.zeros(n_all, dtype=np.int64)
    lo_v = np.zeros(n_all, dtype=np.float32)
    for v in range(n_all):
        axis[v], lo_v[v] = edge_axis_and_lo32(int(edge_id[v]), W, float(x0), float(y0),
                                              float(pixel))
    px = float(pixel)
    lam32, m_lo, m_hi = f(lam), f(margin * px), f((1.0 - margin) * px)
    half = f(0.5)
    for _ in range(int(iterations)):
        nxt = cur.copy()
        for L in range(len(loop_off) - 1):
            a, b = int(loop_off[L]), int(loop_off[L + 1])
            n = b - a
            if n < 3:
                continue
            for q in range(n):
                v = a + q
                p = a + (q - 1) % n
                s = a + (q + 1) % n
                k = int(axis[v])
                av = cur[v, k]
                m = half * f(cur[p, k] + cur[s, k])
                an = f(av + f(lam32 * f(m - av)))
                lo = lo_v[v]
                an = min(max(an, f(lo + m_lo)), f(lo + m_hi))
                nxt[v, k] = an
        cur = nxt
    return cur
