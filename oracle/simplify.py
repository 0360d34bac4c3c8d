"""Topology-preserving simplification of marching-squares contours (the
paper smooths and simplifies its marching-squares boundaries without creating
intersections before writing tool paths, Sec. 4; the method it cites is not
restated there, so this is a rule of our own, written from the grid
structure of marching squares).

TEST INFRASTRUCTURE ONLY: used by the tests, never by the product package.

Every contour vertex lies on a grid edge e, and its loop runs from the cell on
one side of e into the cell on the other. A vertex v (loop position q, its
loop's first vertex being q = 0) is dropped when
  S1 q is odd and the loop has at least 5 vertices (its neighbours stay, and
     the loop keeps at least 3),
  S2 neither cell beside e is a saddle cell, i.e. no edge of either cell other
     than the loop's own two carries a crossing (a non-saddle cell holds only
     this loop's one segment, and the two cells form a convex 1 x 2 block,
     so the chord from v's predecessor to its successor stays inside that
     block and meets no other contour piece),
  S3 v lies within `tol` of the line through its predecessor and successor
     (which are not at the same point).
Loops and their order are unchanged; each keeps its first vertex.

Edge ids follow marching squares' padded grid of width W = nx + 2:
horizontal 2 (J W + I) between samples (I, J) and (I + 1, J), vertical + 1
between (I, J) and (I, J + 1).
"""
from __future__ import annotations

import math

import numpy as np


def edge_cells(eid: int, W: int):
    """The two cells (I, J) beside grid edge eid (a cell spans samples I..I+1,
    J..J+1)."""
    base, vert = divmod(int(eid), 2)
    J, I = divmod(base, W)
    if vert:
        return (I - 1, J), (I, J)
    return (I, J - 1), (I, J)


def cell_edges(I: int, J: int, W: int):
    """The four grid edges of cell (I, J): bottom, top, left, right."""
    return (2 * (J * W + I), 2 * ((J + 1) * W + I), 2 * (J * W + I) + 1,
            2 * (J * W + I + 1) + 1)


def simplify_layer(loop_off, edge_id, xy, nx: int, tol: float):
    """One layer's loops (loop_off[n_loops+1] into edge_id / xy). Returns the
    new (loop_off, edge_id, xy) and the kept mask."""
    W = int(nx) + 2
    present = set(int(e) for e in edge_id)
    keep = np.ones(len(edge_id), dtype=bool)
    for L in range(len(loop_off) - 1):
        a, b = int(loop_off[L]), int(loop_off[L + 1])
        n = b - a
        if n < 5:
            continue
        for q in range(1, n, 2):
            v = a + q
            p = a + q - 1
            nx_ = a + (q + 1) % n
            own = {int(edge_id[p]), int(edge_id[v]), int(edge_id[nx_])}
            saddle = False
            for cell in edge_cells(int(edge_id[v]), W):
                for e in cell_edges(cell[0], cell[1], W):
                    if e not in own and e in present:
                        saddle = True
            if saddle:
                continue
            px, py = float(xy[p][0]), float(xy[p][1])
            qx, qy = float(xy[nx_][0]), float(xy[nx_][1])
            vx, vy = float(xy[v][0]), float(xy[v][1])
            dx, dy = qx - px, qy - py
            L2 = dx * dx + dy * dy
            if L2 == 0.0:
                continue
            cross = (vx - px) * dy - (vy - py) * dx
            if abs(cross) <= tol * math.sqrt(L2):
                keep[v] = False
    new_off = [0]
    for L in range(len(loop_off) - 1):
        new_off.append(new_off[-1] + int(keep[int(loop_off[L]):int(loop_off[L + 1])].sum()))
    return (np.array(new_off, dtype=np.int64), np.asarray(edge_id)[keep],
            np.asarray(xy)[keep], keep)
