"""Zigzag infill of layer contours (Sec. 6: after the binary image and its
boundary contours, a zigzag toolpath fills the interior) -- the definition,
evaluated plainly. TEST INFRASTRUCTURE ONLY (tests, never the product).

Scan lines y_m = y0 + m * spacing (m < n_lines), computed in double and rounded
once to float32. An edge a -> b of a closed loop crosses line m when
min(a_y, b_y) <= y_m < max(a_y, b_y), compared in float32 (the precision in
which the GPU takes the same decision); the crossing abscissa is
x = a_x + t (b_x - a_x), t = (y_m - a_y) / (b_y - a_y), in float64. Along a
line the crossings sorted by x pair up into inside segments (even-odd rule).
The toolpath of a layer takes the lines in increasing m; on even lines the
segments in increasing x, each from low to high x; on odd lines in decreasing
x, each from high to low x."""
from __future__ import annotations

import numpy as np


def line_ys(y0: float, spacing: float, n_lines: int) -> np.ndarray:
    return np.array([y0 + m * spacing for m in range(n_lines)], dtype=np.float64).astype(np.float32)


def hatch_layer(loops, y0: float, spacing: float, n_lines: int):
    """loops: iterable of (n, 2) float32 vertex arrays, each a closed polygon.
    Returns an (n_segments, 3) float64 array of (x_from, x_to, y) in toolpath order."""
    ys = line_ys(y0, spacing, n_lines)
    per_line = [[] for _ in range(n_lines)]
    for P in loops:
        P = np.asarray(P, dtype=np.float32)
        if len(P) == 0:
            continue
        A, B = P, np.roll(P, -1, axis=0)
        lo = np.minimum(A[:, 1], B[:, 1])
        hi = np.maximum(A[:, 1], B[:, 1])
        m0 = np.searchsorted(ys, lo, side="left")   # first line with y >= lo
        m1 = np.searchsorted(ys, hi, side="left")   # first line with y >= hi
        for k in np.nonzero(m1 > m0)[0]:
            ax, ay = float(A[k, 0]), float(A[k, 1])
            bx, by = float(B[k, 0]), float(B[k, 1])
            for m in range(int(m0[k]), int(m1[k])):
                t = (float(ys[m]) - ay) / (by - ay)
                per_line[m].append(ax + t * (bx - ax))
    out = []
    for m in range(n_lines):
        xs = sorted(per_line[m])
        if len(xs) % 2:
            raise ValueError(f"line {m}: odd number of crossings (open contour)")
        pairs = [(xs[2 * i], xs[2 * i + 1]) for i in range(len(xs) // 2)]
        if m % 2:
            pairs = [(b, a) for a, b in reversed(pairs)]
        out += [(a, b, float(ys[m])) for a, b in pairs]
    return np.array(out, dtype=np.float64).reshape(-1, 3)


def hatch_contours(layer_loop_off, loop_vert_off, xy, y0, spacing, n_lines):
    """All layers of a contour set (offset arrays as csl_contours). Returns
    (layer_seg_off[n_layers + 1], seg[n_segments, 3])."""
    n_layers = len(layer_loop_off) - 1
    offs, segs = [0], []
    for k in range(n_layers):
        loops = [xy[loop_vert_off[li]:loop_vert_off[li + 1]]
                 for li in range(layer_loop_off[k], layer_loop_off[k + 1])]
        s = hatch_layer(loops, y0, spacing, n_lines)
        segs.append(s)
        offs.append(offs[-1] + len(s))
    seg = np.concatenate(segs) if segs else np.zeros((0, 3))
    return np.array(offs, dtype=np.int64), seg
