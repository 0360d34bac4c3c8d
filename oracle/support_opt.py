"""Vertex position optimisation for self-support (Sec. 5.3.2, Eq. 16-17).

TEST INFRASTRUCTURE ONLY: used by the tests and bench.py's CPU legs, never by
the product package. Plain Python/numpy in double precision.

Each interior vertex v of a tetrahedral mesh is moved to lower
  J(v) = sum_{e at v} r_e L_e g(theta_e) / sum_{e at v} r_e L_e      (Eq. 16)
with theta_e = arccos |u_e . t_P| (Eq. 11) and g the risky fraction of Eq. 12
(0 for theta <= alpha), within the inscribed sphere of the polyhedron its
neighbours form (Eq. 17). Readings of what the paper leaves open:
  P1 order: the paper visits the interior vertices one by one in random order;
     here a greedy colouring (vertices in index order, each takes the smallest
     colour unused by its neighbours) fixes the order: colour by colour,
     vertices by index. Vertices of one colour share no edge, so a colour's
     moves are independent of one another.
  P2 the sphere of Eq. 17 is the inscribed sphere of the vertex's star in the
     mesh as given: centre o = its initial position, radius ball * tau0, tau0
     the smallest distance from o to the faces opposite it in its tetrahedra.
     So that no tetrahedron flips however the neighbours move, a position is
     also rejected when an incident tetrahedron would change orientation or
     keep less than min_volume of its initial volume.
  P3 a move goes along -grad J (the analytic gradient of Eq. 16 where g is
     smooth; at |u . t_P| = 0 the derivative of |cos| takes its + side) by
     step * tau0, halved up to `backtracks` times until the position is
     allowed and J decreases; a vertex with a zero gradient stays.
  P4 rounds repeat until no vertex moves or `max_rounds` rounds have run.
  P5 boundary vertices (on a face that belongs to one tetrahedron) stay.
"""
from __future__ import annotations

import math

import numpy as np

from .support import PAPER_A

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))   # face opposite vertex k


def g_and_dg(theta: float, alpha: float, a) -> tuple[float, float]:
    """g(theta) of Eq. 12 and its derivative (0 for theta <= alpha)."""
    if theta <= alpha:
        return 0.0, 0.0
    g = 0.0
    dg = 0.0
    for i in range(len(a) - 1, -1, -1):     # Horner
        dg = dg * theta + g
        g = g * theta + a[i]
    return g, dg


def mesh_edges(tets):
    keys = set()
    for t in np.asarray(tets, dtype=np.int64):
        for p, q in LOCAL_EDGES:
            a, b = int(t[p]), int(t[q])
            keys.add((min(a, b), max(a, b)))
    return np.array(sorted(keys), dtype=np.int64).reshape(-1, 2)


def boundary_vertices(tets, n_nodes: int) -> np.ndarray:
    count = {}
    for t in np.asarray(tets, dtype=np.int64):
        for f in FACES:
            key = tuple(sorted(int(t[k]) for k in f))
            count[key] = count.get(key, 0) + 1
    on = np.zeros(n_nodes, dtype=bool)
    for key, c in count.items():
        if c == 1:
            on[list(key)] = True
    return on


def greedy_colours(edges, n_nodes: int) -> np.ndarray:
    nbr = [[] for _ in range(n_nodes)]
    for a, b in edges:
        nbr[a].append(b)
        nbr[b].append(a)
    col = np.full(n_nodes, -1, dtype=np.int64)
    for v in range(n_nodes):
        used = {int(col[w]) for w in nbr[v] if col[w] >= 0}
        c = 0
        while c in used:
            c += 1
        col[v] = c
    return col


def local_J(v, others, radii, t, alpha, a):
    """J(v) of Eq. 16 and its gradient for a vertex at v with edges to
    `others` (scalar double arithmetic, one fixed order)."""
    N = 0.0
    D = 0.0
    dN = [0.0, 0.0, 0.0]
    dD = [0.0, 0.0, 0.0]
    vx, vy, vz = float(v[0]), float(v[1]), float(v[2])
    tx, ty, tz = float(t[0]), float(t[1]), float(t[2])
    for w, r in zip(others, radii):
        r = float(r)
        d = (vx - float(w[0]), vy - float(w[1]), vz - float(w[2]))
        L = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
        if L == 0.0:
            continue
        s = d[0] * tx + d[1] * ty + d[2] * tz
        c = min(abs(s) / L, 1.0)
        theta = math.acos(c)
        g, dg = g_and_dg(theta, alpha, a)
        dL = (d[0] / L, d[1] / L, d[2] / L)
        N += r * L * g
        D += r * L
        for k in range(3):
            dD[k] += r * dL[k]
        if g != 0.0 or dg != 0.0:
            sg = math.copysign(1.0, s)
            s2 = math.sqrt(max(1.0 - c * c, 1e-300))
            tk = (tx, ty, tz)
            for k in range(3):
                dc = (sg * tk[k] - c * dL[k]) / L      # d|cos| / dv
                dtheta = -dc / s2
                dN[k] += r * (dL[k] * g + L * dg * dtheta)
    if D == 0.0:
        return 0.0, np.zeros(3)
    grad = np.array([(dN[k] * D - N * dD[k]) / (D * D) for k in range(3)])
    return N / D, grad


def orient(a, b, c, d) -> float:
    """Six times the signed volume of (a, b, c, d) (scalar double arithmetic)."""
    ax = float(b[0]) - float(a[0])
    ay = float(b[1]) - float(a[1])
    az = float(b[2]) - float(a[2])
    bx = float(c[0]) - float(a[0])
    by = float(c[1]) - float(a[1])
    bz = float(c[2]) - float(a[2])
    cx = float(d[0]) - float(a[0])
    cy = float(d[1]) - float(a[1])
    cz = float(d[2]) - float(a[2])
    return ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx)


def plane_distance(p, a, b, c) -> float:
    """Distance from p to the plane through a, b, c (scalar double arithmetic)."""
    ux, uy, uz = float(b[0]) - float(a[0]), float(b[1]) - float(a[1]), float(b[2]) - float(a[2])
    wx, wy, wz = float(c[0]) - float(a[0]), float(c[1]) - float(a[1]), float(c[2]) - float(a[2])
    nx = uy * wz - uz * wy
    ny = uz * wx - ux * wz
    nz = ux * wy - uy * wx
    nn = math.sqrt(nx * nx + ny * ny + nz * nz)
    if nn == 0.0:
        return 0.0
    px, py, pz = float(p[0]) - float(a[0]), float(p[1]) - float(a[1]), float(p[2]) - float(a[2])
    return abs(px * nx + py * ny + pz * nz) / nn


class Star:
    """The per-vertex data of the optimisation on the mesh as given: incident
    edges (in edge order) with radii, incident tetrahedra, boundary flags,
    colours, the initial positions o, tau0 and the tetrahedra's volumes."""

    def __init__(self, nodes, tets, radius=None, *, t_p=(0.0, 0.0, 1.0), alpha=math.pi / 4,
                 a=PAPER_A, step=0.25, ball=0.5, min_volume=0.1, backtracks=8):
        x = np.asarray(nodes, dtype=np.float32).astype(np.float64).copy()
        self.tets = np.asarray(tets, dtype=np.int64).reshape(-1, 4)
        n = x.shape[0]
        self.edges = mesh_edges(self.tets)
        r = (np.ones(self.edges.shape[0]) if radius is None
             else np.asarray(radius, np.float32).astype(np.float64))
        t0 = [float(v) for v in t_p]
        tn = math.sqrt(t0[0] * t0[0] + t0[1] * t0[1] + t0[2] * t0[2])
        self.t = (t0[0] / tn, t0[1] / tn, t0[2] / tn)
        self.alpha, self.a = alpha, a
        self.step, self.ball, self.min_volume, self.backtracks = step, ball, min_volume, backtracks
        self.inc = [[] for _ in range(n)]          # (other vertex, radius)
        for (p, q), rr in zip(self.edges, r):
            self.inc[p].append((int(q), rr))
            self.inc[q].append((int(p), rr))
        self.vt = [[] for _ in range(n)]           # (tetrahedron, local index)
        for ti, tt in enumerate(self.tets):
            for k in range(4):
                self.vt[int(tt[k])].append((ti, k))
        self.fixed = boundary_vertices(self.tets, n)
        self.colours = greedy_colours(self.edges, n)
        self.order = [v for c in range(int(self.colours.max()) + 1 if n else 0) for v in range(n)
                      if self.colours[v] == c and not self.fixed[v]]
        self.vol0 = [orient(*(x[int(i)] for i in tt)) for tt in self.tets]
        self.o = x
        self.tau0 = np.zeros(n)
        for v in self.order:
            self.tau0[v] = min(plane_distance(x[v], *(x[self.tets[ti][k2]] for k2 in FACES[k]))
                               for ti, k in self.vt[v])

    def allowed(self, v, p, x):
        o = self.o[v]
        dx, dy, dz = p[0] - o[0], p[1] - o[1], p[2] - o[2]
        if math.sqrt(dx * dx + dy * dy + dz * dz) > self.ball * self.tau0[v]:
            return False
        for ti, k in self.vt[v]:
            q = [p if j == k else x[int(self.tets[ti][j])] for j in range(4)]
            vol = orient(*q)
            if not (vol * self.vol0[ti] > 0.0 and abs(vol) >= self.min_volume * abs(self.vol0[ti])):
                return False
        return True

    def move(self, v, x):
        """The new position of vertex v given the positions x, or None."""
        others = [x[w] for w, _ in self.inc[v]]
        radii = [rr for _, rr in self.inc[v]]
        J0, grad = local_J(x[v], others, radii, self.t, self.alpha, self.a)
        gn = math.sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2])
        if gn == 0.0:
            return None
        u = [grad[k] / gn for k in range(3)]
        s = self.step * self.tau0[v]
        for _ in range(self.backtracks + 1):
            cand = np.array([x[v][k] - s * u[k] for k in range(3)])
            if self.allowed(v, cand, x):
                J1, _ = local_J(cand, others, radii, self.t, self.alpha, self.a)
                if J1 < J0:
                    return cand
            s *= 0.5
        return None


def optimize(nodes, tets, radius=None, *, t_p=(0.0, 0.0, 1.0), alpha=math.pi / 4, a=PAPER_A,
             step=0.25, ball=0.5, min_volume=0.1, backtracks=8, max_rounds=100):
    """Returns dict(nodes float64 [N, 3], rounds, moves per round, colours, fixed, edges)."""
    st = Star(nodes, tets, radius, t_p=t_p, alpha=alpha, a=a, step=step, ball=ball,
              min_volume=min_volume, backtracks=backtracks)
    x = st.o.copy()
    moves = []
    for _ in range(max_rounds):
        moved = 0
        for v in st.order:
            p = st.move(v, x)
            if p is not None:
                x[v] = p
                moved += 1
        moves.append(moved)
        if moved == 0:
            break
    return dict(nodes=x, rounds=len(moves), moves=moves, colours=st.colours, fixed=st.fixed,
                edges=st.edges)
