"""Pins of the vertex position optimisation oracle (Sec. 5.3.2, Eq. 16-17):
the gradient against finite differences, g against the pinned Eq. 12 code,
symmetry, the colouring, and the invariants a valid optimisation keeps."""
import math

import numpy as np
import pytest

import synth
from oracle import support as S
from oracle import support_opt as P

A = S.PAPER_A
T = np.array([0.0, 0.0, 1.0])


def test_g_matches_eq12_and_its_derivative():
    for th in np.linspace(0.8, 1.55, 16):
        g, dg = P.g_and_dg(th, math.pi / 4, A)
        assert abs(g - S.g_theta(th)) <= 1e-14
        h = 1e-6
        num = (P.g_and_dg(th + h, math.pi / 4, A)[0] - P.g_and_dg(th - h, math.pi / 4, A)[0]) / (2 * h)
        assert abs(dg - num) <= 1e-7
    assert P.g_and_dg(0.5, math.pi / 4, A) == (0.0, 0.0)


def test_gradient_of_J_against_central_differences():
    r = synth.rng(21)
    for _ in range(30):
        v = r.uniform(-0.2, 0.2, 3)
        others = [r.uniform(-1, 1, 3) for _ in range(7)]
        radii = r.uniform(0.1, 0.4, 7)
        J, grad = P.local_J(v, others, radii, T, math.pi / 4, A)
        # skip stars with an edge within reach of the kink at alpha
        h = 1e-6
        kink = False
        for w in others:
            d = v - w
            th = math.acos(min(abs(d @ T) / np.linalg.norm(d), 1.0))
            kink |= abs(th - math.pi / 4) < 1e-3
        if kink:
            continue
        num = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            num[k] = (P.local_J(v + e, others, radii, T, math.pi / 4, A)[0]
                      - P.local_J(v - e, others, radii, T, math.pi / 4, A)[0]) / (2 * h)
        assert np.abs(grad - num).max() <= 1e-6 * max(1.0, np.abs(num).max())


def test_symmetric_star_climbs_to_its_ball():
    """An octahedral star around the printing axis: its four horizontal edges
    sit at the cusp theta = pi/2, where the derivative of |cos| takes its +
    side, so the centre climbs along +z (x, y stay 0 by symmetry): first by
    step x tau0, tau0 = 1/sqrt(3) (its distance to the faces x + y + z = 1),
    then by halved steps up to the ball of radius ball x tau0, which no
    further step may leave (readings P2, P3)."""
    nodes = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1],
                      [0, 0, -1]], np.float32)
    tets = []
    for xs in (1, 2):
        for ys in (3, 4):
            for zs in (5, 6):
                tets.append([0, xs, ys, zs])
    tau0 = 1.0 / math.sqrt(3.0)
    res = P.optimize(nodes, np.array(tets), step=0.25, ball=0.5, max_rounds=1)
    assert abs(res["nodes"][0, 2] - 0.25 * tau0) <= 1e-15
    res = P.optimize(nodes, np.array(tets), step=0.25, ball=0.5, max_rounds=50)
    z = res["nodes"][0, 2]
    assert res["nodes"][0, 0] == 0.0 and res["nodes"][0, 1] == 0.0
    assert 0.5 * tau0 * (1 - 2.0 ** -8) <= z <= 0.5 * tau0
    assert res["moves"][:2] == [1, 1] and res["moves"][-1] == 0
    assert np.array_equal(res["nodes"][1:], nodes[1:].astype(np.float64))


@pytest.fixture(scope="module")
def mesh():
    nodes, tets = synth.kuhn_tet_mesh((3, 3, 3), 4.0, 0.15, seed=synth.SEED_BASE + 7)
    return nodes, tets


def _orient(x, t):
    a, b, c, d = (x[i] for i in t)
    return float(np.dot(b - a, np.cross(c - a, d - a)))


def test_colouring_is_proper_and_greedy(mesh):
    nodes, tets = mesh
    edges = P.mesh_edges(tets)
    col = P.greedy_colours(edges, nodes.shape[0])
    for a, b in edges:
        assert col[a] != col[b]
    # greedy: every colour below a vertex's is used by an earlier neighbour
    nbr = [set() for _ in range(nodes.shape[0])]
    for a, b in edges:
        nbr[a].add(b)
        nbr[b].add(a)
    for v in range(nodes.shape[0]):
        earlier = {col[w] for w in nbr[v] if w < v}
        assert all(c in earlier for c in range(col[v]))


def test_optimisation_keeps_the_mesh_valid_and_lowers_gamma(mesh):
    nodes, tets = mesh
    res = P.optimize(nodes, tets, max_rounds=20)
    x0 = nodes.astype(np.float64)
    x1 = res["nodes"]
    # boundary vertices stay; every tetrahedron keeps its orientation
    assert np.array_equal(x1[res["fixed"]], x0[res["fixed"]])
    assert res["fixed"].sum() == 4 ** 3 - 2 ** 3
    for t in tets:
        assert _orient(x0, t) * _orient(x1, t) > 0
    assert res["moves"][0] > 0 and res["rounds"] >= 2
    # the paper's metrics improve (Eq. 13-14)
    edges = res["edges"]
    rad = np.full(edges.shape[0], 0.2, np.float32)
    g0, p0 = S.support_metrics(x0, edges, rad)
    g1, p1 = S.support_metrics(x1, edges, rad)
    assert g1 < g0 and p1 > p0
    # every vertex's J is no larger than before (moves only accepted on decrease,
    # and a vertex's J depends on its own position and its neighbours')
    assert np.all(np.isfinite(x1))
