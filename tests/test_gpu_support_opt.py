"""Vertex re-positioning on the GPU (csl_support_optimize) against the FP64
oracle: the same moves round by round, the same positions, and the paper's
metrics before and after."""

import numpy as np
import pytest

import synth
from oracle import support as S
from oracle import support_opt as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _compare(nodes, tets, radius=None, **kw):
    import paper_2101_05031_gb300 as cs
    ref = P.optimize(nodes, tets, radius, **kw)
    got = cs.support_optimize(nodes, tets, radius, **kw)
    assert got["moves_per_round"] == ref["moves"]
    assert got["n_colours"] == int(ref["colours"].max()) + 1
    x = ref["nodes"]
    assert np.all(np.abs(got["nodes"].astype(np.float64) - x) <= 1e-6 * np.abs(x) + 1e-6)
    edges = ref["edges"]
    rad = np.ones(edges.shape[0]) if radius is None else np.asarray(radius, np.float32)
    t_p = kw.get("t_p", (0.0, 0.0, 1.0))
    g0, p0 = S.support_metrics(nodes.astype(np.float64), edges, rad, t_p=t_p)
    g1, p1 = S.support_metrics(x, edges, rad, t_p=t_p)
    assert abs(got["gamma_before"] - g0) <= 1e-12 and abs(got["psi_before"] - p0) <= 1e-10
    assert abs(got["gamma_after"] - g1) <= 1e-9 and abs(got["psi_after"] - p1) <= 1e-7
    return ref, got


def test_kuhn_mesh_matches_the_oracle():
    nodes, tets = synth.kuhn_tet_mesh((6, 6, 6), 4.0, 0.15, seed=synth.SEED_BASE + 7)
    ref, got = _compare(nodes, tets, max_rounds=100)
    assert got["rounds"] >= 3 and got["moves_per_round"][-1] == 0
    assert got["gamma_after"] < got["gamma_before"] and got["psi_after"] > got["psi_before"]


def test_radii_and_a_tilted_direction():
    nodes, tets = synth.kuhn_tet_mesh((4, 5, 3), 3.0, 0.12, seed=synth.SEED_BASE + 8)
    n_e = P.mesh_edges(tets).shape[0]
    radius = synth.rng(9).uniform(0.1, 0.4, n_e).astype(np.float32)
    t = (0.2, -0.1, 1.0)
    _compare(nodes, tets, radius, t_p=t, step=0.3, ball=0.4, max_rounds=30)


def test_symmetric_star_and_empty_mesh():
    import paper_2101_05031_gb300 as cs
    nodes = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1],
                      [0, 0, -1]], np.float32)
    tets = np.array([[0, xs, ys, zs] for xs in (1, 2) for ys in (3, 4) for zs in (5, 6)])
    _compare(nodes, tets, max_rounds=50)
    got = cs.support_optimize(np.zeros((0, 3), np.float32), np.zeros((0, 4), np.int32))
    assert got["rounds"] == 0 and got["nodes"].shape == (0, 3)


def _volumes(x, tets):
    a, b, c, d = (x[tets[:, k]] for k in range(4))
    return np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a)


def test_full_workload_first_round_sampled():
    """The bench's 50^3-cube mesh (750,000 tetrahedra), one round. A vertex of
    the first colour moves from the mesh as given, so 300 of them are
    recomputed by the oracle one by one from the synthetic input alone. For
    every vertex, without the oracle: boundary vertices unmoved, every move
    inside its inscribed-ball limit, and every tetrahedron's orientation kept
    with at least min_volume of its volume (its last vertex to move checked
    it against the others' final positions)."""
    import paper_2101_05031_gb300 as cs
    nodes, tets = synth.kuhn_tet_mesh((50, 50, 50), 2.0, 0.15, seed=synth.SEED_BASE + 7)
    got = cs.support_optimize(nodes, tets, max_rounds=1)
    st = P.Star(nodes, tets)
    x0 = nodes.astype(np.float64)
    x1 = got["nodes"].astype(np.float64)
    assert got["n_colours"] == int(st.colours.max()) + 1
    assert np.array_equal(x1[st.fixed], x0[st.fixed])
    first = [v for v in st.order if st.colours[v] == 0]
    r = synth.rng(23)
    n_moved = 0
    for v in r.choice(first, 300, replace=False):
        p = st.move(int(v), x0)
        ref = x0[v] if p is None else p
        assert np.all(np.abs(x1[v] - ref) <= 1e-5 * np.abs(ref) + 1e-5), v
        n_moved += p is not None
    assert n_moved > 250
    dist = np.linalg.norm(x1 - x0, axis=1)
    assert np.all(dist <= st.ball * st.tau0 * (1 + 1e-5) + 1e-6)
    assert np.count_nonzero(dist) > 0.5 * len(st.order)
    t = np.asarray(tets, dtype=np.int64).reshape(-1, 4)
    v0, v1 = _volumes(x0, t), _volumes(x1, t)
    assert np.all(v0 * v1 > 0.0)
    assert np.all(np.abs(v1) >= st.min_volume * np.abs(v0) * (1 - 1e-3))
