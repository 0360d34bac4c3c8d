"""Pins of the self-support metrics reference (no GPU)."""
import numpy as np
import pytest

from oracle import support
import synth


def test_single_struts_closed_forms():
    nodes = np.array([[0, 0, 0], [0, 0, 2], [3, 0, 0], [1, 1, 1]], np.float32)
    # vertical: supported, Gamma 0, Psi 100
    assert support.support_metrics(nodes, np.array([[0, 1]]), [0.3]) == (0.0, 100.0)
    # horizontal: theta = pi/2, Gamma = g(pi/2) = sum a_i (pi/2)^i, Psi 0
    g, p = support.support_metrics(nodes, np.array([[0, 2]]), [0.3])
    assert g == pytest.approx(sum(a * (np.pi / 2) ** i for i, a in enumerate(support.PAPER_A)))
    assert p == 0.0
    # body diagonal: theta = arccos(1/sqrt 3) > pi/4
    g, p = support.support_metrics(nodes, np.array([[0, 3]]), [0.3])
    th = np.arccos(1 / np.sqrt(3))
    assert g == pytest.approx(sum(a * th ** i for i, a in enumerate(support.PAPER_A))) and p == 0.0
    # 45 degrees: supported when alpha reaches theta (up to the rounding of arccos)
    n45 = np.array([[0, 0, 0], [1, 0, 1]], np.float64)
    assert support.support_metrics(n45, np.array([[0, 1]]), [0.3], alpha=np.pi / 4 + 1e-12) == (0.0, 100.0)
    g, p = support.support_metrics(n45, np.array([[0, 1]]), [0.3], alpha=np.pi / 4 - 1e-9)
    assert p == 0.0 and g == pytest.approx(support.g_theta(np.pi / 4, alpha=0.0))


def test_weighting_and_direction():
    """Gamma weights by r L, Psi by L; turning the printing direction swaps the roles."""
    nodes = np.array([[0, 0, 0], [0, 0, 1], [2, 0, 0]], np.float32)
    edges = np.array([[0, 1], [0, 2]])
    r = np.array([0.5, 0.25])
    g, p = support.support_metrics(nodes, edges, r)
    gh = support.g_theta(np.pi / 2)
    assert g == pytest.approx(0.25 * 2 * gh / (0.5 * 1 + 0.25 * 2))
    assert p == pytest.approx(100 * 1 / 3)
    g2, p2 = support.support_metrics(nodes, edges, r, t_p=(1, 0, 0))
    assert g2 == pytest.approx(0.5 * 1 * gh / (0.5 * 1 + 0.25 * 2))
    assert p2 == pytest.approx(100 * 2 / 3)


def test_cubic_bcc_lattice():
    """4^3 cubic+BCC cells along z: the vertical edges (80 of length 5) are the
    only supported ones; the 200 horizontal and 512 diagonal struts are not."""
    nodes, edges, radius = synth.cubic_bcc(4, 5.0, 0.5)
    g, p = support.support_metrics(nodes, edges, radius)
    d = nodes[edges[:, 1]] - nodes[edges[:, 0]]
    L = np.linalg.norm(d, axis=1)
    vert = np.abs(d[:, 2]) / L > 0.99
    assert p == pytest.approx(100 * L[vert].sum() / L.sum())
    th_h, th_d = np.pi / 2, np.arccos(1 / np.sqrt(3))
    horiz = np.abs(d[:, 2]) < 1e-6
    diag = ~vert & ~horiz
    num = (radius[horiz] * L[horiz]).sum() * support.g_theta(th_h) + \
        (radius[diag] * L[diag]).sum() * support.g_theta(th_d)
    assert g == pytest.approx(num / (radius * L).sum())
