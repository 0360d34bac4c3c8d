"""Pins of the zigzag-infill reference against closed forms (no GPU)."""
import numpy as np
import pytest

from oracle import hatch


def test_square_segments_and_zigzag_order():
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)   # counter-clockwise
    seg = hatch.hatch_layer([sq], y0=0.05, spacing=0.1, n_lines=10)
    assert seg.shape == (10, 3)
    ys = hatch.line_ys(0.05, 0.1, 10).astype(np.float64)
    assert np.array_equal(seg[:, 2], ys)
    for m in range(10):
        a, b = (0.0, 1.0) if m % 2 == 0 else (1.0, 0.0)
        assert seg[m, 0] == pytest.approx(a, abs=1e-12) and seg[m, 1] == pytest.approx(b, abs=1e-12)


def test_annulus_two_segments_through_the_hole():
    outer = np.array([[0, 0], [4, 0], [4, 4], [0, 4]], np.float32)
    inner = np.array([[1, 1], [1, 3], [3, 3], [3, 1]], np.float32)   # clockwise hole
    seg = hatch.hatch_layer([outer, inner], y0=0.5, spacing=1.0, n_lines=4)
    # lines y = 0.5, 1.5, 2.5, 3.5
    expect = [(0, 4, 0.5), (4, 3, 1.5), (1, 0, 1.5), (0, 1, 2.5), (3, 4, 2.5), (4, 0, 3.5)]
    assert np.allclose(seg, np.array(expect, np.float64))


def test_vertex_on_a_line_counts_once():
    """Half-open rule: a vertex on the line belongs to the edge that leaves upwards."""
    tri = np.array([[0, 0], [2, 1], [0, 2]], np.float32)
    seg = hatch.hatch_layer([tri], y0=1.0, spacing=1.0, n_lines=1)
    assert np.allclose(seg, [[0.0, 2.0, 1.0]])
    # a horizontal edge on the line adds nothing
    rect = np.array([[0, 1], [3, 1], [3, 2], [0, 2]], np.float32)
    seg = hatch.hatch_layer([rect], y0=1.0, spacing=1.0, n_lines=1)
    assert np.allclose(seg, [[0.0, 3.0, 1.0]])


def test_polygon_circle_chords():
    """Chords of a regular 720-gon of radius 5 match 2 sqrt(r^2 - y^2) within the
    polygon's sagitta."""
    th = np.linspace(0, 2 * np.pi, 720, endpoint=False)
    circ = np.stack([5 * np.cos(th), 5 * np.sin(th)], 1).astype(np.float32)
    seg = hatch.hatch_layer([circ], y0=-4.95, spacing=0.1, n_lines=100)
    assert len(seg) == 100
    chord = np.abs(seg[:, 1] - seg[:, 0])
    exact = 2 * np.sqrt(25 - seg[:, 2] ** 2)
    sagitta = 5 * (1 - np.cos(np.pi / 720))
    assert np.all(exact - chord <= 2 * sagitta / np.sqrt(np.maximum(1 - (seg[:, 2] / 5) ** 2, 1e-3)) + 1e-5)
    assert np.all(chord <= exact + 1e-5)


def test_no_loops_no_segments():
    seg = hatch.hatch_layer([], 0.5, 1.0, 3)
    assert seg.shape == (0, 3)
    off, seg = hatch.hatch_contours(np.array([0, 0, 0]), np.array([0]), np.zeros((0, 2), np.float32),
                                    0.5, 1.0, 3)
    assert list(off) == [0, 0, 0] and seg.shape == (0, 3)
