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


# ---- Eq. 12 (the quintic) against values worked out by hand from the printed
# coefficients a = [-0.02, -0.31, 1.44, -1.11, 0.58, -0.16] ----

def test_quintic_hand_values():
    # theta = 1: every power is 1, so g = sum of the coefficients
    #   -0.02 - 0.31 + 1.44 - 1.11 + 0.58 - 0.16 = 0.42
    assert support.g_theta(1.0) == pytest.approx(0.42, abs=1e-12)
    # theta = 2 (outside the physical range, but it fixes the coefficient order):
    #   -0.02 - 0.31*2 + 1.44*4 - 1.11*8 + 0.58*16 - 0.16*32
    #   = -0.02 - 0.62 + 5.76 - 8.88 + 9.28 - 5.12 = 0.40
    assert support.g_theta(2.0) == pytest.approx(0.40, abs=1e-12)
    # theta = pi/2 = 1.5707963: powers 2.4674011, 3.8757846, 6.0880682, 9.5631152
    #   -0.02 - 0.4869469 + 3.5530576 - 4.3021209 + 3.5310796 - 1.5300984 = 0.7449710
    assert support.g_theta(np.pi / 2) == pytest.approx(0.7449710, abs=2e-7)
    # just above theta = pi/4 = 0.7853982: powers 0.6168503, 0.4844730, 0.3805042, 0.2988479
    #   -0.02 - 0.2434734 + 0.8882644 - 0.5377650 + 0.2206924 - 0.0478157 = 0.2599027
    assert support.g_theta(np.pi / 4 + 1e-12) == pytest.approx(0.2599027, abs=2e-7)
    # at and below alpha the strut is self-supported
    assert support.g_theta(np.pi / 4) == 0.0 and support.g_theta(0.3) == 0.0


# ---- Appendix II (the exact ratio) ----

def _risky_share_brute(theta, alpha, n=400001):
    """The risky share measured from the geometry alone: the unit bottom circle
    rotated about x by theta, p(phi) = (cos phi, sin phi cos theta, sin phi
    sin theta), its normal n = p, printing direction z; over the facing-down
    half (n_z < 0), the projected (x, y) polyline length where n_z < -sin(alpha)
    against the whole half's length (segments classified at their midpoints,
    so each end of the arc is placed within half a segment: about 8e-6 of the
    share at this n)."""
    phi = np.linspace(np.pi, 2 * np.pi, n)
    x, y = np.cos(phi), np.sin(phi) * np.cos(theta)
    seg = np.hypot(np.diff(x), np.diff(y))
    mid = 0.5 * (phi[1:] + phi[:-1])
    risky = np.sin(mid) * np.sin(theta) < -np.sin(alpha)
    return seg[risky].sum() / seg.sum()


@pytest.mark.parametrize("alpha", [np.pi / 4, np.pi / 6, np.pi / 3])
@pytest.mark.parametrize("theta", [0.9, 1.0, 1.2, 1.4, np.pi / 2 - 0.01])
def test_exact_ratio_matches_brute_force(theta, alpha):
    if np.sin(theta) <= np.sin(alpha):
        assert support.g_exact(theta, alpha) == 0.0
        return
    assert support.g_exact(theta, alpha) == pytest.approx(_risky_share_brute(theta, alpha),
                                                          abs=2e-5)


def test_exact_ratio_closed_forms():
    # theta = pi/2: the ellipse degenerates to the x axis, the element is
    # |sin phi|, and the share is cos(phi0) = cos(alpha)
    for alpha in (np.pi / 4, np.pi / 6, np.pi / 3):
        assert support.g_exact(np.pi / 2, alpha) == pytest.approx(np.cos(alpha), abs=1e-12)
    # alpha = 0: the whole facing-down half needs support
    for theta in (0.3, 1.0, np.pi / 2):
        assert support.g_exact(theta, 0.0) == pytest.approx(1.0, abs=1e-12)
    # self-supported at and below alpha, and continuous there (no jump)
    assert support.g_exact(np.pi / 4) == 0.0 and support.g_exact(0.5) == 0.0
    assert support.g_exact(np.pi / 4 + 1e-9) < 1e-3
    # monotone in theta
    th = np.linspace(np.pi / 4 + 1e-3, np.pi / 2, 40)
    assert np.all(np.diff(support.g_exact(th)) > 0)


def test_quintic_departs_from_the_exact_ratio():
    """Eq. 12 approximates Appendix II well away from alpha (within 0.04 for
    theta >= 0.9) but starts at 0.26 where the exact ratio starts at 0."""
    th = np.linspace(0.9, np.pi / 2, 30)
    assert np.max(np.abs(support.g_theta(th) - support.g_exact(th))) < 0.04
    near = np.pi / 4 + 1e-6
    assert support.g_theta(near) - support.g_exact(near) > 0.25


def test_metrics_with_the_exact_ratio():
    nodes = np.array([[0, 0, 0], [3, 0, 0]], np.float32)
    g, p = support.support_metrics(nodes, np.array([[0, 1]]), [0.3], g="exact")
    assert g == pytest.approx(np.cos(np.pi / 4), abs=1e-12) and p == 0.0
