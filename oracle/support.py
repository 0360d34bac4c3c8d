"""Self-support metrics of a lattice (Sec. 5.3, Eq. 11-14), evaluated plainly
in float64. TEST INFRASTRUCTURE ONLY (tests, never the product).

theta_j = arccos |u_j . t_P| (Eq. 11); edges with theta_j <= alpha are fully
self-supported; g(theta) = sum_i a_i theta^i for theta > alpha, else 0
(Eq. 12, a = the paper's quintic for alpha = pi/4); Gamma = sum over the
unsupported edges of r L g / sum of r L (Eq. 13); Psi = 100 x sum over the
supported edges of L / sum of L (Eq. 14).

g_exact is the ratio the quintic approximates (Appendix II): the share of the
projected bottom circle's arc length on which the surface normal n satisfies
n . t_P < -sin(alpha). Reading of the appendix: the circle of a strut tilted
by theta projects to the ellipse (cos phi, cos(theta) sin phi), whose arc
length element is sqrt(sin^2 phi + cos^2(theta) cos^2 phi), and the risky arc
is phi in [phi0, pi/2] of the quarter, phi0 = arcsin(sin(alpha)/sin(theta)).
The appendix prints sin^2(theta) in the element and integrates over
[0, phi0]; taken literally that ratio is 1 at theta = alpha (a jump from 0)
and 1/2 at theta = pi/2, while the quintic gives 0.26 and 0.745 and follows
this reading within 0.04 for theta >= 0.9. Pinned by a brute-force polyline
length of the risky arc computed from the geometric definition."""
from __future__ import annotations

import numpy as np

PAPER_A = (-0.02, -0.31, 1.44, -1.11, 0.58, -0.16)


def g_theta(theta, alpha=np.pi / 4, a=PAPER_A):
    theta = np.asarray(theta, dtype=np.float64)
    poly = sum(a[i] * theta ** i for i in range(6))
    return np.where(theta > alpha, poly, 0.0)


def g_exact(theta, alpha=np.pi / 4):
    """Appendix II: risky share of the projected ellipse's arc length; 0 when
    sin(theta) <= sin(alpha). Quadrature of the arc length element (scipy)."""
    from scipy.integrate import quad

    def one(th):
        st = np.sin(th)
        if st <= np.sin(alpha):
            return 0.0
        phi0 = np.arcsin(np.sin(alpha) / st)
        c2 = np.cos(th) ** 2

        def ds(phi):
            return np.sqrt(np.sin(phi) ** 2 + c2 * np.cos(phi) ** 2)

        risky = quad(ds, phi0, np.pi / 2, epsabs=0.0, epsrel=1e-13, limit=200)[0]
        total = quad(ds, 0.0, np.pi / 2, epsabs=0.0, epsrel=1e-13, limit=200)[0]
        return risky / total

    theta = np.asarray(theta, dtype=np.float64)
    return np.vectorize(one, otypes=[np.float64])(theta)


def support_metrics(nodes, edges, radius, t_p=(0.0, 0.0, 1.0), alpha=np.pi / 4, a=PAPER_A,
                    g="quintic"):
    """g = "quintic" (Eq. 12 with coefficients a) or "exact" (Appendix II)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    edges = np.asarray(edges)
    r = np.asarray(radius, dtype=np.float64)
    t = np.asarray(t_p, dtype=np.float64)
    t = t / np.linalg.norm(t)
    d = nodes[edges[:, 1]] - nodes[edges[:, 0]]
    L = np.linalg.norm(d, axis=1)
    cs = np.zeros_like(L)
    nz = L > 0
    cs[nz] = np.abs(d[nz] @ t) / L[nz]
    theta = np.arccos(np.minimum(cs, 1.0))
    supported = theta <= alpha
    gv = g_theta(theta, alpha, a) if g == "quintic" else g_exact(theta, alpha)
    gamma = np.sum((r * L * gv)[~supported]) / np.sum(r * L)
    psi = 100.0 * np.sum(L[supported]) / np.sum(L)
    return float(gamma), float(psi)
