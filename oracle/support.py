"""Self-support metrics of a lattice (Sec. 5.3, Eq. 11-14), evaluated plainly
in float64. TEST INFRASTRUCTURE ONLY (tests, never the product).

theta_j = arccos |u_j . t_P| (Eq. 11); edges with theta_j <= alpha are fully
self-supported; g(theta) = sum_i a_i theta^i for theta > alpha, else 0
(Eq. 12, a = the paper's quintic for alpha = pi/4); Gamma = sum over the
unsupported edges of r L g / sum of r L (Eq. 13); Psi = 100 x sum over the
supported edges of L / sum of L (Eq. 14)."""
from __future__ import annotations

import numpy as np

PAPER_A = (-0.02, -0.31, 1.44, -1.11, 0.58, -0.16)


def g_theta(theta, alpha=np.pi / 4, a=PAPER_A):
    theta = np.asarray(theta, dtype=np.float64)
    poly = sum(a[i] * theta ** i for i in range(6))
    return np.where(theta > alpha, poly, 0.0)


def support_metrics(nodes, edges, radius, t_p=(0.0, 0.0, 1.0), alpha=np.pi / 4, a=PAPER_A):
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
    gamma = np.sum((r * L * g_theta(theta, alpha, a))[~supported]) / np.sum(r * L)
    psi = 100.0 * np.sum(L[supported]) / np.sum(L)
    return float(gamma), float(psi)
