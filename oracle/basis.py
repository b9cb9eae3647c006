"""Gauss-Lobatto-Legendre nodes and Lagrange basis on the reference interval [-1, 1].

Section 2.3 (FE discretization): the fields are expanded in C0-continuous piecewise
Lagrange polynomials of degree p interpolating on Gauss-Lobatto-Legendre (GLL) points.
The GLL points of degree p are -1, +1 and the p-1 roots of P_p'(xi); their quadrature
weights are 2 / (p (p+1) P_p(xi)^2).
"""
import numpy as np
from numpy.polynomial import legendre as leg


def gll(p):
    """GLL nodes (ascending) and weights for polynomial degree p >= 1."""
    if p < 1:
        raise ValueError("p must be >= 1")
    c = np.zeros(p + 1)
    c[p] = 1.0
    dc = leg.legder(c)
    if p >= 2:
        inner = np.sort(np.real(leg.legroots(dc)))
        # two Newton steps on P_p' to polish the companion-matrix roots
        ddc = leg.legder(dc)
        for _ in range(2):
            inner = inner - leg.legval(inner, dc) / leg.legval(inner, ddc)
        x = np.concatenate([[-1.0], inner, [1.0]])
    else:
        x = np.array([-1.0, 1.0])
    w = 2.0 / (p * (p + 1) * leg.legval(x, c) ** 2)
    return x, w


def lagrange_values(nodes, pts):
    """B[a, i] = l_i(pts[a]) for the Lagrange polynomials l_i on ``nodes``."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.atleast_1d(np.asarray(pts, dtype=np.float64))
    n = len(nodes)
    B = np.ones((len(pts), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                B[:, i] *= (pts - nodes[j]) / (nodes[i] - nodes[j])
    return B


def lagrange_derivs(nodes, pts):
    """D[a, i] = l_i'(pts[a]) by the product rule."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.atleast_1d(np.asarray(pts, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(pts), n))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.full(len(pts), 1.0 / (nodes[i] - nodes[k]))
            for j in range(n):
                if j != i and j != k:
                    term *= (pts - nodes[j]) / (nodes[i] - nodes[j])
            D[:, i] += term
    return D


def gauss_legendre(q):
    """Gauss-Legendre points and weights (exact for degree <= 2q-1)."""
    return leg.leggauss(q)
