"""Gauss-Lobatto-Legendre (GLL) nodes, weights and derivative matrix.

Sec. 5.1: each hexahedron is mapped to [-1, 1]^3 and the solution is stored at
the tensor-product grid of GLL nodes of degree N (called ``p`` here), with
Np = (p+1)^3 nodes per element.  Standard textbook definitions are used:

* nodes: -1, the p-1 roots of P_p'(x), +1  (P_p the Legendre polynomial);
* weights: w_i = 2 / (p (p+1) P_p(x_i)^2);
* derivative matrix D_ij = l_j'(x_i) for the Lagrange basis l_j on the nodes.
"""
import numpy as np
from numpy.polynomial import legendre as L


def legendre_p(n, x):
    """P_n(x) by numpy's Legendre series evaluation (library primitive)."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    return L.legval(x, c)


def gll_nodes_weights(p):
    """GLL nodes (ascending) and quadrature weights for degree p >= 1."""
    if p < 1:
        raise ValueError("p must be >= 1")
    c = np.zeros(p + 1)
    c[p] = 1.0
    interior = np.sort(np.real(L.legroots(L.legder(c)))) if p >= 2 else np.empty(0)
    x = np.concatenate(([-1.0], interior, [1.0]))
    w = 2.0 / (p * (p + 1) * legendre_p(p, x) ** 2)
    return x, w


def gll_derivative(p):
    """D_ij = l_j'(x_i), the nodal differentiation matrix on the GLL nodes.

    Closed form for GLL points: D_ij = P_p(x_i) / (P_p(x_j) (x_i - x_j)) for
    i != j, D_00 = -p(p+1)/4, D_pp = +p(p+1)/4, other diagonal entries 0.
    """
    x, _ = gll_nodes_weights(p)
    P = legendre_p(p, x)
    n = p + 1
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = P[i] / (P[j] * (x[i] - x[j]))
    D[0, 0] = -p * (p + 1) / 4.0
    D[p, p] = p * (p + 1) / 4.0
    return D
