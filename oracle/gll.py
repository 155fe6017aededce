"""Gauss-Legendre-Lobatto nodal basis (remark "Basis functions, geometry and
numerical integration", Sec. 2.2).

The 1D basis of degree p is the Lagrange basis on the p+1 GLL points; the same
points give the collocation quadrature used for all volume and face integrals.

Pins (tests/test_oracle_gll.py): printed closed-form nodes/weights for p=1..4,
exactness of the quadrature up to degree 2p-1, exact differentiation of
polynomials of degree <= p.
"""
import numpy as np


def legendre(p, x):
    """P_p(x) and P_p'(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    P0, P1 = np.ones_like(x), x.copy()
    if p == 0:
        return P0, np.zeros_like(x)
    for n in range(2, p + 1):
        P0, P1 = P1, ((2 * n - 1) * x * P1 - (n - 1) * P0) / n
    # derivative from (1-x^2) P_p' = p (P_{p-1} - x P_p)
    with np.errstate(divide="ignore", invalid="ignore"):
        dP = p * (P0 - x * P1) / (1.0 - x * x)
    end = np.abs(x) == 1.0
    dP = np.where(end, 0.5 * p * (p + 1) * x ** (p + 1), dP)
    return P1, dP


def gll(p):
    """GLL nodes (ascending) and weights for degree p >= 1.

    Interior nodes are the roots of P_p'; weights w_i = 2 / (p (p+1) P_p(x_i)^2).
    """
    if p < 1:
        raise ValueError("p >= 1")
    x = -np.cos(np.pi * np.arange(p + 1) / p)  # Chebyshev-Lobatto start
    for _ in range(100):
        P, dP = legendre(p, x)
        # Newton on q(x) = (1 - x^2) P_p'(x) = p (P_{p-1} - x P_p), interior only
        Pm1 = legendre(p - 1, x)[0]
        q = p * (Pm1 - x * P)
        # q'(x) = -p (p+1) P_p(x)  (Legendre ODE)
        dq = -p * (p + 1) * P
        step = np.zeros_like(x)
        step[1:-1] = q[1:-1] / dq[1:-1]
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    x = 0.5 * (x - x[::-1])  # exact symmetry
    P, _ = legendre(p, x)
    w = 2.0 / (p * (p + 1) * P * P)
    return x, w


def lagrange_eval(nodes, x):
    """L[q, j] = l_j(x_q): Lagrange basis on `nodes` evaluated at points x."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_deriv_eval(nodes, x):
    """Ld[q, j] = l_j'(x_q), by the product rule applied to the product formula."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    Ld = np.zeros((len(x), n))
    for j in range(n):
        denom = 1.0
        for m in range(n):
            if m != j:
                denom *= nodes[j] - nodes[m]
        for k in range(n):
            if k == j:
                continue
            term = np.ones_like(x)
            for m in range(n):
                if m != j and m != k:
                    term *= x - nodes[m]
            Ld[:, j] += term
        Ld[:, j] /= denom
    return Ld


def diff_matrix(p):
    """D[i, j] = l_j'(xi_i) on the GLL nodes of degree p."""
    x, _ = gll(p)
    return lagrange_deriv_eval(x, x)


def interp_matrix(p_from, x_to):
    """Evaluate a degree-p_from GLL nodal polynomial at points x_to."""
    x, _ = gll(p_from)
    return lagrange_eval(x, x_to)
