"""Oracle pins for the GLL basis (remark of Sec. 2.2)."""
import os

import numpy as np
import pytest
from numpy import sqrt  # noqa: F401  (used by the golden expressions)

from oracle.gll import gll, diff_matrix, lagrange_eval

GOLD = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        p, xs, ws = line.split("|")
        rows.append((int(p), [eval(x) for x in xs.split(",")], [eval(w) for w in ws.split(",")]))
    return rows


@pytest.mark.parametrize("p,xs,ws", _golden())
def test_closed_form_nodes_weights(p, xs, ws):
    x, w = gll(p)
    np.testing.assert_allclose(x, xs, atol=1e-15)
    np.testing.assert_allclose(w, ws, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 12, 16])
def test_quadrature_exact_to_2p_minus_1(p):
    x, w = gll(p)
    for k in range(2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    # degree 2p is not integrated exactly (the collocation mass is lumped)
    assert abs(np.sum(w * x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-12


@pytest.mark.parametrize("p", [1, 2, 4, 7, 8, 10])
def test_derivative_exact_for_degree_p(p):
    x, _ = gll(p)
    D = diff_matrix(p)
    for k in range(p + 1):
        np.testing.assert_allclose(D @ x ** k, k * x ** max(k - 1, 0) * (k > 0), atol=1e-11)


def test_lagrange_cardinal():
    x, _ = gll(6)
    np.testing.assert_allclose(lagrange_eval(x, x), np.eye(7), atol=1e-14)
