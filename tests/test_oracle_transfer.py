"""Oracle pins for the transfer operators (Sec. 3.2)."""
import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from oracle import transfer
from oracle.geometry import node_geometry


def _pair(kind, p_c, p_f):
    V = wl.uniform_vertices(4)
    if kind == "p":
        levels = wl.hierarchy(V, [p_f, p_c])
    else:
        levels = wl.hierarchy(V, [p_f], h_root=2)
    return levels[0], levels[1]


@pytest.mark.parametrize("kind,pc,pf", [("p", 1, 2), ("p", 2, 4), ("p", 4, 8), ("p", 3, 7),
                                         ("h", 1, 1), ("h", 2, 2), ("h", 3, 3), ("h", 4, 4)])
def test_projection_inverts_interpolation(kind, pc, pf):
    lc, lf = _pair(kind, pc, pf)
    T = transfer.Transfer(lc, lf)
    uc = np.random.default_rng(0).standard_normal(lc["corners"].shape[0] * (pc + 1) ** 3)
    np.testing.assert_allclose(T.project(T.interpolate(uc)), uc, atol=1e-13)


@pytest.mark.parametrize("kind,pc,pf", [("p", 2, 4), ("p", 3, 7), ("h", 2, 2), ("h", 3, 3)])
def test_interpolation_reproduces_coarse_polynomials(kind, pc, pf):
    lc, lf = _pair(kind, pc, pf)
    T = transfer.Transfer(lc, lf)
    f = lambda X: X[..., 0] ** pc * X[..., 1] + X[..., 2] ** pc - X[..., 1] * X[..., 2]
    uc = f(node_geometry(lc["corners"], pc)["x"]).reshape(-1)
    uf = f(node_geometry(lf["corners"], pf)["x"]).reshape(-1)
    np.testing.assert_allclose(T.interpolate(uc), uf, atol=1e-13)


@pytest.mark.parametrize("kind,pc,pf", [("p", 2, 4), ("p", 3, 7), ("h", 2, 2), ("h", 3, 3)])
def test_restriction_is_transpose(kind, pc, pf):
    """<R r, u> = <r, I u> for random pairs (R is the transpose of I)."""
    lc, lf = _pair(kind, pc, pf)
    T = transfer.Transfer(lc, lf)
    nc = lc["corners"].shape[0] * (pc + 1) ** 3
    nf = lf["corners"].shape[0] * (pf + 1) ** 3
    rng = np.random.default_rng(7)
    for _ in range(5):
        uc, rf = rng.standard_normal(nc), rng.standard_normal(nf)
        a, b = T.restrict(rf) @ uc, rf @ T.interpolate(uc)
        assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))


@pytest.mark.parametrize("p,shared", [(2, True), (3, False), (4, True)])
def test_h_projection_averages_only_for_even_p(p, shared):
    lc, lf = _pair("h", p, p)
    T = transfer.Transfer(lc, lf)
    # a field that is constant per child: projection averages at shared nodes
    N = p + 1
    uf = np.repeat(lf["octant"].astype(float), N ** 3)
    uc = T.project(uf).reshape(-1, N, N, N)
    half = (N - 1) // 2
    has_fraction = np.any(np.abs(uc - np.round(uc)) > 1e-12)
    assert has_fraction == shared
    if shared:
        assert abs(uc[0, half, half, half] - 3.5) < 1e-14   # mean of octants 0..7
