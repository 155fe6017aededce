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


# ---------------------------------------------------------------- L2 projection variant
@pytest.mark.parametrize("kind,pc,pf", [("p", 1, 2), ("p", 2, 4), ("p", 4, 8), ("p", 3, 7),
                                         ("h", 1, 1), ("h", 2, 2), ("h", 3, 3), ("h", 4, 4)])
def test_l2_projection_inverts_interpolation(kind, pc, pf):
    lc, lf = _pair(kind, pc, pf)
    T = transfer.Transfer(lc, lf, "l2")
    uc = np.random.default_rng(1).standard_normal(lc["corners"].shape[0] * (pc + 1) ** 3)
    np.testing.assert_allclose(T.project(T.interpolate(uc)), uc, atol=1e-12)


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 4), (3, 7), (4, 8), (5, 10)])
def test_l2_p_projection_is_the_legendre_truncation(pc, pf):
    """p-coarsening: the fine GLL rule integrates u_f times a coarse polynomial
    exactly (degree pf + pc <= 2 pf - 1), so the discrete L2 projection is the
    exact one, i.e. the fine polynomial's Legendre series cut after degree pc
    (computed here from the Legendre expansion, not from the quadrature)."""
    from numpy.polynomial import legendre as leg
    from oracle.gll import gll
    lc, lf = _pair("p", pc, pf)
    T = transfer.Transfer(lc, lf, "l2")
    xf, _ = gll(pf)
    xc, _ = gll(pc)
    rng = np.random.default_rng(2)
    for _ in range(3):
        vals = rng.standard_normal(pf + 1)             # a fine polynomial by its nodal values
        coef = leg.legfit(xf, vals, pf)                # exact (pf + 1 points, degree pf)
        want = leg.legval(xc, coef[:pc + 1])
        got = T.P1[0] @ vals
        np.testing.assert_allclose(got, want, atol=1e-12 * max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_l2_h_projection_residual_is_orthogonal_to_the_parent_space(p):
    """h-coarsening: u_f - I P u_f is orthogonal to every parent polynomial in
    the children's quadrature inner product (each child half of the parent)."""
    from oracle.gll import gll
    lc, lf = _pair("h", p, p)
    T = transfer.Transfer(lc, lf, "l2")
    _, w = gll(p)
    rng = np.random.default_rng(3)
    for _ in range(3):
        vf = rng.standard_normal((2, p + 1))           # two children's nodal values (1D)
        uc = T.P1[0] @ vf[0] + T.P1[1] @ vf[1]
        res = [vf[s] - T.I1[s] @ uc for s in range(2)]
        for k in range(p + 1):                         # every parent basis function
            e = np.zeros(p + 1)
            e[k] = 1.0
            ip = sum(0.5 * (T.I1[s] @ e) @ (w * res[s]) for s in range(2))
            assert abs(ip) < 1e-13


def test_l2_and_interpolation_agree_on_coarse_polynomials_and_differ_otherwise():
    lc, lf = _pair("h", 3, 3)
    Ti, Tl = transfer.Transfer(lc, lf), transfer.Transfer(lc, lf, "l2")
    rng = np.random.default_rng(4)
    uc = rng.standard_normal(lc["corners"].shape[0] * 64)
    np.testing.assert_allclose(Tl.project(Ti.interpolate(uc)), Ti.project(Ti.interpolate(uc)),
                               atol=1e-12)
    uf = rng.standard_normal(lf["corners"].shape[0] * 64)
    assert np.abs(Tl.project(uf) - Ti.project(uf)).max() > 1e-3
