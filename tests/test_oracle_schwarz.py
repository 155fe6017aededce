"""Oracle pins for the Schwarz / fast-diagonalization smoother (Sec. 4.3.1)."""
import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from oracle import sip, schwarz


@pytest.mark.parametrize("p,delta,m", [(4, .04, 1), (4, .08, 1), (4, .16, 1),
                                       (8, .04, 1), (8, .08, 2), (8, .16, 2),
                                       (16, .04, 2), (16, .08, 3), (16, .16, 5),
                                       (7, .08, 2), (1, .08, 1)])
def test_overlap_layers(p, delta, m):
    assert schwarz.overlap_layers(p, delta) == m


@pytest.mark.parametrize("p", [1, 4, 7, 8])
def test_generalized_eigenpairs(p):
    T = schwarz.FDTables(p, 0.08, 5.0)
    for v, t in T.tab.items():
        S, M, L, lam = t["S"], t["M"], t["L"], t["lam"]
        np.testing.assert_allclose(S.T @ M @ S, np.eye(len(lam)), atol=1e-12)
        np.testing.assert_allclose(S.T @ L @ S, np.diag(lam), atol=1e-10 * max(1, lam.max()))
        n = p + 1 + schwarz.overlap_layers(p, 0.08) * ((v[0] == "i") + (v[1] == "i"))
        assert len(lam) == n


@pytest.mark.parametrize("kind", ["cart", "pert"])
def test_fd_equals_dense_inverse_of_surrogate(kind):
    V = wl.uniform_vertices(3) if kind == "cart" else wl.perturbed_vertices(3, 0.2, np.random.default_rng(4))
    lev = wl.level_from_vertices(V, 3)
    sw = schwarz.Schwarz(lev, 0.08, 5.0)
    rng = np.random.default_rng(0)
    for e in (0, 4, 13, 26):
        shape = sw.restriction(e).shape
        rs = rng.standard_normal(shape)
        y = sw.fd_solve(e, rs).reshape(-1)
        ref = np.linalg.solve(sw.surrogate_matrix(e), rs.reshape(-1))
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("p", [2, 4])
def test_uniform_cartesian_surrogate_is_exact(p):
    lev = wl.level_from_vertices(wl.uniform_vertices(3), p)
    ops = sip.LevelOps(lev, 2.0)
    A = sip.assemble(ops).toarray()
    sw = schwarz.Schwarz(lev, 0.08, 2.0)
    rng = np.random.default_rng(1)
    for e in range(ops.ne):  # all 27 subdomains: interior, face, edge, corner
        idx = sw.restriction(e)
        As = A[np.ix_(idx.reshape(-1), idx.reshape(-1))]
        assert np.abs(As - sw.surrogate_matrix(e)).max() <= 1e-12 * np.abs(As).max()
        rs = rng.standard_normal(idx.shape)
        y = sw.fd_solve(e, rs).reshape(-1)
        ref = np.linalg.solve(As, rs.reshape(-1))
        assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("p,delta", [(2, .08), (4, .08), (8, .08), (8, .16), (7, .3)])
def test_weights_partition_of_unity(p, delta):
    lev = wl.level_from_vertices(wl.uniform_vertices(3), p)
    sw = schwarz.Schwarz(lev, delta, 2.0)
    pu = np.zeros(sw.ne * sw.N ** 3)
    for e in range(sw.ne):
        idx = sw.restriction(e)
        np.add.at(pu, idx[idx >= 0], sw.weights(e)[idx >= 0])
    np.testing.assert_allclose(pu, 1.0, atol=1e-14)


def test_surrogate_widths_box_exact_and_trilinear_coefficients():
    c = wl.level_from_vertices(wl.uniform_vertices(1, hi=(0.3, 0.5, 2.0)), 1)["corners"][0]
    np.testing.assert_allclose(schwarz.surrogate_widths(c), [0.3, 0.5, 2.0], rtol=1e-14)
    g = schwarz.surrogate_coeffs(np.array([0.3, 0.5, 2.0]))
    np.testing.assert_allclose(g[1:], [0.5 * 2.0 / 0.6, 2.0 * 0.3 / 1.0, 0.3 * 0.5 / 4.0])
    # P1 Legendre coefficient of a trilinear map == its L2 projection by quadrature
    from oracle.geometry import map_and_jacobian
    from oracle.gll import gll
    rng = np.random.default_rng(5)
    corners = c + 0.05 * rng.standard_normal(c.shape)
    x, w = gll(4)
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    pts, _ = map_and_jacobian(corners, X1, X2, X3)
    W3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    for i, Xi in enumerate((X1, X2, X3)):
        a_quad = np.einsum("kji,kjia->a", W3 * Xi, pts) / (8.0 / 3.0)
        a_closed = sum((1.0 if (cc >> i) & 1 else -1.0) * corners[cc] / 8.0 for cc in range(8))
        np.testing.assert_allclose(a_quad, a_closed, atol=1e-14)
