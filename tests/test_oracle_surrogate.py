"""Oracle pins for the Kronecker-sum fits and the MLP (learned surrogate)."""
import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from oracle import mlp, surrogate as su
from oracle.geometry import node_geometry, volume_metric, face_factors, h_perp
from oracle.gll import gll, diff_matrix
from oracle.schwarz import side_of


def _lines(level, mu_star):
    p = level["p"]
    geo = node_geometry(level["corners"], p)
    G = volume_metric(geo)
    W, c = face_factors(geo)
    mu = mu_star * p * (p + 1) / (2.0 * h_perp(geo, W))
    ne = level["nbr"].shape[0]
    sides = np.array([[side_of(level["nbr"][e, f]) for f in range(6)] for e in range(ne)])
    return [su.line_entries(G, c, W, mu, diff_matrix(p), gll(p)[1], sides, d) for d in range(3)]


@pytest.mark.parametrize("p", [1, 2, 3])
def test_line_entries_equal_dense_element_block(p):
    V = wl.perturbed_vertices(3, 0.2, np.random.default_rng(3))
    lev = wl.level_from_vertices(V, p)
    N = p + 1
    Es = _lines(lev, 5.0)
    for e in (0, 4, 13, 26):   # corner, edge, interior elements: Dirichlet and interior faces
        A = su.element_block_dense(lev, e, 5.0).reshape(N, N, N, N, N, N)
        refs = [np.einsum("kjikjm->kjim", A), np.einsum("kjikmi->kijm", A),
                np.einsum("kjimji->ijkm", A)]
        for d in range(3):
            assert np.abs(Es[d][e] - refs[d]).max() <= 1e-13 * np.abs(refs[d]).max()


def test_fit_is_exact_on_boxes():
    lev = wl.level_from_vertices(wl.uniform_vertices(3, hi=(1.0, 0.5, 2.0)), 4)
    gf, gg = su.fit_coefficients(lev, 5.0)
    np.testing.assert_allclose(gf, gg, rtol=1e-12)


def test_fit_equals_dense_lstsq():
    """Normal equations == least squares on the dense, scaled, vectorised matrices."""
    p = 2
    N = p + 1
    lev = wl.level_from_vertices(wl.perturbed_vertices(3, 0.2, np.random.default_rng(5)), p)
    gf, _ = su.fit_coefficients(lev, 5.0)
    _, w = gll(p)
    K = lambda a, b, c: np.kron(a, np.kron(b, c))
    M = np.diag(w)
    s = 1.0 / np.sqrt(np.diag(K(M, M, M)))
    for e in (0, 13):
        sides = [side_of(lev["nbr"][e, f]) for f in range(6)]
        Lc = su.central_blocks(p, 5.0, sides)
        Ks = [K(M, M, Lc[0]), K(M, Lc[1], M), K(Lc[2], M, M)]
        A = su.element_block_dense(lev, e, 5.0)
        cols = np.stack([(s[:, None] * Kk * s[None, :]).reshape(-1) for Kk in Ks], 1)
        ref = np.linalg.lstsq(cols, (s[:, None] * A * s[None, :]).reshape(-1), rcond=None)[0]
        np.testing.assert_allclose(gf[e], ref, rtol=1e-10)


def test_fit_translation_invariant_and_scales_with_h():
    rng = np.random.default_rng(9)
    cr = su.training_elements(6, rng)
    lv = dict(p=3, corners=cr, nbr=np.zeros((6, 6), np.int32))
    g0, _ = su.fit_coefficients(lv, 10.0)
    lv2 = dict(p=3, corners=cr * 3.0 + np.array([1.0, -2.0, 0.5]), nbr=lv["nbr"])
    g1, _ = su.fit_coefficients(lv2, 10.0)
    np.testing.assert_allclose(g1, 3.0 * g0, rtol=1e-11)    # g ~ h for nu = 1
    X0, X1 = su.mlp_inputs(cr), su.mlp_inputs(lv2["corners"])
    np.testing.assert_allclose(X0, X1, atol=1e-12)


def test_targets_decode_to_fit():
    rng = np.random.default_rng(4)
    cr = su.training_elements(5, rng)
    lv = dict(p=3, corners=cr, nbr=np.zeros((5, 6), np.int32))
    gf, _ = su.fit_coefficients(lv, 10.0)
    Y = su.mlp_targets(cr, gf)
    vol = np.array([su._vol(c) for c in cr])
    np.testing.assert_allclose(su.coeffs_from_outputs(Y, vol), gf, rtol=1e-12)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    th = mlp.init(rng)
    X = rng.standard_normal((7, 24))
    Y = rng.standard_normal((7, 6))
    g = mlp.grad(th, X, Y)
    idx = rng.choice(th.size, 40, replace=False)
    for i in idx:
        e = np.zeros_like(th)
        e[i] = 1e-6
        fd = (mlp.loss(th + e, X, Y) - mlp.loss(th - e, X, Y)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9


def test_adam_step_textbook():
    rng = np.random.default_rng(1)
    th, g = rng.standard_normal(5), rng.standard_normal(5)
    m, v = np.zeros(5), np.zeros(5)
    th1, m1, v1 = mlp.adam_step(th, g, m, v, 1, lr=0.01)
    # first step: m_hat = g, v_hat = g^2  ->  th - lr * g / (|g| + eps)
    np.testing.assert_allclose(th1, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
