"""The algebra the FP32 curvilinear operator relies on when it recomputes the
volume metric instead of reading it (Sec. 2.2 geometric factors): from the
trilinear map written in monomial form x = a0 + a1 xi + a2 eta + a3 zeta +
a4 xi eta + a5 xi zeta + a6 eta zeta + a7 xi eta zeta, with
a_k = 1/8 sum_c (product of the corner's signs in the monomial) x_c, the
Jacobian's columns J_d = dx/dxi_d are affine in zeta along a z-line, the rows
of adj(J) are C_0 = J_1 x J_2, C_1 = J_2 x J_0, C_2 = J_0 x J_1, and
  G_df = nu w_i w_j w_k (C_d . C_f) / det J,
  c_t  = s nu w_a w_b (C_d . C_t) / det J,   W = w_a w_b |C_d|
equal the oracle's definitions nu w det J grad xi_d . grad xi_f and its face
factors (from the inverse Jacobian).  Run in FP64 here; the kernel evaluates
the same expressions in FP32."""
import numpy as np

from oracle import geometry
from paper_2608_14123_b300 import workloads as wl


def _monomial_coefficients(corners):
    """[8, 3] corners -> a1..a7 [7, 3] (the set-up's table, restated)."""
    a = np.zeros((7, 3))
    for c in range(8):
        s0, s1, s2 = [1.0 if (c >> d) & 1 else -1.0 for d in range(3)]
        sg = [s0, s1, s2, s0 * s1, s0 * s2, s1 * s2, s0 * s1 * s2]
        for k in range(7):
            a[k] += 0.125 * sg[k] * corners[c]
    return a


def _columns(a, xi, eta, zeta):
    a1, a2, a3, a4, a5, a6, a7 = a
    J0 = (a1 + a4 * eta) + (a5 + a7 * eta) * zeta
    J1 = (a2 + a4 * xi) + (a6 + a7 * xi) * zeta
    J2 = a3 + a5 * xi + a6 * eta + a7 * xi * eta
    return J0, J1, J2


def _cases():
    rng = np.random.default_rng(wl.SEED_BASE + 31)
    V = wl.perturbed_vertices(2, 0.2, rng)
    out = []
    for p in (1, 3, 7):
        lev = wl.level_from_vertices(V, p, -1, False)
        out.append((lev["corners"], p))
    return out


def test_metric_from_monomial_form_equals_oracle():
    nu = 1.7
    for corners, p in _cases():
        geo = geometry.node_geometry(corners, p)
        G_ref = geometry.volume_metric(geo, nu)          # [e, k, j, i, d, f]
        xi, w = geo["xi"], geo["w"]
        N = p + 1
        for e in range(corners.shape[0]):
            a = _monomial_coefficients(corners[e])
            for k in range(N):
                for j in range(N):
                    for i in range(N):
                        J0, J1, J2 = _columns(a, xi[i], xi[j], xi[k])
                        C = [np.cross(J1, J2), np.cross(J2, J0), np.cross(J0, J1)]
                        det = J0 @ C[0]
                        np.testing.assert_allclose(det, geo["detJ"][e, k, j, i], rtol=1e-13)
                        s = nu * w[i] * w[j] * w[k] / det
                        G = np.array([[s * (C[d] @ C[f]) for f in range(3)] for d in range(3)])
                        scale = np.abs(G_ref[e, k, j, i]).max()
                        assert np.abs(G - G_ref[e, k, j, i]).max() <= 1e-13 * scale


def test_face_factors_from_monomial_form_equal_oracle():
    nu = 0.9
    for corners, p in _cases():
        geo = geometry.node_geometry(corners, p)
        W_ref, c_ref = geometry.face_factors(geo, nu)    # [e, f, b, a], [e, f, b, a, t]
        xi, w = geo["xi"], geo["w"]
        N = p + 1
        for e in range(corners.shape[0]):
            a = _monomial_coefficients(corners[e])
            for f in range(6):
                d, sgn = f // 2, (1.0 if f % 2 else -1.0)
                K, J, I = geometry.face_node_index(N, f)
                for bb in range(N):
                    for aa in range(N):
                        k, j, i = K[bb, aa], J[bb, aa], I[bb, aa]
                        J0, J1, J2 = _columns(a, xi[i], xi[j], xi[k])
                        C = [np.cross(J1, J2), np.cross(J2, J0), np.cross(J0, J1)]
                        det = J0 @ C[0]
                        wab = w[aa] * w[bb]
                        W = wab * np.linalg.norm(C[d])
                        c = [sgn * nu * wab * (C[d] @ C[t]) / det for t in range(3)]
                        np.testing.assert_allclose(W, W_ref[e, f, bb, aa], rtol=1e-13)
                        scale = np.abs(c_ref[e, f, bb, aa]).max()
                        assert np.abs(np.array(c) - c_ref[e, f, bb, aa]).max() <= 1e-13 * scale


def test_monomial_form_reproduces_the_corners():
    """x(+-1, +-1, +-1) of the monomial form returns the 8 corners (a0 from
    the corner average), the form's own consistency check."""
    for corners, _ in _cases():
        for e in range(corners.shape[0]):
            a = _monomial_coefficients(corners[e])
            a0 = corners[e].mean(axis=0)
            for c in range(8):
                x, y, z = [1.0 if (c >> d) & 1 else -1.0 for d in range(3)]
                X = (a0 + a[0] * x + a[1] * y + a[2] * z + a[3] * x * y + a[4] * x * z
                     + a[5] * y * z + a[6] * x * y * z)
                np.testing.assert_allclose(X, corners[e, c], atol=1e-14)
