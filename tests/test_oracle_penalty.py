"""Oracle pins of the penalty length h_perp (Sec. 2.2: the element extension
perpendicular to the interface).

On curved elements the paper does not say how h_perp is measured; the
reading taken is the smallest local extent 2 / |grad xi_d| over the face's
GLL nodes.  Pins: on boxes it is the edge length exactly (the paper's h); on a
valid mesh with a nearly folded corner the face's mean extent |Omega| / |face|
leaves the SIP operator indefinite at mu_star = 5 (the penalty cannot control
the flux next to the corner), the local reading keeps it positive definite;
and the graded, strongly perturbed workload's operator is positive definite
at mu_star = 5 on its small variant."""
import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from oracle import geometry, sip


def _mean_extent(geo, W):
    vol = np.sum(geo["W3"] * geo["detJ"], axis=(1, 2, 3))
    return vol[:, None] / np.sum(W, axis=(2, 3))


def _near_folded_block(p):
    """2^3 cells of [0,1]^3 whose shared centre vertex is moved 0.3 cells
    towards the far corner: the cell at that corner keeps positive corner
    Jacobians (smallest / largest = 0.10) but is close to folding."""
    V = wl.uniform_vertices(2)
    V[1, 1, 1] += 0.15
    return V, wl.level_from_vertices(V, p)


def test_h_perp_is_the_edge_length_on_boxes():
    V = wl.uniform_vertices(2, 3, 4, hi=(0.5, 1.5, 2.0))
    lv = wl.level_from_vertices(V, 4)
    geo = geometry.node_geometry(lv["corners"], 4)
    W, _ = geometry.face_factors(geo, 1.0)
    hp = geometry.h_perp(geo, W)
    h = np.array([0.25, 0.5, 0.5])
    np.testing.assert_allclose(hp, np.repeat(h, 2)[None, :].repeat(len(hp), 0), rtol=1e-13)


@pytest.mark.parametrize("p", [1, 3])
def test_local_extent_keeps_operator_spd_next_to_a_nearly_folded_corner(p):
    V, lv = _near_folded_block(p)
    assert 0.09 < wl.corner_jacobian_ratio(V).min() < 0.11
    A = sip.assemble(sip.LevelOps(lv, 5.0)).toarray()
    assert np.linalg.eigvalsh(A)[0] > 0.0
    # the face's mean extent: indefinite at the same mu_star
    orig = sip.h_perp
    try:
        sip.h_perp = _mean_extent
        Am = sip.assemble(sip.LevelOps(lv, 5.0)).toarray()
    finally:
        sip.h_perp = orig
    assert np.linalg.eigvalsh(Am)[0] < 0.0


def test_graded_perturbed_workload_spd_at_mu5():
    """The small variant of the graded, +-0.25h perturbed workload (4^3 cells,
    every cell's corner-Jacobian ratio >= 0.2): SPD on its p = 1 and p = 3
    levels at mu_star = 5."""
    cfg = wl.config(3, small=True)
    for lv in cfg["levels"]:
        if lv["p"] > 3:
            continue
        A = sip.assemble(sip.LevelOps(lv, 5.0)).toarray()
        assert np.linalg.eigvalsh(A)[0] > 0.0, lv["p"]


def test_quality_redraw_bounds_the_corner_jacobian_ratio():
    cfg = wl.config(3)
    lv = cfg["levels"][-1]
    n = lv["shape"][0]
    V = np.zeros((n + 1,) * 3 + (3,))
    for c in range(8):
        o = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        q = lv["ijk"] + o
        V[q[:, 0], q[:, 1], q[:, 2]] = lv["corners"][:, c]
    assert wl.corner_jacobian_ratio(V).min() >= wl.MIN_JACOBIAN_RATIO
