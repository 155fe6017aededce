"""Oracle pins for the FAS with local refinement (Sec. 3.1, 3.3, Alg. 2)."""
import numpy as np

from paper_2608_14123_b300 import workloads as wl
from oracle import fas, sip


def _small(buffer):
    rng = np.random.default_rng(wl.SEED_BASE + 4)
    spec = wl.front_spec(rng)
    levels = wl.refined_hierarchy(spec, n_base=4, n_ref=1, n_root=2, buffer=buffer)
    return spec, levels


def _rhs(H, spec):
    out = []
    for op in H.ops:
        X = op.geo["x"]
        out.append(sip.rhs(op, wl.eval_front_f(spec, X), wl.eval_front_u(spec, X)).reshape(-1))
    return out


class _Exact(fas.LocalHierarchy):
    """Exact solves of the active equations of each level in place of smoothing."""

    def smooth(self, l, u, g, n):
        import scipy.sparse.linalg as spla
        if n == 0:
            return u
        if not hasattr(self, "_lu"):
            self._lu = {}
        if l not in self._lu:
            A = sip.assemble(self.ops[l]).tocsr()
            act = np.repeat(self.active[l], self.ops[l].N ** 3)
            self._lu[l] = (spla.splu(A[act][:, act].tocsc()), A[act][:, ~act], act)
        lu, Aaf, act = self._lu[l]
        u = u.copy()
        u[act] = lu.solve(g[act] - Aaf @ u[~act])
        return u


def test_exact_level_solves_converge_to_the_fas_fixed_point():
    """With exact level solves in place of the smoother the FAS iteration is a
    block iteration between the levels; it converges to the fixed point of
    Eq. (6): twigs hold the projection of the finer level (6b), frozen
    elements the interpolation of the parent leaves (6a), and every leaf
    residual vanishes (6c)."""
    spec, levels = _small(2.0)
    assert any(np.any(lv["cls"] == 2) for lv in levels)
    H = _Exact(levels, 5.0, 0.08, 2, 2, 4)
    f = _rhs(H, spec)
    u = [np.zeros(op.ndof) for op in H.ops]
    u, hist = H.solve_local(u, f, rtol=1e-9, max_cycles=15)
    assert hist[-1] <= 1e-9 * hist[0]
    for l in range(1, H.L + 1):
        up, recv = H.tr[l].project_active(u[l], u[l - 1], H.cls[l])
        tw = np.repeat(H.cls[l - 1] == 1, H.ops[l - 1].N ** 3)
        uu = H.tr[l].interpolate(u[l - 1])
        fr = np.repeat(H.cls[l] == 2, H.ops[l].N ** 3)
        scale = np.abs(u[l]).max()
        if tw.any():
            assert np.abs(up - u[l - 1])[tw].max() <= 1e-7 * scale
        if fr.any():
            assert np.abs(uu - u[l])[fr].max() <= 1e-7 * scale


def test_full_coverage_equals_global_refinement():
    spec, levels = _small(100.0)      # every cell refined: no frozen elements, no coarse leaves
    assert not any(np.any(lv["cls"] == 2) for lv in levels)
    H = fas.LocalHierarchy(levels, 5.0, 0.08, 2, 2, 4)
    f = _rhs(H, spec)
    u = [np.zeros(op.ndof) for op in H.ops]
    u[-1] = np.random.default_rng(3).uniform(-1, 1, H.ops[-1].ndof)
    a, _ = H.fas_vcycle_local(u, f)
    b, _ = H.fas_vcycle(u, f[-1])
    np.testing.assert_allclose(a[-1], b[-1], rtol=0, atol=1e-12 * np.abs(b[-1]).max())


def test_local_refinement_converges_with_schwarz_smoother():
    spec, levels = _small(2.0)
    H = fas.LocalHierarchy(levels, 5.0, 0.08, 2, 2, 4)
    f = _rhs(H, spec)
    u = [np.zeros(op.ndof) for op in H.ops]
    u, hist = H.solve_local(u, f, rtol=1e-8, max_cycles=15)
    assert hist[-1] <= 1e-8 * hist[0]
