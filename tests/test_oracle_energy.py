"""Oracle pins of the element error indicators and the composite energy norm
of the adaptive loop (Sec. 6.1 energy norm, Sec. 6.4 indicators and marking).

* The sum of the leaf indicators of a single level equals eps^T A eps with A
  assembled explicitly (sparse matrix, independent of the matrix-free apply).
* The energy norm of the error of the exact discrete solution against the
  nodal interpolant of a smooth manufactured solution falls with the mesh width
  at (at least) the rate p of the energy norm.
* Marking keeps exactly the leaves above 0.7 of the largest indicator.
"""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import fas, sip
from paper_2608_14123_b300 import workloads as wl


def _one_level(n, p):
    V = wl.uniform_vertices(n)
    levels = wl.hierarchy(V, [p])
    return fas.LocalHierarchy(levels, 2.0, 0.08, 1, 1, 1), levels


def test_indicators_sum_to_the_quadratic_form():
    H, _ = _one_level(3, 2)
    rng = np.random.default_rng(4)
    eps = rng.standard_normal(H.ops[0].ndof)
    A = sip.assemble(H.ops[0])
    assert abs(H.energy_error([eps]) ** 2 - eps @ (A @ eps)) <= 1e-10 * abs(eps @ (A @ eps))


def test_energy_error_converges_at_rate_p():
    p = 2
    spec = wl.sine_rhs_spec()
    errs = []
    for n in (2, 4, 8):
        H, levels = _one_level(n, p)
        op = H.ops[0]
        X = op.geo["x"]
        b = sip.rhs(op, wl.eval_f(spec, X), np.zeros(X.shape[:-1])).reshape(-1)
        uh = spla.spsolve(sip.assemble(op).tocsc(), b)
        ui = wl.eval_u(spec, X).reshape(-1)
        errs.append(H.energy_error([uh - ui]))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] >= p - 0.3, rates


def test_marking_keeps_the_leaves_above_the_fraction():
    ind = [np.array([1.0, 5.0, 9.0]), np.array([10.0, 6.0, 7.5])]
    leaf = [np.array([True, True, False]), np.array([True, True, True])]
    m = fas.LocalHierarchy.mark_for_refinement(ind, leaf, 0.7)
    assert m[0].tolist() == [False, False, False]   # 9.0 is not a leaf
    assert m[1].tolist() == [True, False, True]     # > 7.0
