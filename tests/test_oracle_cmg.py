"""Oracle pins of the cascadic startup (Alg. 3, FAS-CMG).

* Closed form: on box elements SIP-DG with GLL collocation reproduces linear
  functions exactly (the discrete solution of -lap u = 0 with linear
  Dirichlet data u_D is u_D at the nodes; on curved elements the collocated
  metric terms make it only approximate), the root solve then returns u_D
  on the root, the interpolation between levels is exact for linear
  functions and smoothing leaves an exact solution unchanged: the CMG start
  equals u_D on every level, for any n_sc.
* Structure: with many smoothing steps per level, level L-1 converges to the
  discrete solution of its own right-hand side, so the start value is
  I_L (A_{L-1}^{-1} f_{L-1}) with A_{L-1} assembled explicitly and solved by a
  sparse direct solver (independent of the smoother and transfer code).  A
  wrong right-hand side per level or a missing final interpolation fails it.
* Use: started from the CMG value, the V-cycles need fewer cycles to reach
  1e-10 of the zero start's residual than from zero.
"""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import fas, sip
from paper_2608_14123_b300 import workloads as wl


def _setup(cid, small, uD=None, f=None):
    cfg = wl.config(cid, small=small)
    pr = cfg["params"]
    H = fas.Hierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    fl = []
    for op in H.ops:
        X = op.geo["x"]
        fn = wl.eval_f(cfg["rhs"], X) if f is None else f(X)
        ud = np.zeros(X.shape[:-1]) if uD is None else uD(X)
        fl.append(sip.rhs(op, fn, ud).reshape(-1))
    return H, fl


def _linear(X):
    return 0.3 + 1.1 * X[..., 0] - 0.7 * X[..., 1] + 0.4 * X[..., 2]


def test_cmg_reproduces_a_linear_solution_on_every_level():
    for cid, small in ((1, False), (2, True)):
        H, fl = _setup(cid, small, uD=_linear, f=lambda X: np.zeros(X.shape[:-1]))
        for sc in (0, 2):
            u = H.cmg(fl, sc=sc)
            for l, op in enumerate(H.ops):
                ex = _linear(op.geo["x"]).reshape(-1)
                assert np.abs(u[l] - ex).max() <= 1e-10 * np.abs(ex).max(), (cid, sc, l)


def test_cmg_with_converged_levels_is_the_interpolated_discrete_solution():
    H, fl = _setup(1, False)
    L = H.L
    u = H.cmg(fl, sc=400)
    ref = spla.spsolve(sip.assemble(H.ops[L - 1]).tocsc(), fl[L - 1])
    assert np.abs(u[L - 1] - ref).max() <= 1e-8 * np.abs(ref).max()
    top = H.tr[L].interpolate(ref)
    assert np.abs(u[L] - top).max() <= 1e-8 * np.abs(top).max()


def test_cmg_start_saves_cycles():
    H, fl = _setup(1, False)
    L = H.L
    u_c = H.cmg(fl)[L]
    r_zero = np.linalg.norm(fl[L])
    r_c = np.linalg.norm(H.residual(L, u_c, fl[L]))
    assert r_c < r_zero
    _, h_c = H.solve(u_c, fl[L], rtol=1e-10 * r_zero / r_c)
    _, h_zero = H.solve(np.zeros_like(u_c), fl[L], rtol=1e-10)
    assert h_c[-1] <= 1e-10 * r_zero and len(h_c) < len(h_zero)
