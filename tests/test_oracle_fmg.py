"""Oracle pins of the full multigrid startup (Alg. 4, FAS-FMG).

* Structure: with many V-cycles per level the sub-hierarchy cycles converge,
  so the start value must equal I_L (A_{L-1}^{-1} f_{L-1}) -- the level-(L-1)
  discrete solution of its own right-hand side, interpolated to the top --
  with A_{L-1} assembled explicitly and solved by a sparse direct solver
  (independent of the cycle code).  A wrong right-hand side per level, a
  missing final interpolation or a cycle that does not treat level l as the
  top all fail it.
* Closed form: with linear Dirichlet data on box meshes the start is that
  linear function (SIP-DG reproduces it, every step preserves it).
* Use: started from the FMG value, the V-cycles reach 1e-10 of the residual
  of a zero start in fewer cycles than from the zero start itself.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fas, sip
from paper_2608_14123_b300 import workloads as wl


def _setup(cid, small):
    cfg = wl.config(cid, small=small)
    pr = cfg["params"]
    H = fas.Hierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    fl = []
    for op in H.ops:
        X = op.geo["x"]
        fl.append(sip.rhs(op, wl.eval_f(cfg["rhs"], X), np.zeros(X.shape[:-1])).reshape(-1))
    return H, fl


def test_fmg_with_converged_levels_is_the_interpolated_discrete_solution():
    H, fl = _setup(1, False)
    L = H.L
    u = H.fmg(fl, cycles=30)
    ref = H.tr[L].interpolate(spla.spsolve(sip.assemble(H.ops[L - 1]).tocsc(), fl[L - 1]))
    assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()


def test_fmg_start_saves_cycles():
    H, fl = _setup(1, False)
    L = H.L
    u_fmg = H.fmg(fl, cycles=1)
    r_zero = np.linalg.norm(fl[L])
    r_fmg = np.linalg.norm(H.residual(L, u_fmg, fl[L]))
    assert r_fmg < r_zero
    _, h_fmg = H.solve(u_fmg, fl[L], rtol=1e-10 * r_zero / r_fmg)
    _, h_zero = H.solve(np.zeros_like(u_fmg), fl[L], rtol=1e-10)
    assert h_fmg[-1] <= 1e-10 * r_zero and h_zero[-1] <= 1e-10 * r_zero
    assert len(h_fmg) < len(h_zero)


def test_local_fmg_equals_global_fmg_without_local_refinement():
    """On a globally refined hierarchy the local variant reproduces Alg. 4."""
    H, fl = _setup(1, False)
    cfg = wl.config(1)
    pr = cfg["params"]
    HL = fas.LocalHierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    u_loc = HL.fmg_local(fl, cycles=1)
    u_glob = H.fmg(fl, cycles=1)
    assert np.abs(u_loc[-1] - u_glob).max() <= 1e-12 * np.abs(u_glob).max()


def test_local_fmg_start_saves_cycles():
    cfg = wl.config4(small=True)
    pr = cfg["params"]
    H = fas.LocalHierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    f = []
    for op in H.ops:
        X = op.geo["x"]
        f.append(sip.rhs(op, wl.eval_front_f(cfg["rhs"], X), wl.eval_front_u(cfg["rhs"], X)).reshape(-1))
    zero = [np.zeros(op.ndof) for op in H.ops]
    r_zero = H.composite_residual(zero, f)
    u_f = H.fmg_local(f, cycles=1)
    r_f = H.composite_residual(u_f, f)
    assert r_f < r_zero
    _, h_f = H.solve_local(u_f, f, rtol=1e-10 * r_zero / r_f)
    _, h_z = H.solve_local(zero, f, rtol=1e-10)
    assert h_f[-1] <= 1e-10 * r_zero * (1 + 1e-9) and len(h_f) < len(h_z)


def test_fmg_reproduces_a_linear_solution():
    """Closed form: on box elements the SIP-DG solution of -lap u = 0 with
    linear Dirichlet data is that linear function at the nodes, the root is
    solved exactly, interpolation is exact for it and a V-cycle leaves an
    exact solution unchanged: the FMG start is the linear function."""
    def lin(X):
        return 0.3 + 1.1 * X[..., 0] - 0.7 * X[..., 1] + 0.4 * X[..., 2]
    for cid, small in ((1, False), (2, True)):
        cfg = wl.config(cid, small=small)
        pr = cfg["params"]
        H = fas.Hierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
        fl = [sip.rhs(op, np.zeros(op.geo["x"].shape[:-1]), lin(op.geo["x"])).reshape(-1)
              for op in H.ops]
        u = H.fmg(fl, cycles=1)
        ex = lin(H.ops[-1].geo["x"]).reshape(-1)
        assert np.abs(u - ex).max() <= 1e-10 * np.abs(ex).max(), cid
