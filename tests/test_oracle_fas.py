"""Oracle pins for the multigrid cycles (Algs. 1, 2, 5, 6)."""
import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from oracle import fas, sip


def _setup(cid=1, small=False):
    cfg = wl.config(cid, small=small)
    pr = cfg["params"]
    H = fas.Hierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    top = H.ops[-1]
    X = top.geo["x"]
    b = sip.rhs(top, wl.eval_f(cfg["rhs"], X), np.zeros(X.shape[:-1])).reshape(-1)
    return cfg, H, b


def test_fas_equals_cs_for_linear_problem():
    cfg, H, b = _setup(1)
    u = H.zero_levels(cfg["u0"])
    for _ in range(2):
        u, _ = H.fas_vcycle(u, b)
    uc = cfg["u0"].copy()
    for _ in range(2):
        uc = H.cs_vcycle(uc, b)
    assert np.abs(u[-1] - uc).max() <= 1e-12 * np.abs(uc).max()


def test_exact_smoother_gives_one_cycle_convergence():
    cfg, H, b = _setup(1)
    A = sip.assemble(H.ops[-1]).toarray()
    L = H.L
    ex = np.linalg.solve(A, b)
    H.was = lambda l, u, g, n, _A=A, _H=H: (np.linalg.solve(sip.assemble(_H.ops[l]).toarray(), g)
                                          if n > 0 else u)
    u, _ = H.fas_vcycle(H.zero_levels(cfg["u0"]), b)
    assert np.abs(u[L] - ex).max() <= 1e-10 * np.abs(ex).max()


def test_config1_solve_reaches_1e10_and_discretization_error():
    cfg, H, b = _setup(1)
    u, hist = H.solve(cfg["u0"], b)
    assert hist[-1] <= 1e-10 * hist[0]
    assert len(hist) - 1 <= 8
    rates = [hist[k + 1] / hist[k] for k in range(len(hist) - 1)]
    assert max(rates[1:]) < 0.1
    X = H.ops[-1].geo["x"]
    e = u - wl.eval_u(cfg["rhs"], X).reshape(-1)
    assert np.sqrt(np.sum(H.ops[-1].mass.reshape(-1) * e * e)) < 1e-5


def test_scg_beats_was_as_one_level_iteration():
    """Krylov acceleration (Alg. 6) of the Schwarz sweep converges faster than
    the plain sweep (Alg. 5) used as a one-level iteration."""
    cfg, H, b = _setup(1)
    L = H.L
    u0 = cfg["u0"]
    r0 = np.linalg.norm(b - H.A(L, u0))
    r_scg = np.linalg.norm(b - H.A(L, H.scg(L, u0, b, 30, 0.0))) / r0
    r_was = np.linalg.norm(b - H.A(L, H.was(L, u0, b, 30))) / r0
    assert r_scg < 1e-5 and r_scg < 1e-2 * r_was
    # r_max exit: stops as soon as the residual falls below the bound
    u = H.scg(L, u0, b, 100, 1e-3 * r0)
    assert np.linalg.norm(b - H.A(L, u)) <= 1e-3 * r0
