"""Oracle pins for SCG (Alg. 6, Sec. 4.3.2): the inexact preconditioned CG
that the method adopts reduces to textbook CG / PCG for a fixed symmetric
preconditioner, converges in one step with the exact inverse as
preconditioner, leaves at the first step with |r| <= r_max, and the reading of
its first search direction (p = z) is the one under which the SCG-smoothed
V-cycle converges in the handful of cycles the paper prints."""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_2608_14123_b300 import workloads as wl
from oracle import fas, sip


def _setup(cid=1, small=False, **kw):
    cfg = wl.config(cid, small=small)
    pr = cfg["params"]
    H = fas.Hierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                      **kw)
    top = H.ops[-1]
    X = top.geo["x"]
    b = sip.rhs(top, wl.eval_f(cfg["rhs"], X), np.zeros(X.shape[:-1])).reshape(-1)
    return cfg, H, b


def _textbook_pcg(Aop, b, x, Minv, n):
    """Hestenes-Stiefel PCG with the Fletcher-Reeves coefficient, written out
    independently of the oracle: the iterates x_1..x_n."""
    r = b - Aop(x)
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    xs = []
    for _ in range(n):
        q = Aop(p)
        a = rz / (p @ q)
        x = x + a * p
        r = r - a * q
        z = Minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        xs.append(x.copy())
    return xs


@pytest.mark.parametrize("first", ["z", "r"])
def test_identity_preconditioner_gives_textbook_cg(first):
    """z = r: both readings of the first direction coincide with CG."""
    cfg, H, b = _setup(1)
    l = 1
    A = lambda v: H.A(l, v)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(H.ops[l].ndof)
    x0 = rng.standard_normal(H.ops[l].ndof)
    ref = _textbook_pcg(A, g, x0.copy(), lambda r: r.copy(), 8)
    for n in (1, 2, 5, 8):
        got = H.scg(l, x0.copy(), g, n, 0.0, precond=lambda r: r.copy(), first=first)
        np.testing.assert_allclose(got, ref[n - 1], rtol=0, atol=1e-9 * np.abs(ref[n - 1]).max())


def test_jacobi_preconditioner_gives_textbook_pcg():
    """A fixed SPD preconditioner (the inverse diagonal): the reading p = z
    reproduces textbook PCG step by step (the Polak-Ribiere beta of Alg. 6
    equals Fletcher-Reeves when z^T r0 = 0); the printed p = r does not."""
    cfg, H, b = _setup(1)
    l = 1
    Ad = sip.assemble(H.ops[l]).toarray()
    dinv = 1.0 / np.diag(Ad)
    M = lambda r: dinv * r
    A = lambda v: Ad @ v
    rng = np.random.default_rng(4)
    g = rng.standard_normal(Ad.shape[0])
    x0 = np.zeros_like(g)
    ref = _textbook_pcg(A, g, x0.copy(), M, 6)
    for n in (1, 3, 6):
        got = H.scg(l, x0.copy(), g, n, 0.0, precond=M, first="z")
        np.testing.assert_allclose(got, ref[n - 1], rtol=0, atol=1e-9 * np.abs(ref[n - 1]).max())
    bad = H.scg(l, x0.copy(), g, 1, 0.0, precond=M, first="r")
    assert np.abs(bad - ref[0]).max() > 1e-3 * np.abs(ref[0]).max()


def test_exact_preconditioner_converges_in_one_step():
    """With z = A^-1 r the first step p = z, alpha = z.r / z.A z = 1 lands on
    the solution; the printed first direction p = r does not."""
    cfg, H, b = _setup(1)
    l = 1
    Ad = sip.assemble(H.ops[l]).toarray()
    ch = sla.cho_factor(Ad)
    M = lambda r: sla.cho_solve(ch, r)
    rng = np.random.default_rng(5)
    g = rng.standard_normal(Ad.shape[0])
    ex = sla.cho_solve(ch, g)
    got = H.scg(l, np.zeros_like(g), g, 1, 0.0, precond=M, first="z")
    assert np.abs(got - ex).max() <= 1e-12 * np.abs(ex).max()
    bad = H.scg(l, np.zeros_like(g), g, 1, 0.0, precond=M, first="r")
    assert np.abs(bad - ex).max() > 1e-2 * np.abs(ex).max()


def test_exit_test_stops_at_first_step_below_r_max():
    """r_max: the iterate after the first step whose residual is <= r_max (the
    textbook CG iterate of that step), unchanged by a larger step cap."""
    cfg, H, b = _setup(1)
    l = 1
    A = lambda v: H.A(l, v)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(H.ops[l].ndof)
    ref = _textbook_pcg(A, g, np.zeros_like(g), lambda r: r.copy(), 40)
    res = [np.linalg.norm(g - A(x)) for x in ref]
    r_max = 0.5 * (res[9] + res[10]) if res[10] < res[9] else 0.999 * res[10]
    k = next(i for i, v in enumerate(res) if v <= r_max)
    got = H.scg(l, np.zeros_like(g), g, 40, r_max, precond=lambda r: r.copy())
    np.testing.assert_allclose(got, ref[k], rtol=0, atol=1e-9 * np.abs(ref[k]).max())


def test_first_direction_reading_matches_paper_cycle_counts():
    """The paper prints 3-4 V-cycles to 1e-10 for the SCG(2,2,4) multigrid
    methods on uniform Cartesian meshes at p = 4 (Table 1: CS-MG-SCG n10 = 4,
    FAS-CMG-SCG 3-4).  On the Cartesian p = 4 workload (p 4 -> 2 -> 1, dense
    root) the reading p = z converges in that range; the printed p = r
    diverges."""
    cfg, H, b = _setup(1, smoother="scg", scg_first="z")
    u, hist = H.solve(cfg["u0"], b, max_cycles=12)
    assert hist[-1] <= 1e-10 * hist[0] and len(hist) - 1 <= 5
    cfg, H, b = _setup(1, smoother="scg", scg_first="r")
    u, hist = H.solve(cfg["u0"], b, max_cycles=6)
    assert hist[-1] > hist[0]


def test_scg_root_with_tight_tolerance_equals_exact_root():
    """The SCG root solve (Alg. 6 as the coarse solver) run to a tight
    tolerance gives the same V-cycle as the exact dense root."""
    cfg, He, b = _setup(1)
    cfg, Hs, _ = _setup(1, coarse="scg", root_rtol=1e-13, root_steps=400)
    ue, _ = He.fas_vcycle(He.zero_levels(cfg["u0"]), b)
    us, _ = Hs.fas_vcycle(Hs.zero_levels(cfg["u0"]), b)
    assert np.abs(us[-1] - ue[-1]).max() <= 1e-9 * np.abs(ue[-1]).max()


def test_scg_root_visit_reduces_root_residual_by_rtol():
    """One visit of the SCG root leaves |g0 - A0 u0| <= root_rtol |r_start| (or
    spends its step cap)."""
    cfg, H, b = _setup(1, coarse="scg", root_rtol=1e-4, root_steps=200)
    rng = np.random.default_rng(8)
    g0 = rng.standard_normal(H.ops[0].ndof)
    u0 = rng.standard_normal(H.ops[0].ndof)
    r0 = np.linalg.norm(g0 - H.A(0, u0))
    u = H.root_solve(g0, u0.copy())
    assert np.linalg.norm(g0 - H.A(0, u)) <= 1e-4 * r0
