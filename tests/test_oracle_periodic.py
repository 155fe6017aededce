"""Oracle on the periodic box of the paper's uniform Cartesian study: the
constants span the null space of the SIP operator (kappa = 0, no Dirichlet
faces), the root is solved in its complement, and the FAS V-cycle converges
for a consistent right-hand side (zero mean)."""
import numpy as np

from oracle import fas, sip
from paper_2608_14123_b300 import workloads as wl


def _small(kind="h", p=2, n=4):
    cfg = wl.paper_cartesian_periodic(p, kind, n=n)
    pr = cfg["params"]
    H = fas.Hierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    return cfg, H


def test_constants_are_the_null_space():
    cfg, H = _small()
    for l, op in enumerate(H.ops):
        one = np.ones(op.ndof)
        Au = H.A(l, one)
        A = sip.assemble(op)
        assert np.abs(Au).max() <= 1e-11 * abs(A).max()


def test_root_solve_in_the_complement():
    cfg, H = _small()
    assert H.nullspace
    rng = np.random.default_rng(3)
    g = rng.standard_normal(H.ops[0].ndof)
    g -= g.mean()
    x = H.root_solve(g)
    A0 = sip.assemble(H.ops[0]).toarray()
    assert np.abs(A0 @ x - g).max() <= 1e-10 * np.abs(g).max()
    assert abs(x.sum()) <= 1e-9 * np.abs(x).max() * x.size


def test_vcycles_converge_for_consistent_rhs():
    cfg, H = _small()
    top = H.ops[-1]
    X = top.geo["x"]
    f = sip.rhs(top, wl.eval_f(cfg["rhs"], X), np.zeros(X.shape[:-1])).reshape(-1)
    f -= f.mean()
    _, hist = H.solve(cfg["u0"].copy(), f, rtol=1e-10, max_cycles=40)
    assert hist[-1] <= 1e-10 * hist[0]


def test_periodic_topology_is_symmetric():
    """Every face neighbour sees the element back through the opposite face,
    and the 27-neighbourhood of each element is its periodic block."""
    cfg = wl.paper_cartesian_periodic(4, "h", n=4)
    for lv in cfg["levels"]:
        nbr, nbr27, ijk = lv["nbr"], lv["nbr27"], lv["ijk"]
        n = lv["shape"][0]
        assert (nbr >= 0).all()
        for e in range(nbr.shape[0]):
            for f in range(6):
                assert nbr[nbr[e, f], f ^ 1] == e
            for oz in (-1, 0, 1):
                for oy in (-1, 0, 1):
                    for ox in (-1, 0, 1):
                        q = nbr27[e, (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)]
                        want = (ijk[e] + np.array([ox, oy, oz])) % n
                        assert (ijk[q] == want).all()
