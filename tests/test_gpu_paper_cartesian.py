"""The paper's uniform Cartesian study on the GPU: periodic box, constant null
space, parity of the V-cycle with the oracle on a small periodic hierarchy,
and the cycle counts n10 printed by the paper for h-multigrid (its L = 4
levels, p = 4 and 8; tests/golden/paper_uniform_cartesian_n10.txt), which pin
the smoother, the weights reading and the FAS cycle as a whole."""
import os

import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import rel, torch_cuda

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_uniform_cartesian_n10.txt")


def _paper_rows():
    """(kind, p, s1, s2, sc, start, smoother, P) -> n10 as printed by the paper."""
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        kind, p, s1, s2, sc, start, sm, P, n10 = line.split()
        out[(kind, int(p), int(s1), int(s2), int(sc), start, sm, P)] = int(n10)
    return out


def _paper_n10():
    return {k[:5]: v for k, v in _paper_rows().items() if k[5:] == ("mg", "was", "I")}


def _solver(cfg, s1, s2, sc, prec, smoother=dgfas.DGFAS_WAS, projection=dgfas.DGFAS_P_INTERP):
    return dgfas.Solver(cfg["levels"], cfg["params"]["mu_star"], cfg["params"]["delta"], s1, s2, sc,
                        precision=prec, smoother=smoother, projection=projection)


def _level_rhs(cfg, S):
    """Each level's own right-hand side, projected to zero sum (the full
    multigrid startup's inputs on the periodic box)."""
    torch = torch_cuda()
    out = []
    for l in range(S.n_levels):
        xyz = S.node_coords(l)
        fn = torch.from_numpy(wl.eval_f(cfg["rhs"], xyz.cpu().numpy())).cuda()
        b = torch.empty_like(fn)
        S.dgfas_assemble_rhs_level(l, fn, None, b)
        out.append(b - b.mean())
    return out


def n10_of(kind, p, s1, s2, sc, start, smoother, P, prec=dgfas.DGFAS_FP64):
    """Cycles to reduce the residual by 1e10 on the paper's periodic workload:
    from the random start, or from the full multigrid (Alg. 4) or cascadic
    (Alg. 3) start value, measured against the random start's residual (the
    reference of the paper's counts)."""
    torch = torch_cuda()
    cfg = wl.paper_cartesian_periodic(p, kind)
    S = _solver(cfg, s1, s2, sc, prec,
                dgfas.DGFAS_SCG if smoother == "scg" else dgfas.DGFAS_WAS,
                dgfas.DGFAS_P_L2 if P == "L" else dgfas.DGFAS_P_INTERP)
    b = _rhs(cfg, S)
    u = torch.from_numpy(cfg["u0"]).cuda()
    r = torch.empty_like(u)
    S.dgfas_apply_op(-1, u, b, r)
    r_rand = S.dgfas_norm(-1, r)
    if start in ("fmg", "cmg"):
        if start == "fmg":
            S.dgfas_fmg(_level_rhs(cfg, S), u, 1)
        else:   # the paper's CMG runs n_s0 = n_s1 + n_s2 smoothing steps per level
            S.dgfas_cmg(_level_rhs(cfg, S), u, s1 + s2)
        S.dgfas_apply_op(-1, u, b, r)
        rtol = 1e-10 * r_rand / S.dgfas_norm(-1, r)
    else:
        rtol = 1e-10
    info = S.dgfas_solve(u, b, rtol, 60)
    S.close()
    return info["cycles"]


def _rhs(cfg, S):
    torch = torch_cuda()
    xyz = S.node_coords(-1)
    fn = torch.from_numpy(wl.eval_f(cfg["rhs"], xyz.cpu().numpy())).cuda()
    b = torch.empty_like(fn)
    S.dgfas_assemble_rhs(fn, None, b)
    return b - b.mean()   # consistent with the constant null space


def test_periodic_vcycle_matches_oracle():
    torch = torch_cuda()
    from oracle import fas, sip
    cfg = wl.paper_cartesian_periodic(2, "h", n=4)
    pr = cfg["params"]
    S = _solver(cfg, pr["s1"], pr["s2"], pr["sc"], dgfas.DGFAS_FP64)
    H = fas.Hierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    top = H.ops[-1]
    X = top.geo["x"]
    f_or = sip.rhs(top, wl.eval_f(cfg["rhs"], X), np.zeros(X.shape[:-1])).reshape(-1)
    f_or -= f_or.mean()
    b = _rhs(cfg, S)
    assert rel(b.cpu().numpy(), f_or) < 1e-12
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    S.dgfas_fas_vcycle(u, b)
    u_or, _ = H.fas_vcycle(H.zero_levels(cfg["u0"].copy()), f_or)
    assert rel(u.cpu().numpy(), u_or[-1]) < 1e-11
    one = torch.ones_like(u)
    Au = torch.empty_like(u)
    S.dgfas_apply_op(-1, one, None, Au)
    assert float(Au.abs().max()) < 1e-10


@pytest.mark.parametrize("s", [(1, 1, 2), (2, 2, 4)])
@pytest.mark.parametrize("p,prec", [(4, dgfas.DGFAS_FP64), (4, dgfas.DGFAS_BF16),
                                    (8, dgfas.DGFAS_FP64)])
def test_h_multigrid_cycle_counts_match_the_paper(p, prec, s):
    torch = torch_cuda()
    cfg = wl.paper_cartesian_periodic(p, "h")
    S = _solver(cfg, *s, prec)
    b = _rhs(cfg, S)
    u = torch.from_numpy(cfg["u0"]).cuda()
    info = S.dgfas_solve(u, b, 1e-10, 60)
    # p = 4 (overlap of one node layer) reproduces the paper's counts exactly;
    # at p = 8 two layers carry the weights' transition, whose function the
    # paper does not print (reading), and the counts agree within one cycle
    tol = 0 if p == 4 else 1
    assert abs(info["cycles"] - _paper_n10()[("h", p) + s]) <= tol


@pytest.mark.parametrize("p,s", [(4, (1, 1, 2)), (4, (2, 2, 4)), (8, (1, 1, 2)), (8, (2, 2, 4))])
def test_p_multigrid_cycle_counts_near_the_paper(p, s):
    """p-multigrid p, p/2, ..., 1: the paper solves the p = 1 level with SCG to
    a tolerance, this hierarchy continues with h-levels down to a 2^3 root (one
    V-cycle there instead of a converged solve), which moves n10 by at most
    two cycles."""
    torch = torch_cuda()
    cfg = wl.paper_cartesian_periodic(p, "p")
    S = _solver(cfg, *s, dgfas.DGFAS_FP64)
    b = _rhs(cfg, S)
    u = torch.from_numpy(cfg["u0"]).cuda()
    info = S.dgfas_solve(u, b, 1e-10, 60)
    assert abs(info["cycles"] - _paper_n10()[("p", p) + s]) <= 2


# SCG smoother from the random start: every row of the paper's table at p = 4
# and 8 (mu_star = 2, delta = 0.08).  Tolerances (cycles): h-multigrid one
# cycle, p-multigrid two (the paper solves the p = 1 level by SCG to a
# tolerance, this hierarchy continues with h-levels to an exact 2^3 root).
SCG_ROWS = [k for k in _paper_rows() if k[5:] == ("mg", "scg", "I")]
# Full multigrid startup (Alg. 4) with embedded interpolation or L2 projection.
# With the exact root solve the startup leaves a residual 1e-8 .. 1e-9 of the
# random start's on these problems, so the solve needs at most the paper's
# cycles (measured: equal at h-multigrid p = 8, one to four fewer elsewhere;
# the paper's root solve is SCG with a step budget, Sec. 4.4).
FMG_ROWS = [k for k in _paper_rows() if k[5] == "fmg"]
# Cascadic startup (Alg. 3) with n_s0 = n_s1 + n_s2 smoothing steps per level
# (the study's setting): with the exact root the start leaves a smaller
# residual than the paper's, and the solve needs at most the paper's cycles
# (measured: equal at p-multigrid p = 4 SCG, one to six fewer elsewhere).
CMG_ROWS = [k for k in _paper_rows() if k[5] == "cmg"]


@pytest.mark.parametrize("row", SCG_ROWS, ids=lambda k: "-".join(str(x) for x in k))
def test_scg_rows_match_the_paper(row):
    want = _paper_rows()[row]
    got = n10_of(*row)
    tol = 2 if row[0] == "p" else 1
    assert abs(got - want) <= tol, (row, got, want)


@pytest.mark.parametrize("row", FMG_ROWS, ids=lambda k: "-".join(str(x) for x in k))
def test_fmg_rows_within_the_paper_counts(row):
    want = _paper_rows()[row]
    got = n10_of(*row)
    assert 1 <= got <= want, (row, got, want)


@pytest.mark.parametrize("row", CMG_ROWS, ids=lambda k: "-".join(str(x) for x in k))
def test_cmg_rows_within_the_paper_counts(row):
    want = _paper_rows()[row]
    got = n10_of(*row)
    assert 1 <= got <= want, (row, got, want)
