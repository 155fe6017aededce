"""GPU parity of the full multigrid startup (Alg. 4) with the oracle: the FP64
start value on configs 1 and 2 (small), the mixed-precision start followed by
V-cycles to 1e-10, and the rejection of locally refined hierarchies."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import make_oracle, make_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _level_rhs(cfg, S, H):
    """Each level's own right-hand side, assembled by each side from the same
    nodal f (homogeneous Dirichlet data)."""
    torch = torch_cuda()
    from oracle import sip
    f_or, f_gpu = [], []
    for l, op in enumerate(H.ops):
        X = op.geo["x"]
        f_or.append(sip.rhs(op, wl.eval_f(cfg["rhs"], X), np.zeros(X.shape[:-1])).reshape(-1))
        xyz = S.node_coords(l).cpu().numpy()
        fn = torch.from_numpy(wl.eval_f(cfg["rhs"], xyz)).cuda()
        b = torch.empty_like(fn)
        S.dgfas_assemble_rhs_level(l, fn, None, b)
        f_gpu.append(b)
    torch.cuda.synchronize()
    return f_or, f_gpu


@pytest.mark.parametrize("cid,small", [(1, False), (2, True)])
def test_fmg_start_matches_oracle_fp64(cid, small):
    torch = torch_cuda()
    cfg = wl.config(cid, small=small)
    S, H = make_solver(cfg, precision=dgfas.DGFAS_FP64), make_oracle(cfg)
    f_or, f_gpu = _level_rhs(cfg, S, H)
    for l in range(S.n_levels):
        assert rel(f_gpu[l].cpu().numpy(), f_or[l]) < 1e-12, l
    u = torch.zeros(S.ndof(-1), dtype=torch.float64, device="cuda")
    S.dgfas_fmg(f_gpu, u)
    u_or = H.fmg(f_or, cycles=1)
    assert rel(u.cpu().numpy(), u_or) < 1e-11


def test_fmg_then_mixed_solve_reaches_1e10():
    torch = torch_cuda()
    cfg = wl.config(2, small=True)
    S, H = make_solver(cfg, precision=dgfas.DGFAS_BF16), make_oracle(cfg)
    _, f_gpu = _level_rhs(cfg, S, H)
    b = f_gpu[-1]
    r_zero = float(torch.linalg.norm(b))
    u = torch.zeros_like(b)
    S.dgfas_fmg(f_gpu, u)
    r = torch.empty_like(b)
    S.dgfas_apply_op(-1, u, b, r)   # r = b - A u of the FMG value
    r_fmg = S.dgfas_norm(-1, r)
    assert r_fmg < r_zero
    info = S.dgfas_solve(u, b, 1e-10 * r_zero / r_fmg, 40)
    assert info["r_final"] <= 1e-10 * r_zero * (1 + 1e-9)


def test_fmg_on_local_refinement_matches_oracle():
    """Config 4 (small): the FP64 FMG start on every level (the top's and the
    level solutions left for the composite solve) against the oracle, then
    the mixed-precision solve from it reaches 1e-10 of the zero start's
    composite residual."""
    torch = torch_cuda()
    from oracle import fas, sip
    cfg = wl.config4(small=True)
    pr = cfg["params"]
    H = fas.LocalHierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    f_or = []
    for op in H.ops:
        X = op.geo["x"]
        f_or.append(sip.rhs(op, wl.eval_front_f(cfg["rhs"], X),
                            wl.eval_front_u(cfg["rhs"], X)).reshape(-1))
    u_or = H.fmg_local(f_or, cycles=1)
    for prec in (dgfas.DGFAS_FP64, dgfas.DGFAS_FP32):
        S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                         precision=prec)
        L = S.n_levels - 1
        f_gpu = []
        for l in range(S.n_levels):
            xyz = S.node_coords(l).cpu().numpy()
            fn = torch.from_numpy(wl.eval_front_f(cfg["rhs"], xyz)).cuda()
            un = torch.from_numpy(wl.eval_front_u(cfg["rhs"], xyz)).cuda()
            b = torch.empty_like(fn)
            S.dgfas_assemble_rhs_level(l, fn, un, b)
            if l < L:
                S.dgfas_set_level_rhs(l, b)
            f_gpu.append(b)
        u = torch.zeros_like(f_gpu[-1])
        S.dgfas_fmg(f_gpu, u)
        if prec == dgfas.DGFAS_FP64:
            assert rel(u.cpu().numpy(), u_or[L]) < 1e-11
            for l in range(L):
                ul = torch.empty(S.ndof(l), dtype=torch.float64, device="cuda")
                S.dgfas_get_level_solution(l, ul)
                assert rel(ul.cpu().numpy(), u_or[l]) < 1e-11, l
        else:
            r_zero = H.composite_residual([np.zeros(op.ndof) for op in H.ops], f_or)
            r_f = S.dgfas_composite_residual(u, f_gpu[-1])
            info = S.dgfas_solve(u, f_gpu[-1], 1e-10 * r_zero / r_f, 40)
            assert info["r_final"] <= 1e-10 * r_zero * (1 + 1e-9)


@pytest.mark.parametrize("cid,small,root,smoother", [(1, False, None, "was"), (2, True, None, "was"),
                                                     (5, True, "p1", "scg")])
def test_cmg_start_matches_oracle_fp64(cid, small, root, smoother):
    """Cascadic startup (Alg. 3): the top start value and the level solutions
    it leaves below the top match the oracle's (FP64; WAS, and SCG with the
    SCG root at p = 1), for n_sc = 0 (interpolation only) and the workload's
    n_sc."""
    torch = torch_cuda()
    cfg = wl.config(cid, small=small, root=root)
    sm = dgfas.DGFAS_SCG if smoother == "scg" else dgfas.DGFAS_WAS
    S = make_solver(cfg, precision=dgfas.DGFAS_FP64, smoother=sm)
    H = make_oracle(cfg, smoother=smoother)
    f_or, f_gpu = _level_rhs(cfg, S, H)
    for sc in (0, cfg["params"]["sc"]):
        u = torch.zeros(S.ndof(-1), dtype=torch.float64, device="cuda")
        S.dgfas_cmg(f_gpu, u, sc)
        u_or = H.cmg(f_or, sc=sc)
        assert rel(u.cpu().numpy(), u_or[-1]) < 1e-10, sc
        for l in range(S.n_levels - 1):
            ul = torch.empty(S.ndof(l), dtype=torch.float64, device="cuda")
            S.dgfas_get_level_solution(l, ul)
            assert rel(ul.cpu().numpy(), u_or[l]) < 1e-10, (sc, l)


def test_cmg_then_mixed_solve_reaches_1e10():
    torch = torch_cuda()
    cfg = wl.config(2, small=True)
    S, H = make_solver(cfg, precision=dgfas.DGFAS_BF16), make_oracle(cfg)
    _, f_gpu = _level_rhs(cfg, S, H)
    b = f_gpu[-1]
    r_zero = float(torch.linalg.norm(b))
    u = torch.zeros_like(b)
    S.dgfas_cmg(f_gpu, u, cfg["params"]["sc"])
    r = torch.empty_like(b)
    S.dgfas_apply_op(-1, u, b, r)
    r_c = S.dgfas_norm(-1, r)
    assert r_c < r_zero
    info = S.dgfas_solve(u, b, 1e-10 * r_zero / r_c, 40)
    assert info["r_final"] <= 1e-10 * r_zero * (1 + 1e-9)
