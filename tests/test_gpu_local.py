"""GPU parity on a locally refined multilevel mesh (Sec. 3.1, config 4 small):
twigs, leaves and frozen elements on the refinement levels, leaf right-hand
sides on every level, composite residual (Sec. 6.1)."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import rel, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = torch_cuda()
    from oracle import fas, sip
    cfg = wl.config4(small=True)
    pr = cfg["params"]
    S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    H = fas.LocalHierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    f_or, f_gpu = [], []
    for l, op in enumerate(H.ops):
        X = op.geo["x"]
        f_or.append(sip.rhs(op, wl.eval_front_f(cfg["rhs"], X), wl.eval_front_u(cfg["rhs"], X)).reshape(-1))
        xyz = S.node_coords(l).cpu().numpy()
        fn = torch.from_numpy(wl.eval_front_f(cfg["rhs"], xyz)).cuda()
        un = torch.from_numpy(wl.eval_front_u(cfg["rhs"], xyz)).cuda()
        b = torch.empty_like(fn)
        S.dgfas_assemble_rhs_level(l, fn, un, b)
        if l < S.n_levels - 1:
            S.dgfas_set_level_rhs(l, b)
        f_gpu.append(b)
    torch.cuda.synchronize()
    return cfg, S, H, f_or, f_gpu


def test_level_rhs(setup):
    cfg, S, H, f_or, f_gpu = setup
    for l in range(S.n_levels):
        assert rel(f_gpu[l].cpu().numpy(), f_or[l]) < 1e-12, l


def test_apply_and_sweep_every_level(setup):
    cfg, S, H, f_or, f_gpu = setup
    torch = torch_cuda()
    rng = np.random.default_rng(21)
    for l in range(S.n_levels):
        n = S.ndof(l)
        u = rng.uniform(-1, 1, n)
        g = rng.uniform(-1, 1, n)
        ud, gd = torch.from_numpy(u).cuda(), torch.from_numpy(g).cuda()
        out = torch.empty_like(ud)
        S.dgfas_apply_op(l, ud, gd, out)
        ref = g - H.A(l, u)
        ref[np.repeat(H.cls[l] == 2, H.ops[l].N ** 3)] = 0.0     # r^f = 0 (Eq. (4d))
        assert rel(out.cpu().numpy(), ref) < 1e-12, l
        if l > 0:
            S.dgfas_schwarz_smooth(l, ud, gd, 1)
            ref = H.was(l, u, g, 1)
            assert rel(ud.cpu().numpy() - u, ref - u) < 1e-10, l


def test_vcycles_and_solve(setup):
    cfg, S, H, f_or, f_gpu = setup
    torch = torch_cuda()
    L = S.n_levels - 1
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    uo = [np.zeros(op.ndof) for op in H.ops]
    uo[L] = cfg["u0"].copy()
    for k in range(2):
        S.dgfas_fas_vcycle(u, f_gpu[L])
        uo, _ = H.fas_vcycle_local(uo, f_or)
        assert rel(u.cpu().numpy(), uo[L]) < 1e-10, k
        for l in range(1, L):
            ul = torch.empty(S.ndof(l), dtype=torch.float64, device="cuda")
            S.dgfas_get_level_solution(l, ul)
            assert rel(ul.cpu().numpy(), uo[l]) < 1e-10, (k, l)
    r_gpu = S.dgfas_composite_residual(u, f_gpu[L])
    r_or = H.composite_residual(uo, f_or)
    assert abs(r_gpu - r_or) <= 1e-10 * r_or


def test_solve_reaches_1e10_like_oracle():
    torch = torch_cuda()
    from oracle import fas, sip
    cfg = wl.config4(small=True)
    pr = cfg["params"]
    for prec in (dgfas.DGFAS_FP64, dgfas.DGFAS_FP32):
        S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                         precision=prec)
        L = S.n_levels - 1
        fl = None
        for l in range(S.n_levels):
            xyz = S.node_coords(l).cpu().numpy()
            fn = torch.from_numpy(wl.eval_front_f(cfg["rhs"], xyz)).cuda()
            un = torch.from_numpy(wl.eval_front_u(cfg["rhs"], xyz)).cuda()
            b = torch.empty_like(fn)
            S.dgfas_assemble_rhs_level(l, fn, un, b)
            if l < L:
                S.dgfas_set_level_rhs(l, b)
            fl = b
        u = torch.from_numpy(cfg["u0"].copy()).cuda()
        info = S.dgfas_solve(u, fl, 1e-10, 40)
        assert info["r_final"] <= 1e-10 * info["r0"]
        if prec == dgfas.DGFAS_FP64:
            H = fas.LocalHierarchy(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"],
                                   pr["sc"])
            f_or = []
            for op in H.ops:
                X = op.geo["x"]
                f_or.append(sip.rhs(op, wl.eval_front_f(cfg["rhs"], X),
                                    wl.eval_front_u(cfg["rhs"], X)).reshape(-1))
            uo = [np.zeros(op.ndof) for op in H.ops]
            uo[L] = cfg["u0"].copy()
            uo, hist = H.solve_local(uo, f_or)
            assert info["cycles"] == len(hist) - 1
