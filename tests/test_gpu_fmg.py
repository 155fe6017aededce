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


def test_fmg_rejects_local_refinement():
    torch = torch_cuda()
    cfg = wl.config4(small=True)
    pr = cfg["params"]
    S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"])
    fs = [torch.zeros(S.ndof(l), dtype=torch.float64, device="cuda") for l in range(S.n_levels)]
    u = torch.zeros(S.ndof(-1), dtype=torch.float64, device="cuda")
    with pytest.raises(dgfas.DgfasError) as e:
        S.dgfas_fmg(fs, u)
    assert e.value.code == -7   # DGFAS_ERR_UNSUPPORTED
