"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 operator applies 1e-12 relative (max-norm over the vector,
relative to its max entry); one smoother sweep and one V-cycle 1e-10; solves
reach r_2 <= 1e-10 r_2^0.  The FP32 smoother is checked by the solve reaching
1e-10 (the FP64 outer cycle acts as iterative refinement) and by its sweep
agreeing with the FP64 sweep to FP32 accuracy."""
import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import make_oracle, make_solver, rel, rhs_both, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [(1, False), (2, True), (3, True), (5, True)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"cfg{c[0]}{'s' if c[1] else ''}")
def pair(request):
    cid, small = request.param
    cfg = wl.config(cid, small=small)
    return cfg, make_solver(cfg), make_oracle(cfg)


def test_node_coords_and_rhs(pair):
    cfg, S, H = pair
    torch = torch_cuda()
    xyz = S.node_coords(-1).cpu().numpy()
    assert rel(xyz, H.ops[-1].geo["x"].reshape(-1, 3)) < 1e-14
    b, b_or = rhs_both(cfg, S, H)
    assert rel(b.cpu().numpy(), b_or) < 1e-12


def test_apply_every_level(pair):
    cfg, S, H = pair
    torch = torch_cuda()
    rng = np.random.default_rng(11)
    for l in range(S.n_levels):
        n = S.ndof(l)
        u = rng.uniform(-1, 1, n)
        g = rng.uniform(-1, 1, n)
        ud, gd = torch.from_numpy(u).cuda(), torch.from_numpy(g).cuda()
        out = torch.empty_like(ud)
        S.dgfas_apply_op(l, ud, None, out)
        Au = H.A(l, u)
        assert rel(out.cpu().numpy(), Au) < 1e-12, l
        S.dgfas_apply_op(l, ud, gd, out)
        assert rel(out.cpu().numpy(), g - Au) < 1e-12, l


def test_apply32_every_level(pair):
    """The FP32 operator of the smoothers (on curvilinear levels with the
    metric recomputed in FP32 from the trilinear map) against the oracle's
    FP64 operator on the same FP32 input: out = g - A u and A u to 3e-5 of
    max |A u| (random u: no cancellation, FP32 rounding of a few dozen terms
    per entry; a missing or wrong term errs by percents)."""
    cfg, S, H = pair
    torch = torch_cuda()
    rng = np.random.default_rng(13)
    for l in range(S.n_levels):
        n = S.ndof(l)
        u = rng.uniform(-1, 1, n).astype(np.float32)
        g = rng.uniform(-1, 1, n)
        ud, gd = torch.from_numpy(u).cuda(), torch.from_numpy(g).cuda()
        out = torch.empty_like(ud)
        Au = H.A(l, u.astype(np.float64))
        scale = np.abs(Au).max()
        S.dgfas_apply_op32(l, ud, None, out)
        assert np.abs(out.cpu().numpy() - Au).max() <= 3e-5 * scale, l
        S.dgfas_apply_op32(l, ud, gd, out)
        assert np.abs(out.cpu().numpy() - (g - Au)).max() <= 3e-5 * (scale + 1.0), l


def test_one_sweep_each_level(pair):
    cfg, S, H = pair
    torch = torch_cuda()
    rng = np.random.default_rng(12)
    for l in range(1, S.n_levels):
        n = S.ndof(l)
        u = rng.uniform(-1, 1, n)
        g = rng.uniform(-1, 1, n)
        ud, gd = torch.from_numpy(u).cuda(), torch.from_numpy(g).cuda()
        S.dgfas_schwarz_smooth(l, ud, gd, 1)
        ref = H.was(l, u, g, 1)
        assert rel(ud.cpu().numpy() - u, ref - u) < 1e-10, l


def test_vcycle_iterates(pair):
    cfg, S, H = pair
    torch = torch_cuda()
    b, b_or = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    uo = H.zero_levels(cfg["u0"])
    for k in range(2):
        rn = S.dgfas_fas_vcycle(u, b)
        uo, rno = H.fas_vcycle(uo, b_or)
        assert abs(rn - rno) <= 1e-10 * rno
        assert rel(u.cpu().numpy(), uo[-1]) < 1e-10, k


def test_fp32_sweep_close_to_fp64():
    cfg = wl.config(2, small=True)
    torch = torch_cuda()
    S64, S32 = make_solver(cfg, precision=0), make_solver(cfg, precision=1)
    rng = np.random.default_rng(3)
    L = S64.n_levels - 1
    n = S64.ndof(L)
    u = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    g = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    u64, u32 = u.clone(), u.clone()
    S64.dgfas_schwarz_smooth(L, u64, g, 1)
    S32.dgfas_schwarz_smooth(L, u32, g, 1)
    d64, d32 = (u64 - u).cpu().numpy(), (u32 - u).cpu().numpy()
    assert rel(d32, d64) < 1e-4


@pytest.mark.parametrize("cid,small,prec", [(1, False, 0), (1, False, 1), (2, True, 0), (2, True, 1)])
def test_solve_reaches_1e10(cid, small, prec):
    cfg = wl.config(cid, small=small)
    torch = torch_cuda()
    S, H = make_solver(cfg, precision=prec), make_oracle(cfg)
    b, b_or = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    info = S.dgfas_solve(u, b, 1e-10, 40)
    assert info["r_final"] <= 1e-10 * info["r0"]
    uo, hist = H.solve(cfg["u0"], b_or)
    if prec == 0:
        assert info["cycles"] == len(hist) - 1
        assert rel(u.cpu().numpy(), uo) < 1e-9
    else:
        assert info["cycles"] <= len(hist) - 1 + 2
        assert rel(u.cpu().numpy(), uo) < 1e-8


def test_graph_replay_matches_direct_launches():
    cfg = wl.config(1)
    torch = torch_cuda()
    S1, S2 = make_solver(cfg, precision=1), make_solver(cfg, precision=1)
    S2.dgfas_use_graph(True)
    H = make_oracle(cfg)
    b, _ = rhs_both(cfg, S1, H)
    u1 = torch.from_numpy(cfg["u0"].copy()).cuda()
    u2 = u1.clone()
    for _ in range(3):
        r1 = S1.dgfas_fas_vcycle(u1, b)
        r2 = S2.dgfas_fas_vcycle(u2, b)
    assert r1 == r2
    assert torch.equal(u1, u2)
    i1 = S1.dgfas_solve(u1.clone(), b, 1e-10, 30)
    i2 = S2.dgfas_solve(u2.clone(), b, 1e-10, 30)
    assert i1["cycles"] == i2["cycles"] and i1["history"] == i2["history"]


@pytest.mark.parametrize("cid,small", CASES, ids=lambda c: str(c))
def test_vcycle_iterates_l2_projection(cid, small):
    """The L2 projection variant of P (Sec. 3.2): V-cycle iterates match the
    oracle's with the same variant (p- and h-transfers)."""
    cfg = wl.config(cid, small=small)
    torch = torch_cuda()
    S = make_solver(cfg, projection="l2")
    H = make_oracle(cfg, projection="l2")
    b, b_or = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    uo = H.zero_levels(cfg["u0"])
    for k in range(2):
        rn = S.dgfas_fas_vcycle(u, b)
        uo, rno = H.fas_vcycle(uo, b_or)
        assert abs(rn - rno) <= 1e-10 * rno
        assert rel(u.cpu().numpy(), uo[-1]) < 1e-10, k
