"""GPU parity of SCG (Alg. 6) through the C ABI against the FP64 oracle.

The CUDA path keeps every scalar of the recurrence on the device; these tests
compare its iterates with the oracle's step by step (1e-10 relative, FP64),
V-cycle by V-cycle with SCG as smoother and as the root solver of the
p-multigrid hierarchies of the curvilinear workloads (p 7 -> 3 -> 1, root SCG
at p = 1), check that solves reach 1e-10 with the oracle's cycle count and
solution, and that the CUDA-graph replay of an SCG cycle is bit-identical to
direct launches."""
import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import make_oracle, make_solver, rel, rhs_both, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [(1, False, None), (3, True, None), (5, True, None), (3, True, "p1"), (5, True, "p1")]


def _ids(c):
    return f"cfg{c[0]}{'s' if c[1] else ''}{'-' + c[2] if c[2] else ''}"


@pytest.fixture(scope="module", params=CASES, ids=_ids)
def pair(request):
    cid, small, root = request.param
    cfg = wl.config(cid, small=small, root=root)
    return cfg, make_solver(cfg, smoother=1), make_oracle(cfg, smoother="scg")


def test_scg_steps_each_level(pair):
    """n = 1..4 SCG steps on every level from a random start: the iterate
    matches the oracle's (the correction u_n - u_0, 1e-10 relative)."""
    cfg, S, H = pair
    torch = torch_cuda()
    rng = np.random.default_rng(21)
    for l in range(1, S.n_levels):
        nd = S.ndof(l)
        u = rng.uniform(-1, 1, nd)
        g = rng.uniform(-1, 1, nd)
        gd = torch.from_numpy(g).cuda()
        for n in (1, 2, 3, 4):
            ud = torch.from_numpy(u).cuda()
            S.dgfas_schwarz_smooth(l, ud, gd, n)
            ref = H.scg(l, u, g, n, 0.0)
            assert rel(ud.cpu().numpy() - u, ref - u) < 1e-10, (l, n)


def test_scg_vcycle_iterates(pair):
    cfg, S, H = pair
    torch = torch_cuda()
    b, b_or = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    uo = H.zero_levels(cfg["u0"])
    for k in range(2):
        rn = S.dgfas_fas_vcycle(u, b)
        uo, rno = H.fas_vcycle(uo, b_or)
        assert abs(rn - rno) <= 1e-10 * rno, k
        assert rel(u.cpu().numpy(), uo[-1]) < 1e-10, k


def test_scg_solve_matches_oracle(pair):
    cfg, S, H = pair
    torch = torch_cuda()
    b, b_or = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    info = S.dgfas_solve(u, b, 1e-10, 40)
    uo, hist = H.solve(cfg["u0"], b_or, max_cycles=40)
    assert info["r_final"] <= 1e-10 * info["r0"]
    assert info["cycles"] == len(hist) - 1
    assert rel(u.cpu().numpy(), uo) < 1e-9


def test_scg_root_from_zero_in_fmg_matches_oracle():
    """The SCG root from a zero start (the first step of the full multigrid
    startup, Alg. 4) and the startup's sub-hierarchy cycles: the FMG start
    value of the top level matches the oracle's."""
    cfg = wl.config(5, small=True, root="p1")
    torch = torch_cuda()
    S, H = make_solver(cfg, smoother=1), make_oracle(cfg, smoother="scg")
    rng = np.random.default_rng(5)
    f = [rng.uniform(-1, 1, S.ndof(l)) for l in range(S.n_levels)]
    ref = H.fmg(f)
    u_top = torch.empty(S.ndof(), dtype=torch.float64, device="cuda")
    S.dgfas_fmg([torch.from_numpy(x).cuda() for x in f], u_top, 1)
    assert rel(u_top.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("prec", [1, 2])
def test_scg_graph_replay_bit_identical(prec):
    cfg = wl.config(5, small=True, root="p1")
    torch = torch_cuda()
    S1, S2 = make_solver(cfg, precision=prec, smoother=1), make_solver(cfg, precision=prec,
                                                                       smoother=1)
    S2.dgfas_use_graph(True)
    H = make_oracle(cfg, smoother="scg")
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


@pytest.mark.parametrize("case,prec", [((3, True, "p1"), 1), ((3, True, "p1"), 2),
                                       ((5, True, "p1"), 1), ((5, True, "p1"), 2)])
def test_scg_mixed_precision_solve_cycles(case, prec):
    """SCG in correction form on FP32 vectors (FP32 operator, FP32 / BF16
    Schwarz sweep) inside the FP64 outer cycle: the solve reaches 1e-10 in at
    most two cycles more than the FP64 oracle (the solutions at 1e-12 are
    compared in test_gpu_mixed_precision)."""
    cid, small, root = case
    cfg = wl.config(cid, small=small, root=root)
    torch = torch_cuda()
    S, H = make_solver(cfg, precision=prec, smoother=1), make_oracle(cfg, smoother="scg")
    b, b_or = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    info = S.dgfas_solve(u, b, 1e-10, 40)
    uo, hist = H.solve(cfg["u0"], b_or, max_cycles=40)
    assert info["r_final"] <= 1e-10 * info["r0"]
    assert info["cycles"] <= len(hist) - 1 + 2



@pytest.mark.parametrize("steps,rtol,reached", [(200, 1e-6, True), (2, 1e-14, False)])
def test_scg_root_reports_whether_it_reached_its_tolerance(steps, rtol, reached):
    """The root SCG's step cap and exit test (Sec. 4.3.2): with the Schwarz
    smoother the root solve is the last SCG block of a V-cycle, and
    dgfas_scg_info reports its steps, final |r|^2 and whether it stopped at
    |r| <= root_rtol |r_start| (reached) or at its step cap; the steps and
    |r|^2 match the oracle's loop from the same projected start."""
    torch = torch_cuda()
    cfg = wl.config(5, small=True, root="p1")
    S = make_solver(cfg, smoother=0, coarse="scg", root_steps=steps, root_rtol=rtol)
    H = make_oracle(cfg, smoother="was", coarse="scg", root_steps=steps, root_rtol=rtol)
    calls = [0]
    sweep = H.sw[0].correction

    def counted(r):
        calls[0] += 1
        return sweep(r)

    H.sw[0].correction = counted
    last = {}
    scg = H.scg

    def scg_rr(l, u, f, n, r_max, precond=None, first=None):
        out = scg(l, u, f, n, r_max, precond, first)
        if l == 0:
            calls_then = calls[0]
            last.update(steps=calls_then, rr=float(np.sum((f - H.A(0, out)) ** 2)),
                        r_max=r_max)
            calls[0] = 0
        return out

    H.scg = scg_rr
    b, b_or = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    S.dgfas_fas_vcycle(u, b)
    H.fas_vcycle(H.zero_levels(cfg["u0"]), b_or)
    rr, n, done = S.dgfas_scg_info()
    assert done == reached
    assert n == last["steps"] == (n if reached else steps)
    # the device's |r|^2 is the recursive residual's, the oracle's the true
    # one; they part by about steps * eps * |A| |u|, 1e-5 of |r|^2 here
    assert abs(rr - last["rr"]) <= 1e-3 * last["rr"]
    if reached:
        assert rr <= last["r_max"] ** 2 * (1 + 1e-9)
    S.close()
