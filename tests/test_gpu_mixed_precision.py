"""Mixed-precision smoothing on the CUDA path against the FP64 oracle.

Sweep bound.  A BF16 tensor-core sweep rounds, in each of the six mode
products of the fast-diagonalization solve, the data operand and the matrix
operand to BF16 (unit roundoff u = 2^-8) and accumulates in FP32.  To first
order each product then adds 2u times the product of the absolute values, so
the computed correction differs from the exact one by at most

    12 u * sum_e R^T W (|S3| x |S2| x |S1|) |D|^-1 (|S3|^T x |S2|^T x |S1|^T) R |r|

node by node (W >= 0, D > 0).  The test evaluates that chain with the oracle's
tables in absolute value and allows 13 u (second-order terms) plus an FP32
allowance.  Levels whose subdomains are narrower than the tensor-core tiles
run the FP32 SIMT solve in BF16 mode: there u = 2^-24 and the FP32 sums of
up to 16 terms add 16 u per product.

Solve.  FP32 and BF16 smoothers inside the FP64 outer cycle (iterative
refinement) solved to r_2 <= 1e-12 r_2^0 agree with the oracle's FP64 solution
to 1e-8 of its largest entry (both solutions lie within 1e-12 r_2^0 / sigma_min
of the discrete solution)."""
import copy

import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import make_oracle, make_solver, rel, rhs_both, torch_cuda

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8
U_FP32 = 2.0 ** -24


def _abs_chain(sw, r):
    """sum_e R^T W (|S| x |S| x |S|) |D|^-1 (|S|^T x ...) R |r| with the oracle's tables."""
    a = copy.copy(sw)
    a.tables = copy.copy(sw.tables)
    a.tables.tab = {k: dict(v, S=np.abs(v["S"])) for k, v in sw.tables.tab.items()}
    return a.correction(np.abs(r))


@pytest.mark.parametrize("cid,small", [(2, True), (3, True), (5, True)])
def test_bf16_sweep_within_rounding_bound(cid, small):
    cfg = wl.config(cid, small=small)
    torch = torch_cuda()
    S = make_solver(cfg, precision=2)
    H = make_oracle(cfg)
    rng = np.random.default_rng(31)
    for l in range(1, S.n_levels):
        nd = S.ndof(l)
        u = rng.uniform(-1, 1, nd)
        g = rng.uniform(-1, 1, nd)
        ud, gd = torch.from_numpy(u).cuda(), torch.from_numpy(g).cuda()
        S.dgfas_schwarz_smooth(l, ud, gd, 1)
        got = ud.cpu().numpy() - u
        ref = H.was(l, u, g, 1) - u
        r = g - H.A(l, u)
        chain = _abs_chain(H.sw[l], r)
        N, m = H.sw[l].N, H.sw[l].m
        tc = N + 2 * m >= 12
        ub = U_BF16 if tc else U_FP32
        k = 13.0 if tc else 13.0 + 6 * 16
        bound = k * ub * chain + 1e-5 * np.abs(ref).max()
        err = np.abs(got - ref)
        assert np.all(err <= bound), (l, float((err / bound).max()))
        # measured, in the max norm of the level's correction: BF16 tensor-core
        # sweeps within a few percent, FP32 sweeps within 1e-4
        assert err.max() <= (0.1 if tc else 1e-4) * np.abs(ref).max(), l


@pytest.mark.parametrize("cid,small,root,smoother,prec", [
    (1, False, None, 0, 1), (1, False, None, 0, 2),
    (2, True, None, 0, 1), (2, True, None, 0, 2),
    (3, True, "p1", 1, 1), (3, True, "p1", 1, 2),
    (5, True, "p1", 1, 1), (5, True, "p1", 1, 2)])
def test_mixed_solve_matches_fp64_oracle(cid, small, root, smoother, prec):
    cfg = wl.config(cid, small=small, root=root)
    torch = torch_cuda()
    S = make_solver(cfg, precision=prec, smoother=smoother)
    H = make_oracle(cfg, smoother="scg" if smoother else "was")
    b, b_or = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    info = S.dgfas_solve(u, b, 1e-12, 60)
    uo, hist = H.solve(cfg["u0"], b_or, rtol=1e-12, max_cycles=60)
    assert info["r_final"] <= 1e-12 * info["r0"]
    assert hist[-1] <= 1e-12 * hist[0]
    assert rel(u.cpu().numpy(), uo) < 1e-8
