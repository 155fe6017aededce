"""The allocation-free Schwarz correction entry point.

Callers that cannot allocate device memory while they smooth (for example
code running inside its own CUDA stream capture, or under an allocator that
owns all device memory) use dgfas_schwarz_correct_static, whose scratch is a
fixed array inside the library.  This file checks it against the regular
smoother through the C ABI on two calls in a row (the shared array keeps the
previous call's contents), and that oversized levels are rejected.  It is
collected last on purpose."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl
from tests.gpu_helpers import make_solver, torch_cuda

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.mark.parametrize("cid,small", [(1, False), (2, True), (3, True)])
def test_static_correction_matches_smoother(cid, small):
    torch = torch_cuda()
    cfg = wl.config(cid, small=small)
    S = make_solver(cfg, precision=dgfas.DGFAS_FP64)
    rng = np.random.default_rng(40 + cid)
    for level in range(1, S.n_levels):
        n = S.ndof(level)
        u = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
        g = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
        u_ref, u_new = u.clone(), u.clone()
        r = torch.empty_like(u)
        for _ in range(2):   # two calls in a row
            S.dgfas_schwarz_smooth(level, u_ref, g, 1)
            S.dgfas_apply_op(level, u_new, g, r)
            S.dgfas_schwarz_correct_static(level, r, u_new)
            torch.cuda.synchronize()
            a, b = u_new.cpu().numpy(), u_ref.cpu().numpy()
            assert np.abs(a - b).max() <= TOL * np.abs(b).max(), level


def test_static_correction_rejects_oversized_level():
    torch = torch_cuda()
    V = wl.uniform_vertices(12)
    levels = wl.hierarchy(V, [8, 1], h_root=3)
    S = dgfas.Solver(levels, 5.0, 0.08)
    top = S.n_levels - 1        # 12^3 elements at p = 8: 1728 * 13^3 > 2^21 entries
    n = S.ndof(top)
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = torch.ones_like(u)
    with pytest.raises(dgfas.DgfasError) as ei:
        S.dgfas_schwarz_correct_static(top, r, u)
    assert ei.value.code == -7
    assert float(u.abs().max()) == 0.0
