"""Tensor-core (tcgen05, BF16 -> FP32 in TMEM) building block of the FD solve."""
import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas

pytestmark = pytest.mark.gpu


def test_tcgen05_mma_selftest():
    D, timed_out = dgfas.dgfas_tc_selftest()
    assert not timed_out
    r = np.arange(128)[:, None]
    k = np.arange(16)[None, :]
    A = ((r + 2 * k) % 7 - 3).astype(np.float64)
    n = np.arange(16)[:, None]
    B = ((3 * n + k) % 5 - 2).astype(np.float64)
    np.testing.assert_array_equal(D, A @ B.T)


def _sweep(cfg, prec, level, seed=3):
    from tests.gpu_helpers import make_solver, torch_cuda
    torch = torch_cuda()
    S = make_solver(cfg, precision=prec)
    rng = np.random.default_rng(seed)
    n = S.ndof(level)
    u = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    g = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    u1 = u.clone()
    S.dgfas_schwarz_smooth(level, u1, g, 1)
    assert S.dgfas_tc_error() == 0
    return (u1 - u).cpu().numpy()


@pytest.mark.parametrize("cid,small", [(1, False), (2, True), (3, True)])
def test_bf16_tensor_core_sweep_matches_fp32(cid, small):
    """One Schwarz sweep with the tensor-core FD (BF16 operands, FP32
    accumulation) against the FP32 SIMT FD: BF16 rounding of the six mode
    products bounds the difference (~1e-2 of the correction)."""
    from paper_2608_14123_b300 import workloads as wl
    cfg = wl.config(cid, small=small)
    for level in range(1, len(cfg["levels"])):
        d32 = _sweep(cfg, dgfas.DGFAS_FP32, level)
        d16 = _sweep(cfg, dgfas.DGFAS_BF16, level)
        err = np.linalg.norm(d16 - d32) / np.linalg.norm(d32)
        assert err < 3e-2, (level, err)


@pytest.mark.parametrize("cid,small", [(1, False), (2, True)])
def test_bf16_smoother_solve_reaches_1e10(cid, small):
    from paper_2608_14123_b300 import workloads as wl
    from tests.gpu_helpers import make_oracle, make_solver, rhs_both, torch_cuda
    torch = torch_cuda()
    cfg = wl.config(cid, small=small)
    S, H = make_solver(cfg, precision=dgfas.DGFAS_BF16), make_oracle(cfg)
    b, _ = rhs_both(cfg, S, H)
    u = torch.from_numpy(cfg["u0"].copy()).cuda()
    info = S.dgfas_solve(u, b, 1e-10, 40)
    assert info["r_final"] <= 1e-10 * info["r0"]
    assert S.dgfas_tc_error() == 0


def test_tcgen05_mn_major_operand_selftest():
    """MN-major A operand (the layout the FD kernel writes without transposing
    in shared memory): leading byte offset = core-matrix stride along K, stride
    byte offset = core-matrix stride along M."""
    import ctypes
    lib = dgfas.load()
    out = np.zeros(2 * 128 * 16, dtype=np.float32)
    to = ctypes.c_int(0)
    assert lib.dgfas_tc_selftest_mn(out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(to)) == 0
    assert to.value == 0
    r = np.arange(128)[:, None]
    k = np.arange(16)[None, :]
    A = ((r + 2 * k) % 7 - 3).astype(np.float64)
    n = np.arange(16)[:, None]
    B = ((3 * n + k) % 5 - 2).astype(np.float64)
    np.testing.assert_array_equal(out.reshape(2, 128, 16)[1], A @ B.T)


def test_bf16_sweep_many_elements_per_cta():
    """The tensor-core FD keeps one CTA per SM slot and walks several elements
    per CTA (about 3.5 here: 4096 elements, p = 7, curvilinear), reusing its
    shared operand buffers; the small workloads give most CTAs one element.
    The sweep must stay finite and within BF16 rounding of the FP32 SIMT sweep
    on every node block, and a BF16 SCG solve must reach 1e-10."""
    from paper_2608_14123_b300 import workloads as wl
    from tests.gpu_helpers import torch_cuda
    torch = torch_cuda()
    rng = np.random.default_rng(wl.SEED_BASE + 5)
    V = wl.perturbed_vertices(16, 0.15, rng)
    levels = wl.hierarchy(V, [7, 3, 1], h_root=4)
    top = len(levels) - 1
    n = levels[top]["corners"].shape[0] * 8 ** 3
    u = rng.uniform(-1, 1, n)
    g = rng.uniform(-1, 1, n)
    d = {}
    for prec in (dgfas.DGFAS_FP32, dgfas.DGFAS_BF16):
        S = dgfas.Solver(levels, 5.0, 0.08, 2, 2, 4, precision=prec, smoother=dgfas.DGFAS_SCG)
        ud = torch.from_numpy(u).cuda()
        S.dgfas_schwarz_smooth(top, ud, torch.from_numpy(g).cuda(), 1)
        assert S.dgfas_tc_error() == 0
        d[prec] = ud.cpu().numpy() - u
        S.close()
    d16, d32 = d[dgfas.DGFAS_BF16], d[dgfas.DGFAS_FP32]
    assert np.all(np.isfinite(d16))
    # per element: BF16 rounding of the six mode products, well below 10%
    e16, e32 = d16.reshape(-1, 512), d32.reshape(-1, 512)
    per = np.linalg.norm(e16 - e32, axis=1) / np.linalg.norm(e32, axis=1)
    assert per.max() < 0.1, per.max()
    S = dgfas.Solver(levels, 5.0, 0.08, 2, 2, 4, precision=dgfas.DGFAS_BF16,
                     smoother=dgfas.DGFAS_SCG)
    b = torch.from_numpy(g).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = S.dgfas_solve(x, b, 1e-10, 20)
    assert info["r_final"] <= 1e-10 * info["r0"]
    assert S.dgfas_tc_error() == 0
    S.close()
